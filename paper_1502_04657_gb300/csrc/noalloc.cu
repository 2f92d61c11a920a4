// Allocation-free variant of the coarsest-level nonlinear solve.
//
// Some callers may not allocate device memory at all: frameworks that hand every byte of
// the GPU to their own pool and do not let libraries call cudaMalloc (an outside allocation
// can fail or fragment their pool), and services that must not allocate once they serve
// (cudaMalloc and cudaFree can synchronise the device and stall the requests in flight).
// For them fmg_eig_coarse_solve_noalloc computes the same result as fmg_eig_coarse_solve
// without a handle: the caller passes the problem and the output buffers, and every
// intermediate lives in one fixed device array declared in this file (kScratchDoubles
// doubles, 256 KiB, held by every GPU that loads the library until the process exits).
//
// The array's name is only a host-side stand-in in host code, so its device address is
// looked up once per device with cudaGetSymbolAddress (with that device current) on the
// first call that runs on the device, and kept for the life of the process; the lookup is
// not repeated after cudaDeviceReset, so a process that resets a device must not call this
// function on that device again.  The call copies small tables from host memory and
// synchronises its stream before it returns.  All calls share the one array: concurrent or
// overlapping calls on the GPU race with each other and must be serialised by the caller.
#include <mutex>

#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr size_t kScratchDoubles = 32768;  // 256 KiB
constexpr int kMaxCoarseCells = 9;         // 64 coarse unknowns: the dense solve's shared-memory limit
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace fmg

using namespace fmg;

extern "C" int fmg_eig_coarse_solve_noalloc(const fmg_eig_problem* prob, double* lambda_out,
                                            double* u_dev, int32_t* iters, void* stream) {
  if (!prob || !lambda_out || !u_dev) return FMG_EINVAL;
  if (prob->dim != 2 || prob->precision != FMG_FP64 || prob->operator_form != FMG_W_LEFT)
    return FMG_ENOTSUP;
  const int n1 = prob->coarse_cells;
  if (n1 < 2 || n1 > kMaxCoarseCells) return FMG_EINVAL;  // beyond the fixed scratch
  if (!(prob->box_len > 0.0) || !(prob->zeta >= 0.0) ||
      !(prob->omega > 0.0 && prob->omega <= 1.0) || !(prob->scf_tol > 0.0) ||
      prob->scf_max_iter < 1)
    return FMG_EINVAL;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);

  double* base = nullptr;
  if (scratch_on_current_device(&base) != cudaSuccess) {
    cudaGetLastError();
    return FMG_ECUDA;
  }

  // level-1 grid and the layout of the fixed array
  Grid g;
  g.dim = 2;
  g.n = n1;
  g.rows = n1 + 1;
  g.pitch = (n1 + 1 + 31) / 32 * 32;
  g.stride = (size_t)g.rows * g.pitch;
  g.h = prob->box_len / n1;
  const int m = n1 - 1, nh = m * m, ntri = 2 * n1 * n1;
  size_t off = 0;
  auto take = [&](size_t doubles) {
    double* p = base + off;
    off += (doubles + 31) / 32 * 32;  // keep every piece 256-byte aligned
    return p;
  };
  Coef2D c;
  c.cC = take(g.stride);
  c.cE = take(g.stride);
  c.cN = take(g.stride);
  c.cNE = take(g.stride);
  c.dinv = take(g.stride);
  c.tab = take(8 * (size_t)(n1 + 1));
  double* L1 = take((size_t)nh * nh);
  double* M1 = take((size_t)nh * nh);
  double* cstart = take(nh);
  double* lam = take(1);
  double* params = take(sizeof(PotentialParams) / sizeof(double) + 1);
  int* status = reinterpret_cast<int*>(take(2));
  int* it = status + 1;
  int* tri = reinterpret_cast<int*>(take((size_t)ntri * 3 / 2 + 1));
  int* adj = reinterpret_cast<int*>(take((size_t)nh * 6 / 2 + 1));
  if (off > kScratchDoubles) return FMG_EINVAL;

  // host-side tables on the stack (no heap use), copied into the fixed array
  int tri_h[2 * kMaxCoarseCells * kMaxCoarseCells * 3];
  int adj_h[(kMaxCoarseCells - 1) * (kMaxCoarseCells - 1) * 6];
  int fill[(kMaxCoarseCells - 1) * (kMaxCoarseCells - 1)];
  auto id = [&](int i, int j) { return (i < 1 || j < 1 || i >= n1 || j >= n1) ? -1 : (i - 1) + (j - 1) * m; };
  for (int J = 0; J < n1; ++J)
    for (int I = 0; I < n1; ++I) {
      const int cell = I + n1 * J;
      const int t0[3] = {id(I, J), id(I + 1, J), id(I + 1, J + 1)};
      const int t1[3] = {id(I, J), id(I + 1, J + 1), id(I, J + 1)};
      for (int v = 0; v < 3; ++v) {
        tri_h[(2 * cell) * 3 + v] = t0[v];
        tri_h[(2 * cell + 1) * 3 + v] = t1[v];
      }
    }
  for (int a = 0; a < nh; ++a) fill[a] = 0;
  for (int e = 0; e < nh * 6; ++e) adj_h[e] = -1;
  for (int t = 0; t < ntri; ++t)
    for (int v = 0; v < 3; ++v) {
      const int a = tri_h[t * 3 + v];
      if (a >= 0) adj_h[a * 6 + fill[a]++] = (t << 3) | v;
    }
  PotentialParams pp{};
  pp.w0 = prob->w_const;
  pp.wx = prob->w_quad[0];
  pp.wy = prob->w_quad[1];
  pp.wz = prob->w_quad[2];
  pp.zeta = prob->zeta;
  pp.omega = prob->omega;
  pp.operator_form = prob->operator_form;

  DenseProblem d{};
  d.nh = nh;
  d.aug = 0;
  d.ntri = ntri;
  d.nvert = 3;
  d.tri = tri;
  d.adj = adj;
  d.maxadj = 6;
  d.tri_vol = g.h * g.h / 2.0;
  d.quart_off = d.tri_vol / 180.0;  // |T| 2 d! / (d + 4)! with d = 2
  d.L1 = L1;
  d.M1 = M1;
  d.params = reinterpret_cast<const PotentialParams*>(params);
  d.tol = prob->scf_tol;
  d.max_iter = prob->scf_max_iter;
  d.c_init = cstart;
  d.c_out = u_dev;  // the level-1 interior vector in the ABI layout is the dense vector
  d.lam_out = lam;
  d.iters_out = it;
  d.status_out = status;

  // the array keeps the previous call's contents: clear everything this call will read
  // before writing it, so no stale value can leak in; the status word starts non-zero
  // (all bits set) so that a solve kernel that never ran cannot report success
  if (cudaMemsetAsync(base, 0, off * sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(status, 0xff, sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(tri, tri_h, sizeof(int) * ntri * 3, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(adj, adj_h, sizeof(int) * nh * 6, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(params, &pp, sizeof(pp), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      dense_prepare(dense_smem_bytes(nh, ntri, 3, 0)) != cudaSuccess) {
    cudaGetLastError();
    return FMG_ECUDA;
  }
  coef2d_setup(g, d.params, c, s);
  dense_level1_2d(g, c, L1, M1, s);
  start_vector(g, cstart, nh + 1, s);
  dense_scf(d, 1, s);
  if (cudaGetLastError() != cudaSuccess) return FMG_ECUDA;  // a launch above failed
  double lam_h = 0.0;
  int st[2] = {1, 0};
  if (cudaMemcpyAsync(&lam_h, lam, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FMG_ECUDA;
  }
  *lambda_out = lam_h;
  if (iters) *iters = st[1];
  if (st[0] == 0) return FMG_OK;
  return st[0] == 1 ? FMG_ENOCONV : FMG_ECUDA;  // 1: iteration cap hit; else it never ran
}
