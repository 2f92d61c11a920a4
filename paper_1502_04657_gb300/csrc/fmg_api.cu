// C ABI of libfmg_eig: level hierarchy, the full multigrid scheme (Algorithm 3.2) as one
// CUDA graph per handle, and the component entry points used to check each step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fmg_internal.h"

using namespace fmg;

namespace {

struct Level {
  Grid g;
  Coef2D c{};
  double *x = nullptr, *xt = nullptr, *f = nullptr, *r = nullptr, *u = nullptr,
         *y = nullptr, *z = nullptr;
};

// Symmetric 6-point rule of degree 4 on a triangle: two orbits of barycentric points
// (a, b, b), b = (1 - a)/2, three points each with weight w_k / 3 (w_1 + w_2 = 1).  The three
// parameters solve the exactness conditions for lambda_1^2, lambda_1 lambda_2 lambda_3 and
// lambda_1^4, whose exact means over a triangle are 2 alpha! / (|alpha| + 2)!; with the
// orbit symmetry these imply exactness for every polynomial of degree <= 4.
bool six_point_rule(double out[4]) {
  const double t[3] = {1.0 / 6.0, 1.0 / 60.0, 1.0 / 15.0};
  double x[3] = {0.1, 0.8, 0.2};  // a1, a2, w1
  auto eval = [&](const double* v, double* f) {
    double m[2][3];
    for (int o = 0; o < 2; ++o) {
      const double a = v[o], b = 0.5 * (1.0 - a);
      m[o][0] = (a * a + 2 * b * b) / 3.0;
      m[o][1] = a * b * b;
      m[o][2] = (a * a * a * a + 2 * b * b * b * b) / 3.0;
    }
    for (int q = 0; q < 3; ++q) f[q] = v[2] * m[0][q] + (1.0 - v[2]) * m[1][q] - t[q];
  };
  for (int it = 0; it < 100; ++it) {
    double f[3], jac[3][3];
    eval(x, f);
    for (int c = 0; c < 3; ++c) {
      double xp[3] = {x[0], x[1], x[2]}, fp[3];
      const double hstep = 1e-7;
      xp[c] += hstep;
      eval(xp, fp);
      for (int q = 0; q < 3; ++q) jac[q][c] = (fp[q] - f[q]) / hstep;
    }
    // solve jac d = -f (3x3 Cramer)
    auto det3 = [](double m[3][3]) {
      return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
             m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
             m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    };
    const double d = det3(jac);
    if (d == 0.0) return false;
    double step[3];
    for (int c = 0; c < 3; ++c) {
      double m[3][3];
      for (int q = 0; q < 3; ++q)
        for (int k = 0; k < 3; ++k) m[q][k] = k == c ? -f[q] : jac[q][k];
      step[c] = det3(m) / d;
    }
    for (int c = 0; c < 3; ++c) x[c] += step[c];
    if (fabs(step[0]) + fabs(step[1]) + fabs(step[2]) < 1e-16) break;
  }
  double f[3];
  eval(x, f);
  if (fabs(f[0]) + fabs(f[1]) + fabs(f[2]) > 1e-15) return false;
  out[0] = x[0];
  out[1] = x[2];
  out[2] = x[1];
  out[3] = 1.0 - x[2];
  return true;
}

enum ProfId { kProfJacobi, kProfResidual, kProfRestrict, kProfProlong, kProfRhs,
              kProfMoments, kProfDense, kProfVcycle, kProfCount };

double factorial(int k) {
  double r = 1.0;
  for (int i = 2; i <= k; ++i) r *= i;
  return r;
}

}  // namespace

struct fmg_eig_handle {
  fmg_eig_problem prob{};
  int dev = 0;
  cudaStream_t stream = nullptr;
  std::vector<Level> lv;  // lv[0] = level 1
  std::vector<void*> allocs;
  int nh = 0, ntri = 0, nvert = 3, maxadj = 6;
  double tri_vol = 0.0;
  double rule[4] = {0, 0, 0, 0};
  double *L1 = nullptr, *M1 = nullptr, *L1inv = nullptr, *q4 = nullptr;
  int *tri = nullptr, *adj = nullptr;
  double *lam = nullptr, *c = nullptr, *cstart = nullptr, *auu = nullptr, *buu = nullptr, *partials = nullptr,
         *mom = nullptr, *mom_partials = nullptr, *lam_levels = nullptr, *scal = nullptr,
         *uout = nullptr;
  int *iters = nullptr, *status = nullptr;
  PotentialParams* dparams = nullptr;  // device copy read by the kernels
  PotentialParams* hparams = nullptr;  // pinned host staging, uploaded at every solve
  // profiling: event pairs around the first finest-level launch of each profiled step
  cudaEvent_t prof[kProfCount][2] = {};
  bool prof_armed[kProfCount] = {};
  int kernel_nodes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  size_t dense_smem = 0;

  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    allocs.push_back(p);
    cudaMemset(p, 0, count * sizeof(T));
    return static_cast<T*>(p);
  }
  ~fmg_eig_handle() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (int i = 0; i < kProfCount; ++i)
      for (int j = 0; j < 2; ++j)
        if (prof[i][j]) cudaEventDestroy(prof[i][j]);
    for (void* p : allocs) cudaFree(p);
    if (hparams) cudaFreeHost(hparams);
    if (stream) cudaStreamDestroy(stream);
  }
  Level& L(int k) { return lv[k - 1]; }
  int levels() const { return prob.levels; }
};

namespace {

#define CK(expr)                                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) {                         \
      return FMG_ECUDA;                              \
    }                                                \
  } while (0)

int validate(const fmg_eig_problem* p) {
  if (!p) return FMG_EINVAL;
  if (p->dim != 2 && p->dim != 3) return FMG_EINVAL;
  if (p->coarse_cells < 2 || p->levels < 1 || p->levels > FMG_MAX_LEVELS) return FMG_EINVAL;
  if (p->nu_pre < 0 || p->nu_post < 0 || p->vcycles < 1 || p->corrections < 1)
    return FMG_EINVAL;
  if (!(p->box_len > 0.0) || !(p->zeta >= 0.0) || !(p->omega > 0.0 && p->omega <= 1.0))
    return FMG_EINVAL;
  if (!(p->scf_tol > 0.0) || p->scf_max_iter < 1) return FMG_EINVAL;
  const double cells = (double)p->coarse_cells * pow(2.0, p->levels - 1);
  if (cells > (p->dim == 2 ? 32768.0 : 1024.0)) return FMG_EINVAL;
  if (p->smoother != FMG_SMOOTH_JACOBI) return FMG_ENOTSUP;
  if (p->dim != 2 || p->precision != FMG_FP64 || p->operator_form != FMG_W_LEFT)
    return FMG_ENOTSUP;
  return FMG_OK;
}

PotentialParams potential(const fmg_eig_problem& p) {
  PotentialParams q{};
  q.w0 = p.w_const;
  q.wx = p.w_quad[0];
  q.wy = p.w_quad[1];
  q.wz = p.w_quad[2];
  q.zeta = p.zeta;
  q.omega = p.omega;
  q.operator_form = p.operator_form;
  return q;
}

void build_levels(fmg_eig_handle* h) {
  const fmg_eig_problem& p = h->prob;
  h->lv.resize(p.levels);
  for (int k = 1; k <= p.levels; ++k) {
    Level& l = h->L(k);
    l.g.dim = 2;
    l.g.n = p.coarse_cells << (k - 1);
    l.g.rows = l.g.n + 1;
    l.g.pitch = (l.g.n + 1 + 31) / 32 * 32;
    l.g.stride = (size_t)l.g.rows * l.g.pitch;
    l.g.h = p.box_len / l.g.n;
    const size_t s = l.g.stride;
    l.c.cC = h->alloc<double>(s);
    l.c.cE = h->alloc<double>(s);
    l.c.cN = h->alloc<double>(s);
    l.c.cNE = h->alloc<double>(s);
    l.c.dinv = h->alloc<double>(s);
    l.x = h->alloc<double>(s);
    l.xt = h->alloc<double>(s);
    l.f = h->alloc<double>(s);
    l.r = h->alloc<double>(s);
    l.u = h->alloc<double>(s);
    l.y = h->alloc<double>(s);
    l.z = h->alloc<double>(s);
  }
}

void build_coarse(fmg_eig_handle* h) {
  const int n1 = h->prob.coarse_cells;
  const int m = n1 - 1;
  h->nh = m * m;
  h->nvert = 3;
  h->ntri = 2 * n1 * n1;
  h->maxadj = 6;
  const double H = h->prob.box_len / n1;
  h->tri_vol = H * H / 2.0;
  std::vector<int> tri(h->ntri * 3), adj(h->nh * h->maxadj, -1);
  auto id = [&](int i, int j) { return (i < 1 || j < 1 || i >= n1 || j >= n1) ? -1 : (i - 1) + (j - 1) * m; };
  for (int J = 0; J < n1; ++J)
    for (int I = 0; I < n1; ++I) {
      const int cell = I + n1 * J;
      const int t0[3] = {id(I, J), id(I + 1, J), id(I + 1, J + 1)};
      const int t1[3] = {id(I, J), id(I + 1, J + 1), id(I, J + 1)};
      for (int v = 0; v < 3; ++v) {
        tri[(2 * cell) * 3 + v] = t0[v];
        tri[(2 * cell + 1) * 3 + v] = t1[v];
      }
    }
  std::vector<int> fill(h->nh, 0);
  for (int t = 0; t < h->ntri; ++t)
    for (int v = 0; v < 3; ++v) {
      const int a = tri[t * 3 + v];
      if (a >= 0) adj[a * h->maxadj + fill[a]++] = (t << 3) | v;
    }
  // q4[a][b][c][d] = int_T mu_a mu_b mu_c mu_d / |T| = 2! alpha! / (4 + 2)!
  std::vector<double> q4(81);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          int cnt[3] = {0, 0, 0};
          cnt[a]++;
          cnt[b]++;
          cnt[c]++;
          cnt[d]++;
          q4[((a * 3 + b) * 3 + c) * 3 + d] =
              2.0 * factorial(cnt[0]) * factorial(cnt[1]) * factorial(cnt[2]) / factorial(6);
        }
  h->tri = h->alloc<int>(tri.size());
  h->adj = h->alloc<int>(adj.size());
  h->q4 = h->alloc<double>(q4.size());
  cudaMemcpy(h->tri, tri.data(), tri.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(h->adj, adj.data(), adj.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(h->q4, q4.data(), q4.size() * sizeof(double), cudaMemcpyHostToDevice);
  h->L1 = h->alloc<double>((size_t)h->nh * h->nh);
  h->M1 = h->alloc<double>((size_t)h->nh * h->nh);
  h->L1inv = h->alloc<double>((size_t)h->nh * h->nh);
  h->lam = h->alloc<double>(1);
  h->c = h->alloc<double>(h->nh + 1);
  h->cstart = h->alloc<double>(h->nh + 1);
  h->auu = h->alloc<double>(1);
  h->buu = h->alloc<double>(1);
  h->scal = h->alloc<double>(8);
  h->partials = h->alloc<double>(kReduceBlocks);
  h->mom = h->alloc<double>((size_t)h->ntri * kMom);
  h->mom_partials =
      h->alloc<double>(std::max<size_t>(1, moments2d_partials(h->L(h->levels()).g, n1)));
  h->lam_levels = h->alloc<double>(FMG_MAX_LEVELS);
  h->iters = h->alloc<int>(FMG_MAX_LEVELS);
  h->status = h->alloc<int>(FMG_MAX_LEVELS);
  h->uout = h->alloc<double>(h->L(h->levels()).g.interior());
  h->dense_smem = dense_smem_bytes(h->nh + 1, h->ntri, h->nvert);
}

// ---- enqueue helpers (all work in stream order on s) ---------------------------------------
void prof_begin(fmg_eig_handle* h, int id, int level, cudaStream_t s) {
  if (level == h->levels() && h->prof_armed[id])
    cudaEventRecordWithFlags(h->prof[id][0], s, cudaEventRecordExternal);
}
void prof_end(fmg_eig_handle* h, int id, int level, cudaStream_t s) {
  if (level == h->levels() && h->prof_armed[id]) {
    cudaEventRecordWithFlags(h->prof[id][1], s, cudaEventRecordExternal);
    h->prof_armed[id] = false;
  }
}

void enqueue_setup(fmg_eig_handle* h, cudaStream_t s) {
  for (int k = 1; k <= h->levels(); ++k) coef2d_setup(h->L(k).g, h->dparams, h->L(k).c, s);
  dense_level1_2d(h->L(1).g, h->L(1).c, h->L1, h->M1, s);
  dense_spd_inverse(h->L1, h->L1inv, h->nh, s);
}

DenseProblem dense_base(fmg_eig_handle* h) {
  DenseProblem d{};
  d.nh = h->nh;
  d.ntri = h->ntri;
  d.nvert = h->nvert;
  d.tri = h->tri;
  d.adj = h->adj;
  d.maxadj = h->maxadj;
  d.q4 = h->q4;
  d.tri_vol = h->tri_vol;
  d.L1 = h->L1;
  d.M1 = h->M1;
  d.n1 = h->prob.coarse_cells;
  d.pitch1 = h->L(1).g.pitch;
  d.params = h->dparams;
  d.tol = h->prob.scf_tol;
  d.max_iter = h->prob.scf_max_iter;
  d.c_out = h->c;
  d.lam_out = h->lam;
  return d;
}

// Algorithm 3.2 step 1 into L(1).u and h->lam
void enqueue_coarse(fmg_eig_handle* h, cudaStream_t s) {
  Level& l1 = h->L(1);
  start_vector(l1.g, h->prob.box_len, h->cstart, s);
  DenseProblem d = dense_base(h);
  d.aug = 0;
  d.c_init = h->cstart;
  d.iters_out = h->iters;
  d.status_out = h->status;
  dense_scf(d, s);
  scatter_level1(l1.g, h->c, l1.u, s);
}

// One V-cycle on level j for L_j x = f (x, f in L(j).x, L(j).f).
void enqueue_vcycle(fmg_eig_handle* h, int j, bool x_zero, cudaStream_t s) {
  Level& l = h->L(j);
  if (j == 1) {
    coarse_matvec2d(l.g, h->L1inv, l.f, l.x, s);
    return;
  }
  const fmg_eig_problem& p = h->prob;
  bool zero = x_zero;
  prof_begin(h, kProfVcycle, j, s);
  for (int it = 0; it < p.nu_pre; ++it) {
    const bool prof = !zero;
    if (prof) prof_begin(h, kProfJacobi, j, s);
    jacobi2d(l.g, l.c, l.f, l.x, l.xt, zero, s);
    if (prof) prof_end(h, kProfJacobi, j, s);
    std::swap(l.x, l.xt);
    zero = false;
  }
  if (zero) cudaMemsetAsync(l.x, 0, l.g.stride * sizeof(double), s);
  Level& lc = h->L(j - 1);
  prof_begin(h, kProfResidual, j, s);
  residual2d(l.g, l.c, l.f, l.x, l.r, s);
  prof_end(h, kProfResidual, j, s);
  prof_begin(h, kProfRestrict, j, s);
  restrict2d(l.g, lc.g, l.r, lc.f, s);
  prof_end(h, kProfRestrict, j, s);
  enqueue_vcycle(h, j - 1, true, s);
  prof_begin(h, kProfProlong, j, s);
  prolong2d(l.g, lc.g, lc.x, l.x, true, nullptr, nullptr, s);
  prof_end(h, kProfProlong, j, s);
  for (int it = 0; it < p.nu_post; ++it) {
    jacobi2d(l.g, l.c, l.f, l.x, l.xt, false, s);
    std::swap(l.x, l.xt);
  }
  prof_end(h, kProfVcycle, j, s);
}

void enqueue_multigrid(fmg_eig_handle* h, int k, cudaStream_t s) {
  for (int it = 0; it < h->prob.vcycles; ++it) enqueue_vcycle(h, k, false, s);
}

// One correction step (Algorithm 3.1) on level k: (h->lam, L(k).u) -> (h->lam, L(k).u);
// u~ stays in L(k).x.
void enqueue_correction(fmg_eig_handle* h, int k, cudaStream_t s) {
  Level& l = h->L(k);
  // step 1: auxiliary problem, m V-cycles from u
  prof_begin(h, kProfRhs, k, s);
  rhs2d(l.g, h->lam, h->dparams, l.u, l.f, s);
  prof_end(h, kProfRhs, k, s);
  cudaMemcpyAsync(l.x, l.u, l.g.stride * sizeof(double), cudaMemcpyDeviceToDevice, s);
  enqueue_multigrid(h, k, s);
  const double* ut = l.x;
  // step 2: augmented space V_H + span{u~}
  apply2d(l.g, l.c, ut, l.y, s);
  mass2d(l.g, ut, l.z, s);
  dot(ut, l.y, l.g.stride, h->partials, h->auu, s);
  dot(ut, l.z, l.g.stride, h->partials, h->buu, s);
  for (int j = k; j >= 2; --j) {
    restrict2d(h->L(j).g, h->L(j - 1).g, h->L(j).y, h->L(j - 1).y, s);
    restrict2d(h->L(j).g, h->L(j - 1).g, h->L(j).z, h->L(j - 1).z, s);
  }
  prof_begin(h, kProfMoments, k, s);
  moments2d(l.g, h->prob.coarse_cells, ut, h->mom_partials, h->mom, h->rule, s);
  prof_end(h, kProfMoments, k, s);
  DenseProblem d = dense_base(h);
  d.aug = 1;
  d.gA = h->L(1).y;
  d.gM = h->L(1).z;
  d.auu = h->auu;
  d.buu = h->buu;
  d.mom = h->mom;
  d.c_init = nullptr;
  d.iters_out = h->iters + (k - 1);
  d.status_out = h->status + (k - 1);
  prof_begin(h, kProfDense, k, s);
  dense_scf(d, s);
  prof_end(h, kProfDense, k, s);
  // u = P_{k<-1} c_H + c_u u~
  scatter_level1(h->L(1).g, h->c, h->L(1).y, s);
  for (int j = 2; j < k; ++j)
    prolong2d(h->L(j).g, h->L(j - 1).g, h->L(j - 1).y, h->L(j).y, false, nullptr, nullptr, s);
  prolong2d(l.g, h->L(k - 1).g, h->L(k - 1).y, l.u, false, ut, h->c + h->nh, s);
}

void enqueue_fmg(fmg_eig_handle* h, cudaStream_t s) {
  enqueue_setup(h, s);
  enqueue_coarse(h, s);
  cudaMemcpyAsync(h->lam_levels, h->lam, sizeof(double), cudaMemcpyDeviceToDevice, s);
  for (int k = 2; k <= h->levels(); ++k) {
    prolong2d(h->L(k).g, h->L(k - 1).g, h->L(k - 1).u, h->L(k).u, false, nullptr, nullptr, s);
    for (int it = 0; it < h->prob.corrections; ++it) enqueue_correction(h, k, s);
    cudaMemcpyAsync(h->lam_levels + (k - 1), h->lam, sizeof(double), cudaMemcpyDeviceToDevice,
                    s);
  }
}

cudaStream_t pick(fmg_eig_handle* h, void* stream) {
  return stream ? static_cast<cudaStream_t>(stream) : h->stream;
}

bool level_ok(const fmg_eig_handle* h, int k) { return h && k >= 1 && k <= h->prob.levels; }

}  // namespace

extern "C" {

const char* fmg_eig_strerror(int code) {
  switch (code) {
    case FMG_OK: return "ok";
    case FMG_EINVAL: return "invalid argument";
    case FMG_ENOMEM: return "out of device memory";
    case FMG_ENOCONV: return "nonlinear solve hit its iteration cap";
    case FMG_ECUDA: return "CUDA runtime error";
    case FMG_ETIMEOUT: return "bounded device wait gave up";
    case FMG_ENOTSUP: return "option combination not supported";
    default: return "unknown error";
  }
}

int fmg_eig_create(const fmg_eig_problem* prob, fmg_eig_handle** out) {
  if (!out) return FMG_EINVAL;
  *out = nullptr;
  const int v = validate(prob);
  if (v != FMG_OK) return v;
  fmg_eig_handle* h = new (std::nothrow) fmg_eig_handle();
  if (!h) return FMG_ENOMEM;
  h->prob = *prob;
  if (!six_point_rule(h->rule)) {
    delete h;
    return FMG_ECUDA;
  }
  if (cudaGetDevice(&h->dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FMG_ECUDA;
  }
  try {
    build_levels(h);
    build_coarse(h);
    h->dparams = h->alloc<PotentialParams>(1);
  } catch (const std::bad_alloc&) {
    delete h;
    return FMG_ENOMEM;
  }
  if (cudaMallocHost(&h->hparams, sizeof(PotentialParams)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FMG_ENOMEM;
  }
  *h->hparams = potential(*prob);
  for (int i = 0; i < kProfCount; ++i)
    for (int j = 0; j < 2; ++j)
      if (cudaEventCreate(&h->prof[i][j]) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return FMG_ECUDA;
      }
  cudaMemcpy(h->dparams, h->hparams, sizeof(PotentialParams), cudaMemcpyHostToDevice);
  if (h->dense_smem > kDenseSmemLimit) {  // the small dense solve keeps everything in shared memory
    delete h;
    return FMG_ENOTSUP;
  }
  if (dense_prepare(h->dense_smem) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FMG_ECUDA;
  }
  // component entry points need the operators; the solve graph recomputes them itself
  enqueue_setup(h, h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FMG_ECUDA;
  }
  for (int i = 0; i < kProfCount; ++i) h->prof_armed[i] = true;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_fmg(h, h->stream);
    e = cudaStreamEndCapture(h->stream, &h->graph);
  }
  for (int i = 0; i < kProfCount; ++i) h->prof_armed[i] = false;
  if (e == cudaSuccess) {
    size_t count = 0;
    e = cudaGraphGetNodes(h->graph, nullptr, &count);
    std::vector<cudaGraphNode_t> nodes(count);
    if (e == cudaSuccess && count) e = cudaGraphGetNodes(h->graph, nodes.data(), &count);
    for (size_t i = 0; e == cudaSuccess && i < count; ++i) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      if (t == cudaGraphNodeTypeKernel) h->kernel_nodes++;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, h->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FMG_ECUDA;
  }
  *out = h;
  return FMG_OK;
}

size_t fmg_eig_level_size(const fmg_eig_handle* h, int32_t level) {
  if (!level_ok(h, level)) return 0;
  return h->lv[level - 1].g.interior();
}

void fmg_eig_destroy(fmg_eig_handle* h) { delete h; }

int fmg_eig_set_params(fmg_eig_handle* h, const fmg_eig_problem* prob) {
  if (!h || !prob) return FMG_EINVAL;
  const int v = validate(prob);
  if (v != FMG_OK) return v;
  const fmg_eig_problem& a = h->prob;
  if (prob->dim != a.dim || prob->coarse_cells != a.coarse_cells || prob->levels != a.levels ||
      prob->nu_pre != a.nu_pre || prob->nu_post != a.nu_post || prob->vcycles != a.vcycles ||
      prob->corrections != a.corrections || prob->precision != a.precision ||
      prob->operator_form != a.operator_form || prob->smoother != a.smoother ||
      prob->box_len != a.box_len || prob->scf_tol != a.scf_tol ||
      prob->scf_max_iter != a.scf_max_iter)
    return FMG_EINVAL;
  // the pinned staging copy is read by the next solve's upload, in stream order
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return FMG_ECUDA;
  h->prob.w_const = prob->w_const;
  for (int d = 0; d < 3; ++d) h->prob.w_quad[d] = prob->w_quad[d];
  h->prob.zeta = prob->zeta;
  h->prob.omega = prob->omega;
  *h->hparams = potential(h->prob);
  if (cudaMemcpyAsync(h->dparams, h->hparams, sizeof(PotentialParams), cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return FMG_ECUDA;
  enqueue_setup(h, h->stream);  // keep the component entry points' operators current
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return FMG_ECUDA;
  return FMG_OK;
}

int fmg_eig_kernel_count(const fmg_eig_handle* h) { return h ? h->kernel_nodes : 0; }

int fmg_eig_profile(fmg_eig_handle* h, double* ms, int32_t count) {
  if (!h || !ms || count < 1) return FMG_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return FMG_ECUDA;
  const int n = count < kProfCount ? count : kProfCount;
  for (int i = 0; i < n; ++i) {
    float t = 0.f;
    ms[i] = cudaEventElapsedTime(&t, h->prof[i][0], h->prof[i][1]) == cudaSuccess ? t : -1.0;
  }
  cudaGetLastError();
  return n;
}

int fmg_eig_solve_dev(fmg_eig_handle* h, double* lambda_dev, double* u_dev, size_t u_len,
                      void* stream) {
  if (!h || !lambda_dev) return FMG_EINVAL;
  const Level& fine = h->L(h->levels());
  if (u_dev && u_len != fine.g.interior()) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  CK(cudaMemcpyAsync(h->dparams, h->hparams, sizeof(PotentialParams), cudaMemcpyHostToDevice, s));
  CK(cudaGraphLaunch(h->exec, s));
  CK(cudaMemcpyAsync(lambda_dev, h->lam, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (u_dev) unpack_interior(fine.g, fine.u, u_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_solve(fmg_eig_handle* h, double* lambda, double* u_host, size_t u_len,
                  fmg_eig_stats* stats) {
  if (!h || !lambda) return FMG_EINVAL;
  const Level& fine = h->L(h->levels());
  if (u_host && u_len != fine.g.interior()) return FMG_EINVAL;
  cudaStream_t s = h->stream;
  CK(cudaEventRecord(h->ev0, s));
  CK(cudaMemcpyAsync(h->dparams, h->hparams, sizeof(PotentialParams), cudaMemcpyHostToDevice, s));
  CK(cudaGraphLaunch(h->exec, s));
  CK(cudaEventRecord(h->ev1, s));
  double lam = 0.0;
  CK(cudaMemcpyAsync(&lam, h->lam, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (u_host) {
    unpack_interior(fine.g, fine.u, h->uout, s);
    CK(cudaMemcpyAsync(u_host, h->uout, u_len * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  int st[FMG_MAX_LEVELS];
  CK(cudaMemcpyAsync(st, h->status, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *lambda = lam;
  int rc = FMG_OK;
  for (int k = 0; k < h->levels(); ++k)
    if (st[k] != 0) rc = FMG_ENOCONV;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->lambda = lam;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    stats->solve_ms = ms;
    stats->levels = h->levels();
    stats->status = rc;
    CK(cudaMemcpy(stats->lambda_levels, h->lam_levels, sizeof(double) * h->levels(),
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(stats->scf_iters, h->iters, sizeof(int) * h->levels(), cudaMemcpyDeviceToHost));
    // b(u,u) - 1 and lambda - a(u,u) - (Wu,u) - zeta int u^4 on the finest level
    Level& l = h->L(h->levels());
    apply2d(l.g, l.c, l.u, l.y, s);
    mass2d(l.g, l.u, l.z, s);
    nload2d(l.g, l.u, l.r, s);
    dot(l.u, l.y, l.g.stride, h->partials, h->scal + 0, s);
    dot(l.u, l.z, l.g.stride, h->partials, h->scal + 1, s);
    dot(l.u, l.r, l.g.stride, h->partials, h->scal + 2, s);
    double sc[3];
    CK(cudaMemcpyAsync(sc, h->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    stats->norm_defect = sc[1] - 1.0;
    stats->identity_defect = lam - (sc[0] + h->prob.zeta * sc[2]);
  }
  return rc;
}

// ---- component entry points ------------------------------------------------------------
int fmg_eig_apply_operator(fmg_eig_handle* h, int32_t level, const double* x_dev,
                           double* y_dev, void* stream) {
  if (!level_ok(h, level) || !x_dev || !y_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  pack_interior(l.g, x_dev, l.r, s);
  apply2d(l.g, l.c, l.r, l.y, s);
  unpack_interior(l.g, l.y, y_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_apply_mass(fmg_eig_handle* h, int32_t level, const double* x_dev, double* y_dev,
                       void* stream) {
  if (!level_ok(h, level) || !x_dev || !y_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  pack_interior(l.g, x_dev, l.r, s);
  mass2d(l.g, l.r, l.y, s);
  unpack_interior(l.g, l.y, y_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_jacobi(fmg_eig_handle* h, int32_t level, const double* f_dev,
                   const double* x_in_dev, double* x_out_dev, void* stream) {
  if (!level_ok(h, level) || !f_dev || !x_in_dev || !x_out_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  pack_interior(l.g, f_dev, l.f, s);
  pack_interior(l.g, x_in_dev, l.r, s);
  jacobi2d(l.g, l.c, l.f, l.r, l.y, false, s);
  unpack_interior(l.g, l.y, x_out_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_residual_restrict(fmg_eig_handle* h, int32_t level, const double* f_dev,
                              const double* x_dev, double* rc_dev, void* stream) {
  if (!level_ok(h, level) || level < 2 || !f_dev || !x_dev || !rc_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  Level& lc = h->L(level - 1);
  pack_interior(l.g, f_dev, l.f, s);
  pack_interior(l.g, x_dev, l.z, s);
  residual2d(l.g, l.c, l.f, l.z, l.r, s);
  restrict2d(l.g, lc.g, l.r, lc.y, s);
  unpack_interior(lc.g, lc.y, rc_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_prolong_add(fmg_eig_handle* h, int32_t level, const double* ec_dev, double* x_dev,
                        void* stream) {
  if (!level_ok(h, level) || level < 2 || !ec_dev || !x_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  Level& lc = h->L(level - 1);
  pack_interior(lc.g, ec_dev, lc.y, s);
  pack_interior(l.g, x_dev, l.y, s);
  prolong2d(l.g, lc.g, lc.y, l.y, true, nullptr, nullptr, s);
  unpack_interior(l.g, l.y, x_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_nonlinear_load(fmg_eig_handle* h, int32_t level, const double* u_dev,
                           double* n_dev, void* stream) {
  if (!level_ok(h, level) || !u_dev || !n_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  pack_interior(l.g, u_dev, l.r, s);
  nload2d(l.g, l.r, l.y, s);
  unpack_interior(l.g, l.y, n_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_aux_rhs(fmg_eig_handle* h, int32_t level, double lambda, const double* u_dev,
                    double* f_dev, void* stream) {
  if (!level_ok(h, level) || !u_dev || !f_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(h->scal + 7, &lambda, sizeof(double), cudaMemcpyHostToDevice));
  pack_interior(l.g, u_dev, l.r, s);
  rhs2d(l.g, h->scal + 7, h->dparams, l.r, l.y, s);
  unpack_interior(l.g, l.y, f_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_multigrid(fmg_eig_handle* h, int32_t level, const double* f_dev, double* x_dev,
                      void* stream) {
  if (!level_ok(h, level) || !f_dev || !x_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  Level& l = h->L(level);
  pack_interior(l.g, f_dev, l.f, s);
  pack_interior(l.g, x_dev, l.x, s);
  enqueue_multigrid(h, level, s);
  unpack_interior(l.g, l.x, x_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_correction(fmg_eig_handle* h, int32_t level, double lambda_in,
                       const double* u_in_dev, double* lambda_out, double* u_out_dev,
                       double* u_tilde_dev, int32_t* iters) {
  if (!level_ok(h, level) || level < 2 || !u_in_dev || !lambda_out || !u_out_dev)
    return FMG_EINVAL;
  cudaStream_t s = h->stream;
  Level& l = h->L(level);
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(h->lam, &lambda_in, sizeof(double), cudaMemcpyHostToDevice));
  pack_interior(l.g, u_in_dev, l.u, s);
  enqueue_correction(h, level, s);
  unpack_interior(l.g, l.u, u_out_dev, s);
  if (u_tilde_dev) unpack_interior(l.g, l.x, u_tilde_dev, s);
  int st = 0, it = 0;
  CK(cudaMemcpyAsync(lambda_out, h->lam, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, h->status + (level - 1), sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&it, h->iters + (level - 1), sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  return st == 0 ? FMG_OK : FMG_ENOCONV;
}

int fmg_eig_coarse_solve(fmg_eig_handle* h, double* lambda_out, double* u_dev, int32_t* iters) {
  if (!h || !lambda_out || !u_dev) return FMG_EINVAL;
  cudaStream_t s = h->stream;
  enqueue_coarse(h, s);
  unpack_interior(h->L(1).g, h->L(1).u, u_dev, s);
  int st = 0, it = 0;
  CK(cudaMemcpyAsync(lambda_out, h->lam, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&it, h->iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  return st == 0 ? FMG_OK : FMG_ENOCONV;
}

}  // extern "C"
