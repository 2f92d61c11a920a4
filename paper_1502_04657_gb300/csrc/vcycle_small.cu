// The small levels of a 2D V-cycle in one kernel: one CTA per instance runs the whole V-cycle
// from an entry level with at most 32 cells per side down to the exact solve on level 1 and
// back, with every level's x, f and residual in shared memory.
//
// On these levels a sweep has at most 961 nodes, so the separate launches of the V-cycle
// (about 17 from 32 cells per side down and up again) cost their launch latency, not their
// work.  In one CTA the FP64 work runs on one SM, a few microseconds per sweep, with a
// barrier between steps.  Every step evaluates the same expressions in the same order as the
// separate kernels (grid2d.cu: damped Jacobi, residual, P^T, P; dense.cu: the level-1 inverse
// applied row by row with a warp butterfly), so the results are bit-identical.
#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr int kVThreads = 512;
constexpr int kVWarps = kVThreads / 32;

__device__ __forceinline__ double warp_sum_xor(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// f - L x at interior node (i, j) as grid2d.cu's defect(): coefficients from the level's
// global arrays (index kg), x from a shared-memory plane of row length w = n + 1 (zero
// boundary ring)
__device__ __forceinline__ double defect_small(const Coef2D& c, size_t kg, int pitch, double f,
                                               const double* x, int e, int w) {
  double r = fma(-c.cC[kg], x[e], f);
  r = fma(-c.cE[kg], x[e + 1], r);
  r = fma(-c.cE[kg - 1], x[e - 1], r);
  r = fma(-c.cN[kg], x[e + w], r);
  r = fma(-c.cN[kg - pitch], x[e - w], r);
  r = fma(-c.cNE[kg], x[e + w + 1], r);
  r = fma(-c.cNE[kg - pitch - 1], x[e - w - 1], r);
  return r;
}

__global__ void __launch_bounds__(kVThreads) k_vcycle_small2d(SmallVcycle v) {
  extern __shared__ double sm[];
  const int ib = blockIdx.x, tid = threadIdx.x;
  const int L = v.levels;
  double *X[kSmallMaxLevels], *XT[kSmallMaxLevels], *F[kSmallMaxLevels], *R[kSmallMaxLevels];
  size_t off = 0;
  for (int j = 0; j < L; ++j) {
    const size_t m = (size_t)(v.lv[j].n + 1) * (v.lv[j].n + 1);
    X[j] = sm + off;
    XT[j] = X[j] + m;
    F[j] = XT[j] + m;
    R[j] = F[j] + m;
    off += 4 * m;
  }
  for (size_t e = tid; e < off; e += kVThreads) sm[e] = 0.0;
  __syncthreads();
  {  // entry level: f, and x unless it starts at zero
    const SmallLevel2D& t = v.lv[L - 1];
    const int n = t.n, w = n + 1, m = n - 1;
    for (int q = tid; q < m * m; q += kVThreads) {
      const int i = 1 + q % m, j = 1 + q / m;
      const size_t kg = ib * t.stride + (size_t)j * t.pitch + i;
      F[L - 1][j * w + i] = v.f[kg];
      if (!v.x_zero) X[L - 1][j * w + i] = v.x[kg];
    }
  }
  __syncthreads();

  // damped Jacobi sweeps on level index j (as k_jacobi2d / k_jacobi2d_zero)
  auto smooth = [&](int j, int nu, bool zero) {
    const SmallLevel2D& t = v.lv[j];
    const int n = t.n, w = n + 1, m = n - 1;
    for (int it = 0; it < nu; ++it) {
      for (int q = tid; q < m * m; q += kVThreads) {
        const int i = 1 + q % m, jj = 1 + q / m;
        const int e = jj * w + i;
        const size_t kg = ib * t.stride + (size_t)jj * t.pitch + i;
        XT[j][e] = zero ? t.c.dinv[kg] * F[j][e]
                        : fma(t.c.dinv[kg], defect_small(t.c, kg, t.pitch, F[j][e], X[j], e, w),
                              X[j][e]);
      }
      double* tmp = X[j];
      X[j] = XT[j];
      XT[j] = tmp;
      zero = false;
      __syncthreads();
    }
  };

  // descent
  for (int j = L - 1; j >= 1; --j) {
    const SmallLevel2D& t = v.lv[j];
    const int n = t.n, w = n + 1, m = n - 1;
    smooth(j, v.nu_pre, j == L - 1 ? v.x_zero != 0 : true);
    // (with no pre-smoothing a zero start leaves X at its zero fill)
    for (int q = tid; q < m * m; q += kVThreads) {  // residual (k_residual2d)
      const int i = 1 + q % m, jj = 1 + q / m;
      const int e = jj * w + i;
      const size_t kg = ib * t.stride + (size_t)jj * t.pitch + i;
      R[j][e] = defect_small(t.c, kg, t.pitch, F[j][e], X[j], e, w);
    }
    __syncthreads();
    const int nc = v.lv[j - 1].n, wc = nc + 1, mc = nc - 1;
    for (int q = tid; q < mc * mc; q += kVThreads) {  // P^T (k_restrict2d)
      const int I = 1 + q % mc, J = 1 + q / mc;
      const double* rf = R[j];
      const int kf = 2 * J * w + 2 * I;
      const double s = ((rf[kf + 1] + rf[kf - 1]) + (rf[kf + w] + rf[kf - w])) +
                       (rf[kf + w + 1] + rf[kf - w - 1]);
      F[j - 1][J * wc + I] = fma(0.5, s, rf[kf]);
    }
    __syncthreads();
  }
  {  // level 1: x = L1^{-1} f (k_coarse_matvec)
    const int n = v.lv[0].n, w = n + 1, m = n - 1, nh = m * m;
    const double* Linv = v.Linv + (size_t)ib * nh * nh;
    double* xs = R[0];  // f in the level-1 unknown order (R[0] is free here)
    for (int q = tid; q < nh; q += kVThreads) xs[q] = F[0][(1 + q / m) * w + 1 + q % m];
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int p = warp; p < nh; p += kVWarps) {
      const double* row = Linv + (size_t)p * nh;
      double s = 0.0;
      for (int q = lane; q < nh; q += 32) s = fma(row[q], xs[q], s);
      s = warp_sum_xor(s);
      if (lane == 0) X[0][(1 + p / m) * w + 1 + p % m] = s;
    }
    __syncthreads();
  }
  // ascent
  for (int j = 1; j < L; ++j) {
    const SmallLevel2D& t = v.lv[j];
    const int n = t.n, w = n + 1, m = n - 1;
    const int wc = v.lv[j - 1].n + 1;
    const double* ec = X[j - 1];
    for (int q = tid; q < m * m; q += kVThreads) {  // x += P e (k_prolong2d)
      const int i = 1 + q % m, jj = 1 + q / m;
      const int ai = i & 1, aj = jj & 1;
      const int kc = (jj >> 1) * wc + (i >> 1);
      const double a = ec[kc];
      const double x = X[j][jj * w + i];
      X[j][jj * w + i] = (ai | aj) ? fma(0.5, a + ec[kc + ai + aj * wc], x) : a + x;
    }
    __syncthreads();
    smooth(j, v.nu_post, false);
  }
  {  // entry level's x back to global memory
    const SmallLevel2D& t = v.lv[L - 1];
    const int n = t.n, w = n + 1, m = n - 1;
    for (int q = tid; q < m * m; q += kVThreads) {
      const int i = 1 + q % m, j = 1 + q / m;
      v.x[ib * t.stride + (size_t)j * t.pitch + i] = X[L - 1][j * w + i];
    }
  }
}

}  // namespace

size_t vcycle_small_smem(const SmallVcycle& v) {
  size_t m = 0;
  for (int j = 0; j < v.levels; ++j) m += 4 * (size_t)(v.lv[j].n + 1) * (v.lv[j].n + 1);
  return m * sizeof(double);
}

cudaError_t vcycle_small(const SmallVcycle& v, int nb, cudaStream_t s) {
  const size_t bytes = vcycle_small_smem(v);
  if (bytes > kSmallSmemLimit) return cudaErrorInvalidValue;
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_vcycle_small2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmemLimit);
  if (attr != cudaSuccess) return attr;
  k_vcycle_small2d<<<nb, kVThreads, bytes, s>>>(v);
  return cudaSuccess;
}

}  // namespace fmg
