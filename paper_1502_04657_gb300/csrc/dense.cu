// Small dense FP64 solves: the nonlinear eigenproblem on V_{h_1} (Algorithm 3.2 step 1) and
// on the augmented space V_H + span{u~} (Algorithm 3.1 step 2), plus the coarsest-level
// inverse used by the V-cycle.
//
// The nonlinear problem on an n-dimensional space with basis psi is
//     F(c, lambda) = (K0 + zeta G(c)) c - lambda M c = 0,   c^T M c = 1,
// G(c)_ij = int w^2 psi_i psi_j, w = sum_j c_j psi_j.  Section 3.2 allows self-consistent
// or Newton-type iterations; both converge to the same ground state, which is what the
// result is.  This kernel takes inverse-power steps c <- (K0 + zeta G(c))^{-1} M c while the
// relative residual is large (they pull any positive start into the ground state's basin),
// then Newton steps on the bordered system
//     [K0 + 3 zeta G(c) - lambda M   -M c] [dc]   [-F]
//     [-(M c)^T                        0 ] [dl] = [ 0]
// (d/dc of G(c) c is 3 G(c) for the cubic term), which converge quadratically.  lambda is
// reported as c^T (K0 + zeta G(c)) c at the final c.
//
// G(c) is assembled per coarse simplex T from the moments of u~ (see moments2d.cu) and the
// exact quartic table q4 of the coarse barycentrics:
//   int_T w^2 mu_a mu_b  = |T| sum w_c w_d q4_abcd + 2 c_u sum w_c T3_abc + c_u^2 T2_ab
//   int_T w^2 mu_a u~    = sum w_c w_d T3_acd + 2 c_u sum w_c T2_ac + c_u^2 T1_a
//   int_T w^2 u~^2       = sum w_c w_d T2_cd  + 2 c_u sum w_c T1_c  + c_u^2 T0
// with w_c the coarse coefficients at T's vertices (0 on the boundary), c_u that of u~.
//
// One CTA of 256 threads per problem, everything in shared memory, fixed-order reductions.
// The iteration count is bounded by max_iter; hitting it sets status 1.
#include <math.h>

#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxVert = 4;
constexpr double kSwitch = 1e-2;  // relative residual below which Newton takes over

struct Smem {
  double *K0, *MM, *G, *J, *c, *Mc, *Hc, *x, *loc, *red;
  int n, nh, n1p, L;
};

__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// y = A c for an n x n row-major matrix
__device__ void matvec(const double* A, const double* c, double* y, int n) {
  for (int a = threadIdx.x; a < n; a += kThreads) {
    double s = 0.0;
    const double* row = A + (size_t)a * n;
    for (int b = 0; b < n; ++b) s = fma(row[b], c[b], s);
    y[a] = s;
  }
}

__device__ double dotv(const double* a, const double* b, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) s = fma(a[i], b[i], s);
  return block_sum(s, red);
}

__device__ __forceinline__ int sym2(int a, int b, int nv) {
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  return a * nv - a * (a - 1) / 2 + (b - a);
}

__device__ __forceinline__ int sym3(int a, int b, int c, int nv) {
  // sort a <= b <= c, then count lexicographically smaller sorted triples
  if (a > b) { const int t = a; a = b; b = t; }
  if (b > c) { const int t = b; b = c; c = t; }
  if (a > b) { const int t = a; a = b; b = t; }
  int idx = 0;
  for (int x = 0; x < a; ++x) idx += (nv - x) * (nv - x + 1) / 2;
  for (int y = a; y < b; ++y) idx += nv - y;
  return idx + (c - b);
}

__device__ void build_G(const DenseProblem& p, Smem& s) {
  const int nv = p.nvert, L = s.L, nh = s.nh, n = s.n;
  const int nmom = 1 + nv + nv * (nv + 1) / 2 + nv * (nv + 1) * (nv + 2) / 6;
  const int o2 = 1 + nv, o3 = o2 + nv * (nv + 1) / 2;
  for (int t = threadIdx.x; t < p.ntri; t += kThreads) {
    double w[kMaxVert];
    for (int v = 0; v < nv; ++v) {
      const int id = p.tri[t * nv + v];
      w[v] = id >= 0 ? s.c[id] : 0.0;
    }
    const double cu = p.aug ? s.c[nh] : 0.0;
    const double* mom = p.aug ? p.mom + (size_t)t * nmom : nullptr;
    double* lt = s.loc + (size_t)t * L * L;
    for (int a = 0; a < nv; ++a) {
      for (int b = a; b < nv; ++b) {
        double q = 0.0;
        for (int c = 0; c < nv; ++c)
          for (int d = 0; d < nv; ++d)
            q = fma(w[c] * w[d], p.q4[((a * nv + b) * nv + c) * nv + d], q);
        double v = p.tri_vol * q;
        if (p.aug) {
          double t3 = 0.0;
          for (int c = 0; c < nv; ++c) t3 = fma(w[c], mom[o3 + sym3(a, b, c, nv)], t3);
          v = fma(2.0 * cu, t3, v);
          v = fma(cu * cu, mom[o2 + sym2(a, b, nv)], v);
        }
        lt[a * L + b] = v;
        lt[b * L + a] = v;
      }
    }
    if (p.aug) {
      for (int a = 0; a < nv; ++a) {
        double t3 = 0.0, t2 = 0.0;
        for (int c = 0; c < nv; ++c) {
          t2 = fma(w[c], mom[o2 + sym2(a, c, nv)], t2);
          for (int d = 0; d < nv; ++d) t3 = fma(w[c] * w[d], mom[o3 + sym3(a, c, d, nv)], t3);
        }
        const double v = fma(cu * cu, mom[1 + a], fma(2.0 * cu, t2, t3));
        lt[a * L + nv] = v;
        lt[nv * L + a] = v;
      }
      double t2 = 0.0, t1 = 0.0;
      for (int c = 0; c < nv; ++c) {
        t1 = fma(w[c], mom[1 + c], t1);
        for (int d = 0; d < nv; ++d) t2 = fma(w[c] * w[d], mom[o2 + sym2(c, d, nv)], t2);
      }
      lt[nv * L + nv] = fma(cu * cu, mom[0], fma(2.0 * cu, t1, t2));
    }
  }
  for (int e = threadIdx.x; e < n * n; e += kThreads) s.G[e] = 0.0;
  __syncthreads();
  // rows of coarse nodes: each thread owns one row, sums its incident simplices in order
  for (int a = threadIdx.x; a < nh; a += kThreads) {
    double* row = s.G + (size_t)a * n;
    double au = 0.0;
    for (int e = 0; e < p.maxadj; ++e) {
      const int code = p.adj[a * p.maxadj + e];
      if (code < 0) break;
      const int t = code >> 3, la = code & 7;
      const double* lt = s.loc + (size_t)t * L * L;
      for (int lb = 0; lb < nv; ++lb) {
        const int vb = p.tri[t * nv + lb];
        if (vb >= 0) row[vb] += lt[la * L + lb];
      }
      if (p.aug) au += lt[la * L + nv];
    }
    if (p.aug) row[nh] = au;
  }
  if (p.aug && threadIdx.x == kThreads - 1) {
    double uu = 0.0;
    for (int t = 0; t < p.ntri; ++t) uu += s.loc[(size_t)t * L * L + nv * L + nv];
    s.G[(size_t)nh * n + nh] = uu;
  }
  __syncthreads();
  if (p.aug)
    for (int a = threadIdx.x; a < nh; a += kThreads) s.G[(size_t)nh * n + a] = s.G[(size_t)a * n + nh];
  __syncthreads();
}

// In-place Cholesky of the n x n matrix A (lower triangle).  Returns false if not SPD.
__device__ bool cholesky(double* A, int n, double* red) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[k * n + k];
      if (!(d > 0.0)) fail = 1;
      else A[k * n + k] = sqrt(d);
    }
    __syncthreads();
    if (fail) return false;
    const double dk = A[k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += kThreads) A[i * n + k] /= dk;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = threadIdx.x; e < m * m; e += kThreads) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) A[i * n + j] = fma(-A[i * n + k], A[j * n + k], A[i * n + j]);
    }
    __syncthreads();
  }
  return true;
}

// Solve (L L^T) x = b in place (x holds b on entry); warp 0 works, others wait.
__device__ void chol_solve(const double* A, int n, double* x) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = lane; j < i; j += 32) s = fma(A[i * n + j], x[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) x[i] = (x[i] - s) / A[i * n + i];
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = 0.0;
      for (int j = i + 1 + lane; j < n; j += 32) s = fma(A[j * n + i], x[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) x[i] = (x[i] - s) / A[i * n + i];
      __syncwarp();
    }
  }
  __syncthreads();
}

// Gaussian elimination with partial pivoting on the m x m matrix A, right-hand side x.
__device__ bool lu_solve(double* A, int m, double* x) {
  __shared__ int piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < m; i += 32) {
        const double v = fabs(A[i * m + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        piv = bi;
        if (!(best > 0.0)) bad = 1;
      }
    }
    __syncthreads();
    if (bad) return false;
    const int pk = piv;
    if (pk != k) {
      for (int j = threadIdx.x; j < m; j += kThreads) {
        const double t = A[k * m + j];
        A[k * m + j] = A[pk * m + j];
        A[pk * m + j] = t;
      }
      if (threadIdx.x == 0) {
        const double t = x[k];
        x[k] = x[pk];
        x[pk] = t;
      }
    }
    __syncthreads();
    const double d = A[k * m + k];
    for (int i = k + 1 + threadIdx.x; i < m; i += kThreads) A[i * m + k] /= d;
    __syncthreads();
    const int r = m - k - 1;
    for (int e = threadIdx.x; e < r * r; e += kThreads) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      A[i * m + j] = fma(-A[i * m + k], A[k * m + j], A[i * m + j]);
    }
    for (int i = k + 1 + threadIdx.x; i < m; i += kThreads) x[i] = fma(-A[i * m + k], x[k], x[i]);
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = m - 1; i >= 0; --i) {
      double s = 0.0;
      for (int j = i + 1 + lane; j < m; j += 32) s = fma(A[i * m + j], x[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) x[i] = (x[i] - s) / A[i * m + i];
      __syncwarp();
    }
  }
  __syncthreads();
  return true;
}

__device__ void normalise_and_sign(const DenseProblem& p, Smem& s) {
  matvec(s.MM, s.c, s.Mc, s.n);
  __syncthreads();
  const double cmc = dotv(s.c, s.Mc, s.n, s.red);
  double sg;
  if (p.aug) {
    sg = s.c[s.nh];
  } else {
    double t = 0.0;
    for (int i = threadIdx.x; i < s.n; i += kThreads) t += s.c[i];
    sg = block_sum(t, s.red);
  }
  __syncthreads();  // every thread has read c before any thread rescales it
  const double f = (sg < 0.0 ? -1.0 : 1.0) / sqrt(cmc);
  for (int i = threadIdx.x; i < s.n; i += kThreads) s.c[i] *= f;
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_dense_scf(DenseProblem p) {
  extern __shared__ double sm[];
  Smem s;
  s.nh = p.nh;
  s.n = p.nh + p.aug;
  s.n1p = s.n + 1;
  s.L = p.nvert + 1;
  const int n = s.n, nh = s.nh;
  s.K0 = sm;
  s.MM = s.K0 + n * n;
  s.G = s.MM + n * n;
  s.J = s.G + n * n;
  s.c = s.J + s.n1p * s.n1p;
  s.Mc = s.c + n;
  s.Hc = s.Mc + n;
  s.x = s.Hc + n;
  s.loc = s.x + s.n1p;
  s.red = s.loc + (size_t)p.ntri * s.L * s.L;

  const int m1 = p.n1 - 1;
  const double zeta = p.params->zeta;
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    const int a = e / n, b = e % n;
    double kv, mv;
    if (a < nh && b < nh) {
      kv = p.L1[a * nh + b];
      mv = p.M1[a * nh + b];
    } else if (a == nh && b == nh) {
      kv = p.auu[0];
      mv = p.buu[0];
    } else {
      const int q = a < nh ? a : b;
      const size_t pad = (size_t)(1 + q / m1) * p.pitch1 + 1 + q % m1;
      kv = p.gA[pad];
      mv = p.gM[pad];
    }
    s.K0[e] = kv;
    s.MM[e] = mv;
  }
  for (int i = threadIdx.x; i < n; i += kThreads)
    s.c[i] = p.c_init ? p.c_init[i] : (i == nh ? 1.0 : 0.0);
  __syncthreads();
  normalise_and_sign(p, s);

  int it = 0, status = 1;
  double lam = 0.0;
  for (;; ++it) {
    build_G(p, s);
    // H c, M c, lambda, residual
    for (int a = threadIdx.x; a < n; a += kThreads) {
      double hk = 0.0, hg = 0.0, mc = 0.0;
      const double* kr = s.K0 + (size_t)a * n;
      const double* gr = s.G + (size_t)a * n;
      const double* mr = s.MM + (size_t)a * n;
      for (int b = 0; b < n; ++b) {
        hk = fma(kr[b], s.c[b], hk);
        hg = fma(gr[b], s.c[b], hg);
        mc = fma(mr[b], s.c[b], mc);
      }
      s.Hc[a] = fma(zeta, hg, hk);
      s.Mc[a] = mc;
    }
    __syncthreads();
    lam = dotv(s.c, s.Hc, n, s.red);
    double rr = 0.0, mm = 0.0;
    for (int a = threadIdx.x; a < n; a += kThreads) {
      const double r = fma(-lam, s.Mc[a], s.Hc[a]);
      rr = fma(r, r, rr);
      mm = fma(s.Mc[a], s.Mc[a], mm);
    }
    rr = block_sum(rr, s.red);
    mm = block_sum(mm, s.red);
    const double rn = sqrt(rr) / (fabs(lam) * sqrt(mm));
    if (rn <= p.tol) {
      status = 0;
      break;
    }
    if (it >= p.max_iter) break;
    if (rn > kSwitch) {
      // inverse-power step: c <- (K0 + zeta G)^{-1} M c
      for (int e = threadIdx.x; e < n * n; e += kThreads) s.J[e] = fma(zeta, s.G[e], s.K0[e]);
      for (int a = threadIdx.x; a < n; a += kThreads) s.x[a] = s.Mc[a];
      __syncthreads();
      if (!cholesky(s.J, n, s.red)) break;
      chol_solve(s.J, n, s.x);
      for (int a = threadIdx.x; a < n; a += kThreads) s.c[a] = s.x[a];
      __syncthreads();
    } else {
      const int m = s.n1p;
      for (int e = threadIdx.x; e < m * m; e += kThreads) {
        const int a = e / m, b = e % m;
        double v;
        if (a < n && b < n)
          v = fma(3.0 * zeta, s.G[a * n + b], fma(-lam, s.MM[a * n + b], s.K0[a * n + b]));
        else if (a == n && b == n)
          v = 0.0;
        else
          v = -s.Mc[a < n ? a : b];
        s.J[e] = v;
      }
      for (int a = threadIdx.x; a < m; a += kThreads)
        s.x[a] = a < n ? -fma(-lam, s.Mc[a], s.Hc[a]) : 0.0;
      __syncthreads();
      if (!lu_solve(s.J, m, s.x)) break;
      for (int a = threadIdx.x; a < n; a += kThreads) s.c[a] += s.x[a];
      __syncthreads();
    }
    normalise_and_sign(p, s);
  }
  for (int a = threadIdx.x; a < n; a += kThreads) p.c_out[a] = s.c[a];
  if (threadIdx.x == 0) {
    p.lam_out[0] = lam;
    p.iters_out[0] = it;
    p.status_out[0] = status;
  }
}

__global__ void __launch_bounds__(kThreads) k_spd_inverse(const double* L, double* Linv, int n) {
  extern __shared__ double sm[];
  double* A = sm;
  double* red = A + n * n;
  for (int e = threadIdx.x; e < n * n; e += kThreads) A[e] = L[e];
  __syncthreads();
  if (!cholesky(A, n, red)) {
    for (int e = threadIdx.x; e < n * n; e += kThreads) Linv[e] = nan("");
    return;
  }
  // column j of the inverse: forward then backward substitution, one thread per column
  for (int j = threadIdx.x; j < n; j += kThreads) {
    for (int i = 0; i < n; ++i) {
      double s = i == j ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s = fma(-A[i * n + k], Linv[k * n + j], s);
      Linv[i * n + j] = s / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = Linv[i * n + j];
      for (int k = i + 1; k < n; ++k) s = fma(-A[k * n + i], Linv[k * n + j], s);
      Linv[i * n + j] = s / A[i * n + i];
    }
  }
}

__global__ void k_coarse_matvec2d(int n, int pitch, const double* __restrict__ Linv,
                                  const double* __restrict__ x, double* __restrict__ y) {
  const int m = n - 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m * m) return;
  const double* row = Linv + (size_t)p * m * m;
  double s = 0.0;
  for (int q = 0; q < m * m; ++q) s = fma(row[q], x[(size_t)(1 + q / m) * pitch + 1 + q % m], s);
  y[(size_t)(1 + p / m) * pitch + 1 + p % m] = s;
}

}  // namespace

size_t dense_smem_bytes(int n, int ntri, int nvert) {
  const int n1p = n + 1, L = nvert + 1;
  return sizeof(double) * ((size_t)3 * n * n + (size_t)n1p * n1p + 3 * n + n1p +
                           (size_t)ntri * L * L + kThreads);
}

void dense_scf(const DenseProblem& p, cudaStream_t s) {
  const int n = p.nh + p.aug;
  k_dense_scf<<<1, kThreads, dense_smem_bytes(n, p.ntri, p.nvert), s>>>(p);
}

// The attribute is per function, shared by every handle in the process, so it is always set
// to the ceiling every caller is validated against (never to one caller's smaller need).
cudaError_t dense_prepare(size_t need) {
  if (need > kDenseSmemLimit) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_dense_scf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kDenseSmemLimit);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_spd_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kDenseSmemLimit);
}

void dense_spd_inverse(const double* L, double* Linv, int n, cudaStream_t s) {
  k_spd_inverse<<<1, kThreads, sizeof(double) * ((size_t)n * n + kThreads), s>>>(L, Linv, n);
}

void coarse_matvec2d(const Grid& g, const double* Linv, const double* x, double* y,
                     cudaStream_t s) {
  const int m = g.n - 1;
  k_coarse_matvec2d<<<(m * m + 63) / 64, 64, 0, s>>>(g.n, g.pitch, Linv, x, y);
}

}  // namespace fmg
