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
// then Newton steps, which converge quadratically.  A Newton step solves the bordered system
//     [A    -M c] [dc]   [-r]        A = K0 + 3 zeta G(c) - lambda M,  r = F(c, lambda)
//     [-c^T M  0] [dl] = [ 0]        (d/dc of G(c) c is 3 G(c) for the cubic term)
// by block elimination with A' = A + lambda (M c)(M c)^T: the constraint (M c)^T dc = 0 makes
// A' dc = A dc, and A' is positive definite near the ground state (A is semidefinite there,
// singular only along c), so an LDL^T factorisation without pivoting applies:
//     y1 = A'^{-1} r,  y2 = A'^{-1} M c,  dl = (Mc.y1)/(Mc.y2),  dc = -y1 + dl y2.
// lambda is reported as c^T (K0 + zeta G(c)) c at the final c.
//
// G(c) is assembled per coarse simplex T from the exact integrals of products of its
// barycentrics (local_G) and, on the augmented space (w = w_H + c_u u~), from the fine-pass
// integrals (augment2d.cu): T3^T (per simplex), B1 = int u~^2 phi phi, t1 = int u~^3 phi,
// T0 = int u~^4:
//   G_ab = sum_T [int_T w_H^2 mu_a mu_b + 2 c_u sum w_c T3_abc] + c_u^2 B1_ab
//   G_au = sum_T sum w_c w_d T3_acd + 2 c_u (B1 c_H)_a + c_u^2 t1_a
//   G_uu = c_H^T B1 c_H + 2 c_u t1.c_H + c_u^2 T0
// with w_c the coarse coefficients at T's vertices (0 on the boundary).
//
// One CTA of 256 threads per problem, a batch of problems one CTA each (measured against 128
// and 512: the solve is bound by barriers and latency on one SM, and 256 threads balance the
// work per thread against the cost of each block-wide barrier),
// everything in shared memory, fixed-order reductions, one barrier per elimination step and
// warp-synchronous triangular solves.  The iteration count is bounded by max_iter; hitting it
// sets status 1.
#include <math.h>
#include <stdint.h>

#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr int kThreads = 256;

// the simplex-local blocks (ntri (nvert + 1)^2 doubles) fit in the n x n work matrix A
__host__ __device__ inline bool loc_in_A(int n, int ntri, int nvert) {
  return (size_t)ntri * (nvert + 1) * (nvert + 1) <= (size_t)n * n;
}
constexpr int kWarps = kThreads / 32;
constexpr int kMaxVert = 4;
constexpr double kSwitch = 1e-2;  // relative residual below which Newton takes over
// refinement steps of the linear solves (single-precision inverse, FP64 residuals).  The
// single-precision inverse leaves a relative error of about 7e-7 in a solve and one step
// squares it (~5e-13); a Newton correction is as large as the current error, so its own error
// is then far below FP64 rounding of c (two steps gave the same iteration counts and the same
// eigenvalues to 3e-16).  While the residual is above kRefineBelow the step needs no
// refinement at all: its error, about 7e-7 of the correction, is then below a tenth of the
// quadratic term C e^2 (C ~ 10) that the step leaves anyway.  An inverse-power step needs
// only a direction.
constexpr int kRefineNewton = 1;
constexpr double kRefineBelow = 1e-6;
constexpr int kRefinePower = 1;

struct Smem {
  double *K0, *MM, *G, *A, *loc;
  const double* B1;
  double *c, *Mc, *Hc, *Gc, *r, *y1, *y2, *dinv, *red, *sv;
  int* sym3;  // nv^3 table of sorted-triple indices
  int *tri, *adj;  // shared copies of the simplex and adjacency tables
  double *t3, *t1;  // shared copies of the fine-pass integrals (augmented problem)
  int n, nh, L;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order: butterfly within each warp, then warp 0 adds the warp
// totals in the same butterfly order (two barriers).  Every thread gets the result.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = (threadIdx.x & 31) < kWarps ? red[threadIdx.x & 31] : 0.0;
  t = warp_sum(t);
  __syncthreads();  // red may be reused right away
  return t;
}

// 1 / d by Newton's iteration from the hardware's approximate reciprocal (about 2^-20 relative
// error; two steps reach FP64 rounding).
__device__ __forceinline__ double recip(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  y = fma(y, fma(-d, y, 1.0), y);
  y = fma(y, fma(-d, y, 1.0), y);
  return y;
}

// Two block-wide sums at once, each in block_sum's order (so each result is bit-identical to
// its own block_sum), for the price of one: the second reduces in red[kWarps ..].
__device__ double2 block_sum2(double a, double b, double* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = a;
    red[kWarps + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  const int l = threadIdx.x & 31;
  double ta = l < kWarps ? red[l] : 0.0, tb = l < kWarps ? red[kWarps + l] : 0.0;
  ta = warp_sum(ta);
  tb = warp_sum(tb);
  __syncthreads();
  return make_double2(ta, tb);
}

__device__ double dotv(const double* a, const double* b, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) s = fma(a[i], b[i], s);
  return block_sum(s, red);
}

// y_q = sum_b X_q[a][b] x_b for up to three symmetric n x n matrices X_q and every row a:
// thread t takes row a = t % n and the columns b = part, part + parts, ... (part = t / n), so
// the lanes of a warp read consecutive rows of one column (conflict-free, X symmetric); the
// row's thread then adds the parts in a fixed order.  `red` holds parts * n * 3 doubles.
template <int NM>
__device__ void symv(const double* const* X, const double* x, double* const* y, int n,
                     double* red) {
  const int parts = n <= kThreads ? kThreads / n : 1;
  const int t = threadIdx.x;
  const int a = t % n, part = t / n;
  if (part < parts && t < parts * n) {
    double acc[NM];
#pragma unroll
    for (int q = 0; q < NM; ++q) acc[q] = 0.0;
    for (int b = part; b < n; b += parts) {
      const double xb = x[b];
#pragma unroll
      for (int q = 0; q < NM; ++q) acc[q] = fma(X[q][(size_t)b * n + a], xb, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < NM; ++q) red[((size_t)q * parts + part) * n + a] = acc[q];
  }
  __syncthreads();
  for (int r = t; r < n; r += kThreads) {
#pragma unroll
    for (int q = 0; q < NM; ++q) {
      double v = 0.0;
      for (int pp = 0; pp < parts; ++pp) v += red[((size_t)q * parts + pp) * n + r];
      y[q][r] = v;
    }
  }
  __syncthreads();
}

// rows of (K0 c, G c); M c is kept up to date by normalise_and_sign
__device__ void apply_all(Smem& s) {
  const double* X[2] = {s.K0, s.G};
  double* Y[2] = {s.Hc, s.Gc};
  symv<2>(X, s.c, Y, s.n, s.sv);
}

// Local contributions of each simplex T (one thread per simplex): the pair entries
// int_T w^2 mu_a mu_b (+ 2 c_u sum_c w_c T3_abc) and, on the augmented space, the coupling
// sum_cd w_c w_d T3_acd of vertex a with u~.  By the barycentric monomial rule
// int_T mu^alpha = d! |T| alpha! / (|alpha| + d)!,
//   int_T w^2 mu_a mu_b = |T| 2 d! / (d + 4)! h_2(w_1 .. w_nv, w_a, w_b)   (a != b),
// and twice that for a = b, with h_2 the complete homogeneous symmetric polynomial of degree
// 2 (the count of ways to share the exponent of w_a between the copies of w_a is exactly the
// factor alpha_a + 1 the rule produces), so a simplex needs h_1 = sum w, h_2 and a few
// products per pair.  The u~ coupling reuses the pair sums x3_ac = sum_d w_d T3_acd.
template <int NV>
__device__ void local_G(const DenseProblem& p, Smem& s, double cu) {
  const int L = s.L;
  for (int t = threadIdx.x; t < p.ntri; t += kThreads) {
    double wv[NV], sq[NV];
    double h1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int id = s.tri[t * NV + v];
      wv[v] = id >= 0 ? s.c[id] : 0.0;
      sq[v] = wv[v] * wv[v];
      h1 += wv[v];
      s2 += sq[v];
    }
    const double h2 = 0.5 * fma(h1, h1, s2);  // sum_{i <= j} w_i w_j
    const double* t3 = s.t3 + (size_t)t * p.nt3;
    double* lt = s.loc + (size_t)t * L * L;
    double ucp[NV];  // sum_b w_b x3_ab, accumulated pair by pair (x3 is symmetric)
#pragma unroll
    for (int a = 0; a < NV; ++a) ucp[a] = 0.0;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int b = a; b < NV; ++b) {
        double v;
        if (a == b) v = 2.0 * p.quart_off * fma(3.0, sq[a], fma(2.0 * wv[a], h1, h2));
        else v = p.quart_off * (fma(wv[a] + wv[b], h1, h2) + fma(wv[a], wv[b], sq[a] + sq[b]));
        if (p.aug) {
          double x = 0.0;  // x3_ab = sum_c w_c T3_abc
#pragma unroll
          for (int c = 0; c < NV; ++c) x = fma(wv[c], t3[s.sym3[(a * NV + b) * NV + c]], x);
          ucp[a] = fma(wv[b], x, ucp[a]);
          if (b != a) ucp[b] = fma(wv[a], x, ucp[b]);
          v = fma(2.0 * cu, x, v);
        }
        lt[a * L + b] = v;
        lt[b * L + a] = v;
      }
    if (p.aug) {
#pragma unroll
      for (int a = 0; a < NV; ++a) lt[a * L + NV] = ucp[a];
    }
  }
}

__device__ void build_G(const DenseProblem& p, Smem& s) {
  const int nv = p.nvert, L = s.L, nh = s.nh, n = s.n;
  const double cu = p.aug ? s.c[nh] : 0.0;
  if (p.aug) {
    // w = c_u u~ (the start of every augmented solve: c_H = 0 exactly): every simplex term
    // vanishes and G is c_u^2 [B1 t1; t1^T T0], which the general path below also reaches
    // (its sums then add only zeros), so the results are identical
    bool any = false;
    for (int a = threadIdx.x; a < nh; a += kThreads) any |= s.c[a] != 0.0;
    if (!__syncthreads_or(any)) {
      const double cu2 = cu * cu;
      for (int e = threadIdx.x; e < nh * nh; e += kThreads) {
        const int a = e / nh, b = e - a * nh;
        s.G[(size_t)a * n + b] = __dmul_rn(cu2, s.B1[e]);
      }
      for (int a = threadIdx.x; a < nh; a += kThreads) {
        const double g = __dmul_rn(cu2, s.t1[a]);
        s.G[(size_t)a * n + nh] = g;
        s.G[(size_t)nh * n + a] = g;
      }
      if (threadIdx.x == 0) s.G[(size_t)nh * n + nh] = __dmul_rn(cu * cu, p.t0[0]);
      __syncthreads();
      return;
    }
  }
  if (p.nvert == 3) local_G<3>(p, s, cu);
  else local_G<4>(p, s, cu);
  __syncthreads();
  if (p.aug) {  // Hc <- B1 c_H (scratch; recomputed by apply_all afterwards)
    const double* X[1] = {s.B1};
    double* Y[1] = {s.Hc};
    symv<1>(X, s.c, Y, nh, s.sv);
  }
  const double cu2 = cu * cu;
  // coarse block: every entry starts as [c_u^2 B1_ab] (rounded on its own, no contraction)
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = warp; a < nh; a += kWarps) {
      double* row = s.G + (size_t)a * n;
      const double* brow = p.aug ? s.B1 + (size_t)a * nh : nullptr;
      for (int b = lane; b < nh; b += 32) row[b] = p.aug ? __dmul_rn(cu2, brow[b]) : 0.0;
    }
  }
  __syncthreads();
  if (p.gent) {
    // then each structurally nonzero entry adds its simplex contributions, one thread per
    // entry, in the order of the gather list (a's adjacency order, then vertex order)
    for (int q = threadIdx.x; q < p.npat; q += kThreads) {
      const int e = __ldg(p.gent + q), k1 = __ldg(p.gstart + q + 1);
      const int a = e / nh, b = e - a * nh;
      double* g = s.G + (size_t)a * n + b;
      double v = *g;
      for (int k = __ldg(p.gstart + q); k < k1; ++k) v += s.loc[__ldg(p.gidx + k)];
      *g = v;
    }
  } else {
    // no gather lists: each row's thread walks its simplices and adds into its row
    for (int a = threadIdx.x; a < nh; a += kThreads) {
      double* row = s.G + (size_t)a * n;
      for (int k = 0; k < p.maxadj; ++k) {
        const int code = s.adj[a * p.maxadj + k];
        if (code < 0) break;
        const int t = code >> 3, la = code & 7;
        const double* lt = s.loc + (size_t)t * L * L;
        for (int lb = 0; lb < nv; ++lb) {
          const int vb = s.tri[t * nv + lb];
          if (vb >= 0) row[vb] += lt[la * L + lb];
        }
      }
    }
  }
  if (p.aug) {
    // coupling of row a with u~, on the threads with the least work above (the last ones)
    for (int a = kThreads - 1 - threadIdx.x; a < nh; a += kThreads) {
      double au = 0.0;
      for (int k = 0; k < p.maxadj; ++k) {
        const int code = s.adj[a * p.maxadj + k];
        if (code < 0) break;
        const int t = code >> 3, la = code & 7;
        au += s.loc[(size_t)t * L * L + la * L + nv];
      }
      s.G[(size_t)a * n + nh] = fma(cu2, s.t1[a], fma(2.0 * cu, s.Hc[a], au));
    }
  }
  if (p.aug) {
    double part = 0.0;
    for (int a = threadIdx.x; a < nh; a += kThreads)
      part = fma(s.c[a], fma(2.0 * cu, s.t1[a], s.Hc[a]), part);
    const double tot = block_sum(part, s.red);  // also orders the row writes above
    if (threadIdx.x == 0) s.G[(size_t)nh * n + nh] = fma(cu * cu, p.t0[0], tot);
    for (int a = threadIdx.x; a < nh; a += kThreads) s.G[(size_t)nh * n + a] = s.G[(size_t)a * n + nh];
  }
  __syncthreads();
}

// In-place symmetric elimination A = L D L^T (no pivoting) on the lower triangle: after it,
// A_kk = D_k and A_ik = L_ik D_k (i > k); dinv[k] = 1 / D_k.  At step k every thread updates
// its elements (i >= j > k) of the trailing triangle, and the thread that updates the next
// pivot also forms its reciprocal, so each step needs one barrier.  Returns false at a
// non-positive pivot (every thread reads the same pivot, so all return together).
__device__ bool ldlt(double* A, int n, double* dinv) {
  if (threadIdx.x == 0) dinv[0] = A[0] > 0.0 ? recip(A[0]) : 0.0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const double d = A[k * n + k];
    if (!(d > 0.0)) return false;
    const double inv = dinv[k];
    const int m = n - k - 1;
    const int tri = m * (m + 1) / 2;
    for (int e = threadIdx.x; e < tri; e += kThreads) {
      // e -> (r, c), c <= r, rows of the trailing lower triangle in order
      int r = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      while ((r + 1) * (r + 2) / 2 <= e) ++r;
      while (r * (r + 1) / 2 > e) --r;
      const int c = e - r * (r + 1) / 2;
      const int i = k + 1 + r, j = k + 1 + c;
      const double v = fma(-(A[i * n + k] * inv), A[j * n + k], A[i * n + j]);
      A[i * n + j] = v;
      if (e == 0) dinv[k + 1] = v > 0.0 ? recip(v) : 0.0;  // (k+1, k+1): the next pivot
    }
    __syncthreads();
  }
  return true;
}

// Solve (L D L^T) x = b for x held in `x` (b on entry), by one warp, column by column: once
// an entry is final, the lanes update the remaining ones (only warp-level synchronisation).
// Reads the lower triangle written by ldlt.
__device__ void ldlt_solve_warp(const double* A, const double* dinv, int n, double* x) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < n; ++k) {  // forward: w_k = z_k / D_k, z_i -= A_ik w_k (i > k)
    const double wk = x[k] * dinv[k];
    __syncwarp();
    if (lane == 0) x[k] = wk;
    for (int i = k + 1 + lane; i < n; i += 32) x[i] = fma(-A[i * n + k], wk, x[i]);
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {  // backward: x_i -= (A_ki / D_i) x_k (i < k)
    const double xk = x[k];
    for (int i = lane; i < k; i += 32) x[i] = fma(-A[k * n + i] * dinv[i], xk, x[i]);
    __syncwarp();
  }
}

// Inverse of an SPD n x n matrix in single precision by the sweep operator (Gauss-Jordan
// elimination without pivoting, stable for SPD matrices).  Sweeping a set P of indices maps
// M to M' with H = (M_PP)^{-1}:
//     M'_PP = -H,  M'_Pj = H M_Pj,  M'_iP = M_iP H,  M'_ij = M_ij - M_iP H M_Pj  (i, j not in P),
// and after sweeping every index the matrix is -A^{-1}.  Sweeping P at once equals sweeping
// its indices one after another, so the indices go in blocks of 4 (the matrix padded to a
// multiple of 4 with an identity block, which sweeps to itself): one barrier per block.  The
// sweep keeps M symmetric, so the pivot columns are read from the pivot rows.  Each row
// belongs to 256 / R threads (R = 64 rows for n <= 64, 32 for n <= 32), each keeping
// C = R / (256 / R) contiguous columns in registers for the whole elimination; the owners of
// the next pivot rows publish them to shared memory (rowb: 2 x 4 rows of 64 floats,
// double-buffered, 16-byte aligned).  Every thread inverts the 4 x 4 pivot block itself, by
// four scalar sweeps in registers with fast approximate reciprocals (their error is one more
// single-precision rounding, which the refinement removes).
template <int R>
__device__ __forceinline__ void sweep_rows(const double* __restrict__ A, float* __restrict__ M,
                                           float* __restrict__ rowb, int n, bool& ok) {
  constexpr int T = kThreads / R;  // threads per row
  constexpr int C = R / T;         // columns per thread (T C = R >= n), a multiple of 4
  const int i = threadIdx.x / T, jb = (threadIdx.x % T) * C;
  const int np = (n + 3) & ~3;     // padded size, <= R
  float v[C];
#pragma unroll
  for (int q = 0; q < C; ++q) {
    const int j = jb + q;
    v[q] = i < n && j < n ? (float)A[i * n + j] : (i == j ? 1.0f : 0.0f);
  }
  if (i < 4) {
#pragma unroll
    for (int q = 0; q < C; q += 4)
      *reinterpret_cast<float4*>(rowb + i * 64 + jb + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
  }
  __syncthreads();
  for (int k = 0; k < np; k += 4) {
    const float* rb = rowb + ((k >> 2) & 1) * 256;  // rows k .. k + 3
    // H = (M_PP)^{-1}: four scalar sweeps of the pivot block give -H
    float h[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) h[r][c] = rb[r * 64 + k + c];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float d = h[m][m];
      if (!(d > 0.0f)) {
        ok = false;
        return;
      }
      const float inv = __fdividef(1.0f, d);
      float g[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (r == m) g[r][c] = c == m ? -inv : h[m][c] * inv;
          else g[r][c] = c == m ? h[r][m] * inv : fmaf(-h[r][m] * inv, h[m][c], h[r][c]);
        }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) h[r][c] = g[r][c];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) h[r][c] = -h[r][c];  // the sweeps left -H
    float f[4];  // M_iP H, with M_iP = M_Pi from the pivot rows
    {
      float mi[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) mi[r] = rb[r * 64 + i];
#pragma unroll
      for (int c = 0; c < 4; ++c)
        f[c] = fmaf(mi[0], h[0][c], fmaf(mi[1], h[1][c], fmaf(mi[2], h[2][c], mi[3] * h[3][c])));
    }
    const bool prow = i >= k && i < k + 4;
#pragma unroll
    for (int q = 0; q < C; q += 4) {
      float4 a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = *reinterpret_cast<const float4*>(rb + r * 64 + jb + q);
      const float ak[4][4] = {{a[0].x, a[1].x, a[2].x, a[3].x}, {a[0].y, a[1].y, a[2].y, a[3].y},
                              {a[0].z, a[1].z, a[2].z, a[3].z}, {a[0].w, a[1].w, a[2].w, a[3].w}};
      if (jb + q == k) {  // the pivot columns: M_iP H, or -H on the pivot rows
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float hv = 0.0f;
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (i == k + r) hv = -h[r][e];
          v[q + e] = prow ? hv : f[e];
        }
      } else if (prow) {  // the pivot rows: H M_Pj
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float hv = 0.0f;
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (i == k + r)
              hv = fmaf(h[r][0], ak[e][0], fmaf(h[r][1], ak[e][1], fmaf(h[r][2], ak[e][2], h[r][3] * ak[e][3])));
          v[q + e] = hv;
        }
      } else {  // M_ij - M_iP H M_Pj
#pragma unroll
        for (int e = 0; e < 4; ++e)
          v[q + e] = fmaf(-f[0], ak[e][0], fmaf(-f[1], ak[e][1], fmaf(-f[2], ak[e][2], fmaf(-f[3], ak[e][3], v[q + e]))));
      }
    }
    if (k + 4 < np && i >= k + 4 && i < k + 8) {  // publish rows k + 4 .. k + 7
      float* rn = rowb + (((k >> 2) + 1) & 1) * 256 + (i - k - 4) * 64;
#pragma unroll
      for (int q = 0; q < C; q += 4)
        *reinterpret_cast<float4*>(rn + jb + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    }
    __syncthreads();
  }
  if (i < n) {
#pragma unroll
    for (int q = 0; q < C; ++q)
      if (jb + q < n) M[i * n + jb + q] = v[q];
  }
  __syncthreads();
}

// -A^{-1} into M (n x n floats, row-major) for an SPD FP64 n x n matrix A, n <= 64; false at
// a non-positive pivot or for n > 64 (every thread reads the same pivots, so all return
// together).  rowb: 512 floats, 16-byte aligned.
__device__ __forceinline__ bool sweep_inverse(const double* __restrict__ A, float* __restrict__ M,
                                              float* __restrict__ rowb, int n) {
  bool ok = true;
  if (n <= 32) sweep_rows<32>(A, M, rowb, n, ok);
  else if (n <= 64) sweep_rows<64>(A, M, rowb, n, ok);
  else ok = false;
  return ok;
}

// y_v = X x_v (v < NV) for one symmetric FP64 n x n matrix X and NV FP64 vectors, with the
// row/part split of symv.  red: parts * n * NV doubles.
template <int NV>
__device__ void symv_vec(const double* X, const double* const* x, double* const* y, int n,
                         double* red) {
  const int parts = n <= kThreads ? kThreads / n : 1;
  const int t = threadIdx.x;
  const int a = t % n, part = t / n;
  if (part < parts && t < parts * n) {
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int b = part; b < n; b += parts) {
      const double xab = X[(size_t)b * n + a];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fma(xab, x[v][b], acc[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) red[((size_t)v * parts + part) * n + a] = acc[v];
  }
  __syncthreads();
  for (int r = t; r < n; r += kThreads) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double w = 0.0;
      for (int pp = 0; pp < parts; ++pp) w += red[((size_t)v * parts + pp) * n + r];
      y[v][r] = w;
    }
  }
  __syncthreads();
}

// y_v (FP64) = -X x_v for the single-precision symmetric matrix X = -A^{-1} of the sweep
// operator and NV vectors x_v (FP64), all in single precision: the vectors are rounded to
// FP32 once into xf (NV n floats), the parts summed in FP32 in redf (parts n NV floats), and
// only the n NV results converted back.  (Conversions between FP64 and FP32 issue at the
// FP64 rate, so none sits inside the n^2 loop.)
template <int NV>
__device__ void symv_f32(const float* X, const double* const* x, double* const* y, int n,
                         float* xf, float* redf) {
  for (int r = threadIdx.x; r < n; r += kThreads) {
#pragma unroll
    for (int v = 0; v < NV; ++v) xf[v * n + r] = (float)x[v][r];
  }
  __syncthreads();
  const int parts = n <= kThreads ? kThreads / n : 1;
  const int t = threadIdx.x;
  const int a = t % n, part = t / n;
  if (part < parts && t < parts * n) {
    float acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0f;
    for (int b = part; b < n; b += parts) {
      const float xab = X[(size_t)b * n + a];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fmaf(xab, xf[v * n + b], acc[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) redf[((size_t)v * parts + part) * n + a] = acc[v];
  }
  __syncthreads();
  for (int r = t; r < n; r += kThreads) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float w = 0.0f;
      for (int pp = 0; pp < parts; ++pp) w += redf[((size_t)v * parts + pp) * n + r];
      y[v][r] = -(double)w;
    }
  }
  __syncthreads();
}

// Solve A y_v = b_v (v < NV) for the SPD FP64 matrix A (kept intact) to FP64 accuracy:
// A^{-1} in single precision by the sweep operator (in the two float buffers P0, P1), then
// `refine` steps of iterative refinement with FP64 residuals e = b - A y.  Each step cuts the
// error by about cond(A) 2^-24 (cond(A) is of order 10^3 for these coarse spaces), so two
// steps reach FP64 rounding.  b_v is read, y_v written, e_v is scratch; false (nothing
// written) when the single-precision elimination meets a non-positive pivot.
template <int NV>
__device__ __forceinline__ bool solve_refined(const double* A, float* Ainv, int n,
                                              const double* const* b, double* const* y,
                                              double* const* e, int refine, double* red) {
  // single-precision staging in the reduction scratch (3 kThreads doubles = 1536 floats):
  // the sweep's pivot rows (512 floats + alignment), then NV n floats of vectors
  // and parts n NV <= kThreads NV floats of partial sums (n <= 64 here); symv_vec's use of
  // it never overlaps
  float* xf = reinterpret_cast<float*>(red);
  // the pivot row is read as float4: 16-byte alignment (red is only 8-byte aligned)
  float* rowb = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(red) + 15) & ~uintptr_t(15));
  if (!sweep_inverse(A, Ainv, rowb, n)) return false;
  float* redf = xf + NV * n;
  symv_f32<NV>(Ainv, b, y, n, xf, redf);  // y = A^{-1} b
  for (int it = 0; it < refine; ++it) {
    symv_vec<NV>(A, y, e, n, red);  // e = A y
    for (int r = threadIdx.x; r < n; r += kThreads) {
#pragma unroll
      for (int v = 0; v < NV; ++v) e[v][r] = b[v][r] - e[v][r];
    }
    __syncthreads();
    symv_f32<NV>(Ainv, e, e, n, xf, redf);  // correction A^{-1} e, in place of e
    for (int r = threadIdx.x; r < n; r += kThreads) {
#pragma unroll
      for (int v = 0; v < NV; ++v) y[v][r] += e[v][r];
    }
    __syncthreads();
  }
  return true;
}

__device__ void normalise_and_sign(const DenseProblem& p, Smem& s) {
  const int n = s.n;
  {
    const double* X[1] = {s.MM};
    double* Y[1] = {s.Mc};
    symv<1>(X, s.c, Y, n, s.sv);
  }
  double cmc, sg;
  if (p.aug) {
    cmc = dotv(s.c, s.Mc, n, s.red);
    sg = s.c[s.nh];
  } else {
    double d = 0.0, t = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      d = fma(s.c[i], s.Mc[i], d);
      t += s.c[i];
    }
    const double2 dt = block_sum2(d, t, s.red);
    cmc = dt.x;
    sg = dt.y;
  }
  __syncthreads();  // every thread has read c before any thread rescales it
  const double f = (sg < 0.0 ? -1.0 : 1.0) / sqrt(cmc);
  for (int i = threadIdx.x; i < n; i += kThreads) {
    s.c[i] *= f;
    s.Mc[i] *= f;  // M c of the rescaled c
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 2) k_dense_scf(DenseProblem p) {
  extern __shared__ double sm[];
  if (blockIdx.x) {  // instance blockIdx.x of a batch: its slices of the per-instance arrays
    const size_t b = blockIdx.x, nh = p.nh, cs = nh + 1;
    p.L1 += b * nh * nh;
    p.M1 += b * nh * nh;
    p.params += b;
    p.c_out += b * cs;
    p.lam_out += b;
    p.iters_out += b;
    p.status_out += b;
    if (p.c_init) p.c_init += b * cs;
    if (p.aug) {
      p.gA += b * nh;
      p.gM += b * nh;
      p.t1 += b * nh;
      p.B1 += b * nh * nh;
      p.t3 += b * (size_t)p.ntri * p.nt3;
      p.auu += b;
      p.buu += b;
      p.t0 += b;
    }
  }
  __shared__ int sym3_tab[kMaxVert * kMaxVert * kMaxVert];
  // the layout is computed by every thread, then kept in shared memory (published by thread
  // 0), so its ~25 pointers need not stay in registers through the iteration
  __shared__ Smem s_layout;
  Smem sl;
  sl.nh = p.nh;
  sl.n = p.nh + p.aug;
  sl.L = p.nvert + 1;
  const int n = sl.n, nh = sl.nh, nv = p.nvert;
  double* q = sm;
  sl.K0 = q; q += (size_t)n * n;
  sl.MM = q; q += (size_t)n * n;
  sl.G = q; q += (size_t)n * n;
  sl.A = q; q += (size_t)n * n;
  // the simplex-local blocks are only live inside build_G, when A is free: they share its
  // space when they fit (2D), which with B1 read from global memory keeps a 2D CTA under
  // half the shared memory of an SM (two instances of a batch per SM)
  if (loc_in_A(n, p.ntri, p.nvert)) {
    sl.loc = sl.A;
  } else {
    sl.loc = q;
    q += (size_t)p.ntri * sl.L * sl.L;
  }
  sl.c = q; q += n;
  sl.Mc = q; q += n;
  sl.Hc = q; q += n;
  sl.Gc = q; q += n;
  sl.r = q; q += n;
  sl.y1 = q; q += n;
  sl.y2 = q; q += n;
  sl.dinv = q; q += n;
  sl.red = q; q += kThreads;
  sl.sv = q; q += 3 * kThreads;
  sl.t1 = q; q += nh;
  sl.t3 = q; q += p.aug ? (size_t)p.ntri * p.nt3 : 0;
  sl.tri = reinterpret_cast<int*>(q); q += ((size_t)p.ntri * nv + 1) / 2;
  sl.adj = reinterpret_cast<int*>(q); q += ((size_t)nh * p.maxadj + 1) / 2;
  sl.B1 = p.aug ? p.B1 : nullptr;  // nh * nh in global memory (read twice per build_G)
  sl.sym3 = sym3_tab;
  if (threadIdx.x == 0) s_layout = sl;
  __syncthreads();
  Smem& s = s_layout;

  const double zeta = p.params->zeta;
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    const int a = e / n, b = e - (e / n) * n;
    double kv, mv;
    if (a < nh && b < nh) {
      kv = p.L1[a * nh + b];
      mv = p.M1[a * nh + b];
    } else if (a == nh && b == nh) {
      kv = p.auu[0];
      mv = p.buu[0];
    } else {
      const int qq = a < nh ? a : b;
      kv = p.gA[qq];
      mv = p.gM[qq];
    }
    s.K0[e] = kv;
    s.MM[e] = mv;
  }
  if (p.aug) {
    for (int e = threadIdx.x; e < nh; e += kThreads) s.t1[e] = p.t1[e];
    for (int e = threadIdx.x; e < p.ntri * p.nt3; e += kThreads) s.t3[e] = p.t3[e];
  }
  for (int e = threadIdx.x; e < p.ntri * nv; e += kThreads) s.tri[e] = p.tri[e];
  for (int e = threadIdx.x; e < nh * p.maxadj; e += kThreads) s.adj[e] = p.adj[e];
  for (int e = threadIdx.x; e < nv * nv * nv; e += kThreads) {
    int a = e / (nv * nv), b = (e / nv) % nv, c = e % nv;
    if (a > b) { const int t = a; a = b; b = t; }
    if (b > c) { const int t = b; b = c; c = t; }
    if (a > b) { const int t = a; a = b; b = t; }
    int idx = 0;
    for (int x = 0; x < a; ++x) idx += (nv - x) * (nv - x + 1) / 2;
    for (int y = a; y < b; ++y) idx += nv - y;
    sym3_tab[e] = idx + (c - b);
  }
  for (int i = threadIdx.x; i < n; i += kThreads)
    s.c[i] = p.c_init ? p.c_init[i] : (i == nh ? 1.0 : 0.0);
  __syncthreads();
  if (p.K_out) {  // assemble-only mode: K0, M and G(c_init) as given
    build_G(p, s);
    for (int e = threadIdx.x; e < n * n; e += kThreads) {
      p.K_out[e] = s.K0[e];
      p.M_out[e] = s.MM[e];
      p.G_out[e] = s.G[e];
    }
    return;
  }
  normalise_and_sign(p, s);

  int it = 0, status = 1;
  double lam = 0.0;
  for (;; ++it) {
    build_G(p, s);
    apply_all(s);  // Hc = K0 c, Gc = G c (Mc = M c from normalise_and_sign)
    // each thread forms, reads and later overwrites only its own rows of Hc and r here, so
    // the loops need no barrier between them (the block sums order everything after them)
    double lp = 0.0, mm = 0.0;
    for (int a = threadIdx.x; a < n; a += kThreads) {
      const double h = fma(zeta, s.Gc[a], s.Hc[a]);
      s.Hc[a] = h;
      lp = fma(s.c[a], h, lp);
      mm = fma(s.Mc[a], s.Mc[a], mm);
    }
    const double2 lm = block_sum2(lp, mm, s.red);
    lam = lm.x;
    mm = lm.y;
    double rr = 0.0;
    for (int a = threadIdx.x; a < n; a += kThreads) {
      const double r = fma(-lam, s.Mc[a], s.Hc[a]);
      s.r[a] = r;
      rr = fma(r, r, rr);
    }
    rr = block_sum(rr, s.red);
    const double rn = sqrt(rr) / (fabs(lam) * sqrt(mm));
    if (rn <= p.tol) {
      status = 0;
      break;
    }
    if (it >= p.max_iter) break;
    bool newton = rn <= kSwitch;
    // the single-precision inverse of the linear solves below lives in G's space (G is not
    // read again before the next build_G)
    float* Pinv = reinterpret_cast<float*>(s.G);
    bool g_valid = true;
    if (newton) {
      // A' = K0 + 3 zeta G - lambda M + |lambda| (Mc)(Mc)^T, symmetric: the lower triangle
      // in FP64 (|lambda| Mc staged in dinv), then mirrored
      const double tau = fabs(lam), z3 = 3.0 * zeta;
      for (int a = threadIdx.x; a < n; a += kThreads) s.dinv[a] = tau * s.Mc[a];
      __syncthreads();
      for (int e = threadIdx.x; e < n * n; e += kThreads) {
        const int a = e / n, b = e - (e / n) * n;
        if (b <= a)
          s.A[e] = fma(s.dinv[a], s.Mc[b], fma(z3, s.G[e], fma(-lam, s.MM[e], s.K0[e])));
      }
      __syncthreads();
      for (int e = threadIdx.x; e < n * n; e += kThreads) {
        const int a = e / n, b = e - (e / n) * n;
        if (b > a) s.A[e] = s.A[(size_t)b * n + a];
      }
      __syncthreads();
      const double* rhs[2] = {s.r, s.Mc};
      double* sol[2] = {s.y1, s.y2};
      double* scr[2] = {s.Hc, s.Gc};
      g_valid = false;
      const int refine = rn < kRefineBelow ? kRefineNewton : 0;
      if (!solve_refined<2>(s.A, Pinv, n, rhs, sol, scr, refine, s.sv)) {
        // single precision met a non-positive pivot: LDL^T in FP64
        for (int a = threadIdx.x; a < n; a += kThreads) {
          s.y1[a] = s.r[a];
          s.y2[a] = s.Mc[a];
        }
        __syncthreads();
        newton = ldlt(s.A, n, s.dinv);
        if (newton) {
          if ((threadIdx.x >> 5) == 0) ldlt_solve_warp(s.A, s.dinv, n, s.y1);
          else if ((threadIdx.x >> 5) == 1) ldlt_solve_warp(s.A, s.dinv, n, s.y2);
          __syncthreads();
        }
      }
      if (newton) {
        double p1 = 0.0, p2 = 0.0;
        for (int a = threadIdx.x; a < n; a += kThreads) {
          p1 = fma(s.Mc[a], s.y1[a], p1);
          p2 = fma(s.Mc[a], s.y2[a], p2);
        }
        const double2 m12 = block_sum2(p1, p2, s.red);
        const double dl = m12.x / m12.y;
        for (int a = threadIdx.x; a < n; a += kThreads) s.c[a] += fma(dl, s.y2[a], -s.y1[a]);
        __syncthreads();
      }
    }
    if (!newton) {
      // inverse-power step: c <- (K0 + zeta G)^{-1} M c
      if (!g_valid) build_G(p, s);  // the Newton attempt overwrote G
      for (int e = threadIdx.x; e < n * n; e += kThreads) s.A[e] = fma(zeta, s.G[e], s.K0[e]);
      __syncthreads();
      const double* rhs[1] = {s.Mc};
      double* sol[1] = {s.y1};
      double* scr[1] = {s.Hc};
      if (!solve_refined<1>(s.A, Pinv, n, rhs, sol, scr, kRefinePower, s.sv)) {
        for (int a = threadIdx.x; a < n; a += kThreads) s.y1[a] = s.Mc[a];
        __syncthreads();
        if (!ldlt(s.A, n, s.dinv)) break;
        if ((threadIdx.x >> 5) == 0) ldlt_solve_warp(s.A, s.dinv, n, s.y1);
        __syncthreads();
      }
      for (int a = threadIdx.x; a < n; a += kThreads) s.c[a] = s.y1[a];
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

// L^{-1} for an SPD matrix: L = C D C^T, then all columns of C D C^T X = I at once (rows
// sequential, columns spread over the threads), everything in shared memory.
__global__ void __launch_bounds__(kThreads) k_spd_inverse(const double* L, double* Linv, int n) {
  extern __shared__ double sm[];
  L += blockIdx.x * (size_t)n * n;  // instance blockIdx.x
  Linv += blockIdx.x * (size_t)n * n;
  double* A = sm;
  double* Y = A + n * n;
  double* dinv = Y + n * n;
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    A[e] = L[e];
    const int i = e / n, j = e - (e / n) * n;
    Y[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  if (!ldlt(A, n, dinv)) {
    for (int e = threadIdx.x; e < n * n; e += kThreads) Linv[e] = nan("");
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // forward: rows of W with (C D) W = I: W_k = (Y_k - sum_{i<k} A_ki W_i) / D_k
  for (int k = 0; k < n; ++k) {
    const double inv = dinv[k];
    for (int j = threadIdx.x; j < n; j += kThreads) Y[k * n + j] *= inv;
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += kWarps) {
      const double l = A[i * n + k];
      for (int j = lane; j < n; j += 32) Y[i * n + j] = fma(-l, Y[k * n + j], Y[i * n + j]);
    }
    __syncthreads();
  }
  // backward: C^T X = W, X_i = W_i - sum_{k>i} (A_ki / D_i) X_k
  for (int k = n - 1; k >= 0; --k) {
    for (int i = warp; i < k; i += kWarps) {
      const double l = A[k * n + i] * dinv[i];
      for (int j = lane; j < n; j += 32) Y[i * n + j] = fma(-l, Y[k * n + j], Y[i * n + j]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += kThreads) Linv[e] = Y[e];
}

// y = Linv x on the interior of level 1: one CTA, x gathered to shared memory, one warp per
// row with coalesced loads and a shuffle reduction.
__device__ __forceinline__ size_t level1_index(int dim, int m, int pitch, int q) {
  if (dim == 2) return (size_t)(1 + q / m) * pitch + 1 + q % m;
  return ((size_t)(1 + q / (m * m)) * (m + 2) + 1 + (q / m) % m) * pitch + 1 + q % m;
}

__global__ void __launch_bounds__(kThreads) k_coarse_matvec(int dim, int n, int pitch, size_t st,
                                                            const double* __restrict__ Linv,
                                                            const double* __restrict__ x,
                                                            double* __restrict__ y) {
  __shared__ double xs[1024];
  const int m = n - 1, nh = dim == 2 ? m * m : m * m * m;
  Linv += blockIdx.x * (size_t)nh * nh;  // instance blockIdx.x
  x += blockIdx.x * st;
  y += blockIdx.x * st;
  for (int q = threadIdx.x; q < nh; q += kThreads) xs[q] = x[level1_index(dim, m, pitch, q)];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p = warp; p < nh; p += kWarps) {
    const double* row = Linv + (size_t)p * nh;
    double s = 0.0;
    for (int q = lane; q < nh; q += 32) s = fma(row[q], xs[q], s);
    s = warp_sum(s);
    if (lane == 0) y[level1_index(dim, m, pitch, p)] = s;
  }
}

}  // namespace

size_t dense_smem_bytes(int n, int ntri, int nvert, int aug) {
  const int L = nvert + 1, nh = n - aug;
  const size_t nt3 = nvert == 3 ? 10 : 20;
  const size_t maxadj = nvert == 3 ? 6 : 24;
  const size_t loc = loc_in_A(n, ntri, nvert) ? 0 : (size_t)ntri * L * L;
  return sizeof(double) * ((size_t)4 * n * n + loc + 8 * (size_t)n + 4 * kThreads + nh +
                           (aug ? (size_t)ntri * nt3 : 0) + ((size_t)ntri * nvert + 1) / 2 +
                           ((size_t)nh * maxadj + 1) / 2);
}

void dense_scf(const DenseProblem& p, int nb, cudaStream_t s) {
  const int n = p.nh + p.aug;
  k_dense_scf<<<nb, kThreads, dense_smem_bytes(n, p.ntri, p.nvert, p.aug), s>>>(p);
}

// The attribute is per function, shared by every handle in the process, so it is always set
// to the ceiling every caller is validated against (never to one caller's smaller need).
cudaError_t dense_prepare(size_t need) {
  if (need > kDenseSmemLimit) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_dense_scf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kDenseSmemLimit);
  if (e != cudaSuccess) return e;
  // all of the unified L1 as shared memory, so that two small (2D) instances share an SM
  e = cudaFuncSetAttribute(k_dense_scf, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_spd_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kDenseSmemLimit);
}

void dense_spd_inverse(const double* L, double* Linv, int n, int nb, cudaStream_t s) {
  k_spd_inverse<<<nb, kThreads, sizeof(double) * (2 * (size_t)n * n + n), s>>>(L, Linv, n);
}

void coarse_matvec(const Grid& g, const double* Linv, const double* x, double* y,
                   cudaStream_t s) {
  k_coarse_matvec<<<g.nb, kThreads, 0, s>>>(g.dim, g.n, g.pitch, g.stride, Linv, x, y);
}

}  // namespace fmg
