// 2D level kernels: matrix-free P1 stencils on the structured right-triangle mesh.
//
// Mesh (Section 3, regular refinement with beta = 2): squares of side h split by their (1,1)
// diagonal, so node (i,j) couples to E, W, N, S, NE and SW.  With x = i h, y = j h and
// W = w0 + wx x^2 + wy y^2, exact integration of a^(phi_p, phi_q) + (W phi_p, phi_q)
// (Section 2) gives, per node, the stencil
//   C : 4  + h^2 w0/2  + h^4 [wx (9i^2+1)/18          + wy (9j^2+1)/18]
//   E : -1 + h^2 w0/12 + h^4 [wx (10i^2+10i+3)/120    + wy (15j^2+1)/180]
//   N : -1 + h^2 w0/12 + h^4 [wx (15i^2+1)/180        + wy (10j^2+10j+3)/120]
//   NE:      h^2 w0/12 + h^4 [wx (10i^2+10i+3)/120    + wy (10j^2+10j+3)/120]
// with W = E(i-1,j), S = N(i,j-1), SW = NE(i-1,j-1) by symmetry; the mass stencil is
// h^2/12 (6 at C, 1 at the six neighbours).  (Derived once by symbolic integration over the
// six triangles of a node's star.)
//
// FP64 on this part issues at ~1/64 of the FP32 rate, so the kernels trade bandwidth for
// FP64 instructions: the four coupling arrays and omega/D are materialised once per solve
// (40 B/node extra traffic) and every sweep then costs 9 FP64 instructions per node.
#include "fmg_internal.h"
#include "dfloat.cuh"
#include "star2d.cuh"

namespace fmg {
namespace {

__device__ __forceinline__ size_t at(int i, int j, int pitch) { return (size_t)j * pitch + i; }

// The stencil is separable: every coefficient is (constant + part in i) + (part in j).  A 1D
// pass tabulates the eight parts, the 2D pass adds them.  Table layout (n + 1 entries each):
// X_C, X_E, X_N, X_NE (constants folded in) then Y_C, Y_E, Y_N, Y_NE.
__global__ void k_coef1d(int n, double h, const PotentialParams* __restrict__ pp,
                         double* __restrict__ tab) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x > n) return;
  const PotentialParams p = pp[blockIdx.y];
  tab += (size_t)blockIdx.y * 8 * (n + 1);
  const double wl = p.operator_form == FMG_W_LEFT ? 1.0 : 0.0;
  const double h2 = h * h, h4 = h2 * h2;
  const double d = x, m = h2 * p.w0;
  const double sq = (9.0 * d * d + 1.0) / 18.0;            // C
  const double ad = (10.0 * d * d + 10.0 * d + 3.0) / 120.0;  // along the edge direction
  const double ac = (15.0 * d * d + 1.0) / 180.0;           // across the edge direction
  const int s = n + 1;
  tab[0 * s + x] = 4.0 + wl * (m / 2.0 + h4 * p.wx * sq);
  tab[1 * s + x] = -1.0 + wl * (m / 12.0 + h4 * p.wx * ad);
  tab[2 * s + x] = -1.0 + wl * (m / 12.0 + h4 * p.wx * ac);
  tab[3 * s + x] = wl * (m / 12.0 + h4 * p.wx * ad);
  tab[4 * s + x] = wl * h4 * p.wy * sq;
  tab[5 * s + x] = wl * h4 * p.wy * ac;
  tab[6 * s + x] = wl * h4 * p.wy * ad;
  tab[7 * s + x] = wl * h4 * p.wy * ad;
}

// 1 / c by Newton's iteration y <- y (2 - c y) from the hardware's approximate reciprocal
// (rcp.approx.ftz.f64, measured 2^-20 relative error on this part): two steps take it below FP64
// rounding (4 DFMA, no conversions on the FP64 pipe, instead of a full division).
__device__ __forceinline__ double recip(double c) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(c));
  y = fma(y, fma(-c, y, 1.0), y);
  y = fma(y, fma(-c, y, 1.0), y);
  return y;
}

__global__ void k_coef2d(int n, int pitch, size_t st, const double* __restrict__ tab,
                         const PotentialParams* __restrict__ pp, Coef2D c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n || j > n) return;
  const int s = n + 1;
  const int ib = blockIdx.z;
  tab += (size_t)ib * 8 * s;
  pp += ib;
  const size_t k = ib * st + at(i, j, pitch);
  const double cc = tab[i] + tab[4 * s + j];
  c.cC[k] = cc;
  c.cE[k] = tab[s + i] + tab[5 * s + j];
  c.cN[k] = tab[2 * s + i] + tab[6 * s + j];
  c.cNE[k] = tab[3 * s + i] + tab[7 * s + j];
  c.dinv[k] = pp->omega * recip(cc);
}

// (L x)_k: 1 DMUL + 6 DFMA
__device__ __forceinline__ double lop(const Coef2D& c, const double* __restrict__ x, size_t k,
                                      int pitch) {
  double v = c.cC[k] * x[k];
  v = fma(c.cE[k], x[k + 1], v);
  v = fma(c.cE[k - 1], x[k - 1], v);
  v = fma(c.cN[k], x[k + pitch], v);
  v = fma(c.cN[k - pitch], x[k - pitch], v);
  v = fma(c.cNE[k], x[k + pitch + 1], v);
  v = fma(c.cNE[k - pitch - 1], x[k - pitch - 1], v);
  return v;
}

// The defect f - L x at node k as one chain of fused multiply-adds from f: seven FP64
// operations where f - (L x) takes eight (the smoothers are bound by the FP64 pipe)
__device__ __forceinline__ double defect(const Coef2D& c, double f, const double* __restrict__ x,
                                         size_t k, int pitch) {
  double r = fma(-c.cC[k], x[k], f);
  r = fma(-c.cE[k], x[k + 1], r);
  r = fma(-c.cE[k - 1], x[k - 1], r);
  r = fma(-c.cN[k], x[k + pitch], r);
  r = fma(-c.cN[k - pitch], x[k - pitch], r);
  r = fma(-c.cNE[k], x[k + pitch + 1], r);
  r = fma(-c.cNE[k - pitch - 1], x[k - pitch - 1], r);
  return r;
}

// thread (i, j) of instance ib = blockIdx.z; k is its element index in the batched arrays
#define INTERIOR_2D                                             \
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;      \
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;      \
  if (i >= n || j >= n) return;                                 \
  const int ib = blockIdx.z;                                     \
  const size_t k = ib * st + at(i, j, pitch);

__global__ void k_apply2d(int n, int pitch, size_t st, Coef2D c, const double* __restrict__ x,
                          double* __restrict__ y) {
  INTERIOR_2D
  y[k] = lop(c, x, k, pitch);
}

// f -= (Lw - La) u = W u (the potential's mass matrix) for the paper-literal form, whose
// auxiliary operator La = A leaves W u on the right-hand side; Lw = A + W
__global__ void k_sub_wmass2d(int n, int pitch, size_t st, Coef2D cw, Coef2D ca,
                              const double* __restrict__ u, double* __restrict__ f) {
  INTERIOR_2D
  f[k] -= lop(cw, u, k, pitch) - lop(ca, u, k, pitch);
}

__global__ void k_mass2d(int n, int pitch, size_t st, double h2_12, const double* __restrict__ x,
                         double* __restrict__ y) {
  INTERIOR_2D
  const double s = ((x[k + 1] + x[k - 1]) + (x[k + pitch] + x[k - pitch])) +
                   (x[k + pitch + 1] + x[k - pitch - 1]);
  y[k] = h2_12 * fma(6.0, x[k], s);
}

// The same mass apply in double-float arithmetic from the split of x (mixed-precision modes'
// augmented pass): every weight is positive, so the sloppy double-float sums keep ~2^-47 of
// the result; FP64 output.
__global__ void k_mass2d_df(int n, int pitch, size_t st, dfloat h2_12, SplitVec x,
                            double* __restrict__ y) {
  INTERIOR_2D
  auto X = [&](size_t q) { return get<dfloat>(x, q); };
  const dfloat s = ((X(k + 1) + X(k - 1)) + (X(k + pitch) + X(k - pitch))) +
                   (X(k + pitch + 1) + X(k - pitch - 1));
  y[k] = to_double(h2_12 * fma(dfloat(6), X(k), s));
}

__global__ void k_jacobi2d(int n, int pitch, size_t st, Coef2D c, const double* __restrict__ f,
                           const double* __restrict__ x, double* __restrict__ xo) {
  INTERIOR_2D
  xo[k] = fma(c.dinv[k], defect(c, f[k], x, k, pitch), x[k]);
}

// One step of the Chebyshev semi-iteration: d <- alpha d + beta D^{-1} (f - L x), xo = x + d
// (dinv = 1/D for this smoother).  first: d is not read (alpha = 0).  x_zero: x = 0.
__global__ void k_cheb2d(int n, int pitch, size_t st, Coef2D c, const double* __restrict__ f,
                         const double* __restrict__ x, double* __restrict__ d,
                         double* __restrict__ xo, double alpha, double beta, int first,
                         int x_zero) {
  INTERIOR_2D
  const double r = x_zero ? f[k] : defect(c, f[k], x, k, pitch);
  double dn = beta * c.dinv[k] * r;
  if (!first) dn = fma(alpha, d[k], dn);
  d[k] = dn;
  xo[k] = x_zero ? dn : x[k] + dn;
}

__global__ void k_jacobi2d_zero(int n, int pitch, size_t st, Coef2D c, const double* __restrict__ f,
                                double* __restrict__ xo) {
  INTERIOR_2D
  xo[k] = c.dinv[k] * f[k];
}

__global__ void k_residual2d(int n, int pitch, size_t st, Coef2D c, const double* __restrict__ f,
                             const double* __restrict__ x, double* __restrict__ r) {
  INTERIOR_2D
  r[k] = defect(c, f[k], x, k, pitch);
}

// r_c = P^T r_f: a coarse node takes its own fine value plus half of the six fine nodes on
// the coarse edges through it (the (1,1)-diagonal edges included).
// r_c = P^T r_f for coarse nodes (2P, J) and (2P + 1, J) on one thread: fine columns
// 4P - 2 .. 4P + 3 of rows 2J - 1 .. 2J + 1 as three 16-byte loads per row (all inside the
// array: row 2J - 1 >= 1 starts past column 1, and the pitch leaves room past column
// nf + 1), the pair stored as one 16-byte vector when both are interior.
// blockIdx.z = q nb + ib: vector q of vecs, instance ib.
__global__ void k_restrict2d(int nc, int pc, int pf, size_t stc, size_t stf, RestrictVecs vecs,
                             int nb) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (2 * P >= nc || J >= nc) return;
  const int q = blockIdx.z / nb, ib = blockIdx.z - q * nb;
  const double* __restrict__ rf = vecs.rf[q];
  double* __restrict__ rc = vecs.rc[q];
  const double* r0 = rf + ib * stf + at(4 * P - 2, 2 * J - 1, pf);  // column 4P - 2, row 2J - 1
  double v[3][6];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 t = *reinterpret_cast<const double2*>(r0 + (size_t)q * pf + 2 * c);
      v[q][2 * c] = t.x;
      v[q][2 * c + 1] = t.y;
    }
  // coarse node 2P + d: fine centre column 4P + 2d is v[.][2 + 2d]
  double out[2];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const int c = 2 + 2 * d;
    const double sum = ((v[1][c + 1] + v[1][c - 1]) + (v[2][c] + v[0][c])) +
                       (v[2][c + 1] + v[0][c - 1]);
    out[d] = fma(0.5, sum, v[1][c]);
  }
  double* o = rc + ib * stc + at(2 * P, J, pc);  // even: 16-byte aligned
  if (P > 0 && 2 * P + 1 < nc) {
    *reinterpret_cast<double2*>(o) = make_double2(out[0], out[1]);
  } else {
    if (P > 0) o[0] = out[0];
    if (2 * P + 1 < nc) o[1] = out[1];
  }
}

// x_f (+)= P e_c (+ scale * extra): fine node (2I+a, 2J+b) is the midpoint of coarse nodes
// (I,J) and (I+a, J+b), a, b in {0,1}.  One thread per coarse cell (I, J), I, J in
// [0, nc): it reads the cell's four corners once and writes fine columns 2I, 2I + 1 of rows
// 2J and 2J + 1 as 16-byte vectors (column 0 and row 0, on the boundary, are not written).
// scale[ib * scale_stride] is instance ib's factor.
__global__ void k_prolong2d(int nc, int pf, int pc, size_t st, size_t stc,
                            const double* __restrict__ ec, double* __restrict__ xf, int add,
                            const double* __restrict__ extra, const double* __restrict__ scale,
                            int scale_stride) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nc || J >= nc) return;
  const int ib = blockIdx.z;
  const size_t kc = ib * stc + at(I, J, pc);
  const double e00 = ec[kc], e10 = ec[kc + 1], e01 = ec[kc + pc], e11 = ec[kc + pc + 1];
  const double sc = extra ? scale[(size_t)ib * scale_stride] : 0.0;
  const size_t k0 = ib * st + at(2 * I, 2 * J, pf);  // even: the pair is 16-byte aligned
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    if (b == 0 && J == 0) continue;
    const size_t k = k0 + (size_t)b * pf;
    double2 x = make_double2(0.0, 0.0);
    if (add) x = *reinterpret_cast<const double2*>(xf + k);
    // the midpoint value 0.5 (a + b) is added with one FMA (0.5 s is exact, so this rounds
    // exactly as the separate multiply and add would)
    double v0 = b == 0 ? e00 + x.x : fma(0.5, e00 + e01, x.x);
    double v1 = fma(0.5, e00 + (b == 0 ? e10 : e11), x.y);
    if (extra) {
      const double2 t = *reinterpret_cast<const double2*>(extra + k);
      v0 = fma(sc, t.x, v0);
      v1 = fma(sc, t.y, v1);
    }
    if (I > 0) *reinterpret_cast<double2*>(xf + k) = make_double2(v0, v1);
    else xf[k + 1] = v1;
  }
}

// int u^3 phi_p over the six triangles of the star of p, exactly.  With the hexagon of
// neighbours n_0..n_5 = E, NE, N, W, SW, S taken cyclically (each consecutive pair closes one
// triangle with p), summing int_K u^3 lambda_p = |K|/60 sum_{|b|=3} u^b (b_p + 1) gives
//   |K|/60 [24u^3 + 6u^2 S1 + 2u(2 S2 + P) + 2 S3 + Q],
// S_q = sum n_k^q, P = sum n_k n_{k+1}, Q = sum n_k n_{k+1} (n_k + n_{k+1}), |K| = h^2/2.
// Through the pair sums m_k = n_k + n_{k+1} and squares q_k = n_k^2 (2 S1 = M1 = sum m_k,
// 2 (2 S2 + P) = M2 + 2 S2 with M2 = sum m_k^2, 2 S3 + Q = M3 = sum m_k (q_k + q_{k+1})):
//   |K|/60 [u^2 (24u + 3 M1) + u (M2 + 2 S2) + M3].
// This per-node form serves the double-float and single-precision right-hand sides (T =
// dfloat with u read as a SplitVec, or float) and the FP64 kernels of small launches; large
// FP64 launches evaluate the same sums per mesh edge (star2d.cuh), which saves FP64
// instructions but, in double-float arithmetic, loses more to the longer dependency chains
// and lane shuffles than it saves.
// M1 (twice the neighbour sum) is returned through m1_out when given: the mass stencil of
// the right-hand side needs the same sum.
template <typename T, typename U = const double*>
__device__ __forceinline__ T nload_at(const U& u, size_t k, int pitch, T* m1_out = nullptr) {
  const T up = get<T>(u, k);
  const T n0 = get<T>(u, k + 1), n1 = get<T>(u, k + pitch + 1), n2 = get<T>(u, k + pitch);
  const T n3 = get<T>(u, k - 1), n4 = get<T>(u, k - pitch - 1), n5 = get<T>(u, k - pitch);
  const T m0 = n0 + n1, m1 = n1 + n2, m2 = n2 + n3, m3 = n3 + n4, m4 = n4 + n5, m5 = n5 + n0;
  const T q0 = n0 * n0, q1 = n1 * n1, q2 = n2 * n2, q3 = n3 * n3, q4 = n4 * n4, q5 = n5 * n5;
  const T M1 = ((m0 + m1) + (m2 + m3)) + (m4 + m5);
  if (m1_out) *m1_out = M1;
  T M2 = m0 * m0;
  M2 = fma(m1, m1, M2);
  M2 = fma(m2, m2, M2);
  M2 = fma(m3, m3, M2);
  M2 = fma(m4, m4, M2);
  M2 = fma(m5, m5, M2);
  const T S2 = ((q0 + q1) + (q2 + q3)) + (q4 + q5);
  T M3 = m0 * (q0 + q1);
  M3 = fma(m1, q1 + q2, M3);
  M3 = fma(m2, q2 + q3, M3);
  M3 = fma(m3, q3 + q4, M3);
  M3 = fma(m4, q4 + q5, M3);
  M3 = fma(m5, q5 + q0, M3);
  const T u2 = up * up;
  const T v = fma(up, fma(T(2), S2, M2), u2 * fma(T(24), up, T(3) * M1));
  return v + M3;
}

// FP64 node by node, for launches too small to fill the GPU as column walks
__global__ void k_nload2d_node(int n, int pitch, size_t st, double scale,
                               const double* __restrict__ u, double* __restrict__ out) {
  INTERIOR_2D
  out[k] = scale * nload_at<double>(u, k, pitch);
}

__global__ void k_rhs2d_node(int n, int pitch, size_t st, double h2_12, double h2_120,
                             const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
                             const double* __restrict__ u, double* __restrict__ f) {
  INTERIOR_2D
  const double nscale = pp[ib].zeta * h2_120;
  double m1;  // twice the sum of the six neighbours
  const double nl = nload_at<double>(u, k, pitch, &m1);
  const double mu = h2_12 * fma(6.0, u[k], 0.5 * m1);
  f[k] = fma(lam[ib], mu, -nscale * nl);
}

// The FP64 cubic-load kernels below walk columns (star2d.cuh): launch with star2d_grid /
// star2d_block.
__global__ void __launch_bounds__(32 * kStarWarps)
    k_nload2d(int n, int pitch, size_t st, double scale, const double* __restrict__ u,
              double* __restrict__ out) {
  star2d_walk<double>(n, pitch, st, u, [&](size_t k, const Star2D<double>& p) {
    out[k] = scale * star_cubic(p);
  });
}

// f = lambda M u - N(u); the mass stencil h^2/12 (6 u_p + neighbour sum) reuses the cubic
// load's M1 (twice the neighbour sum): h^2/24 (12 u_p + M1)
__global__ void __launch_bounds__(32 * kStarWarps)
    k_rhs2d(int n, int pitch, size_t st, double h2_24, double h2_120,
            const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
            const double* __restrict__ u, double* __restrict__ f) {
  const double nscale = pp[blockIdx.z].zeta * h2_120, l = lam[blockIdx.z];
  star2d_walk<double>(n, pitch, st, u, [&](size_t k, const Star2D<double>& p) {
    const double mu = h2_24 * fma(12.0, p.u, p.M1);
    f[k] = fma(l, mu, -nscale * star_cubic(p));
  });
}

// The same right-hand side in double-float arithmetic from the split u (mixed-precision
// modes): ~2^-47 relative rounding per operation on the FP32 pipes; the FP64 result combines
// the two FP64-converted parts.
// The scales h^2/12 and h^2/120 arrive as double-float constants, so each node spends only
// the two FP64 conversions and the final combination on the FP64 pipe.
__global__ void k_rhs2d_df(int n, int pitch, size_t st, dfloat h2_12, dfloat h2_120,
                           const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
                           SplitVec u, double* __restrict__ f) {
  INTERIOR_2D
  dfloat m1;  // twice the sum of the six neighbours
  const double nl = to_double(h2_120 * nload_at<dfloat>(u, k, pitch, &m1));
  const double mu = to_double(h2_12 * fma(dfloat(6), get<dfloat>(u, k), dfloat(0.5) * m1));
  f[k] = fma(lam[ib], mu, -pp[ib].zeta * nl);
}

// FP32 auxiliary right-hand side of the mixed-precision iteration (same closed forms in
// single precision, FP64 result): the V-cycles that consume it are FP32 as well, and its
// rounding moves u~ by ~1e-7, which reaches lambda only at second order through the
// augmented solve.
__global__ void k_rhs2d_f32(int n, int pitch, size_t st, float h2_12, float h2_120,
                            const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
                            const double* __restrict__ u, double* __restrict__ f) {
  INTERIOR_2D
  const float nscale = (float)pp[ib].zeta * h2_120;
  const float s = (((float)u[k + 1] + (float)u[k - 1]) + ((float)u[k + pitch] + (float)u[k - pitch])) +
                  ((float)u[k + pitch + 1] + (float)u[k - pitch - 1]);
  const float mu = h2_12 * fmaf(6.0f, (float)u[k], s);
  f[k] = f2d_exact(fmaf((float)lam[ib], mu, -nscale * nload_at<float>(u, k, pitch)));
}

__global__ void k_dense_level1_2d(int n, int pitch, size_t st, double h2_12, Coef2D c,
                                  double* L, double* M) {
  const int m = n - 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m * m) return;
  const int i = 1 + p % m, j = 1 + p / m;
  const size_t nn = (size_t)m * m * m * m;
  double* lr = L + blockIdx.y * nn + (size_t)p * m * m;
  double* mr = M + blockIdx.y * nn + (size_t)p * m * m;
  for (int q = 0; q < m * m; ++q) {
    lr[q] = 0.0;
    mr[q] = 0.0;
  }
  const size_t k = blockIdx.y * st + at(i, j, pitch);
  lr[p] = c.cC[k];
  mr[p] = 6.0 * h2_12;
  auto put = [&](int di, int dj, double v) {
    const int ii = i + di, jj = j + dj;
    if (ii < 1 || jj < 1 || ii >= n || jj >= n) return;
    const int q = (ii - 1) + (jj - 1) * m;
    lr[q] = v;
    mr[q] = h2_12;
  };
  put(1, 0, c.cE[k]);
  put(-1, 0, c.cE[k - 1]);
  put(0, 1, c.cN[k]);
  put(0, -1, c.cN[k - pitch]);
  put(1, 1, c.cNE[k]);
  put(-1, -1, c.cNE[k - pitch - 1]);
}

__global__ void k_start2d(int n, double* c, int cstride) {
  const int m = n - 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m * m) return;
  const int i = 1 + p % m, j = 1 + p / m;
  c[(size_t)blockIdx.y * cstride + p] = sinpi((double)i / n) * sinpi((double)j / n);
}

// launch shape over count_x x count_y nodes of every instance of g
dim3 grid_of(const Grid& g, int count_x, int count_y) {
  return dim3((count_x + g.bx - 1) / g.bx, (count_y + g.by - 1) / g.by, g.nb);
}
dim3 block_of(const Grid& g) { return dim3(g.bx, g.by); }

}  // namespace

void coef2d_setup(const Grid& g, const PotentialParams* p, const Coef2D& c, cudaStream_t s) {
  k_coef1d<<<dim3((g.n + 1 + 127) / 128, g.nb), 128, 0, s>>>(g.n, g.h, p, c.tab);
  k_coef2d<<<grid_of(g, g.n + 1, g.n + 1), block_of(g), 0, s>>>(g.n, g.pitch, g.stride, c.tab,
                                                                 p, c);
}

void apply2d(const Grid& g, const Coef2D& c, const double* x, double* y, cudaStream_t s) {
  k_apply2d<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(g.n, g.pitch, g.stride, c, x,
                                                                  y);
}

void sub_wmass2d(const Grid& g, const Coef2D& cw, const Coef2D& ca, const double* u, double* f,
                 cudaStream_t s) {
  k_sub_wmass2d<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(g.n, g.pitch, g.stride, cw,
                                                                     ca, u, f);
}

void mass2d(const Grid& g, const double* x, double* y, cudaStream_t s) {
  k_mass2d<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(g.n, g.pitch, g.stride,
                                                                 g.h * g.h / 12.0, x, y);
}

void mass2d_df(const Grid& g, SplitVec x, double* y, cudaStream_t s) {
  k_mass2d_df<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(
      g.n, g.pitch, g.stride, dfloat(g.h * g.h / 12.0), x, y);
}

void jacobi2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* xo,
              bool x_is_zero, cudaStream_t s) {
  if (x_is_zero)
    k_jacobi2d_zero<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(g.n, g.pitch, g.stride,
                                                                          c, f, xo);
  else
    k_jacobi2d<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(g.n, g.pitch, g.stride, c,
                                                                     f, x, xo);
}

void cheb2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* d,
            double* xo, double alpha, double beta, bool first, bool x_zero, cudaStream_t s) {
  k_cheb2d<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(
      g.n, g.pitch, g.stride, c, f, x, d, xo, alpha, beta, first ? 1 : 0, x_zero ? 1 : 0);
}

void residual2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* r,
                cudaStream_t s) {
  k_residual2d<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(g.n, g.pitch, g.stride, c,
                                                                     f, x, r);
}

void restrict2d(const Grid& fine, const Grid& coarse, const double* rf, double* rc,
                cudaStream_t s, const double* rf2, double* rc2) {
  const RestrictVecs v{{rf, rf2}, {rc, rc2}};
  const int nv = rf2 ? 2 : 1;
  const dim3 block(32, 8);
  const dim3 grid((coarse.n / 2 + 32) / 32, (coarse.n - 1 + 7) / 8, nv * fine.nb);
  k_restrict2d<<<grid, block, 0, s>>>(coarse.n, coarse.pitch, fine.pitch, coarse.stride,
                                      fine.stride, v, fine.nb);
}

void prolong2d(const Grid& fine, const Grid& coarse, const double* ec, double* xf, bool add,
               const double* extra, const double* scale, int scale_stride, cudaStream_t s) {
  const dim3 block(32, 8);
  const dim3 grid((coarse.n + 31) / 32, (coarse.n + 7) / 8, fine.nb);
  k_prolong2d<<<grid, block, 0, s>>>(coarse.n, fine.pitch, coarse.pitch, fine.stride,
                                     coarse.stride, ec, xf, add ? 1 : 0, extra, scale,
                                     scale_stride);
}

void nload2d(const Grid& g, const double* u, double* out, cudaStream_t s) {
  if (!star2d_walks(g)) {
    k_nload2d_node<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(
        g.n, g.pitch, g.stride, g.h * g.h / 120.0, u, out);
    return;
  }
  k_nload2d<<<star2d_grid(g.n, g.nb), star2d_block(), 0, s>>>(g.n, g.pitch, g.stride,
                                                               g.h * g.h / 120.0, u, out);
}

void rhs2d(const Grid& g, const double* lam, const PotentialParams* p, const double* u,
           double* f, cudaStream_t s) {
  if (!star2d_walks(g)) {
    k_rhs2d_node<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(
        g.n, g.pitch, g.stride, g.h * g.h / 12.0, g.h * g.h / 120.0, lam, p, u, f);
    return;
  }
  k_rhs2d<<<star2d_grid(g.n, g.nb), star2d_block(), 0, s>>>(
      g.n, g.pitch, g.stride, g.h * g.h / 24.0, g.h * g.h / 120.0, lam, p, u, f);
}

void rhs2d_f32(const Grid& g, const double* lam, const PotentialParams* p, const double* u,
               double* f, cudaStream_t s) {
  k_rhs2d_f32<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(
      g.n, g.pitch, g.stride, (float)(g.h * g.h / 12.0), (float)(g.h * g.h / 120.0), lam, p, u, f);
}

void rhs2d_df(const Grid& g, const double* lam, const PotentialParams* p, SplitVec u, double* f,
              cudaStream_t s) {
  k_rhs2d_df<<<grid_of(g, g.n - 1, g.n - 1), block_of(g), 0, s>>>(
      g.n, g.pitch, g.stride, dfloat(g.h * g.h / 12.0), dfloat(g.h * g.h / 120.0), lam, p, u, f);
}

void dense_level1_2d(const Grid& g, const Coef2D& c, double* L, double* M, cudaStream_t s) {
  const int m = g.n - 1;
  k_dense_level1_2d<<<dim3((m * m + 63) / 64, g.nb), 64, 0, s>>>(g.n, g.pitch, g.stride,
                                                                 g.h * g.h / 12.0, c, L, M);
}

void start_vector(const Grid& g, double* c, int cstride, cudaStream_t s) {
  const int m = g.n - 1;
  k_start2d<<<dim3((m * m + 63) / 64, g.nb), 64, 0, s>>>(g.n, c, cstride);
}

}  // namespace fmg
