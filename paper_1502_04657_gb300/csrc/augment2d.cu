// Fine-grid pass of the augmented nonlinear problem (Algorithm 3.1 step 2), 2D.
//
// On V_{H,h_k} = V_H + span{u~}, with w = w_H + c_u u~, the nonlinear matrix
// G(c)_ij = int w^2 psi_i psi_j needs four integrals of u~ against coarse hats phi^H:
//   T0    = int u~^4                       = u~ . N(u~),       N(u)_p = int u^3 phi_p
//   T1_a  = int u~^3 phi^H_a               = (P^T ... P^T N(u~))_a   (repeated restriction)
//   T2_ab = int u~^2 phi^H_a phi^H_b       = (P^T ... P^T B(u~) P ... P)_ab,
//           B(u)_pq = int u^2 phi_p phi_q, the FE matrix of a form on V_{h_k}; restricting a
//           form to the nested subspace is exact, level by level (Galerkin coarsening)
//   T3^T_abc = int_T u~ mu_a mu_b mu_c     per coarse triangle T (barycentrics mu of T)
// (the paper re-assembles the augmented matrix with a fine pass per nonlinear iteration,
// Section 3.2; these four quantities make every iteration independent of the fine grid).
//
// T3 is linear in u~: T3^T = sum_v u~_v int_T phi_v q, q = mu_a mu_b mu_c a cubic.  Taylor
// expansion of q about node v is exact, so int_T phi_v q = sum_{i+j<=3} d^{ij}q(v)/(i!j!) m_ij
// with m_ij the moments of phi_v over the fine triangles of v's star that lie in T.  Those
// depend only on v's class (interior of T, one of T's three edges, one of its vertices), so
// T3 follows from monomial sums of u~ per class: 4 FP64 FMAs per interior node.
#include <type_traits>

#include "fmg_internal.h"
#include "reduce_dev.cuh"
#include "dfloat.cuh"
#include "star2d.cuh"

namespace fmg {
namespace {

__device__ __forceinline__ size_t at(int i, int j, int pitch) { return (size_t)j * pitch + i; }

// N(u)_p and the density stencil B(u) at p (coupling to p, E, N, NE).  Star triangles of p
// are the consecutive pairs of its hexagon of neighbours E, NE, N, W, SW, S; on a triangle
// (p, q, r) of area |K|:
//   int u^2 lambda_p^2       = |K|/90  [6u_p^2 + u_q^2 + u_r^2 + 3u_p u_q + 3u_p u_r + u_q u_r]
//   int u^2 lambda_p lambda_q = |K|/180 [3u_p^2 + 3u_q^2 + u_r^2 + 4u_p u_q + 2u_p u_r + 2u_q u_r]
// Summed over the star, and written with the per-edge numbers of the column walk
// (star2d.cuh: s, F = s^2 + a^2 + b^2 of an edge (a, b), M1 and sum F over the opposite
// edges):
//   B_pp = |K|/180 [u_p (72 u_p + 6 M1) + sum F]
//   B_pq = |K|/180 [2 (F_pq + s_pq (s_pq + u_r1 + u_r2)) + u_r1^2 + u_r2^2]
// for the edge p-q shared by the triangles closed by r1 and r2 (E: NE, S; N: NE, W;
// NE: E, N).  s60, s180 = |K| / 60, / 180 (computed on the host: an FP64 division per node
// would cost as much as a quarter of the kernel's arithmetic).
// FP64 mode.
__global__ void __launch_bounds__(32 * kStarWarps)
    k_nload_density2d(int n, int pitch, size_t st, double s60, double s180,
                      const double* __restrict__ u, double* __restrict__ nl,
                      double* __restrict__ bC, double* __restrict__ bE,
                      double* __restrict__ bN, double* __restrict__ bNE) {
  using T = double;
  star2d_walk<T>(n, pitch, st, u, [&](size_t k, const Star2D<T>& p) {
    nl[k] = out_of(s60 * star_cubic(p));
    put_entry(bC, k, s180 * fma(p.u, fma(T(72), p.u, T(6) * p.M1), p.SF));
    put_entry(bE, k, s180 * fma(T(2), fma(p.H.s, p.H.s + (p.uNE + p.uS), p.H.F), p.qNE + p.qS));
    put_entry(bN, k, s180 * fma(T(2), fma(p.V.s, p.V.s + (p.uNE + p.uW), p.V.F), p.qNE + p.qW));
    put_entry(bNE, k, s180 * fma(T(2), fma(p.D.s, p.D.s + (p.uE + p.uN), p.D.F), p.qE + p.qN));
  });
}

// The same quantities node by node: the cubic load through the pair sums
// m_k = n_k + n_{k+1} (nload_at in grid2d.cu) and the density stencil from the two triangle
// formulas above.  T, U: FP64 (double, const double*) for launches too small to fill the GPU
// as column walks, or double-float from the split u (dfloat, SplitVec) in the mixed modes,
// whose entries stay split for the coarsening chain.  s60, s90, s180 = |K| / 60, / 90, / 180.
template <typename T, typename U>
__global__ void k_nload_density2d_node(int n, int pitch, size_t st, T s60, T s90, T s180, U u,
                                       double* __restrict__ nl, double* __restrict__ bC,
                                       double* __restrict__ bE, double* __restrict__ bN,
                                       double* __restrict__ bNE) {
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t k = blockIdx.z * st + at(i, j, pitch);
  const T up = get<T>(u, k);
  const T nE = get<T>(u, k + 1), nNE = get<T>(u, k + pitch + 1), nN = get<T>(u, k + pitch);
  const T nW = get<T>(u, k - 1), nSW = get<T>(u, k - pitch - 1), nS = get<T>(u, k - pitch);
  // the cubic load through the pair sums m_k = n_k + n_{k+1} (see nload_at in grid2d.cu)
  const T m0 = nE + nNE, m1 = nNE + nN, m2 = nN + nW, m3 = nW + nSW, m4 = nSW + nS,
          m5 = nS + nE;
  const T qE = nE * nE, qNE = nNE * nNE, qN = nN * nN, qW = nW * nW, qSW = nSW * nSW,
          qS = nS * nS;
  const T M1 = ((m0 + m1) + (m2 + m3)) + (m4 + m5);  // 2 S1
  T M2 = m0 * m0;
  M2 = fma(m1, m1, M2);
  M2 = fma(m2, m2, M2);
  M2 = fma(m3, m3, M2);
  M2 = fma(m4, m4, M2);
  M2 = fma(m5, m5, M2);
  const T s2 = ((qE + qNE) + (qN + qW)) + (qSW + qS);
  T M3 = m0 * (qE + qNE);
  M3 = fma(m1, qNE + qN, M3);
  M3 = fma(m2, qN + qW, M3);
  M3 = fma(m3, qW + qSW, M3);
  M3 = fma(m4, qSW + qS, M3);
  M3 = fma(m5, qS + qE, M3);
  const T u2 = up * up;
  const T s2p = fma(T(0.5), M2, s2);  // 2 S2 + P
  nl[k] = out_of(s60 * (fma(T(2) * up, s2p, u2 * fma(T(24), up, T(3) * M1)) + M3));
  // density stencil, diagonal: sum over the six triangles
  put_entry(bC, k, s90 * fma(T(36), u2, fma(T(3) * up, M1, s2p)));
  // edge p-q shared by the triangles closed by r1 and r2
  const T u26 = T(6) * u2;
  put_entry(bE, k, s180 * fma(T(6), qE,
                              u26 + fma(T(8) * up, nE, fma(T(2) * (up + nE), nNE + nS, qNE + qS))));
  put_entry(bN, k, s180 * fma(T(6), qN,
                              u26 + fma(T(8) * up, nN, fma(T(2) * (up + nN), nNE + nW, qNE + qW))));
  put_entry(bNE, k, s180 * fma(T(6), qNE,
                               u26 + fma(T(8) * up, nNE, fma(T(2) * (up + nNE), nE + nN, qE + qN))));
}

// Galerkin coarsening of a 7-point stencil: Bc(a,b) = sum_{v,w} P_va P_wb B(v,w).  The
// fine support of coarse hat a is 2a plus the offsets below with weights 1 and 1/2.
__device__ constexpr int kSX[7] = {0, 1, -1, 0, 0, 1, -1};
__device__ constexpr int kSY[7] = {0, 0, 0, 1, -1, 1, -1};

template <typename T>
__device__ __forceinline__ T fine_entry(const double* bC, const double* bE, const double* bN,
                                        const double* bNE, size_t kv, int dx, int dy,
                                        int pitch) {
  if (dx == 0 && dy == 0) return get_entry<T>(bC, kv);
  if (dx == 1 && dy == 0) return get_entry<T>(bE, kv);
  if (dx == -1 && dy == 0) return get_entry<T>(bE, kv - 1);
  if (dx == 0 && dy == 1) return get_entry<T>(bN, kv);
  if (dx == 0 && dy == -1) return get_entry<T>(bN, kv - pitch);
  if (dx == 1 && dy == 1) return get_entry<T>(bNE, kv);
  return get_entry<T>(bNE, kv - pitch - 1);  // dx == dy == -1
}

__host__ __device__ constexpr bool in_stencil(int dx, int dy) {
  return (dx == 0 && dy == 0) || (dx == 1 && dy == 0) || (dx == -1 && dy == 0) ||
         (dx == 0 && dy == 1) || (dx == 0 && dy == -1) || (dx == 1 && dy == 1) ||
         (dx == -1 && dy == -1);
}

// FP64: one FMA per pair.  Double-float: the entries (int u~^2 phi phi) are non-negative, so
// they are summed per weight class (1, 1/2, 1/4) with double-float additions, three
// independent chains, and scaled exactly once at the end.  The diagonal entry (TX = TY = 0)
// pairs both supports with themselves, and (p, q), (q, p) read the same fine entry, so it
// takes each unordered pair once with twice its weight (an exact doubling).
template <typename T, int TX, int TY>
__device__ __forceinline__ T coarse_entry(const double* bC, const double* bE, const double* bN,
                                          const double* bNE, size_t kf, int pf) {
  constexpr bool kDiag = TX == 0 && TY == 0;
  T acc = 0;
  T part[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int p = 0; p < 7; ++p) {
#pragma unroll
    for (int q = kDiag ? p : 0; q < 7; ++q) {
      const int dx = 2 * TX + kSX[q] - kSX[p];
      const int dy = 2 * TY + kSY[q] - kSY[p];
      if (in_stencil(dx, dy)) {
        const size_t kv = kf + (long)kSY[p] * pf + kSX[p];
        const bool twice_w = kDiag && q != p;
        if constexpr (std::is_same<T, dfloat>::value) {
          const dfloat e = fine_entry<T>(bC, bE, bN, bNE, kv, dx, dy, pf);
          part[(p != 0) + (q != 0)] += twice_w ? twice(e) : e;
        } else {
          const T w((twice_w ? 2.0 : 1.0) * (p == 0 ? 1.0 : 0.5) * (q == 0 ? 1.0 : 0.5));
          acc = fma(w, fine_entry<T>(bC, bE, bN, bNE, kv, dx, dy, pf), acc);
        }
      }
    }
  }
  if constexpr (std::is_same<T, dfloat>::value) {
    const dfloat h1(part[1].hi * 0.5f, part[1].lo * 0.5f);
    const dfloat h2(part[2].hi * 0.25f, part[2].lo * 0.25f);
    acc = part[0] + (h1 + h2);
  }
  return acc;
}

// T = double (FP64 mode) or dfloat (mixed modes: entries stored split, see put_entry)
template <typename T>
__global__ void k_coarsen_density2d(int nc, int pc, int pf, size_t stc, size_t stf,
                                    const double* __restrict__ fC,
                                    const double* __restrict__ fE,
                                    const double* __restrict__ fN,
                                    const double* __restrict__ fNE, double* __restrict__ cC,
                                    double* __restrict__ cE, double* __restrict__ cN,
                                    double* __restrict__ cNE) {
  const int I = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nc || J >= nc) return;
  const size_t kf = blockIdx.z * stf + at(2 * I, 2 * J, pf);
  const size_t kc = blockIdx.z * stc + at(I, J, pc);
  put_entry(cC, kc, coarse_entry<T, 0, 0>(fC, fE, fN, fNE, kf, pf));
  // couplings to coarse neighbours outside the interior are never read; skip them so no
  // fine entry beyond the interior is touched
  if (I + 1 < nc) put_entry(cE, kc, coarse_entry<T, 1, 0>(fC, fE, fN, fNE, kf, pf));
  if (J + 1 < nc) put_entry(cN, kc, coarse_entry<T, 0, 1>(fC, fE, fN, fNE, kf, pf));
  if (I + 1 < nc && J + 1 < nc)
    put_entry(cNE, kc, coarse_entry<T, 1, 1>(fC, fE, fN, fNE, kf, pf));
}

// ---- T3 class sums -----------------------------------------------------------------------
// Per coarse triangle, 25 sums in normalised coordinates (sg, tg) = (s, t) / r of the coarse
// cell (s, t the fine offsets from its corner, 0..r):
//   [0..9]   interior: sum u sg^k tg^l, (k,l) in kMono order
//   [10..13] edge A: sum u x^m  (T0: bottom t = 0, x = sg;  T1: left s = 0, x = tg)
//   [14..17] edge B: sum u x^m  (T0: right s = r, x = tg;   T1: top t = r,  x = sg)
//   [18..21] diagonal s = t: sum u sg^m
//   [22..24] vertex values (T0: V00, V10, V11;  T1: V00, V11, V01)
constexpr int kSums = 25;
constexpr int kSumThreads = 256;
constexpr int kSumRows = 1024;

template <int T>
__device__ void t3_sums_body(int pf, int n1, int r, const double* __restrict__ u,
                             const double* __restrict__ pw, double* __restrict__ partials,
                             int col_blocks) {
  // instance blockIdx.z: u and partials arrive offset to it
  __shared__ double sh[kSumThreads];
  const int tri = blockIdx.y;
  const int cell = tri >> 1;
  const int I = cell % n1, J = cell / n1;
  const int cb = blockIdx.x % col_blocks, rb = blockIdx.x / col_blocks;
  const int s = cb * blockDim.x + threadIdx.x;
  const int t0 = rb * kSumRows;
  const int t1 = min(t0 + kSumRows, r + 1);
  double c[4] = {0.0, 0.0, 0.0, 0.0};  // interior: sum_t u tg^l for this column
  double ea = 0.0, eb = 0.0, ed = 0.0;  // per-column edge values (T0: bottom, -, diag)
  double eb_t[4] = {0.0, 0.0, 0.0, 0.0};  // edge varying in t (T0 right / T1 left)
  double vtx[3] = {0.0, 0.0, 0.0};
  if (s <= r) {
    const double* col = u + (size_t)(J * r) * pf + (size_t)(I * r + s);
    // the rows of this column inside the triangle: T0 (lower) t <= s, T1 (upper) t >= s; the
    // rows outside would add nothing.  The lanes of a warp read one row per step (coalesced),
    // so T1 starts at the warp's first column, and its lanes skip the rows above their own.
    const int ta = T == 0 ? t0 : max(t0, s - (int)(threadIdx.x & 31));
    const int tb = T == 0 ? min(t1, s + 1) : t1;
    for (int t = ta; t < tb; ++t) {
      const double val = col[(size_t)t * pf];
      const double* p = pw + 4 * t;  // tg^m, m = 0..3
      if (T == 0) {
        if (t == 0) {
          if (s == 0) vtx[0] = val;
          else if (s == r) vtx[1] = val;
          else ea = val;
        } else if (s == r) {
          if (t == r) vtx[2] = val;
          else {
#pragma unroll
            for (int m = 0; m < 4; ++m) eb_t[m] = fma(val, p[m], eb_t[m]);
          }
        } else if (t == s) {
          ed = val;
        } else if (t < s) {
#pragma unroll
          for (int m = 0; m < 4; ++m) c[m] = fma(val, p[m], c[m]);
        }
      } else {
        if (s == 0) {
          if (t == 0) vtx[0] = val;
          else if (t == r) vtx[2] = val;
          else {
#pragma unroll
            for (int m = 0; m < 4; ++m) eb_t[m] = fma(val, p[m], eb_t[m]);
          }
        } else if (t == r) {
          if (s == r) vtx[1] = val;
          else eb = val;
        } else if (s == t) {
          ed = val;
        } else if (s < t) {
#pragma unroll
          for (int m = 0; m < 4; ++m) c[m] = fma(val, p[m], c[m]);
        }
      }
    }
  }
  double acc[kSums];
  const double* ps = pw + 4 * (s <= r ? s : 0);  // sg^m
  const double ok = s <= r ? 1.0 : 0.0;
  // interior monomials in kMono order: (0,0),(1,0),(0,1),(2,0),(1,1),(0,2),(3,0),(2,1),(1,2),(0,3)
  acc[0] = ok * c[0];
  acc[1] = ok * ps[1] * c[0];
  acc[2] = ok * c[1];
  acc[3] = ok * ps[2] * c[0];
  acc[4] = ok * ps[1] * c[1];
  acc[5] = ok * c[2];
  acc[6] = ok * ps[3] * c[0];
  acc[7] = ok * ps[2] * c[1];
  acc[8] = ok * ps[1] * c[2];
  acc[9] = ok * c[3];
  if (T == 0) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      acc[10 + m] = ok * ps[m] * ea;  // bottom, x = sg
      acc[14 + m] = ok * eb_t[m];     // right, x = tg
      acc[18 + m] = ok * ps[m] * ed;  // diagonal
    }
  } else {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      acc[10 + m] = ok * eb_t[m];     // left, x = tg
      acc[14 + m] = ok * ps[m] * eb;  // top, x = sg
      acc[18 + m] = ok * ps[m] * ed;
    }
  }
  acc[22] = ok * vtx[0];
  acc[23] = ok * vtx[1];
  acc[24] = ok * vtx[2];
  block_sum_to<kSums>(acc, sh, partials + ((size_t)tri * gridDim.x + blockIdx.x) * kSums);
}

__global__ void __launch_bounds__(kSumThreads)
    k_t3_sums2d(int pf, int n1, int r, size_t st, size_t pst, const double* __restrict__ u,
                const double* __restrict__ pw, double* __restrict__ partials, int col_blocks) {
  u += blockIdx.z * st;
  partials += blockIdx.z * pst;
  if (blockIdx.y & 1)
    t3_sums_body<1>(pf, n1, r, u, pw, partials, col_blocks);
  else
    t3_sums_body<0>(pf, n1, r, u, pw, partials, col_blocks);
}

// Finalise: T3^T_e = h^2 sum_m map[T][e][m] S_m, a fixed linear map of the 25 class sums per
// triangle type, built on the host for the level's r (t3_map2d).
__global__ void k_t3_finalize2d(int chunks, double h2, size_t pst, size_t tst,
                                const double* __restrict__ partials,
                                const double* __restrict__ map, double* __restrict__ t3) {
  partials += blockIdx.y * pst;
  t3 += blockIdx.y * tst;
  const int tri = blockIdx.x;
  const int T = tri & 1;
  __shared__ double sums[kSums];
  for (int m = threadIdx.x; m < kSums; m += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partials[((size_t)tri * chunks + c) * kSums + m];
    sums[m] = s;
  }
  __syncthreads();
  const int e = threadIdx.x;
  if (e >= 10) return;
  const double* row = map + ((size_t)T * 10 + e) * kSums;
  double acc = 0.0;
  for (int m = 0; m < kSums; ++m) acc = fma(row[m], sums[m], acc);
  t3[(size_t)tri * 10 + e] = h2 * acc;
}

__global__ void k_gather_level1_2d(int n, int pitch, size_t st, const double* __restrict__ gA_pad,
                                   const double* __restrict__ gM_pad,
                                   const double* __restrict__ t1_pad, Density2D b, int split,
                                   double* __restrict__ gA, double* __restrict__ gM,
                                   double* __restrict__ t1, double* __restrict__ B1) {
  const int m = n - 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m * m) return;
  const int i = 1 + p % m, j = 1 + p / m;
  const size_t nh = (size_t)m * m;
  const size_t k = blockIdx.y * st + at(i, j, pitch);
  const size_t q = blockIdx.y * nh + p;
  gA[q] = gA_pad[k];
  gM[q] = gM_pad[k];
  t1[q] = t1_pad[k];
  double* row = B1 + blockIdx.y * nh * nh + (size_t)p * nh;
  for (int q = 0; q < m * m; ++q) row[q] = 0.0;
  const bool sp = split != 0;  // entries stored as double-float splits (mixed modes)
  row[p] = entry_fp64(b.C, k, sp);
  auto put = [&](int di, int dj, const double* a, size_t ka) {
    const int ii = i + di, jj = j + dj;
    if (ii < 1 || jj < 1 || ii >= n || jj >= n) return;
    row[(ii - 1) + (jj - 1) * m] = entry_fp64(a, ka, sp);
  };
  put(1, 0, b.E, k);
  put(-1, 0, b.E, k - 1);
  put(0, 1, b.N, k);
  put(0, -1, b.N, k - pitch);
  put(1, 1, b.NE, k);
  put(-1, -1, b.NE, k - pitch - 1);
}

// a block takes blockDim.x columns (whole warps, up to kSumThreads) of kSumRows rows
int t3_threads2d(int r) { return warps_for(r + 1, kSumThreads); }
int t3_col_blocks(int r) { return (r + 1 + t3_threads2d(r) - 1) / t3_threads2d(r); }
int t3_row_blocks(int r) { return (r + 1 + kSumRows - 1) / kSumRows; }

dim3 grid_of(const Grid& g, int cx, int cy) {
  return dim3((cx + g.bx - 1) / g.bx, (cy + g.by - 1) / g.by, g.nb);
}

}  // namespace

void nload_density2d(const Grid& g, const double* u, double* nl, const Density2D& b,
                     cudaStream_t s) {
  if (!star2d_walks(g)) {
    k_nload_density2d_node<double, const double*>
        <<<grid_of(g, g.n - 1, g.n - 1), dim3(g.bx, g.by), 0, s>>>(
            g.n, g.pitch, g.stride, g.h * g.h / 120.0, g.h * g.h / 180.0, g.h * g.h / 360.0, u,
            nl, b.C, b.E, b.N, b.NE);
    return;
  }
  k_nload_density2d<<<star2d_grid(g.n, g.nb), star2d_block(), 0, s>>>(
      g.n, g.pitch, g.stride, g.h * g.h / 120.0, g.h * g.h / 360.0, u, nl, b.C, b.E, b.N, b.NE);
}

void nload_density2d_df(const Grid& g, SplitVec u, double* nl, const Density2D& b,
                        cudaStream_t s) {
  k_nload_density2d_node<dfloat, SplitVec><<<grid_of(g, g.n - 1, g.n - 1), dim3(g.bx, g.by), 0, s>>>(
      g.n, g.pitch, g.stride, dfloat(g.h * g.h / 120.0), dfloat(g.h * g.h / 180.0),
      dfloat(g.h * g.h / 360.0), u, nl, b.C, b.E, b.N, b.NE);
}

void coarsen_density2d(const Grid& fine, const Grid& coarse, const Density2D& bf,
                       const Density2D& bc, cudaStream_t s, bool split) {
  const dim3 grid = grid_of(fine, coarse.n - 1, coarse.n - 1), block(fine.bx, fine.by);
  if (split)
    k_coarsen_density2d<dfloat><<<grid, block, 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, bf.C, bf.E, bf.N,
        bf.NE, bc.C, bc.E, bc.N, bc.NE);
  else
    k_coarsen_density2d<double><<<grid, block, 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, bf.C, bf.E, bf.N,
        bf.NE, bc.C, bc.E, bc.N, bc.NE);
}

void gather_level1_2d(const Grid& g1, const double* gA_pad, const double* gM_pad,
                      const double* t1_pad, const Density2D& b1, double* gA, double* gM,
                      double* t1, double* B1, cudaStream_t s, bool split) {
  const int m = g1.n - 1;
  k_gather_level1_2d<<<dim3((m * m + 63) / 64, g1.nb), 64, 0, s>>>(
      g1.n, g1.pitch, g1.stride, gA_pad, gM_pad, t1_pad, b1, split ? 1 : 0, gA, gM, t1, B1);
}

size_t t3_partials2d(const Grid& fine, int n1) {
  const int r = fine.n / n1;
  return (size_t)2 * n1 * n1 * t3_col_blocks(r) * t3_row_blocks(r) * kSums;
}

void t3_moments2d(const Grid& fine, int n1, const double* u, const double* pw,
                  const double* map, double* partials, double* t3, cudaStream_t s) {
  const int r = fine.n / n1;
  const int cb = t3_col_blocks(r), rb = t3_row_blocks(r);
  const size_t pst = t3_partials2d(fine, n1);
  k_t3_sums2d<<<dim3(cb * rb, 2 * n1 * n1, fine.nb), t3_threads2d(r), 0, s>>>(
      fine.pitch, n1, r, fine.stride, pst, u, pw, partials, cb);
  k_t3_finalize2d<<<dim3(2 * n1 * n1, fine.nb), 32, 0, s>>>(
      cb * rb, fine.h * fine.h, pst, (size_t)2 * n1 * n1 * 10, partials, map, t3);
}

// Host: moments m_ij = int_K lambda_v (ds)^i (dt)^j over each star triangle of a node (fine
// units, h = 1), summed per class of each coarse-triangle type.  Exact, from the barycentric
// monomial rule int_K lambda^alpha = 2|K| alpha! / (|alpha| + 2)! with |K| = 1/2.
void t3_class_moments2d(double out[2 * 7 * 10]) {
  // star triangles as neighbour pairs of the hexagon E, NE, N, W, SW, S
  const int nb[6][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 0}, {-1, -1}, {0, -1}};
  auto fact = [](int k) {
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
  };
  auto binom = [&](int n, int k) { return fact(n) / (fact(k) * fact(n - k)); };
  double star[6][10];
  const int mk[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0}, ml[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
  for (int t = 0; t < 6; ++t) {
    const int* q = nb[t];
    const int* rr = nb[(t + 1) % 6];
    for (int m = 0; m < 10; ++m) {
      const int i = mk[m], j = ml[m];
      // lambda_v (q_s lq + r_s lr)^i (q_t lq + r_t lr)^j, expanded
      double acc = 0.0;
      for (int a = 0; a <= i; ++a)
        for (int b = 0; b <= j; ++b) {
          const double coef = binom(i, a) * binom(j, b) * pow((double)q[0], a) *
                              pow((double)rr[0], i - a) * pow((double)q[1], b) *
                              pow((double)rr[1], j - b);
          if (coef == 0.0) continue;
          const int eq = a + b, er = (i - a) + (j - b);  // exponents of lambda_q, lambda_r
          acc += coef * 2.0 * 0.5 * fact(1) * fact(eq) * fact(er) / fact(1 + eq + er + 2);
        }
      star[t][m] = acc;
    }
  }
  // classes: 0 interior, 1 edge A, 2 edge B, 3 diagonal, 4..6 vertices (see t3_sums_body);
  // star triangle t = pair (nb[t], nb[t+1]): 0 (E,NE) 1 (NE,N) 2 (N,W) 3 (W,SW) 4 (SW,S) 5 (S,E)
  const int sets[2][7][6] = {
      {{0, 1, 2, 3, 4, 5}, {0, 1, 2, -1}, {2, 3, 4, -1}, {4, 5, 0, -1}, {0, -1}, {2, -1}, {4, -1}},
      {{0, 1, 2, 3, 4, 5}, {5, 0, 1, -1}, {3, 4, 5, -1}, {1, 2, 3, -1}, {1, -1}, {3, -1}, {5, -1}}};
  for (int T = 0; T < 2; ++T)
    for (int c = 0; c < 7; ++c)
      for (int m = 0; m < 10; ++m) {
        double s = 0.0;
        for (int e = 0; e < 6 && sets[T][c][e] >= 0; ++e) s += star[sets[T][c][e]][m];
        if (c == 0) {
          s = 0.0;
          for (int e = 0; e < 6; ++e) s += star[e][m];
        }
        out[(T * 7 + c) * 10 + m] = s;
      }
}

// Host: table of (x / r)^m, m = 0..3, x = 0..r (exact: r is a power of two times n1-free)
void t3_power_table(int r, double* out) {
  for (int x = 0; x <= r; ++x) {
    const double v = (double)x / r;
    out[4 * x + 0] = 1.0;
    out[4 * x + 1] = v;
    out[4 * x + 2] = v * v;
    out[4 * x + 3] = v * v * v;
  }
}

// Host: the linear map from the 25 class sums to T3 (without the h^2 factor) for one level:
//   T3_abc = sum_class sum_{i+j<=3} m^class_ij r^-(i+j) / (i! j!)
//            sum_{k+l<=3} c^abc_kl (k)_i (l)_j S^class_{k-i, l-j},
// with q_abc(sg, tg) = mu_a mu_b mu_c = sum c_kl sg^k tg^l and (k)_i the falling factorial;
// S^class_{a,b} = sum over the class of u sg^a tg^b, one of the 25 sums or zero.
void t3_map2d(int r, double out[2 * 10 * 25]) {
  double mom[2 * 7 * 10];
  t3_class_moments2d(mom);
  const int mk[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0}, ml[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
  const double fall[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 2, 0}, {1, 3, 6, 6}};
  const double fact[4] = {1, 1, 2, 6};
  // index of S^class_{a,b} among the 25 sums (-1: identically zero); see t3_sums_body
  auto sum_index = [](int T, int cls, int a, int b) -> int {
    switch (cls) {
      case 0: { const int d = a + b; return d * (d + 1) / 2 + b; }
      case 1: return T == 0 ? (b == 0 ? 10 + a : -1) : (a == 0 ? 10 + b : -1);
      case 2: return T == 0 ? 14 + b : 14 + a;
      case 3: return 18 + a + b;
      case 4: return (a == 0 && b == 0) ? 22 : -1;
      case 5: return T == 0 ? (b == 0 ? 23 : -1) : 23;
      default: return T == 0 ? 24 : (a == 0 ? 24 : -1);
    }
  };
  for (int i = 0; i < 2 * 10 * 25; ++i) out[i] = 0.0;
  for (int T = 0; T < 2; ++T) {
    double mu[3][3];
    if (T == 0) {
      const double v[3][3] = {{1, -1, 0}, {0, 1, -1}, {0, 0, 1}};
      for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) mu[x][y] = v[x][y];
    } else {
      const double v[3][3] = {{1, 0, -1}, {0, 1, 0}, {0, -1, 1}};
      for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) mu[x][y] = v[x][y];
    }
    int e = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b)
        for (int c = b; c < 3; ++c, ++e) {
          double cq[4][4] = {};
          cq[0][0] = 1.0;
          const int f3[3] = {a, b, c};
          for (int f = 0; f < 3; ++f) {
            double nq[4][4] = {};
            const double* m = mu[f3[f]];
            for (int k = 0; k < 4; ++k)
              for (int l = 0; l + k < 4; ++l) {
                if (cq[k][l] == 0.0) continue;
                nq[k][l] += cq[k][l] * m[0];
                if (k + l + 1 < 4) {
                  nq[k + 1][l] += cq[k][l] * m[1];
                  nq[k][l + 1] += cq[k][l] * m[2];
                }
              }
            for (int k = 0; k < 4; ++k) for (int l = 0; l < 4; ++l) cq[k][l] = nq[k][l];
          }
          double* row = out + ((size_t)T * 10 + e) * 25;
          for (int cls = 0; cls < 7; ++cls)
            for (int q = 0; q < 10; ++q) {
              const int i = mk[q], j = ml[q];
              const double mij = mom[(T * 7 + cls) * 10 + q];
              if (mij == 0.0) continue;
              const double w = mij * pow((double)r, -(i + j)) / (fact[i] * fact[j]);
              for (int k = i; k < 4; ++k)
                for (int l = j; l + k < 4; ++l) {
                  if (cq[k][l] == 0.0) continue;
                  const int si = sum_index(T, cls, k - i, l - j);
                  if (si >= 0) row[si] += w * cq[k][l] * fall[k][i] * fall[l][j];
                }
            }
        }
  }
}

}  // namespace fmg
