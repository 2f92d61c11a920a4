// 3D level kernels: matrix-free P1 stencils on the structured Kuhn-tetrahedron mesh.
//
// Mesh (Section 3, regular refinement with beta = 2): cubes of side h split into the 6 Kuhn
// tetrahedra {v, v+e_s1, v+e_s1+e_s2, v+(1,1,1)}, s a permutation of the axes; the same
// pattern reappears under regular refinement.  Node p couples to the 14 neighbours p +- d,
// d in {X, Y, Z, XY, XZ, YZ, XYZ} (the nonzero 0/1 vectors), and lies in 24 tetrahedra.
// Exact integration over those (derived once by symbolic integration), with x = i h etc.:
//   C  :  6h + w0 h^3 2/5  + h^5 sum_axes w_a (42 a^2 + 5)/105
//   X  : -h  + w0 h^3 /20  + h^5 [wx (63i^2+63i+19)/1260 + wy (63j^2+5)/1260 + wz (63l^2+5)/1260]
//   XY :       w0 h^3 /30  + h^5 [wx (84i^2+84i+25)/2520 + wy (84j^2+84j+25)/2520 + wz (21l^2+1)/630]
//   XYZ:       w0 h^3 /20  + h^5 [wx (63i^2+63i+19)/1260 + wy (..j..) + wz (..l..)]
// (Y, Z, XZ, YZ by permuting the axes; the coupling to p - d is the one of p - d to p).  The
// mass stencil is h^3 (2/5 at C, 1/20 along axes and the body diagonal, 1/30 along face
// diagonals).  As in 2D, the 8 coupling arrays and omega/D are materialised once per solve.
#include <type_traits>

#include "fmg_internal.h"
#include "dfloat.cuh"
#include "star3d.cuh"

namespace fmg {
namespace {

// neighbour k = 2 d + (0: +d, 1: -d), d = X, Y, Z, XY, XZ, YZ, XYZ
__device__ constexpr int kDir[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                                       {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
// The 24 tetrahedra of a node's star as triples of neighbour indices (from the Kuhn split of
// the 8 cells around the node).
__device__ constexpr int kStar[24][3] = {
    {0, 6, 12},  {0, 8, 12},  {2, 6, 12},  {2, 10, 12}, {4, 8, 12},  {4, 10, 12},
    {5, 0, 6},   {5, 2, 6},   {3, 0, 8},   {3, 4, 8},   {11, 5, 0},  {11, 3, 0},
    {1, 2, 10},  {1, 4, 10},  {9, 5, 2},   {9, 1, 2},   {7, 3, 4},   {7, 1, 4},
    {13, 11, 5}, {13, 11, 3}, {13, 9, 5},  {13, 9, 1},  {13, 7, 3},  {13, 7, 1}};

__device__ __forceinline__ long dir_off(int d, int pitch, long plane) {
  return kDir[d][0] + (long)kDir[d][1] * pitch + (long)kDir[d][2] * plane;
}

// blockIdx.z = ib * (n - 1) + (l - 1): plane l of instance ib; k is the element index of node
// (i, j, l) of instance ib in the batched arrays
#define INTERIOR_3D                                                       \
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;                \
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;                \
  const int ib = blockIdx.z / (n - 1);                                     \
  const int l = 1 + (int)blockIdx.z - ib * (n - 1);                        \
  if (i >= n || j >= n) return;                                           \
  const long plane = (long)(n + 1) * pitch;                               \
  const size_t k = ib * st + (size_t)l * plane + (size_t)j * pitch + i;

// tables (n + 1 entries each), per axis a in {x, y, z}, weighted by w_a h^5:
//   0: C part (42 a^2 + 5)/105, 1: along an axis or the body diagonal (63a^2+63a+19)/1260,
//   2: across an axis direction (63a^2+5)/1260, 3: along a face diagonal (84a^2+84a+25)/2520,
//   4: across a face diagonal (21a^2+1)/630.
__global__ void k_coef1d_3d(int n, double h, const PotentialParams* __restrict__ pp,
                            double* __restrict__ tab) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x > n) return;
  const PotentialParams p = pp[blockIdx.y];
  tab += (size_t)blockIdx.y * 15 * (n + 1);
  const double wl = p.operator_form == FMG_W_LEFT ? 1.0 : 0.0;
  const double h2 = h * h, h5 = h2 * h2 * h;
  const double a = x;
  const double poly[5] = {(42.0 * a * a + 5.0) / 105.0, (63.0 * a * a + 63.0 * a + 19.0) / 1260.0,
                          (63.0 * a * a + 5.0) / 1260.0, (84.0 * a * a + 84.0 * a + 25.0) / 2520.0,
                          (21.0 * a * a + 1.0) / 630.0};
  const double w[3] = {p.wx, p.wy, p.wz};
  const int s = n + 1;
  for (int ax = 0; ax < 3; ++ax)
    for (int q = 0; q < 5; ++q) tab[(ax * 5 + q) * s + x] = wl * h5 * w[ax] * poly[q];
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

// The stencil coefficients of a 3D level, one warp per grid row (j, l) of an instance with its
// lanes over i.  Every coupling is a constant plus one table entry per axis; the constant and
// the y and z entries are summed once per row, so a node adds its x entries (8 additions)
// and forms omega / C: about 15 FP64 operations per node instead of 46 when every node
// formed its constants and sums itself.  Couplings: C (tables 0, 0, 0), the axis
// directions d (table 1 along d, 2 across), the face diagonals opposite axis e (table 3 on
// the two axes of the face, 4 on e) and the body diagonal (table 1 on every axis).
__global__ void k_coef3d(int n, int pitch, size_t st, double h, const double* __restrict__ tab,
                         const PotentialParams* __restrict__ pp, Coef3D c) {
  const int lane = threadIdx.x & 31;
  const int s = n + 1;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // j + (n + 1) l
  if (row >= s * s) return;
  const int j = row % s, l = row / s;
  const int ib = blockIdx.y;
  const PotentialParams p = pp[ib];
  const double* T = tab + (size_t)ib * 15 * s;
  const double wl = p.operator_form == FMG_W_LEFT ? 1.0 : 0.0;
  const double w3 = wl * (h * h * h) * p.w0;
  // table index on the x, y and z axis of each coupling, and its constant
  constexpr int kQ[8][3] = {{0, 0, 0}, {1, 2, 2}, {2, 1, 2}, {2, 2, 1},
                            {3, 3, 4}, {3, 4, 3}, {4, 3, 3}, {1, 1, 1}};
  const double axis = -h + w3 * (1.0 / 20.0), face = w3 * (1.0 / 30.0);
  const double K[8] = {6.0 * h + w3 * 0.4, axis, axis, axis, face, face, face, w3 * (1.0 / 20.0)};
  double R[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    R[q] = (K[q] + T[(5 + kQ[q][1]) * s + j]) + T[(10 + kQ[q][2]) * s + l];
  const size_t base = ib * st + ((size_t)l * s + j) * pitch;
  for (int i = lane; i <= n; i += 32) {
    const size_t k = base + i;
    double cc = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double v = R[q] + T[kQ[q][0] * s + i];
      c.a[q][k] = v;
      if (q == 0) cc = v;
    }
    c.dinv[k] = p.omega * recip(cc);
  }
}

__device__ __forceinline__ double lop3(const Coef3D& c, const double* __restrict__ x, size_t k,
                                       int pitch, long plane) {
  double v = c.a[0][k] * x[k];
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    v = fma(c.a[1 + d][k], x[k + o], v);
    v = fma(c.a[1 + d][k - o], x[k - o], v);
  }
  return v;
}

// f - L x at node k as one chain of fused multiply-adds from f (15 FP64 operations, not 16)
__device__ __forceinline__ double defect3(const Coef3D& c, double f, const double* __restrict__ x,
                                          size_t k, int pitch, long plane) {
  double r = fma(-c.a[0][k], x[k], f);
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    r = fma(-c.a[1 + d][k], x[k + o], r);
    r = fma(-c.a[1 + d][k - o], x[k - o], r);
  }
  return r;
}

__global__ void k_apply3d(int n, int pitch, size_t st, Coef3D c, const double* __restrict__ x,
                          double* __restrict__ y) {
  INTERIOR_3D
  y[k] = lop3(c, x, k, pitch, plane);
}

// f -= (Lw - La) u = W u for the paper-literal form (La = A, Lw = A + W)
__global__ void k_sub_wmass3d(int n, int pitch, size_t st, Coef3D cw, Coef3D ca,
                              const double* __restrict__ u, double* __restrict__ f) {
  INTERIOR_3D
  f[k] -= lop3(cw, u, k, pitch, plane) - lop3(ca, u, k, pitch, plane);
}

__global__ void k_jacobi3d(int n, int pitch, size_t st, Coef3D c, const double* __restrict__ f,
                           const double* __restrict__ x, double* __restrict__ xo) {
  INTERIOR_3D
  xo[k] = fma(c.dinv[k], defect3(c, f[k], x, k, pitch, plane), x[k]);
}

// One step of the Chebyshev semi-iteration (see grid2d.cu)
__global__ void k_cheb3d(int n, int pitch, size_t st, Coef3D c, const double* __restrict__ f,
                         const double* __restrict__ x, double* __restrict__ d,
                         double* __restrict__ xo, double alpha, double beta, int first,
                         int x_zero) {
  INTERIOR_3D
  const double r = x_zero ? f[k] : defect3(c, f[k], x, k, pitch, plane);
  double dn = beta * c.dinv[k] * r;
  if (!first) dn = fma(alpha, d[k], dn);
  d[k] = dn;
  xo[k] = x_zero ? dn : x[k] + dn;
}

__global__ void k_jacobi3d_zero(int n, int pitch, size_t st, Coef3D c, const double* __restrict__ f,
                                double* __restrict__ xo) {
  INTERIOR_3D
  xo[k] = c.dinv[k] * f[k];
}

__global__ void k_residual3d(int n, int pitch, size_t st, Coef3D c, const double* __restrict__ f,
                             const double* __restrict__ x, double* __restrict__ r) {
  INTERIOR_3D
  r[k] = defect3(c, f[k], x, k, pitch, plane);
}

template <typename T = double, typename U = const double*>
__device__ __forceinline__ T mass_at(const U& x, size_t k, int pitch, long plane) {
  T ax = 0, fd = 0;
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    const T s = get<T>(x, k + o) + get<T>(x, k - o);
    if (d >= 3 && d < 6) fd += s;
    else ax += s;
  }
  return fma(T(0.4), get<T>(x, k), fma(T(1.0 / 20.0), ax, fd * T(1.0 / 30.0)));
}

__global__ void k_mass3d(int n, int pitch, size_t st, double h3, const double* __restrict__ x,
                         double* __restrict__ y) {
  INTERIOR_3D
  y[k] = h3 * mass_at(x, k, pitch, plane);
}

// The same in double-float arithmetic from the split of x (mixed-precision modes' augmented
// pass; positive weights, so ~2^-47 of the result); FP64 output.
__global__ void k_mass3d_df(int n, int pitch, size_t st, dfloat h3, SplitVec x,
                            double* __restrict__ y) {
  INTERIOR_3D
  y[k] = to_double(h3 * mass_at<dfloat>(x, k, pitch, plane));
}

// r_c = P^T r_f: own fine value plus half of the 14 fine neighbours along the mesh edges.
// r_c = P^T r_f for coarse nodes (2P, J, L) and (2P + 1, J, L) on one thread: each of the
// seven fine rows the pair touches (rows 2J + dy of planes 2L + dz) is read as 16-byte pairs
// of columns 4P - 2 .. 4P + 3 (inside the array: those rows start past column 1 and have
// room past column nf + 1 or continue in the next row); the pair is stored as one vector
// when both are interior.  Per node the sums run in direction order as a node-by-node
// evaluation would: s = sum_d (r(c + o_d) + r(c - o_d)), r_c = 0.5 s + r(c).
// blockIdx.z = (q nb + ib) (nc - 1) + L - 1: vector q of vecs, instance ib, coarse plane L.
__global__ void k_restrict3d(int nc, int pc, int pf, size_t stc, size_t stf, RestrictVecs vecs,
                             int nb) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int qb = blockIdx.z / (nc - 1);
  const int L = 1 + (int)blockIdx.z - qb * (nc - 1);
  const int q = qb / nb, ib = qb - q * nb;
  const double* __restrict__ rf = vecs.rf[q];
  double* __restrict__ rc = vecs.rc[q];
  if (2 * P >= nc || J >= nc) return;
  const long planef = (long)(2 * nc + 1) * pf;
  const double* base = rf + ib * stf + (size_t)(2 * L) * planef + (size_t)(2 * J) * pf + 4 * P;
  // v[r][c]: fine row (dy, dz) = kRow[r] at column 4P - 2 + c
  constexpr int kRow[7][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}, {-1, 0}, {0, -1}, {-1, -1}};
  double v[7][6];
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const double* row = base + (long)kRow[r][0] * pf + (long)kRow[r][1] * planef - 2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 t = *reinterpret_cast<const double2*>(row + 2 * c);
      v[r][2 * c] = t.x;
      v[r][2 * c + 1] = t.y;
    }
  }
  // row index of (dy, dz) and -(dy, dz) for the seven directions
  constexpr int kPlus[7] = {0, 1, 2, 1, 2, 3, 3};
  constexpr int kMinus[7] = {0, 4, 5, 4, 5, 6, 6};
  constexpr int kDx[7] = {1, 0, 0, 1, 1, 0, 1};
  double out[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int c = 2 + 2 * q;  // fine centre column 4P + 2q
    double sum = 0.0;
#pragma unroll
    for (int d = 0; d < 7; ++d) sum += v[kPlus[d]][c + kDx[d]] + v[kMinus[d]][c - kDx[d]];
    out[q] = fma(0.5, sum, v[0][c]);
  }
  double* o = rc + ib * stc + ((size_t)L * (nc + 1) + J) * pc + 2 * P;  // even: aligned
  if (P > 0 && 2 * P + 1 < nc) {
    *reinterpret_cast<double2*>(o) = make_double2(out[0], out[1]);
  } else {
    if (P > 0) o[0] = out[0];
    if (2 * P + 1 < nc) o[1] = out[1];
  }
}

// x_f (+)= P e_c (+ scale * extra): fine node 2I + a (a in {0,1}^3) is the midpoint of coarse
// nodes I and I + a, which are joined by a mesh edge.  One thread per coarse cell (I, J, L),
// I, J, L in [0, nc): the cell's eight corners read once, fine columns 2I, 2I + 1 of its four
// fine rows written as 16-byte vectors (column, row and plane 0 are not written).
// scale[ib * scale_stride] is instance ib's factor.
__global__ void k_prolong3d(int nc, int pf, int pc, size_t st, size_t stc,
                            const double* __restrict__ ec, double* __restrict__ xf, int add,
                            const double* __restrict__ extra, const double* __restrict__ scale,
                            int scale_stride) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int ib = blockIdx.z / nc;
  const int L = (int)blockIdx.z - ib * nc;
  if (I >= nc || J >= nc) return;
  const long planec = (long)(nc + 1) * pc;
  const long planef = (long)(2 * nc + 1) * pf;
  const size_t kc = ib * stc + (size_t)L * planec + (size_t)J * pc + I;
  double e[2][2][2];  // e[al][aj][ai] = e_c(I + ai, J + aj, L + al)
#pragma unroll
  for (int al = 0; al < 2; ++al)
#pragma unroll
    for (int aj = 0; aj < 2; ++aj)
#pragma unroll
      for (int ai = 0; ai < 2; ++ai) e[al][aj][ai] = ec[kc + ai + (size_t)aj * pc + al * planec];
  const double sc = extra ? scale[(size_t)ib * scale_stride] : 0.0;
#pragma unroll
  for (int al = 0; al < 2; ++al)
#pragma unroll
    for (int aj = 0; aj < 2; ++aj) {
      if ((al == 0 && L == 0) || (aj == 0 && J == 0)) continue;
      const size_t k = ib * st + (size_t)(2 * L + al) * planef + (size_t)(2 * J + aj) * pf + 2 * I;
      double2 x = make_double2(0.0, 0.0);
      if (add) x = *reinterpret_cast<const double2*>(xf + k);
      // the midpoint value 0.5 (a + b) is added with one FMA (0.5 s is exact, so this rounds
      // exactly as the separate multiply and add would)
      const double a = e[0][0][0];
      double v0 = (aj | al) ? fma(0.5, a + e[al][aj][0], x.x) : a + x.x;
      double v1 = fma(0.5, a + e[al][aj][1], x.y);
      if (extra) {
        const double2 t = *reinterpret_cast<const double2*>(extra + k);
        v0 = fma(sc, t.x, v0);
        v1 = fma(sc, t.y, v1);
      }
      if (I > 0) *reinterpret_cast<double2*>(xf + k) = make_double2(v0, v1);
      else xf[k + 1] = v1;
    }
}

// Star sums over the 24 tetrahedra of p (vertex values u_p, u_q, u_r, u_s; |K| = h^3/6):
//   int u^3 lambda_p        = |K|/140 [h3 + u_p (h2 + u_p (s + u_p))]
//   int u^2 lambda_p^2      = |K|/210 [3 u_p^2 + 2 u_p s + h2]
//   int u^2 lambda_p lambda_q = |K|/420 [u_p^2 + u_q^2 + u_p u_q + h2 + (u_p + u_q) s]
// with s, h2, h3 the complete homogeneous symmetric sums of degree 1, 2, 3 of the four
// values.  Writing h_k = sum_{i<=k} u_p^(k-i) h'_i with h'_i those of the three other vertices,
// the sums over the star become sums over its link - the triangulated sphere of the 14
// neighbours whose 24 triangles are the tetrahedra's faces opposite p:
//   sum_T [h3 + u_p h2 + u_p^2 s + u_p^3] = 96 u_p^3 + 3 u_p^2 H1 + 2 u_p H2 + H3,
//   sum_T [3 u_p^2 + 2 u_p s + h2]        = 144 u_p^2 + 3 u_p H1 + H2,
// H1 = sum_n deg_n u_n,  H2 = sum_n deg_n u_n^2 + 2 sum_edges u_m u_n,
// H3 = sum_n deg_n u_n^3 + 2 sum_edges u_m u_n (u_m + u_n) + sum_triangles u_a u_b u_c,
// (deg_n = link triangles at n; every link edge lies in two triangles), and for the edge to a
// neighbour q, whose tetrahedra close with the link edges (r, t) opposite q (U = u_p + u_q):
//   sum [..] = deg_q (U^2 + 2 (u_p^2 + u_p u_q + u_q^2)) + 2 U sum (u_r + u_t)
//              + sum (u_r^2 + u_r u_t + u_t^2).
// This evaluates each link edge and triangle once instead of each tetrahedron's sums.
struct Link {
  int deg[14];
  int edge[36][2];
  int pair[7][6][2];  // link edges opposite the + neighbour 2 d (deg of them)
  int npair[7];
};

constexpr int kStarHost[24][3] = {
    {0, 6, 12},  {0, 8, 12},  {2, 6, 12},  {2, 10, 12}, {4, 8, 12},  {4, 10, 12},
    {5, 0, 6},   {5, 2, 6},   {3, 0, 8},   {3, 4, 8},   {11, 5, 0},  {11, 3, 0},
    {1, 2, 10},  {1, 4, 10},  {9, 5, 2},   {9, 1, 2},   {7, 3, 4},   {7, 1, 4},
    {13, 11, 5}, {13, 11, 3}, {13, 9, 5},  {13, 9, 1},  {13, 7, 3},  {13, 7, 1}};

constexpr Link make_link() {
  Link L{};
  int ne = 0;
  for (int t = 0; t < 24; ++t)
    for (int i = 0; i < 3; ++i) {
      L.deg[kStarHost[t][i]]++;
      for (int j = i + 1; j < 3; ++j) {
        const int a = kStarHost[t][i] < kStarHost[t][j] ? kStarHost[t][i] : kStarHost[t][j];
        const int b = kStarHost[t][i] < kStarHost[t][j] ? kStarHost[t][j] : kStarHost[t][i];
        bool seen = false;
        for (int e = 0; e < ne; ++e) seen = seen || (L.edge[e][0] == a && L.edge[e][1] == b);
        if (!seen) {
          L.edge[ne][0] = a;
          L.edge[ne][1] = b;
          ++ne;
        }
      }
    }
  for (int d = 0; d < 7; ++d)
    for (int t = 0; t < 24; ++t) {
      const int* v = kStarHost[t];
      const int q = 2 * d;
      if (v[0] != q && v[1] != q && v[2] != q) continue;
      int o[2] = {0, 0}, m = 0;
      for (int i = 0; i < 3; ++i)
        if (v[i] != q) o[m++] = v[i];
      L.pair[d][L.npair[d]][0] = o[0];
      L.pair[d][L.npair[d]][1] = o[1];
      L.npair[d]++;
    }
  return L;
}

__device__ constexpr Link kLink = make_link();
static_assert(make_link().npair[0] == 6 && make_link().npair[3] == 4 && make_link().deg[13] == 6,
              "Kuhn star link");

// T is the arithmetic type: double in FP64 mode, double-float (u read as a SplitVec) in the
// mixed-precision modes, float in the FP32 auxiliary right-hand side (k_rhs3d_f32).
template <typename T, bool DENSITY, typename U = const double*>
__device__ __forceinline__ void star3(const U& u, size_t k, int pitch, long plane, T& nl, T* b) {
  T nv[14], sq[14];
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    nv[2 * d] = get<T>(u, k + o);
    nv[2 * d + 1] = get<T>(u, k - o);
  }
  const T up = get<T>(u, k);
  const T u2 = up * up;
  // degree-weighted sums (deg 6 or 4)
  T s6 = 0, s4 = 0, q6 = 0, q4 = 0, c6 = 0, c4 = 0;
#pragma unroll
  for (int n = 0; n < 14; ++n) {
    sq[n] = nv[n] * nv[n];
    if (kLink.deg[n] == 6) {
      s6 += nv[n];
      q6 += sq[n];
      c6 = fma(sq[n], nv[n], c6);
    } else {
      s4 += nv[n];
      q4 += sq[n];
      c4 = fma(sq[n], nv[n], c4);
    }
  }
  T E = 0, EE = 0, Tr = 0;
#pragma unroll
  for (int e = 0; e < 36; ++e) {
    const T m = nv[kLink.edge[e][0]], n = nv[kLink.edge[e][1]];
    const T p = m * n;
    E += p;
    EE = fma(p, m + n, EE);
  }
#pragma unroll
  for (int t = 0; t < 24; ++t)
    Tr = fma(nv[kStar[t][0]] * nv[kStar[t][1]], nv[kStar[t][2]], Tr);
  const T H1 = fma(T(6), s6, T(4) * s4);
  const T H2 = fma(T(6), q6, fma(T(4), q4, T(2) * E));
  const T H3 = fma(T(6), c6, fma(T(4), c4, fma(T(2), EE, Tr)));
  nl = fma(u2, fma(T(96), up, T(3) * H1), fma(T(2) * up, H2, H3));
  if (DENSITY) {
    b[0] = fma(up, fma(T(144), up, T(3) * H1), H2);
#pragma unroll
    for (int d = 0; d < 7; ++d) {
      const T uq = nv[2 * d];
      T sv = 0, sh = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j < kLink.npair[d]) {
          const int r = kLink.pair[d][j][0], t = kLink.pair[d][j][1];
          sv += nv[r] + nv[t];
          sh += fma(nv[r], nv[t], sq[r] + sq[t]);
        }
      }
      const T upq = up + uq;
      const T h2pq = fma(up, uq, u2 + sq[2 * d]);
      b[1 + d] = fma((T)kLink.npair[d], fma(upq, upq, T(2) * h2pq), fma(T(2) * upq, sv, sh));
    }
  }
}

// FP64 node by node through the link sums of star3, for launches too small to fill the GPU
// as plane walks
__global__ void k_nload3d_node(int n, int pitch, size_t st, double scale,
                               const double* __restrict__ u, double* __restrict__ out) {
  INTERIOR_3D
  double nl;
  star3<double, false>(u, k, pitch, plane, nl, nullptr);
  out[k] = scale * nl;
}

__global__ void k_rhs3d_node(int n, int pitch, size_t st, double h3, double nscale,
                             const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
                             const double* __restrict__ u, double* __restrict__ f) {
  INTERIOR_3D
  double nl;
  star3<double, false>(u, k, pitch, plane, nl, nullptr);
  const double mu = h3 * mass_at(u, k, pitch, plane);
  f[k] = fma(lam[ib], mu, -(pp[ib].zeta * nscale) * nl);
}

// Three blocks per SM (74 KB of shared memory each, registers capped at 80) for the walks
// that fit without spills; the FP64 density walk keeps two (at three it spills and measured
// slower: 7.98 against 7.93 ms on the finest 3D level, where the right-hand side went from
// 5.28 to 5.19 ms and the double-float walks from 2.28 / 1.46 to 2.22 / 1.26 ms).
// FP64 kernels from the plane walk (star3d.cuh): 6 x the star sum of
// h3 + u_p h2 + u_p^2 h1 + u_p^3 is S3 + 3 u_p S2 + 6 u_p^2 S1 + 144 u_p^3 in its sums of
// h1, 2 h2, 6 h3; launch with star3_grid / star3_block and kS3Smem bytes.
template <typename T>
__device__ __forceinline__ T star3_cubic6(const Star3T<T>& p) {
  return fma(p.u, fma(p.u, fma(T(144), p.u, T(6) * p.S1), T(3) * p.S2), p.S3);
}

__global__ void __launch_bounds__(kS3X * kS3Y, 3)
    k_nload3d(int n, int pitch, size_t st, double scale6, const double* __restrict__ u,
              double* __restrict__ out) {
  star3_walk<false>(n, pitch, st, u, [&](size_t k, const Star3& p) {
    out[k] = scale6 * star3_cubic6(p);
  });
}

// f = lambda M u - zeta N(u); the mass stencil is h^3/120 (24 u_p + S1)
__global__ void __launch_bounds__(kS3X * kS3Y, 3)
    k_rhs3d(int n, int pitch, size_t st, double h3_120, double nscale6,
            const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
            const double* __restrict__ u, double* __restrict__ f) {
  const int ib = blockIdx.z / star3_zchunks(n);
  const double l = lam[ib], zn = pp[ib].zeta * nscale6;
  star3_walk<false>(n, pitch, st, u, [&](size_t k, const Star3& p) {
    f[k] = fma(l, h3_120 * fma(24.0, p.u, p.S1), -zn * star3_cubic6(p));
  });
}

// N(u~) and the density stencil, FP64: s140_6, s210_2, s420_2 = |K|/140/6, |K|/210/2,
// |K|/420/2 against the sums of h1, 2 h2, 6 h3 (an edge lies in 6 tetrahedra along an axis
// or the body diagonal, 4 along a face diagonal)
__global__ void __launch_bounds__(kS3X * kS3Y, 2)
    k_nload_density3d(int n, int pitch, size_t st, double s140_6, double s210_2,
                      double s420_2, const double* __restrict__ u, double* __restrict__ nl,
                      Density3D b) {
  star3_walk<true>(n, pitch, st, u, [&](size_t k, const Star3& p) {
    nl[k] = s140_6 * star3_cubic6(p);
    b.a[0][k] = s210_2 * fma(p.u, fma(144.0, p.u, 4.0 * p.S1), p.S2);
    const double u2 = twice(p.u);
#pragma unroll
    for (int d = 0; d < 7; ++d) {
      const double t = fma(p.u, p.un[d], p.q + p.qn[d]);  // u_p^2 + u_q^2 + u_p u_q
      const double two_ne = (d >= 3 && d < 6) ? 8.0 : 12.0;
      // 2 (u_p + u_q) in one operation: (u_p + u_q) 2 E1 rounds the same
      b.a[1 + d][k] = s420_2 * fma(two_ne, t, fma(fma(2.0, p.un[d], u2), p.E1[d], p.E2[d]));
    }
  });
}

// The same two walks in double-float arithmetic from the split u (mixed-precision modes): the
// density stencil is stored split (put_entry) for the coarsening chain, N(u~) and the
// right-hand side are combined in FP64.  Forming each tetrahedron's symmetric sums once
// needs about half the double-float operations of the node-by-node form (k_*_node below).
__global__ void __launch_bounds__(kS3X * kS3Y, 3)
    k_nload_density3d_df(int n, int pitch, size_t st, dfloat s140_6, dfloat s210_2,
                         dfloat s420_2, SplitVec u, double* __restrict__ nl, Density3D b) {
  star3_walk<true, dfloat>(n, pitch, st, u, [&](size_t k, const Star3T<dfloat>& p) {
    nl[k] = out_of(s140_6 * star3_cubic6(p));
    put_entry(b.a[0], k, s210_2 * fma(p.u, fma(dfloat(144), p.u, dfloat(4) * p.S1), p.S2));
    const dfloat u2 = twice(p.u);
#pragma unroll
    for (int d = 0; d < 7; ++d) {
      const dfloat t = fma(p.u, p.un[d], p.q + p.qn[d]);  // u_p^2 + u_q^2 + u_p u_q
      const dfloat two_ne((d >= 3 && d < 6) ? 8 : 12);
      put_entry(b.a[1 + d], k,
                s420_2 * fma(two_ne, t, fma(fma(dfloat(2), p.un[d], u2), p.E1[d], p.E2[d])));
    }
  });
}

__global__ void __launch_bounds__(kS3X * kS3Y, 3)
    k_rhs3d_dfw(int n, int pitch, size_t st, dfloat h3_120, dfloat nscale6,
                const double* __restrict__ lam, const PotentialParams* __restrict__ pp, SplitVec u,
                double* __restrict__ f) {
  const int ib = blockIdx.z / star3_zchunks(n);
  const double l = lam[ib], zeta = pp[ib].zeta;
  star3_walk<false, dfloat>(n, pitch, st, u, [&](size_t k, const Star3T<dfloat>& p) {
    const double mu = to_double(h3_120 * fma(dfloat(24), p.u, p.S1));
    f[k] = fma(l, mu, -zeta * to_double(nscale6 * star3_cubic6(p)));
  });
}

// s140, s210, s420 = |K| / 140, / 210, / 420 (host-side: no FP64 division per node)
// FP32 auxiliary right-hand side of the mixed-precision iteration (same closed forms in
// single precision, FP64 result): the V-cycles that consume it are FP32 as well, and its
// rounding moves u~ by ~1e-7, which reaches lambda only at second order through the
// augmented solve.
__global__ void k_rhs3d_f32(int n, int pitch, size_t st, float h3, float nscale,
                            const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
                            const double* __restrict__ u, double* __restrict__ f) {
  INTERIOR_3D
  float nl;
  star3<float, false>(u, k, pitch, plane, nl, nullptr);
  const float mu = h3 * mass_at<float>(u, k, pitch, plane);
  f[k] = f2d_exact(fmaf((float)lam[ib], mu, -((float)pp[ib].zeta * nscale) * nl));
}

// The same right-hand side in double-float arithmetic from the split u (mixed-precision
// modes), combined in FP64.
__global__ void k_rhs3d_df(int n, int pitch, size_t st, dfloat h3, dfloat nscale,
                           const double* __restrict__ lam, const PotentialParams* __restrict__ pp,
                           SplitVec u, double* __restrict__ f) {
  INTERIOR_3D
  dfloat nl;
  star3<dfloat, false>(u, k, pitch, plane, nl, nullptr);
  const double mu = to_double(h3 * mass_at<dfloat>(u, k, pitch, plane));
  f[k] = fma(lam[ib], mu, -pp[ib].zeta * to_double(nscale * nl));
}

// The same node by node through the link sums of star3: T, U = FP64 (double, const double*)
// for launches too small to fill the GPU as plane walks, or double-float from the split u
// (dfloat, SplitVec) in the mixed modes, whose scales come in T so that the only FP64 work is
// the output conversion.  MINB: resident blocks of 256 threads asked of the register
// allocator (the double-float star needs 255 registers otherwise, which leaves 8 warps per SM).
template <typename T, typename U, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_nload_density3d_node(int n, int pitch, size_t st, T s140, T s210, T s420, U u,
                           double* __restrict__ nl, Density3D b) {
  INTERIOR_3D
  T v, e[8];
  star3<T, true>(u, k, pitch, plane, v, e);
  nl[k] = out_of(s140 * v);
  // the density stencil: FP64, or kept split (double-float) for the coarsening
  put_entry(b.a[0], k, s210 * e[0]);
#pragma unroll
  for (int d = 0; d < 7; ++d) put_entry(b.a[1 + d], k, s420 * e[1 + d]);
}

// Galerkin coarsening of the 15-point density stencil: Bc(a, b) = sum P_va P_wb B(v, w) over
// the 15-node fine supports of the coarse hats (weights 1 at 2a, 1/2 at 2a +- d).
__device__ __forceinline__ int nb_of(int dx, int dy, int dz) {
  // index of the neighbour (dx,dy,dz) in {0: self, 1 + 2d: +d, 2 + 2d: -d}, -1 if not one
  if (dx == 0 && dy == 0 && dz == 0) return 0;
  for (int d = 0; d < 7; ++d) {
    if (dx == kDir[d][0] && dy == kDir[d][1] && dz == kDir[d][2]) return 1 + 2 * d;
    if (dx == -kDir[d][0] && dy == -kDir[d][1] && dz == -kDir[d][2]) return 2 + 2 * d;
  }
  return -1;
}

template <typename V>
__device__ __forceinline__ V fine_entry3(const Density3D& f, size_t kv, int code, int pitch,
                                         long plane) {
  if (code == 0) return get_entry<V>(f.a[0], kv);
  const int d = (code - 1) >> 1;
  if (((code - 1) & 1) == 0) return get_entry<V>(f.a[1 + d], kv);
  return get_entry<V>(f.a[1 + d], kv - dir_off(d, pitch, plane));
}

template <typename V, int T>
__device__ __forceinline__ V coarse_entry3(const Density3D& f, size_t kf, int pf, long planef) {
  // target offset in coarse units: T = 0 self, 1 + d for +d
  const int tx = T == 0 ? 0 : kDir[T - 1][0], ty = T == 0 ? 0 : kDir[T - 1][1],
            tz = T == 0 ? 0 : kDir[T - 1][2];
  // FP64: one FMA per pair.  Double-float: the entries (int u~^2 phi phi) are non-negative, so
  // they are summed per weight class (1, 1/2, 1/4) with double-float additions, three
  // independent chains, and scaled exactly once at the end.  The diagonal entry (T = 0) pairs
  // the support with itself, and (p, q), (q, p) read the same fine entry, so it takes each
  // unordered pair once with twice its weight (an exact doubling).
  constexpr bool kDiag = T == 0;
  V acc = 0;
  V part[3] = {V(0), V(0), V(0)};
#pragma unroll
  for (int p = 0; p < 15; ++p) {
    const int px = p == 0 ? 0 : ((p - 1) & 1 ? -kDir[(p - 1) >> 1][0] : kDir[(p - 1) >> 1][0]);
    const int py = p == 0 ? 0 : ((p - 1) & 1 ? -kDir[(p - 1) >> 1][1] : kDir[(p - 1) >> 1][1]);
    const int pz = p == 0 ? 0 : ((p - 1) & 1 ? -kDir[(p - 1) >> 1][2] : kDir[(p - 1) >> 1][2]);
#pragma unroll
    for (int q = kDiag ? p : 0; q < 15; ++q) {
      const int qx = q == 0 ? 0 : ((q - 1) & 1 ? -kDir[(q - 1) >> 1][0] : kDir[(q - 1) >> 1][0]);
      const int qy = q == 0 ? 0 : ((q - 1) & 1 ? -kDir[(q - 1) >> 1][1] : kDir[(q - 1) >> 1][1]);
      const int qz = q == 0 ? 0 : ((q - 1) & 1 ? -kDir[(q - 1) >> 1][2] : kDir[(q - 1) >> 1][2]);
      const int code = nb_of(2 * tx + qx - px, 2 * ty + qy - py, 2 * tz + qz - pz);
      if (code >= 0) {
        const size_t kv = kf + px + (long)py * pf + (long)pz * planef;
        const bool twice_w = kDiag && q != p;
        if constexpr (std::is_same<V, dfloat>::value) {
          const dfloat e = fine_entry3<V>(f, kv, code, pf, planef);
          part[(p != 0) + (q != 0)] += twice_w ? twice(e) : e;
        } else {
          const V w((twice_w ? 2.0 : 1.0) * (p == 0 ? 1.0 : 0.5) * (q == 0 ? 1.0 : 0.5));
          acc = fma(w, fine_entry3<V>(f, kv, code, pf, planef), acc);
        }
      }
    }
  }
  if constexpr (std::is_same<V, dfloat>::value) {
    const dfloat h1(part[1].hi * 0.5f, part[1].lo * 0.5f);
    const dfloat h2(part[2].hi * 0.25f, part[2].lo * 0.25f);
    acc = part[0] + (h1 + h2);
  }
  return acc;
}

// V = double (FP64 mode) or dfloat (mixed modes: entries stored split, see put_entry)
template <typename V>
__global__ void k_coarsen_density3d(int nc, int pc, int pf, size_t stc, size_t stf,
                                    Density3D f, Density3D c) {
  const int I = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int ib = blockIdx.z / (nc - 1);
  const int L = 1 + (int)blockIdx.z - ib * (nc - 1);
  if (I >= nc || J >= nc) return;
  const long planef = (long)(2 * nc + 1) * pf;
  const size_t kf = ib * stf + (size_t)(2 * L) * planef + (size_t)(2 * J) * pf + 2 * I;
  const size_t kc = ib * stc + ((size_t)L * (nc + 1) + J) * pc + I;
  put_entry(c.a[0], kc, coarse_entry3<V, 0>(f, kf, pf, planef));
  // couplings to coarse neighbours outside the interior are never read: skip them
  if (I + 1 < nc) put_entry(c.a[1], kc, coarse_entry3<V, 1>(f, kf, pf, planef));
  if (J + 1 < nc) put_entry(c.a[2], kc, coarse_entry3<V, 2>(f, kf, pf, planef));
  if (L + 1 < nc) put_entry(c.a[3], kc, coarse_entry3<V, 3>(f, kf, pf, planef));
  if (I + 1 < nc && J + 1 < nc) put_entry(c.a[4], kc, coarse_entry3<V, 4>(f, kf, pf, planef));
  if (I + 1 < nc && L + 1 < nc) put_entry(c.a[5], kc, coarse_entry3<V, 5>(f, kf, pf, planef));
  if (J + 1 < nc && L + 1 < nc) put_entry(c.a[6], kc, coarse_entry3<V, 6>(f, kf, pf, planef));
  if (I + 1 < nc && J + 1 < nc && L + 1 < nc)
    put_entry(c.a[7], kc, coarse_entry3<V, 7>(f, kf, pf, planef));
}

// dense level-1 matrices from a 15-point stencil given per node as (C, +d couplings)
// split: the stencil entries are stored as double-float splits (density, mixed modes)
__global__ void k_dense15(int n, int pitch, size_t vst, Stencil15 st, int use_stencil,
                          double* out, double mass_h3, int split = 0) {
  const double* const* a = use_stencil ? st.a : nullptr;
  const int m = n - 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m * m * m) return;
  const int i = 1 + p % m, j = 1 + (p / m) % m, l = 1 + p / (m * m);
  const long plane = (long)(n + 1) * pitch;
  const size_t base = blockIdx.y * vst;
  const size_t k = base + (size_t)l * plane + (size_t)j * pitch + i;
  const size_t nh = (size_t)m * m * m;
  double* row = out + blockIdx.y * nh * nh + (size_t)p * nh;
  for (int q = 0; q < m * m * m; ++q) row[q] = 0.0;
  const bool sp = split != 0;
  row[p] = a ? entry_fp64(a[0], k, sp) : 0.4 * mass_h3;
  for (int d = 0; d < 7; ++d)
    for (int sg = -1; sg <= 1; sg += 2) {
      const int ii = i + sg * kDir[d][0], jj = j + sg * kDir[d][1], ll = l + sg * kDir[d][2];
      if (ii < 1 || jj < 1 || ll < 1 || ii >= n || jj >= n || ll >= n) continue;
      const size_t kn = base + (size_t)ll * plane + (size_t)jj * pitch + ii;
      double v;
      if (a) v = entry_fp64(a[1 + d], sg > 0 ? k : kn, sp);
      else v = mass_h3 * ((d >= 3 && d < 6) ? 1.0 / 30.0 : 1.0 / 20.0);
      row[(ii - 1) + (size_t)(jj - 1) * m + (size_t)(ll - 1) * m * m] = v;
    }
}

__global__ void k_start3d(int n, double* c, int cstride) {
  const int m = n - 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m * m * m) return;
  const int i = 1 + p % m, j = 1 + (p / m) % m, l = 1 + p / (m * m);
  c[(size_t)blockIdx.y * cstride + p] = sinpi((double)i / n) * sinpi((double)j / n) * sinpi((double)l / n);
}

__global__ void k_gather_vec3d(int n, int pitch, size_t st, const double* __restrict__ a,
                               const double* __restrict__ b, const double* __restrict__ c,
                               double* __restrict__ oa, double* __restrict__ ob,
                               double* __restrict__ oc) {
  const int m = n - 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m * m * m) return;
  const int i = 1 + p % m, j = 1 + (p / m) % m, l = 1 + p / (m * m);
  const size_t k = blockIdx.y * st + ((size_t)l * (n + 1) + j) * pitch + i;
  const size_t q = blockIdx.y * (size_t)m * m * m + p;
  oa[q] = a[k];
  ob[q] = b[k];
  oc[q] = c[k];
}

// launch shape over cx x cy x cz nodes of every instance of g (planes and instances share z)
dim3 grid3(const Grid& g, int cx, int cy, int cz) {
  return dim3((cx + g.bx - 1) / g.bx, (cy + g.by - 1) / g.by, cz * g.nb);
}
dim3 block3(const Grid& g) { return dim3(g.bx, g.by); }

}  // namespace

void coef3d_setup(const Grid& g, const PotentialParams* p, const Coef3D& c, cudaStream_t s) {
  k_coef1d_3d<<<dim3((g.n + 1 + 127) / 128, g.nb), 128, 0, s>>>(g.n, g.h, p, c.tab);
  const int rows = (g.n + 1) * (g.n + 1);
  k_coef3d<<<dim3((rows + 7) / 8, g.nb), 256, 0, s>>>(g.n, g.pitch, g.stride, g.h, c.tab, p, c);
}

#define INTERIOR_LAUNCH(g) grid3(g, g.n - 1, g.n - 1, g.n - 1), block3(g), 0, s

void apply3d(const Grid& g, const Coef3D& c, const double* x, double* y, cudaStream_t s) {
  k_apply3d<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, c, x, y);
}

void sub_wmass3d(const Grid& g, const Coef3D& cw, const Coef3D& ca, const double* u, double* f,
                 cudaStream_t s) {
  k_sub_wmass3d<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, cw, ca, u, f);
}

void mass3d(const Grid& g, const double* x, double* y, cudaStream_t s) {
  k_mass3d<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, g.h * g.h * g.h, x, y);
}

void mass3d_df(const Grid& g, SplitVec x, double* y, cudaStream_t s) {
  k_mass3d_df<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, dfloat(g.h * g.h * g.h), x, y);
}

void jacobi3d(const Grid& g, const Coef3D& c, const double* f, const double* x, double* xo,
              bool x_is_zero, cudaStream_t s) {
  if (x_is_zero) k_jacobi3d_zero<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, c, f, xo);
  else k_jacobi3d<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, c, f, x, xo);
}

void cheb3d(const Grid& g, const Coef3D& c, const double* f, const double* x, double* d,
            double* xo, double alpha, double beta, bool first, bool x_zero, cudaStream_t s) {
  k_cheb3d<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, c, f, x, d, xo, alpha, beta,
                                   first ? 1 : 0, x_zero ? 1 : 0);
}

void residual3d(const Grid& g, const Coef3D& c, const double* f, const double* x, double* r,
                cudaStream_t s) {
  k_residual3d<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, c, f, x, r);
}

void restrict3d(const Grid& fine, const Grid& coarse, const double* rf, double* rc,
                cudaStream_t s, const double* rf2, double* rc2) {
  if (rf2 && (long)(coarse.n - 1) * 2 * fine.nb > 65535) {  // grid z limit: one at a time
    restrict3d(fine, coarse, rf, rc, s);
    restrict3d(fine, coarse, rf2, rc2, s);
    return;
  }
  const RestrictVecs v{{rf, rf2}, {rc, rc2}};
  const int nv = rf2 ? 2 : 1;
  const dim3 grid((coarse.n / 2 + 32) / 32, (coarse.n - 1 + 7) / 8,
                  (coarse.n - 1) * nv * fine.nb);
  k_restrict3d<<<grid, dim3(32, 8), 0, s>>>(coarse.n, coarse.pitch, fine.pitch, coarse.stride,
                                            fine.stride, v, fine.nb);
}

void prolong3d(const Grid& fine, const Grid& coarse, const double* ec, double* xf, bool add,
               const double* extra, const double* scale, int scale_stride, cudaStream_t s) {
  const dim3 grid((coarse.n + 31) / 32, (coarse.n + 7) / 8, coarse.n * fine.nb);
  k_prolong3d<<<grid, dim3(32, 8), 0, s>>>(coarse.n, fine.pitch, coarse.pitch, fine.stride,
                                           coarse.stride, ec, xf, add ? 1 : 0, extra, scale,
                                           scale_stride);
}

// the plane-walk kernels take more than the default 48 KB of dynamic shared memory
template <typename K>
static cudaError_t star3_prepare(K* kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kS3Smem);
}

void nload3d(const Grid& g, const double* u, double* out, cudaStream_t s) {
  const double vol = g.h * g.h * g.h / 6.0;
  if (!star3_walks(g)) {
    k_nload3d_node<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, vol / 140.0, u, out);
    return;
  }
  static const cudaError_t attr = star3_prepare(k_nload3d);
  (void)attr;
  k_nload3d<<<star3_grid(g.n, g.nb), star3_block(), kS3Smem, s>>>(g.n, g.pitch, g.stride,
                                                                  vol / 140.0 / 6.0, u, out);
}

void rhs3d(const Grid& g, const double* lam, const PotentialParams* p, const double* u,
           double* f, cudaStream_t s) {
  const double h3 = g.h * g.h * g.h;
  if (!star3_walks(g)) {
    k_rhs3d_node<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, h3, h3 / 6.0 / 140.0, lam, p,
                                         u, f);
    return;
  }
  static const cudaError_t attr = star3_prepare(k_rhs3d);
  (void)attr;
  k_rhs3d<<<star3_grid(g.n, g.nb), star3_block(), kS3Smem, s>>>(
      g.n, g.pitch, g.stride, h3 / 120.0, h3 / 6.0 / 140.0 / 6.0, lam, p, u, f);
}

void rhs3d_f32(const Grid& g, const double* lam, const PotentialParams* p, const double* u,
               double* f, cudaStream_t s) {
  const double h3 = g.h * g.h * g.h;
  k_rhs3d_f32<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, (float)h3,
                                      (float)(h3 / 6.0 / 140.0), lam, p, u, f);
}

void nload_density3d(const Grid& g, const double* u, double* nl, const Density3D& b,
                     cudaStream_t s) {
  const double vol = g.h * g.h * g.h / 6.0;
  if (!star3_walks(g)) {
    k_nload_density3d_node<double, const double*, 1><<<INTERIOR_LAUNCH(g)>>>(
        g.n, g.pitch, g.stride, vol / 140.0, vol / 210.0, vol / 420.0, u, nl, b);
    return;
  }
  static const cudaError_t attr = star3_prepare(k_nload_density3d);
  (void)attr;
  k_nload_density3d<<<star3_grid(g.n, g.nb), star3_block(), kS3Smem, s>>>(
      g.n, g.pitch, g.stride, vol / 140.0 / 6.0, vol / 210.0 / 2.0, vol / 420.0 / 2.0, u, nl, b);
}

void nload_density3d_df(const Grid& g, SplitVec u, double* nl, const Density3D& b,
                        cudaStream_t s) {
  const double vol = g.h * g.h * g.h / 6.0;
  if (star3_walks(g)) {
    static const cudaError_t attr = star3_prepare(k_nload_density3d_df);
    (void)attr;
    k_nload_density3d_df<<<star3_grid(g.n, g.nb), star3_block(), kS3Smem, s>>>(
        g.n, g.pitch, g.stride, dfloat(vol / 140.0 / 6.0), dfloat(vol / 210.0 / 2.0),
        dfloat(vol / 420.0 / 2.0), u, nl, b);
    return;
  }
  k_nload_density3d_node<dfloat, SplitVec, 2><<<INTERIOR_LAUNCH(g)>>>(
      g.n, g.pitch, g.stride, dfloat(vol / 140.0), dfloat(vol / 210.0), dfloat(vol / 420.0), u,
      nl, b);
}

void rhs3d_df(const Grid& g, const double* lam, const PotentialParams* p, SplitVec u, double* f,
              cudaStream_t s) {
  const double h3 = g.h * g.h * g.h;
  if (star3_walks(g)) {
    static const cudaError_t attr = star3_prepare(k_rhs3d_dfw);
    (void)attr;
    k_rhs3d_dfw<<<star3_grid(g.n, g.nb), star3_block(), kS3Smem, s>>>(
        g.n, g.pitch, g.stride, dfloat(h3 / 120.0), dfloat(h3 / 6.0 / 140.0 / 6.0), lam, p, u, f);
    return;
  }
  k_rhs3d_df<<<INTERIOR_LAUNCH(g)>>>(g.n, g.pitch, g.stride, dfloat(h3), dfloat(h3 / 6.0 / 140.0),
                                     lam, p, u, f);
}

void coarsen_density3d(const Grid& fine, const Grid& coarse, const Density3D& bf,
                       const Density3D& bc, cudaStream_t s, bool split) {
  const dim3 grid = grid3(fine, coarse.n - 1, coarse.n - 1, coarse.n - 1);
  if (split)
    k_coarsen_density3d<dfloat><<<grid, block3(fine), 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, bf, bc);
  else
    k_coarsen_density3d<double><<<grid, block3(fine), 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, bf, bc);
}

void dense_level1_3d(const Grid& g, const Coef3D& c, double* L, double* M, cudaStream_t s) {
  const int m = g.n - 1, cnt = m * m * m;
  Stencil15 st;
  for (int q = 0; q < 8; ++q) st.a[q] = c.a[q];
  const dim3 grid((cnt + 63) / 64, g.nb);
  k_dense15<<<grid, 64, 0, s>>>(g.n, g.pitch, g.stride, st, 1, L, 0.0);
  k_dense15<<<grid, 64, 0, s>>>(g.n, g.pitch, g.stride, st, 0, M, g.h * g.h * g.h);
}

void density_dense3d(const Grid& g, const Density3D& b, double* B, cudaStream_t s, bool split) {
  const int m = g.n - 1, cnt = m * m * m;
  Stencil15 st;
  for (int q = 0; q < 8; ++q) st.a[q] = b.a[q];
  k_dense15<<<dim3((cnt + 63) / 64, g.nb), 64, 0, s>>>(g.n, g.pitch, g.stride, st, 1, B, 0.0,
                                                       split ? 1 : 0);
}

void gather_vec3d(const Grid& g, const double* a, const double* b, const double* c, double* oa,
                  double* ob, double* oc, cudaStream_t s) {
  const int m = g.n - 1, cnt = m * m * m;
  k_gather_vec3d<<<dim3((cnt + 63) / 64, g.nb), 64, 0, s>>>(g.n, g.pitch, g.stride, a, b, c, oa,
                                                            ob, oc);
}

void start_vector3d(const Grid& g, double* c, int cstride, cudaStream_t s) {
  const int m = g.n - 1, cnt = m * m * m;
  k_start3d<<<dim3((cnt + 63) / 64, g.nb), 64, 0, s>>>(g.n, c, cstride);
}

}  // namespace fmg
