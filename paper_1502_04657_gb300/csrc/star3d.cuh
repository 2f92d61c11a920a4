// Plane-walked star sums of the 3D cubic load and density stencil (device code of
// grid3d.cu), in FP64 or, for the mixed-precision modes, in double-float arithmetic (T =
// dfloat, u read from its split copy).
//
// On a tetrahedron K with vertex values a, b, c, d let h1, h2, h3 be the complete homogeneous
// symmetric sums of degree 1, 2, 3 of the four values.  Exact integration of P1 functions
// (Section 2, barycentric monomial integrals) gives, for vertices p != q of K,
//   int_K u^3 lambda_p        = |K|/140 [h3 + u_p h2 + u_p^2 h1 + u_p^3]
//   int_K u^2 lambda_p^2      = |K|/210 [h2 + 2 u_p h1 + 3 u_p^2]
//   int_K u^2 lambda_p lambda_q = |K|/420 [h2 + (u_p + u_q) h1 + u_p^2 + u_q^2 + u_p u_q],
// so a node needs, over the 24 tetrahedra of its star, S_k = sum h_k, and each mesh edge
// p-q, over the 6 or 4 tetrahedra that contain it, E_k = sum h_k (k = 1, 2).  h1, h2, h3 of a
// tetrahedron are the same for its four vertices: they are formed once per tetrahedron (from
// the power sums, 2 h2 = p1^2 + p2 and 6 h3 = p1^3 + 3 p1 p2 + 2 p3) instead of once per
// vertex, and the mass stencil comes for free: h^3/120 (24 u_p + S_1).
//
// Kuhn cube with corner v: tetrahedra {v, v + e_a, v + e_a + e_b, v + (1,1,1)}, named by their
// middle vertices (S, D): T0 (X, XY), T1 (X, XZ), T2 (Y, XY), T3 (Y, YZ), T4 (Z, XZ),
// T5 (Z, YZ).  A corner of the cube lies in all six (v, W) or in two: X in T0 + T1, Y in
// T2 + T3, Z in T4 + T5, XY in T0 + T2, XZ in T1 + T4, YZ in T3 + T5.
//
// Layout of the work: a block covers a 32 x 8 tile of columns and walks 16 planes upwards.
// For each plane z it stages u, u^2, u^3 of plane z + 1 (tile and halo) in shared memory,
// forms the 6 tetrahedra of every cube of layer z (corners in planes z and z + 1) into
// shared memory, and then each thread finishes its node of plane z (the four cubes of layer z
// above it; the four of layer z - 1 below it were summed at the previous step) and starts
// the node above it.  Every sum is taken in a fixed order, so the result does not depend on
// the launch shape.
#pragma once
#include "dfloat.cuh"
#include "fmg_internal.h"

namespace fmg {

constexpr int kS3X = 32, kS3Y = 8, kS3Z = 16;   // tile of columns (= threads), planes per block
constexpr int kS3CX = kS3X + 1;                  // cube layer row (cubes x0 - 1 .. x0 + 31)
constexpr int kS3Cubes = (kS3X + 1) * (kS3Y + 1);
constexpr int kS3NX = kS3X + 2;                  // node plane row (nodes x0 - 1 .. x0 + 32)
constexpr int kS3Nodes = (kS3X + 2) * (kS3Y + 2);
constexpr int kS3Vals = 21;  // per cube: 6 tetrahedra x (h1, 2 h2, 6 h3), then their totals
// three plane slots of (u, u^2, u^3) and one cube layer (a double-float value takes the 8
// bytes of a double)
constexpr size_t kS3Smem = sizeof(double) * (9 * (size_t)kS3Nodes + (size_t)kS3Vals * kS3Cubes);
static_assert(sizeof(dfloat) == sizeof(double), "double-float values share the FP64 layout");

// what a node hands to its epilogue: sums over its 24 tetrahedra of h1, 2 h2 and 6 h3, and for
// each edge towards p + d (d = X, Y, Z, XY, XZ, YZ, XYZ) the sums of h1 and 2 h2 over the
// tetrahedra of the edge with the values u, u^2 at p + d (EDGES only)
template <typename T>
struct Star3T {
  T u, q;
  T S1, S2, S3;
  T E1[7], E2[7];
  T un[7], qn[7];
};
using Star3 = Star3T<double>;

__host__ __device__ inline int star3_zchunks(int n) { return (n - 1 + kS3Z - 1) / kS3Z; }
inline dim3 star3_grid(int n, int nb) {
  return dim3((n - 1 + kS3X - 1) / kS3X, (n - 1 + kS3Y - 1) / kS3Y, nb * star3_zchunks(n));
}
inline dim3 star3_block() { return dim3(kS3X, kS3Y); }

// A block's 16 planes are dependent steps on one SM, so a level with few blocks is
// latency-bound (about 0.23 ms for any n <= 64 on one GB300, against 0.025 ms node by node at
// n = 32).  The walk is taken when it gives at least two blocks per SM (single 3D instances
// from n = 128 on); smaller launches run node by node.
// (FMG_FLAG_STAR_WALKS takes it everywhere.)
constexpr unsigned kWalk3MinBlocks = 2 * 152;
inline bool star3_walks(const Grid& lv) {
  const dim3 g = star3_grid(lv.n, lv.nb);
  return lv.walk_all || (size_t)g.x * g.y * g.z >= kWalk3MinBlocks;
}

// blockDim = (kS3X, kS3Y), kS3Smem bytes of dynamic shared memory; instance
// blockIdx.z / star3_zchunks(n).  out(k, star) for every interior node the block produces.
// T: the arithmetic (double, or dfloat with u a SplitVec); the FP64 instantiation evaluates
// exactly the expressions it did before it was templated.
template <bool EDGES, typename T = double, typename U = const double*, typename Out>
__device__ __forceinline__ void star3_walk(int n, int pitch, size_t st, const U u, Out out) {
  extern __shared__ double s3sm[];
  T* const su = reinterpret_cast<T*>(s3sm);  // [3][kS3Nodes]
  T* const sq = su + 3 * kS3Nodes;           // u^2
  T* const sc = sq + 3 * kS3Nodes;           // 2 u^3
  T* const cube = sc + 3 * kS3Nodes;         // [kS3Vals][kS3Cubes]
  const int nzc = star3_zchunks(n);
  const int ib = blockIdx.z / nzc;
  const int z0 = 1 + (int)(blockIdx.z - ib * nzc) * kS3Z;
  const int z1 = min(z0 + kS3Z, n);
  const int x0 = 1 + blockIdx.x * kS3X, y0 = 1 + blockIdx.y * kS3Y;
  const long plane = (long)(n + 1) * pitch;
  const size_t base = (size_t)ib * st;
  const int tid = threadIdx.y * kS3X + threadIdx.x;
  constexpr int kThreads = kS3X * kS3Y;

  auto load_plane = [&](int zp) {
    const int sl = (zp % 3) * kS3Nodes;
    for (int e = tid; e < kS3Nodes; e += kThreads) {
      const int xl = e % kS3NX, yl = e / kS3NX;
      const int x = x0 - 1 + xl, y = y0 - 1 + yl;
      const T v = (x <= n && y <= n) ? get<T>(u, base + zp * plane + (long)y * pitch + x) : T(0);
      const T v2 = v * v;
      su[sl + e] = v;
      sq[sl + e] = v2;
      sc[sl + e] = twice(v2 * v);  // 2 u^3: 6 h3 takes 2 p3, and doubling is exact
    }
  };

  auto cube_layer = [&](int cz) {
    const int s0 = (cz % 3) * kS3Nodes, s1 = ((cz + 1) % 3) * kS3Nodes;
    for (int e = tid; e < kS3Cubes; e += kThreads) {
      const int a = e % kS3CX, b = e / kS3CX;
      const int v0 = s0 + b * kS3NX + a, v1 = s1 + b * kS3NX + a;
      // corners: v, X, Y, XY in plane cz; Z, XZ, YZ, W in plane cz + 1
      const int X = v0 + 1, Y = v0 + kS3NX, XY = v0 + kS3NX + 1;
      const int Z = v1, XZ = v1 + 1, YZ = v1 + kS3NX;
      const T A = su[v0] + su[v1 + kS3NX + 1];
      const T QA = sq[v0] + sq[v1 + kS3NX + 1];
      const T CA = sc[v0] + sc[v1 + kS3NX + 1];
      // the power sums of v, W and the first middle vertex, shared by its two tetrahedra
      const T a1[3] = {A + su[X], A + su[Y], A + su[Z]};
      const T a2[3] = {QA + sq[X], QA + sq[Y], QA + sq[Z]};
      const T a3[3] = {CA + sc[X], CA + sc[Y], CA + sc[Z]};
      T h[6][3];
      auto tet = [&](int t, int m, int iD) {
        const T h1 = a1[m] + su[iD];
        const T p2 = a2[m] + sq[iD];
        const T p3 = a3[m] + sc[iD];
        const T s2 = h1 * h1;
        h[t][0] = h1;
        h[t][1] = s2 + p2;                         // 2 h2
        h[t][2] = fma(h1, fma(T(3), p2, s2), p3);  // 6 h3 (p3 from 2 u^3: 2 p3)
      };
      tet(0, 0, XY);
      tet(1, 0, XZ);
      tet(2, 1, XY);
      tet(3, 1, YZ);
      tet(4, 2, XZ);
      tet(5, 2, YZ);
#pragma unroll
      for (int t = 0; t < 6; ++t)
#pragma unroll
        for (int j = 0; j < 3; ++j) cube[(3 * t + j) * kS3Cubes + e] = h[t][j];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        cube[(18 + j) * kS3Cubes + e] = ((h[0][j] + h[1][j]) + (h[2][j] + h[3][j])) +
                                        (h[4][j] + h[5][j]);
    }
  };

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x <= n - 1 && y <= n - 1;
  // cubes (x-1, y-1), (x, y-1), (x-1, y), (x, y) of a layer
  const int c00 = ty * kS3CX + tx, c10 = c00 + 1, c01 = c00 + kS3CX, c11 = c01 + 1;
  const int nd = (ty + 1) * kS3NX + tx + 1;  // this column's node in a plane slot
  auto G = [&](int t, int j, int c) { return cube[(3 * t + j) * kS3Cubes + c]; };
  auto TOT = [&](int j, int c) { return cube[(18 + j) * kS3Cubes + c]; };

  // contributions of layer z - 1 to the node of plane z: the node is corner Z of cube (x, y),
  // XZ of (x-1, y), YZ of (x, y-1) and W of (x-1, y-1)
  T pS[3], pEX[2], pEY[2], pEXY[2];
  T PZ[3];
  auto pending = [&]() {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T pxz = G(1, j, c01) + G(4, j, c01);
      const T pyz = G(3, j, c10) + G(5, j, c10);
      pS[j] = (PZ[j] + pxz) + (pyz + TOT(j, c00));
      if (EDGES && j < 2) {
        pEX[j] = G(4, j, c11) + pyz;   // edge +X: T4 of (x, y), pair YZ of (x, y-1)
        pEY[j] = G(5, j, c11) + pxz;   // edge +Y: T5 of (x, y), pair XZ of (x-1, y)
        pEXY[j] = PZ[j];               // edge +XY: pair Z of (x, y)
      }
    }
  };

  load_plane(z0 - 1);
  load_plane(z0);
  __syncthreads();
  cube_layer(z0 - 1);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 3; ++j) PZ[j] = G(4, j, c11) + G(5, j, c11);
  pending();

  for (int z = z0; z < z1; ++z) {
    load_plane(z + 1);
    __syncthreads();
    cube_layer(z);
    __syncthreads();
    // layer z: the node of plane z is corner v of cube (x, y), X of (x-1, y), Y of (x, y-1)
    // and XY of (x-1, y-1)
    Star3T<T> p;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T px = G(0, j, c01) + G(1, j, c01);   // pair X of (x-1, y)
      const T py = G(2, j, c10) + G(3, j, c10);   // pair Y of (x, y-1)
      const T pxy = G(0, j, c00) + G(2, j, c00);  // pair XY of (x-1, y-1)
      PZ[j] = G(4, j, c11) + G(5, j, c11);        // pair Z of (x, y)
      const T S = pS[j] + ((TOT(j, c11) + px) + (py + pxy));
      if (j == 0) p.S1 = S;
      else if (j == 1) p.S2 = S;
      else p.S3 = S;
      if (EDGES && j < 2) {
        T* E = j == 0 ? p.E1 : p.E2;
        E[0] = pEX[j] + ((G(0, j, c11) + G(1, j, c11)) + G(2, j, c10));
        E[1] = pEY[j] + ((G(2, j, c11) + G(3, j, c11)) + G(0, j, c01));
        E[2] = (PZ[j] + G(1, j, c01)) + (G(3, j, c10) + pxy);
        E[3] = pEXY[j] + (G(0, j, c11) + G(2, j, c11));
        E[4] = (G(1, j, c11) + G(4, j, c11)) + py;
        E[5] = (G(3, j, c11) + G(5, j, c11)) + px;
        E[6] = TOT(j, c11);
      }
    }
    if (active) {
      const int sz = (z % 3) * kS3Nodes, sz1 = ((z + 1) % 3) * kS3Nodes;
      p.u = su[sz + nd];
      p.q = sq[sz + nd];
      if (EDGES) {
        const int on[7] = {sz + nd + 1,  sz + nd + kS3NX,  sz1 + nd,        sz + nd + kS3NX + 1,
                           sz1 + nd + 1, sz1 + nd + kS3NX, sz1 + nd + kS3NX + 1};
#pragma unroll
        for (int d = 0; d < 7; ++d) {
          p.un[d] = su[on[d]];
          p.qn[d] = sq[on[d]];
        }
      }
      out(base + z * plane + (long)y * pitch + x, p);
    }
    pending();
  }
}

}  // namespace fmg
