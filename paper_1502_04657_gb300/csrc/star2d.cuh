// Column-streamed star sums of the 2D cubic load and density stencil (device code shared by
// grid2d.cu and augment2d.cu).
//
// On the right-triangle mesh the star of node p is the hexagon of neighbours E, NE, N, W,
// SW, S; each consecutive pair (a, b) closes one triangle with p, and (a, b) is an edge of
// the mesh opposite p.  The exact cubic load int u^3 phi_p (Section 2, P1 functions,
// barycentric monomial integrals) is
//   |K|/60 [u^2 (24u + 3 M1) + u sum_e F_e + sum_e E3_e]
// over the six opposite edges e = (a, b), with s_e = a + b, F_e = s_e^2 + a^2 + b^2
// (= 2 (a^2 + ab + b^2)), E3_e = s_e (a^2 + b^2) and M1 = sum_e s_e (twice the neighbour
// sum).  These three numbers depend on the edge alone, and every mesh edge is opposite two
// nodes, so each is computed once per edge instead of once per node that needs it: a node
// owns its edges towards E (H), N (V) and NE (D) and takes the other opposite edges from
// the lanes beside it and the rows below it.
//
// Layout of the work: a warp covers 32 consecutive columns (lanes 1..30 produce, lanes 0 and
// 31 only supply edges and neighbour values) and R consecutive rows, which one thread walks
// upwards; edges of the rows before and after the block come from one extra row at each
// end.  Every node's arithmetic is the same whichever lane and block computes it, so the
// result does not depend on the launch shape.
#pragma once
#include "fmg_internal.h"
#include "dfloat.cuh"

namespace fmg {

template <typename T>
struct StarEdge {
  T s, F, E3;
};

// what a producing node hands to its epilogue
template <typename T>
struct Star2D {
  T u, q;            // u_p and u_p^2
  T M1, SF, SE;      // sums over the six opposite edges of s, F and E3
  StarEdge<T> H, V, D;  // p's own edges towards E, N and NE
  T uE, uN, uW, uS, uNE;  // neighbour values (apexes of the density stencil's edges)
  T qE, qN, qW, qS, qNE;
};

__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_down1(double v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}
__device__ __forceinline__ dfloat shfl_up1(dfloat v) {
  return dfloat(__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1));
}
__device__ __forceinline__ dfloat shfl_down1(dfloat v) {
  return dfloat(__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1));
}
template <typename T>
__device__ __forceinline__ StarEdge<T> shfl_up1(const StarEdge<T>& e) {
  return {shfl_up1(e.s), shfl_up1(e.F), shfl_up1(e.E3)};
}
template <typename T>
__device__ __forceinline__ StarEdge<T> shfl_down1(const StarEdge<T>& e) {
  return {shfl_down1(e.s), shfl_down1(e.F), shfl_down1(e.E3)};
}

template <typename T>
__device__ __forceinline__ StarEdge<T> star_edge(T a, T qa, T b, T qb) {
  const T s = a + b, qs = qa + qb;
  return {s, fma(s, s, qs), s * qs};
}

// the bracket of the cubic load, u^2 (24u + 3 M1) + u sum F + sum E3
template <typename T>
__device__ __forceinline__ T star_cubic(const Star2D<T>& p) {
  return fma(T(3), p.q * fma(T(8), p.u, p.M1), fma(p.u, p.SF, p.SE));
}

constexpr int kStarRows = 16;   // rows one thread walks
constexpr int kStarWarps = 4;   // warps of a block, stacked in y
constexpr int kStarCols = 30;   // producing columns of a warp

inline dim3 star2d_grid(int n, int nb) {
  return dim3((n - 1 + kStarCols - 1) / kStarCols,
              (n - 1 + kStarRows * kStarWarps - 1) / (kStarRows * kStarWarps), nb);
}
inline dim3 star2d_block() { return dim3(32, kStarWarps); }

// A walk is a chain of dependent row steps, and a block's FP64 work lands on one SM, so a
// level with few blocks is latency-bound (about 33 us for any n <= 512 on one GB300, against
// 8 us node by node at n = 128).  The walk is taken when it gives at least two blocks per SM
// (single 2D instances from n = 1024 on); smaller launches run node by node.
// (FMG_FLAG_STAR_WALKS takes it everywhere.)
constexpr unsigned kWalkMinBlocks = 2 * 152;
inline bool star2d_walks(const Grid& lv) {
  const dim3 g = star2d_grid(lv.n, lv.nb);
  return lv.walk_all || (size_t)g.x * g.y * g.z >= kWalkMinBlocks;
}

// Walks the rows of this thread's strip of instance blockIdx.z and calls out(k, star) for
// every interior node it produces (k = the node's index in the batched arrays).  u is read
// through get<T>: FP64 or the split double-float copy.  blockDim = (32, kStarWarps).
template <typename T, typename U, typename Out>
__device__ __forceinline__ void star2d_walk(int n, int pitch, size_t st, const U& u, Out out) {
  const int lane = threadIdx.x;
  const int i = kStarCols * blockIdx.x + lane;  // lane 0 = first produced column - 1
  const int j0 = 1 + kStarRows * (blockIdx.y * blockDim.y + threadIdx.y);
  if (j0 >= n) return;  // uniform over the warp
  const size_t base = blockIdx.z * st;
  const bool produce = lane >= 1 && lane <= kStarCols && i <= n - 1;
  auto ld = [&](int r) -> T {
    return (i <= n && r <= n) ? get<T>(u, base + (size_t)r * pitch + i) : T(0);
  };
  // row r = j0 - 1 + t: u0/q0 this column, u0R/q0R the next one, u0L/q0L the previous one
  T u0 = ld(j0 - 1);
  T q0 = u0 * u0;
  T u0R = shfl_down1(u0), q0R = shfl_down1(q0);
  // state carried from earlier rows (names say which row: m1 = r - 1, m2 = r - 2)
  T um1 = T(0), qm1 = T(0), um2 = T(0), qm2 = T(0);
  T uRm1 = T(0), qRm1 = T(0), uLm1 = T(0), qLm1 = T(0);
  StarEdge<T> Dm1{}, Dm2{}, VLm1{}, VLm2{}, HLm1{}, HLm2{}, DLm1{}, VRm1{}, Hm1{}, Vm1{};
#pragma unroll
  for (int t = 0; t < kStarRows + 2; ++t) {
    const int r = j0 - 1 + t;
    const T u1 = ld(r + 1);
    const T q1 = u1 * u1;
    const T u1R = shfl_down1(u1), q1R = shfl_down1(q1);
    const T u0L = shfl_up1(u0), q0L = shfl_up1(q0);
    const StarEdge<T> V = star_edge(u0, q0, u1, q1);
    const StarEdge<T> H = star_edge(u0, q0, u0R, q0R);
    const StarEdge<T> D = star_edge(u0, q0, u1R, q1R);
    const StarEdge<T> VL = shfl_up1(V), HL = shfl_up1(H), DL = shfl_up1(D), VR = shfl_down1(V);
    if (t >= 2 && produce && r - 1 <= n - 1) {
      // node (i, r - 1): opposite edges D(i, r-2), V(i-1, r-2), H(i-1, r-2), D(i-1, r-1),
      // V(i+1, r-1) and H(i, r)
      Star2D<T> p;
      p.u = um1;
      p.q = qm1;
      p.M1 = ((Dm2.s + VLm2.s) + (HLm2.s + DLm1.s)) + (VRm1.s + H.s);
      p.SF = ((Dm2.F + VLm2.F) + (HLm2.F + DLm1.F)) + (VRm1.F + H.F);
      p.SE = ((Dm2.E3 + VLm2.E3) + (HLm2.E3 + DLm1.E3)) + (VRm1.E3 + H.E3);
      p.H = Hm1;
      p.V = Vm1;
      p.D = Dm1;
      p.uE = uRm1;
      p.qE = qRm1;
      p.uN = u0;
      p.qN = q0;
      p.uW = uLm1;
      p.qW = qLm1;
      p.uS = um2;
      p.qS = qm2;
      p.uNE = u0R;
      p.qNE = q0R;
      out(base + (size_t)(r - 1) * pitch + i, p);
    }
    // shift the rows
    um2 = um1;
    qm2 = qm1;
    um1 = u0;
    qm1 = q0;
    uRm1 = u0R;
    qRm1 = q0R;
    uLm1 = u0L;
    qLm1 = q0L;
    Dm2 = Dm1;
    Dm1 = D;
    VLm2 = VLm1;
    VLm1 = VL;
    HLm2 = HLm1;
    HLm1 = HL;
    DLm1 = DL;
    VRm1 = VR;
    Hm1 = H;
    Vm1 = V;
    u0 = u1;
    q0 = q1;
    u0R = u1R;
    q0R = q1R;
  }
}

}  // namespace fmg
