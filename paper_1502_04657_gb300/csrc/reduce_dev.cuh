// Device-side sums of many values at once (the per-block class sums of the T3 passes).
#pragma once

namespace fmg {

// Every lane holds N <= 32 values; on return lane m holds the sum over the warp of value m
// (lanes m >= N hold 0).  Recursive halving: at offset o (16, 8, 4, 2, 1) a lane keeps the
// half of its current values selected by bit o of its lane index, sends the other half to
// lane ^ o and adds what that lane sends back, so the 32 sums take 31 shuffles and 31 adds
// per lane (a shuffle tree per value would take 5 N).  The order of the additions is fixed.
template <int N>
__device__ __forceinline__ double warp_transpose_sum(const double (&v)[N]) {
  static_assert(N >= 1 && N <= 32, "at most 32 values per lane");
  double a[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) a[i] = i < N ? v[i] : 0.0;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const double send = up ? a[i] : a[i + o];
      const double keep = up ? a[i + o] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return a[0];
}

// Block totals of N values per thread: out[m] = sum over the block's threads of value m,
// written by thread m.  blockDim.x is a multiple of 32 and every thread of the block calls
// this (with zeros if it has nothing to add); sh holds blockDim.x doubles.  The warps'
// totals are added in warp order, so the result does not depend on scheduling.
template <int N>
__device__ __forceinline__ void block_sum_to(const double (&v)[N], double* sh, double* out) {
  const double w = warp_transpose_sum<N>(v);
  sh[threadIdx.x] = w;
  __syncthreads();
  if (threadIdx.x < N) {
    const int warps = blockDim.x >> 5;
    double s = 0.0;
    for (int q = 0; q < warps; ++q) s += sh[q * 32 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Threads per block for `work` independent items, in whole warps, at most `cap`.
inline int warps_for(long work, int cap) {
  const long t = (work + 31) / 32 * 32;
  return (int)(t < 32 ? 32 : (t > cap ? cap : t));
}

}  // namespace fmg
