// Deterministic FP64 dot products: fixed block count and fixed-order trees, so the result
// does not depend on scheduling (no atomics).
#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr int kThreads = 256;

// Fixed-order block reduction for thread 0: lane trees inside each warp, then warp 0 over the
// warp sums.
__device__ double block_sum_warps(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

// instance blockIdx.y: a, b at blockIdx.y * vst, partials at blockIdx.y * kReduceBlocks.
// Block blockIdx.x sums elements [beg, end) of a chunk (an even number of elements, so the
// pairs are 16-byte aligned): each thread takes pairs in a fixed order into two accumulators
// per lane of the pair, then the block tree.
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                              size_t n, size_t vst, size_t chunk, double* __restrict__ partials) {
  __shared__ double sh[kThreads / 32];
  a += blockIdx.y * vst;
  b += blockIdx.y * vst;
  partials += (size_t)blockIdx.y * kReduceBlocks;
  const size_t beg = blockIdx.x * chunk;
  // a block past n (the even chunk may leave the last one empty) contributes 0
  const size_t end = beg >= n ? beg : (beg + chunk < n ? beg + chunk : n);
  const size_t pend = beg + ((end - beg) & ~(size_t)1);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  size_t i = beg + 2 * threadIdx.x;
  for (; i + 2 * kThreads < pend; i += 4 * kThreads) {
    const double2 x0 = *reinterpret_cast<const double2*>(a + i);
    const double2 y0 = *reinterpret_cast<const double2*>(b + i);
    const double2 x1 = *reinterpret_cast<const double2*>(a + i + 2 * kThreads);
    const double2 y1 = *reinterpret_cast<const double2*>(b + i + 2 * kThreads);
    s0 = fma(x0.x, y0.x, s0);
    s1 = fma(x0.y, y0.y, s1);
    s2 = fma(x1.x, y1.x, s2);
    s3 = fma(x1.y, y1.y, s3);
  }
  if (i < pend) {
    const double2 x0 = *reinterpret_cast<const double2*>(a + i);
    const double2 y0 = *reinterpret_cast<const double2*>(b + i);
    s0 = fma(x0.x, y0.x, s0);
    s1 = fma(x0.y, y0.y, s1);
  }
  if (threadIdx.x == 0 && pend < end) s0 = fma(a[pend], b[pend], s0);
  const double t = block_sum_warps((s0 + s1) + (s2 + s3), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_sum_final(const double* __restrict__ partials, int m, double* out) {
  __shared__ double sh[kThreads / 32];
  partials += (size_t)blockIdx.x * kReduceBlocks;  // instance blockIdx.x
  out += blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += kThreads) s += partials[i];
  const double t = block_sum_warps(s, sh);
  if (threadIdx.x == 0) out[0] = t;
}

}  // namespace

void dot(const double* a, const double* b, size_t n, double* partials, double* out,
         cudaStream_t s, int nb, size_t vst) {
  // at least 8192 elements (32 per thread) per block, at most kReduceBlocks blocks: the
  // split depends on n only, so an instance sums in the same order alone and in a batch
  size_t blocks = (n + 8191) / 8192;
  if (blocks > (size_t)kReduceBlocks) blocks = kReduceBlocks;
  if (blocks < 1) blocks = 1;
  size_t chunk = (n + blocks - 1) / blocks;
  chunk += chunk & 1;  // even: every block's pairs start 16-byte aligned
  k_dot_partial<<<dim3((unsigned)blocks, nb), kThreads, 0, s>>>(a, b, n, vst, chunk, partials);
  k_sum_final<<<nb, kThreads, 0, s>>>(partials, (int)blocks, out);
}

namespace {

// Conjugate gradient updates over whole batched level vectors (boundary and padding entries
// are zero in p, q and r and stay zero): instance ib = i / stride, with its scalars
// rr = r.r, pq = p.L p (a zero denominator gives a zero step, as in the oracle).
__global__ void k_cg_update(size_t n, size_t stride, const double* __restrict__ rr,
                            const double* __restrict__ pq, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ x,
                            double* __restrict__ r) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t ib = i / stride;
    const double a = pq[ib] > 0.0 ? rr[ib] / pq[ib] : 0.0;
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}

__global__ void k_cg_direction(size_t n, size_t stride, const double* __restrict__ rr_new,
                               const double* __restrict__ rr_old, const double* __restrict__ r,
                               double* __restrict__ p) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t ib = i / stride;
    const double b = rr_old[ib] > 0.0 ? rr_new[ib] / rr_old[ib] : 0.0;
    p[i] = fma(b, p[i], r[i]);
  }
}

unsigned cg_blocks(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

void cg_update(size_t n, size_t stride, const double* rr, const double* pq, const double* p,
               const double* q, double* x, double* r, cudaStream_t s) {
  k_cg_update<<<cg_blocks(n), 256, 0, s>>>(n, stride, rr, pq, p, q, x, r);
}

void cg_direction(size_t n, size_t stride, const double* rr_new, const double* rr_old,
                  const double* r, double* p, cudaStream_t s) {
  k_cg_direction<<<cg_blocks(n), 256, 0, s>>>(n, stride, rr_new, rr_old, r, p);
}

}  // namespace fmg
