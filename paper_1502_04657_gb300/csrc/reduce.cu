// Deterministic FP64 dot products: fixed block count and fixed-order trees, so the result
// does not depend on scheduling (no atomics).
#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr int kThreads = 256;

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// instance blockIdx.y: a, b at blockIdx.y * vst, partials at blockIdx.y * kReduceBlocks
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                              size_t n, size_t vst, size_t chunk, double* __restrict__ partials) {
  __shared__ double sh[kThreads];
  a += blockIdx.y * vst;
  b += blockIdx.y * vst;
  partials += (size_t)blockIdx.y * kReduceBlocks;
  const size_t beg = blockIdx.x * chunk;
  const size_t end = beg + chunk < n ? beg + chunk : n;
  double s = 0.0;
  for (size_t i = beg + threadIdx.x; i < end; i += kThreads) s = fma(a[i], b[i], s);
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_sum_final(const double* __restrict__ partials, int m, double* out) {
  __shared__ double sh[kThreads];
  partials += (size_t)blockIdx.x * kReduceBlocks;  // instance blockIdx.x
  out += blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += kThreads) s += partials[i];
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = t;
}

}  // namespace

void dot(const double* a, const double* b, size_t n, double* partials, double* out,
         cudaStream_t s, int nb, size_t vst) {
  size_t blocks = (n + 4 * kThreads - 1) / (4 * kThreads);
  if (blocks > (size_t)kReduceBlocks) blocks = kReduceBlocks;
  if (blocks < 1) blocks = 1;
  const size_t chunk = (n + blocks - 1) / blocks;
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
