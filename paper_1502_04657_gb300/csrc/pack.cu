// Conversion between the ABI layout (interior nodes, x fastest) and the padded device layout.
#include "fmg_internal.h"

namespace fmg {
namespace {

__device__ __forceinline__ size_t padded_index(int dim, int n, int pitch, size_t p) {
  const size_t m = (size_t)(n - 1);
  const size_t i = 1 + p % m;
  if (dim == 2) return (1 + p / m) * pitch + i;
  const size_t j = 1 + (p / m) % m;
  const size_t l = 1 + p / (m * m);
  return (l * (size_t)(n + 1) + j) * pitch + i;
}

// instance blockIdx.y: interior vector at blockIdx.y * ist, padded one at blockIdx.y * pst
__global__ void k_pack(int dim, int n, int pitch, size_t count, size_t ist, size_t pst,
                       const double* __restrict__ in, double* __restrict__ out) {
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p < count) out[blockIdx.y * pst + padded_index(dim, n, pitch, p)] = in[blockIdx.y * ist + p];
}

__global__ void k_unpack(int dim, int n, int pitch, size_t count, size_t ist, size_t pst,
                         const double* __restrict__ in, double* __restrict__ out) {
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p < count) out[blockIdx.y * ist + p] = in[blockIdx.y * pst + padded_index(dim, n, pitch, p)];
}

__global__ void k_gather_index(const double* __restrict__ src, const int* __restrict__ idx,
                               double* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

}  // namespace

void gather_by_index(const double* src, const int* idx, double* dst, int n, cudaStream_t s) {
  k_gather_index<<<(n + 255) / 256, 256, 0, s>>>(src, idx, dst, n);
}

void pack_interior(const Grid& g, const double* interior, double* padded, cudaStream_t s) {
  const size_t count = g.interior();
  k_pack<<<dim3((unsigned)((count + 255) / 256), g.nb), 256, 0, s>>>(
      g.dim, g.n, g.pitch, count, count, g.stride, interior, padded);
}

void unpack_interior(const Grid& g, const double* padded, double* interior, cudaStream_t s) {
  const size_t count = g.interior();
  k_unpack<<<dim3((unsigned)((count + 255) / 256), g.nb), 256, 0, s>>>(
      g.dim, g.n, g.pitch, count, count, g.stride, padded, interior);
}

cudaError_t copy_interior_to_host(const Grid& g, const double* padded, double* host,
                                  cudaStream_t s) {
  const size_t m = (size_t)(g.n - 1), row = m * sizeof(double), sp = (size_t)g.pitch * sizeof(double);
  if (g.dim == 2)  // rows 1 .. n - 1, columns 1 .. n - 1
    return cudaMemcpy2DAsync(host, row, padded + g.pitch + 1, sp, row, m,
                             cudaMemcpyDeviceToHost, s);
  cudaMemcpy3DParms q = {};
  q.srcPtr = make_cudaPitchedPtr(const_cast<double*>(padded), sp, sp, (size_t)(g.n + 1));
  q.srcPos = make_cudaPos(sizeof(double), 1, 1);  // element (1, 1, 1)
  q.dstPtr = make_cudaPitchedPtr(host, row, row, m);
  q.extent = make_cudaExtent(row, m, m);
  q.kind = cudaMemcpyDeviceToHost;
  return cudaMemcpy3DAsync(&q, s);
}

void scatter_level1(const Grid& g, const double* c, size_t cstride, double* padded,
                    cudaStream_t s) {
  const size_t count = g.interior();
  k_pack<<<dim3((unsigned)((count + 255) / 256), g.nb), 256, 0, s>>>(
      g.dim, g.n, g.pitch, count, cstride, g.stride, c, padded);
}

}  // namespace fmg
