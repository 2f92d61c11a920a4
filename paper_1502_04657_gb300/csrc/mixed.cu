// Mixed-precision multigrid iteration (precision FMG_MIXED_FP32 / FMG_MIXED_BF16): the m
// multigrid iterations of Algorithm 3.1 step 1 become an FP64 defect correction around
// single-precision V-cycles,
//     r = f - L x  (FP64 operator, stored in S),   e = V32(r),   x <- x + e  (FP64),
// so only the residual and the update touch FP64 arithmetic.  FP32 issues at ~64x the FP64
// rate on this part, which leaves the V-cycle's smoothing, residual and transfer kernels bound
// by HBM bandwidth.  Their vectors and coefficients are stored in S = float or (the storage
// ablation) bfloat16, always computed in FP32; the FP64 residual keeps the outer iteration
// converging to the FP64 solution of L x = f.
#include <cuda_bf16.h>

#include "fmg_internal.h"

namespace fmg {
namespace {

__device__ __forceinline__ size_t at(int i, int j, int pitch) { return (size_t)j * pitch + i; }

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float ld(const float* p, size_t k) { return p[k]; }
__device__ __forceinline__ float ld(const bf16* p, size_t k) { return __bfloat162float(p[k]); }
__device__ __forceinline__ void st(float* p, size_t k, float v) { p[k] = v; }
__device__ __forceinline__ void st(bf16* p, size_t k, float v) { p[k] = __float2bfloat16_rn(v); }

template <typename S>
struct CS2 {
  const S *cC, *cE, *cN, *cNE, *dinv;
};
template <typename S>
struct CS3 {
  const S* a[8];
  const S* dinv;
};

template <typename S>
CS2<S> cs(const CoefF2D& c) {
  return {reinterpret_cast<const S*>(c.cC), reinterpret_cast<const S*>(c.cE),
          reinterpret_cast<const S*>(c.cN), reinterpret_cast<const S*>(c.cNE),
          reinterpret_cast<const S*>(c.dinv)};
}
template <typename S>
CS3<S> cs(const CoefF3D& c) {
  CS3<S> o;
  for (int q = 0; q < 8; ++q) o.a[q] = reinterpret_cast<const S*>(c.a[q]);
  o.dinv = reinterpret_cast<const S*>(c.dinv);
  return o;
}
template <typename S>
S* sp(float* p) {
  return reinterpret_cast<S*>(p);
}
template <typename S>
const S* sp(const float* p) {
  return reinterpret_cast<const S*>(p);
}

// ---- conversions and the FP64 ends of the defect correction ----------------------------
// (contiguous over all instances: the arrays hold the instances back to back)
template <typename S>
__global__ void k_to_s(size_t n, const double* __restrict__ a, S* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    st(b, i, (float)a[i]);
}

template <typename S>
__global__ void k_add_s(size_t n, const S* __restrict__ e, double* __restrict__ x) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] += (double)ld(e, i);
}

// thread (i, j) of instance ib = blockIdx.z; k is its element index in the batched arrays
#define INTERIOR_2D                                        \
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x; \
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y; \
  if (i >= n || j >= n) return;                            \
  const int ib = blockIdx.z;                               \
  const size_t k = ib * st_ + at(i, j, pitch);

template <typename S>
__global__ void k_residual_mixed2d(int n, int pitch, size_t st_, Coef2D c,
                                   const double* __restrict__ f, const double* __restrict__ x,
                                   S* __restrict__ r) {
  INTERIOR_2D
  double v = c.cC[k] * x[k];
  v = fma(c.cE[k], x[k + 1], v);
  v = fma(c.cE[k - 1], x[k - 1], v);
  v = fma(c.cN[k], x[k + pitch], v);
  v = fma(c.cN[k - pitch], x[k - pitch], v);
  v = fma(c.cNE[k], x[k + pitch + 1], v);
  v = fma(c.cNE[k - pitch - 1], x[k - pitch - 1], v);
  st(r, k, (float)(f[k] - v));
}

// ---- single-precision 2D stencil kernels ----------------------------------------------------
template <typename S>
__device__ __forceinline__ float lop32(const CS2<S>& c, const S* __restrict__ x, size_t k,
                                       int pitch) {
  float v = ld(c.cC, k) * ld(x, k);
  v = fmaf(ld(c.cE, k), ld(x, k + 1), v);
  v = fmaf(ld(c.cE, k - 1), ld(x, k - 1), v);
  v = fmaf(ld(c.cN, k), ld(x, k + pitch), v);
  v = fmaf(ld(c.cN, k - pitch), ld(x, k - pitch), v);
  v = fmaf(ld(c.cNE, k), ld(x, k + pitch + 1), v);
  v = fmaf(ld(c.cNE, k - pitch - 1), ld(x, k - pitch - 1), v);
  return v;
}

template <typename S>
__global__ void k_jacobi32_2d(int n, int pitch, size_t st_, CS2<S> c, const S* __restrict__ f,
                              const S* __restrict__ x, S* __restrict__ xo) {
  INTERIOR_2D
  st(xo, k, fmaf(ld(c.dinv, k), ld(f, k) - lop32(c, x, k, pitch), ld(x, k)));
}

template <typename S>
__global__ void k_jacobi32z_2d(int n, int pitch, size_t st_, CS2<S> c, const S* __restrict__ f,
                               S* __restrict__ xo) {
  INTERIOR_2D
  st(xo, k, ld(c.dinv, k) * ld(f, k));
}

template <typename S>
__global__ void k_residual32_2d(int n, int pitch, size_t st_, CS2<S> c, const S* __restrict__ f,
                                const S* __restrict__ x, S* __restrict__ r) {
  INTERIOR_2D
  st(r, k, ld(f, k) - lop32(c, x, k, pitch));
}

template <typename S>
__global__ void k_restrict32_2d(int nc, int pc, int pf, size_t stc, size_t stf,
                                const S* __restrict__ rf, S* __restrict__ rc) {
  const int I = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nc || J >= nc) return;
  const size_t kf = blockIdx.z * stf + at(2 * I, 2 * J, pf);
  const float s = ((ld(rf, kf + 1) + ld(rf, kf - 1)) + (ld(rf, kf + pf) + ld(rf, kf - pf))) +
                  (ld(rf, kf + pf + 1) + ld(rf, kf - pf - 1));
  st(rc, blockIdx.z * stc + at(I, J, pc), fmaf(0.5f, s, ld(rf, kf)));
}

template <typename S>
__global__ void k_prolong32_2d(int nf, int pf, int pc, size_t st_, size_t stc,
                               const S* __restrict__ ec, S* __restrict__ xf) {
  const int n = nf, pitch = pf;
  INTERIOR_2D
  const int ai = i & 1, aj = j & 1;
  const size_t kc = ib * stc + at(i >> 1, j >> 1, pc);
  float e = ld(ec, kc);
  if (ai | aj) e = 0.5f * (e + ld(ec, kc + ai + (size_t)aj * pc));
  st(xf, k, ld(xf, k) + e);
}

// ---- single-precision 3D stencil kernels (Kuhn mesh, see grid3d.cu) --------------------------
__device__ constexpr int kDir[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                                       {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

__device__ __forceinline__ long dir_off(int d, int pitch, long plane) {
  return kDir[d][0] + (long)kDir[d][1] * pitch + (long)kDir[d][2] * plane;
}

// blockIdx.z = ib * (n - 1) + (l - 1): plane l of instance ib
#define INTERIOR_3D                                                  \
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;           \
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;           \
  const int ib = blockIdx.z / (n - 1);                               \
  const int l = 1 + (int)blockIdx.z - ib * (n - 1);                  \
  if (i >= n || j >= n) return;                                      \
  const long plane = (long)(n + 1) * pitch;                          \
  const size_t k = ib * st_ + (size_t)l * plane + (size_t)j * pitch + i;

template <typename S>
__global__ void k_residual_mixed3d(int n, int pitch, size_t st_, Coef3D c,
                                   const double* __restrict__ f, const double* __restrict__ x,
                                   S* __restrict__ r) {
  INTERIOR_3D
  double v = c.a[0][k] * x[k];
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    v = fma(c.a[1 + d][k], x[k + o], v);
    v = fma(c.a[1 + d][k - o], x[k - o], v);
  }
  st(r, k, (float)(f[k] - v));
}

template <typename S>
__device__ __forceinline__ float lop32_3(const CS3<S>& c, const S* __restrict__ x, size_t k,
                                         int pitch, long plane) {
  float v = ld(c.a[0], k) * ld(x, k);
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    v = fmaf(ld(c.a[1 + d], k), ld(x, k + o), v);
    v = fmaf(ld(c.a[1 + d], k - o), ld(x, k - o), v);
  }
  return v;
}

template <typename S>
__global__ void k_jacobi32_3d(int n, int pitch, size_t st_, CS3<S> c, const S* __restrict__ f,
                              const S* __restrict__ x, S* __restrict__ xo) {
  INTERIOR_3D
  st(xo, k, fmaf(ld(c.dinv, k), ld(f, k) - lop32_3(c, x, k, pitch, plane), ld(x, k)));
}

template <typename S>
__global__ void k_jacobi32z_3d(int n, int pitch, size_t st_, CS3<S> c, const S* __restrict__ f,
                               S* __restrict__ xo) {
  INTERIOR_3D
  st(xo, k, ld(c.dinv, k) * ld(f, k));
}

template <typename S>
__global__ void k_residual32_3d(int n, int pitch, size_t st_, CS3<S> c, const S* __restrict__ f,
                                const S* __restrict__ x, S* __restrict__ r) {
  INTERIOR_3D
  st(r, k, ld(f, k) - lop32_3(c, x, k, pitch, plane));
}

template <typename S>
__global__ void k_restrict32_3d(int nc, int pc, int pf, size_t stc, size_t stf,
                                const S* __restrict__ rf, S* __restrict__ rc) {
  const int I = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int ib = blockIdx.z / (nc - 1);
  const int L = 1 + (int)blockIdx.z - ib * (nc - 1);
  if (I >= nc || J >= nc) return;
  const long planef = (long)(2 * nc + 1) * pf;
  const size_t kf = ib * stf + (size_t)(2 * L) * planef + (size_t)(2 * J) * pf + 2 * I;
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pf, planef);
    s += ld(rf, kf + o) + ld(rf, kf - o);
  }
  st(rc, ib * stc + ((size_t)L * (nc + 1) + J) * pc + I, fmaf(0.5f, s, ld(rf, kf)));
}

template <typename S>
__global__ void k_prolong32_3d(int nf, int pf, int pc, size_t st_, size_t stc,
                               const S* __restrict__ ec, S* __restrict__ xf) {
  const int n = nf, pitch = pf;
  INTERIOR_3D
  const int ai = i & 1, aj = j & 1, al = l & 1;
  const int nc = nf / 2;
  const long planec = (long)(nc + 1) * pc;
  const size_t kc = ib * stc + (size_t)(l >> 1) * planec + (size_t)(j >> 1) * pc + (i >> 1);
  float e = ld(ec, kc);
  if (ai | aj | al) e = 0.5f * (e + ld(ec, kc + ai + (size_t)aj * pc + (size_t)al * planec));
  st(xf, k, ld(xf, k) + e);
}

// coarsest level: y = Linv x with x, y single-precision padded level-1 vectors (FP64
// accumulation); one CTA per instance blockIdx.x
template <typename S>
__global__ void k_coarse32(int dim, int n, int pitch, size_t st_, const double* __restrict__ Linv,
                           const S* __restrict__ x, S* __restrict__ y) {
  __shared__ double xs[1024];
  const int m = n - 1, nh = dim == 2 ? m * m : m * m * m;
  x += blockIdx.x * st_;
  y += blockIdx.x * st_;
  Linv += blockIdx.x * (size_t)nh * nh;
  auto idx = [&](int q) -> size_t {
    if (dim == 2) return (size_t)(1 + q / m) * pitch + 1 + q % m;
    return ((size_t)(1 + q / (m * m)) * (m + 2) + 1 + (q / m) % m) * pitch + 1 + q % m;
  };
  for (int q = threadIdx.x; q < nh; q += blockDim.x) xs[q] = (double)ld(x, idx(q));
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  for (int p = warp; p < nh; p += warps) {
    const double* row = Linv + (size_t)p * nh;
    double s = 0.0;
    for (int q = lane; q < nh; q += 32) s = fma(row[q], xs[q], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) st(y, idx(p), (float)s);
  }
}

dim3 grid2(const Grid& g, int cx, int cy) {
  return dim3((cx + g.bx - 1) / g.bx, (cy + g.by - 1) / g.by, g.nb);
}
dim3 grid3(const Grid& g, int cx, int cy, int cz) {
  return dim3((cx + g.bx - 1) / g.bx, (cy + g.by - 1) / g.by, cz * g.nb);
}
dim3 blk(const Grid& g) { return dim3(g.bx, g.by); }
unsigned blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 32 ? b : 152 * 32);
}

template <typename S>
void jacobi_t(const Grid& g, const CoefF2D& c2, const CoefF3D& c3, const float* f,
              const float* x, float* xo, bool zero, cudaStream_t s) {
  if (g.dim == 2) {
    const dim3 gr = grid2(g, g.n - 1, g.n - 1);
    if (zero) k_jacobi32z_2d<S><<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, cs<S>(c2), sp<S>(f), sp<S>(xo));
    else k_jacobi32_2d<S><<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, cs<S>(c2), sp<S>(f), sp<S>(x), sp<S>(xo));
  } else {
    const dim3 gr = grid3(g, g.n - 1, g.n - 1, g.n - 1);
    if (zero) k_jacobi32z_3d<S><<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, cs<S>(c3), sp<S>(f), sp<S>(xo));
    else k_jacobi32_3d<S><<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, cs<S>(c3), sp<S>(f), sp<S>(x), sp<S>(xo));
  }
}

template <typename S>
void residual_t(const Grid& g, const CoefF2D& c2, const CoefF3D& c3, const float* f,
                const float* x, float* r, cudaStream_t s) {
  if (g.dim == 2)
    k_residual32_2d<S><<<grid2(g, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, cs<S>(c2), sp<S>(f), sp<S>(x), sp<S>(r));
  else
    k_residual32_3d<S><<<grid3(g, g.n - 1, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, cs<S>(c3), sp<S>(f), sp<S>(x), sp<S>(r));
}

template <typename S>
void restrict_t(const Grid& fine, const Grid& coarse, const float* rf, float* rc, cudaStream_t s) {
  if (fine.dim == 2)
    k_restrict32_2d<S><<<grid2(fine, coarse.n - 1, coarse.n - 1), blk(fine), 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, sp<S>(rf), sp<S>(rc));
  else
    k_restrict32_3d<S><<<grid3(fine, coarse.n - 1, coarse.n - 1, coarse.n - 1), blk(fine), 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, sp<S>(rf), sp<S>(rc));
}

template <typename S>
void prolong_t(const Grid& fine, const Grid& coarse, const float* ec, float* xf, cudaStream_t s) {
  if (fine.dim == 2)
    k_prolong32_2d<S><<<grid2(fine, fine.n - 1, fine.n - 1), blk(fine), 0, s>>>(
        fine.n, fine.pitch, coarse.pitch, fine.stride, coarse.stride, sp<S>(ec), sp<S>(xf));
  else
    k_prolong32_3d<S><<<grid3(fine, fine.n - 1, fine.n - 1, fine.n - 1), blk(fine), 0, s>>>(
        fine.n, fine.pitch, coarse.pitch, fine.stride, coarse.stride, sp<S>(ec), sp<S>(xf));
}

}  // namespace

size_t mixed_elem_bytes(bool bf16_storage) { return bf16_storage ? sizeof(bf16) : sizeof(float); }

void to_f32(const double* a, float* b, size_t n, cudaStream_t s, bool bf) {
  if (bf) k_to_s<bf16><<<blocks_for(n), 256, 0, s>>>(n, a, sp<bf16>(b));
  else k_to_s<float><<<blocks_for(n), 256, 0, s>>>(n, a, b);
}

void add_f32(const float* e, double* x, size_t n, cudaStream_t s, bool bf) {
  if (bf) k_add_s<bf16><<<blocks_for(n), 256, 0, s>>>(n, sp<bf16>(e), x);
  else k_add_s<float><<<blocks_for(n), 256, 0, s>>>(n, e, x);
}

void residual_mixed(const Grid& g, const Coef2D& c2, const Coef3D& c3, const double* f,
                    const double* x, float* r, cudaStream_t s, bool bf) {
  if (g.dim == 2) {
    if (bf)
      k_residual_mixed2d<bf16><<<grid2(g, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, c2, f, x, sp<bf16>(r));
    else
      k_residual_mixed2d<float><<<grid2(g, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, c2, f, x, r);
  } else {
    if (bf)
      k_residual_mixed3d<bf16><<<grid3(g, g.n - 1, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, c3, f, x, sp<bf16>(r));
    else
      k_residual_mixed3d<float><<<grid3(g, g.n - 1, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, c3, f, x, r);
  }
}

void jacobi32(const Grid& g, const CoefF2D& c2, const CoefF3D& c3, const float* f,
              const float* x, float* xo, bool zero, cudaStream_t s, bool bf) {
  if (bf) jacobi_t<bf16>(g, c2, c3, f, x, xo, zero, s);
  else jacobi_t<float>(g, c2, c3, f, x, xo, zero, s);
}

void residual32(const Grid& g, const CoefF2D& c2, const CoefF3D& c3, const float* f,
                const float* x, float* r, cudaStream_t s, bool bf) {
  if (bf) residual_t<bf16>(g, c2, c3, f, x, r, s);
  else residual_t<float>(g, c2, c3, f, x, r, s);
}

void restrict32(const Grid& fine, const Grid& coarse, const float* rf, float* rc,
                cudaStream_t s, bool bf) {
  if (bf) restrict_t<bf16>(fine, coarse, rf, rc, s);
  else restrict_t<float>(fine, coarse, rf, rc, s);
}

void prolong32_add(const Grid& fine, const Grid& coarse, const float* ec, float* xf,
                   cudaStream_t s, bool bf) {
  if (bf) prolong_t<bf16>(fine, coarse, ec, xf, s);
  else prolong_t<float>(fine, coarse, ec, xf, s);
}

void coarse32(const Grid& g, const double* Linv, const float* x, float* y, cudaStream_t s,
              bool bf) {
  if (bf) k_coarse32<bf16><<<g.nb, 512, 0, s>>>(g.dim, g.n, g.pitch, g.stride, Linv, sp<bf16>(x), sp<bf16>(y));
  else k_coarse32<float><<<g.nb, 512, 0, s>>>(g.dim, g.n, g.pitch, g.stride, Linv, x, y);
}

}  // namespace fmg
