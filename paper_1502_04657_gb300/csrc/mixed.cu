// Mixed-precision multigrid iteration (precision FMG_MIXED_FP32): the m multigrid iterations
// of Algorithm 3.1 step 1 become an FP64 defect correction around FP32 V-cycles,
//     r = f - L x  (FP64 operator, stored as FP32),   e = V32(r),   x <- x + e  (FP64),
// so only the residual and the update touch FP64 arithmetic.  FP32 issues at ~64x the FP64
// rate on this part, which leaves the FP32 smoothing, residual and transfer kernels bound by
// HBM bandwidth.  The smoother in FP32 uses the FP64 coefficients rounded to FP32; the FP64
// residual keeps the outer iteration converging to the FP64 solution of L x = f.
#include "fmg_internal.h"

namespace fmg {
namespace {

__device__ __forceinline__ size_t at(int i, int j, int pitch) { return (size_t)j * pitch + i; }

// ---- conversions and the FP64 ends of the defect correction ----------------------------
// (contiguous over all instances: the arrays hold the instances back to back)
__global__ void k_to_f32(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_add_f32(size_t n, const float* __restrict__ e, double* __restrict__ x) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] += (double)e[i];
}

// thread (i, j) of instance ib = blockIdx.z; k is its element index in the batched arrays
#define INTERIOR_2D                                        \
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x; \
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y; \
  if (i >= n || j >= n) return;                            \
  const int ib = blockIdx.z;                               \
  const size_t k = ib * st + at(i, j, pitch);

__global__ void k_residual_mixed2d(int n, int pitch, size_t st, Coef2D c,
                                   const double* __restrict__ f, const double* __restrict__ x,
                                   float* __restrict__ r) {
  INTERIOR_2D
  double v = c.cC[k] * x[k];
  v = fma(c.cE[k], x[k + 1], v);
  v = fma(c.cE[k - 1], x[k - 1], v);
  v = fma(c.cN[k], x[k + pitch], v);
  v = fma(c.cN[k - pitch], x[k - pitch], v);
  v = fma(c.cNE[k], x[k + pitch + 1], v);
  v = fma(c.cNE[k - pitch - 1], x[k - pitch - 1], v);
  r[k] = (float)(f[k] - v);
}

// ---- FP32 2D stencil kernels ---------------------------------------------------------------
__device__ __forceinline__ float lop32(const CoefF2D& c, const float* __restrict__ x, size_t k,
                                       int pitch) {
  float v = c.cC[k] * x[k];
  v = fmaf(c.cE[k], x[k + 1], v);
  v = fmaf(c.cE[k - 1], x[k - 1], v);
  v = fmaf(c.cN[k], x[k + pitch], v);
  v = fmaf(c.cN[k - pitch], x[k - pitch], v);
  v = fmaf(c.cNE[k], x[k + pitch + 1], v);
  v = fmaf(c.cNE[k - pitch - 1], x[k - pitch - 1], v);
  return v;
}

__global__ void k_jacobi32_2d(int n, int pitch, size_t st, CoefF2D c,
                              const float* __restrict__ f, const float* __restrict__ x,
                              float* __restrict__ xo) {
  INTERIOR_2D
  xo[k] = fmaf(c.dinv[k], f[k] - lop32(c, x, k, pitch), x[k]);
}

__global__ void k_jacobi32z_2d(int n, int pitch, size_t st, CoefF2D c,
                               const float* __restrict__ f, float* __restrict__ xo) {
  INTERIOR_2D
  xo[k] = c.dinv[k] * f[k];
}

__global__ void k_residual32_2d(int n, int pitch, size_t st, CoefF2D c,
                                const float* __restrict__ f, const float* __restrict__ x,
                                float* __restrict__ r) {
  INTERIOR_2D
  r[k] = f[k] - lop32(c, x, k, pitch);
}

__global__ void k_restrict32_2d(int nc, int pc, int pf, size_t stc, size_t stf,
                                const float* __restrict__ rf, float* __restrict__ rc) {
  const int I = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nc || J >= nc) return;
  const size_t kf = blockIdx.z * stf + at(2 * I, 2 * J, pf);
  const float s = ((rf[kf + 1] + rf[kf - 1]) + (rf[kf + pf] + rf[kf - pf])) +
                  (rf[kf + pf + 1] + rf[kf - pf - 1]);
  rc[blockIdx.z * stc + at(I, J, pc)] = fmaf(0.5f, s, rf[kf]);
}

__global__ void k_prolong32_2d(int nf, int pf, int pc, size_t st, size_t stc,
                               const float* __restrict__ ec, float* __restrict__ xf) {
  const int n = nf, pitch = pf;
  INTERIOR_2D
  const int ai = i & 1, aj = j & 1;
  const size_t kc = ib * stc + at(i >> 1, j >> 1, pc);
  float e = ec[kc];
  if (ai | aj) e = 0.5f * (e + ec[kc + ai + (size_t)aj * pc]);
  xf[k] += e;
}

// ---- FP32 3D stencil kernels (Kuhn mesh, see grid3d.cu) ------------------------------------
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
  const size_t k = ib * st + (size_t)l * plane + (size_t)j * pitch + i;

__global__ void k_residual_mixed3d(int n, int pitch, size_t st, Coef3D c,
                                   const double* __restrict__ f, const double* __restrict__ x,
                                   float* __restrict__ r) {
  INTERIOR_3D
  double v = c.a[0][k] * x[k];
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    v = fma(c.a[1 + d][k], x[k + o], v);
    v = fma(c.a[1 + d][k - o], x[k - o], v);
  }
  r[k] = (float)(f[k] - v);
}

__device__ __forceinline__ float lop32_3(const CoefF3D& c, const float* __restrict__ x, size_t k,
                                         int pitch, long plane) {
  float v = c.a[0][k] * x[k];
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    v = fmaf(c.a[1 + d][k], x[k + o], v);
    v = fmaf(c.a[1 + d][k - o], x[k - o], v);
  }
  return v;
}

__global__ void k_jacobi32_3d(int n, int pitch, size_t st, CoefF3D c,
                              const float* __restrict__ f, const float* __restrict__ x,
                              float* __restrict__ xo) {
  INTERIOR_3D
  xo[k] = fmaf(c.dinv[k], f[k] - lop32_3(c, x, k, pitch, plane), x[k]);
}

__global__ void k_jacobi32z_3d(int n, int pitch, size_t st, CoefF3D c,
                               const float* __restrict__ f, float* __restrict__ xo) {
  INTERIOR_3D
  xo[k] = c.dinv[k] * f[k];
}

__global__ void k_residual32_3d(int n, int pitch, size_t st, CoefF3D c,
                                const float* __restrict__ f, const float* __restrict__ x,
                                float* __restrict__ r) {
  INTERIOR_3D
  r[k] = f[k] - lop32_3(c, x, k, pitch, plane);
}

__global__ void k_restrict32_3d(int nc, int pc, int pf, size_t stc, size_t stf,
                                const float* __restrict__ rf, float* __restrict__ rc) {
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
    s += rf[kf + o] + rf[kf - o];
  }
  rc[ib * stc + ((size_t)L * (nc + 1) + J) * pc + I] = fmaf(0.5f, s, rf[kf]);
}

__global__ void k_prolong32_3d(int nf, int pf, int pc, size_t st, size_t stc,
                               const float* __restrict__ ec, float* __restrict__ xf) {
  const int n = nf, pitch = pf;
  INTERIOR_3D
  const int ai = i & 1, aj = j & 1, al = l & 1;
  const int nc = nf / 2;
  const long planec = (long)(nc + 1) * pc;
  const size_t kc = ib * stc + (size_t)(l >> 1) * planec + (size_t)(j >> 1) * pc + (i >> 1);
  float e = ec[kc];
  if (ai | aj | al) e = 0.5f * (e + ec[kc + ai + (size_t)aj * pc + (size_t)al * planec]);
  xf[k] += e;
}

// coarsest level: y = Linv x with x, y FP32 padded level-1 vectors (FP64 accumulation); one
// CTA per instance blockIdx.x
__global__ void k_coarse32(int dim, int n, int pitch, size_t st, const double* __restrict__ Linv,
                           const float* __restrict__ x, float* __restrict__ y) {
  __shared__ double xs[1024];
  const int m = n - 1, nh = dim == 2 ? m * m : m * m * m;
  x += blockIdx.x * st;
  y += blockIdx.x * st;
  Linv += blockIdx.x * (size_t)nh * nh;
  auto idx = [&](int q) -> size_t {
    if (dim == 2) return (size_t)(1 + q / m) * pitch + 1 + q % m;
    return ((size_t)(1 + q / (m * m)) * (m + 2) + 1 + (q / m) % m) * pitch + 1 + q % m;
  };
  for (int q = threadIdx.x; q < nh; q += blockDim.x) xs[q] = (double)x[idx(q)];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  for (int p = warp; p < nh; p += warps) {
    const double* row = Linv + (size_t)p * nh;
    double s = 0.0;
    for (int q = lane; q < nh; q += 32) s = fma(row[q], xs[q], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[idx(p)] = (float)s;
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

}  // namespace

void to_f32(const double* a, float* b, size_t n, cudaStream_t s) {
  k_to_f32<<<blocks_for(n), 256, 0, s>>>(n, a, b);
}

void add_f32(const float* e, double* x, size_t n, cudaStream_t s) {
  k_add_f32<<<blocks_for(n), 256, 0, s>>>(n, e, x);
}

void residual_mixed(const Grid& g, const Coef2D& c2, const Coef3D& c3, const double* f,
                    const double* x, float* r, cudaStream_t s) {
  if (g.dim == 2)
    k_residual_mixed2d<<<grid2(g, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, c2,
                                                                     f, x, r);
  else
    k_residual_mixed3d<<<grid3(g, g.n - 1, g.n - 1, g.n - 1), blk(g), 0, s>>>(
        g.n, g.pitch, g.stride, c3, f, x, r);
}

void jacobi32(const Grid& g, const CoefF2D& c2, const CoefF3D& c3, const float* f,
              const float* x, float* xo, bool zero, cudaStream_t s) {
  if (g.dim == 2) {
    const dim3 gr = grid2(g, g.n - 1, g.n - 1);
    if (zero) k_jacobi32z_2d<<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, c2, f, xo);
    else k_jacobi32_2d<<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, c2, f, x, xo);
  } else {
    const dim3 gr = grid3(g, g.n - 1, g.n - 1, g.n - 1);
    if (zero) k_jacobi32z_3d<<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, c3, f, xo);
    else k_jacobi32_3d<<<gr, blk(g), 0, s>>>(g.n, g.pitch, g.stride, c3, f, x, xo);
  }
}

void residual32(const Grid& g, const CoefF2D& c2, const CoefF3D& c3, const float* f,
                const float* x, float* r, cudaStream_t s) {
  if (g.dim == 2)
    k_residual32_2d<<<grid2(g, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride, c2, f,
                                                                  x, r);
  else
    k_residual32_3d<<<grid3(g, g.n - 1, g.n - 1, g.n - 1), blk(g), 0, s>>>(g.n, g.pitch, g.stride,
                                                                            c3, f, x, r);
}

void restrict32(const Grid& fine, const Grid& coarse, const float* rf, float* rc,
                cudaStream_t s) {
  if (fine.dim == 2)
    k_restrict32_2d<<<grid2(fine, coarse.n - 1, coarse.n - 1), blk(fine), 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, rf, rc);
  else
    k_restrict32_3d<<<grid3(fine, coarse.n - 1, coarse.n - 1, coarse.n - 1), blk(fine), 0, s>>>(
        coarse.n, coarse.pitch, fine.pitch, coarse.stride, fine.stride, rf, rc);
}

void prolong32_add(const Grid& fine, const Grid& coarse, const float* ec, float* xf,
                   cudaStream_t s) {
  if (fine.dim == 2)
    k_prolong32_2d<<<grid2(fine, fine.n - 1, fine.n - 1), blk(fine), 0, s>>>(
        fine.n, fine.pitch, coarse.pitch, fine.stride, coarse.stride, ec, xf);
  else
    k_prolong32_3d<<<grid3(fine, fine.n - 1, fine.n - 1, fine.n - 1), blk(fine), 0, s>>>(
        fine.n, fine.pitch, coarse.pitch, fine.stride, coarse.stride, ec, xf);
}

void coarse32(const Grid& g, const double* Linv, const float* x, float* y, cudaStream_t s) {
  k_coarse32<<<g.nb, 512, 0, s>>>(g.dim, g.n, g.pitch, g.stride, Linv, x, y);
}

}  // namespace fmg
