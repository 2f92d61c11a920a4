// Mixed-precision multigrid iteration (precision FMG_MIXED_FP32 / FMG_MIXED_BF16): the m
// multigrid iterations of Algorithm 3.1 step 1 become an FP64 defect correction around
// single-precision V-cycles,
//     r = f - L x  (FP64 operator, stored in S),   e = V32(r),   x <- x + e  (FP64),
// so only the residual and the update touch FP64 arithmetic.  FP32 issues at ~64x the FP64
// rate on this part, which leaves the V-cycle's smoothing, residual and transfer kernels bound
// by HBM bandwidth.  Their vectors are stored in S = float or (the storage ablation)
// bfloat16, always computed in FP32.  The stencil coefficients are not stored at all: they are
// separable (2D: an x table plus a y table per coupling; 3D: a constant plus one table per
// axis, see grid2d.cu / grid3d.cu), so a sweep rebuilds them in FP32 from the level's small
// tables (L1-resident) and reads only x and f: 12 bytes per node instead of 32 (2D) or 48
// (3D).  The FP64 residual keeps the outer iteration converging to the FP64 solution of
// L x = f.
#include <cuda_bf16.h>

#include "dfloat.cuh"
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
S* sp(float* p) {
  return reinterpret_cast<S*>(p);
}
template <typename S>
const S* sp(const float* p) {
  return reinterpret_cast<const S*>(p);
}

// ---- conversions and the FP64 ends of the defect correction ----------------------------
// (contiguous over all instances: the arrays hold the instances back to back)
// double-float split of an FP64 vector (the nonlinear kernels of the mixed modes read it)
__global__ void k_split_df(size_t n, const double* __restrict__ u, float* __restrict__ hi,
                           float* __restrict__ lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double v = u[i];
    const float h = __double2float_rn(v);
    hi[i] = h;
    lo[i] = __double2float_rn(v - (double)h);
  }
}

// The split of a level vector for the double-float kernels, two elements per thread and step:
// hi = v with its significand cut to 24 bits, formed from the bit pattern by integer
// operations (|v| below the smallest normal float gives hi = 0), and lo = RN(v - hi), whose
// difference is exact: |v - hi - lo| <= 2^-24 |v - hi| <= 2^-47 |v| while lo is a normal
// float (|v| above about 1e-30, as for the rounded split).  That is one FP64-pipe operation
// per element (the subtraction; both conversions run on the integer pipes) where the split
// with hardware conversions takes four, on a pipe that retires about 2 per SM and clock.
__device__ __forceinline__ void split_trunc(double v, float& hi, float& lo) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  double hd = 0.0;
  hi = 0.0f;
  if (e >= 897 && e <= 1150) {  // a normal float exponent
    const unsigned hb = ((unsigned)((unsigned long long)b >> 32) & 0x80000000u) |
                        ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffff);
    hi = __uint_as_float(hb);
    hd = __longlong_as_double(b & ~0x1fffffffLL);
  }
  lo = d2f_rn(v - hd);
}

__global__ void k_split_u(size_t n2, const double2* __restrict__ u, float2* __restrict__ hi,
                          float2* __restrict__ lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2;
       i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = u[i];
    float2 h, l;
    split_trunc(v.x, h.x, l.x);
    split_trunc(v.y, h.y, l.y);
    hi[i] = h;
    lo[i] = l;
  }
}

template <typename S>
__global__ void k_add_s(size_t n, const S* __restrict__ e, double* __restrict__ x) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] += f2d_exact(ld(e, i));
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
  double v = fma(-c.cC[k], x[k], f[k]);  // f - L x as one chain from f
  v = fma(-c.cE[k], x[k + 1], v);
  v = fma(-c.cE[k - 1], x[k - 1], v);
  v = fma(-c.cN[k], x[k + pitch], v);
  v = fma(-c.cN[k - pitch], x[k - pitch], v);
  v = fma(-c.cNE[k], x[k + pitch + 1], v);
  v = fma(-c.cNE[k - pitch - 1], x[k - pitch - 1], v);
  st(r, k, d2f_rn(v));
}

// ---- single-precision 2D stencil kernels -----------------------------------------------------
// Sweep modes: residual r = f - L x; damped Jacobi x' = x + omega D^-1 (f - L x); the same
// from x = 0 (x' = omega D^-1 f, x not read).
enum SweepMode { kResidual = 0, kJacobi = 1, kJacobiZero = 2 };
constexpr int kRows2 = 4;  // rows per thread: four f and six x rows in flight per thread

// A thread takes column i and rows j0 .. j0 + kRows2 - 1 of instance ib = blockIdx.z.  The
// coefficients of node (i, j) come from the instance's tables (X = x tables C, E, N, NE, Y the
// y ones, s = n + 1 entries each): c = X[i] + Y[j]; the W and S couplings are those of
// (i - 1, j) and (i, j - 1).  All loads of the thread are issued before the first result is
// formed; rows past n - 1 are clamped (loaded, never stored).
template <typename S, int MODE>
__global__ void k_sweep32_2d(int n, int pitch, size_t st_, const float* __restrict__ tab,
                             const float* __restrict__ cst, const S* __restrict__ f,
                             const S* __restrict__ x, S* __restrict__ y) {
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = 1 + (blockIdx.y * blockDim.y + threadIdx.y) * kRows2;
  if (i >= n || j0 >= n) return;
  const int ib = blockIdx.z;
  const int s = n + 1;
  const float* X = tab + (size_t)ib * 8 * s;
  const float* Y = X + 4 * s;
  const size_t base = (size_t)ib * st_;
  f += base;
  x += base;
  y += base;
  float fv[kRows2];
#pragma unroll
  for (int q = 0; q < kRows2; ++q) fv[q] = ld(f, at(i, min(j0 + q, n - 1), pitch));
  float xv[kRows2 + 2][3];  // rows j0 - 1 .. j0 + kRows2, columns i - 1 .. i + 1
  if (MODE != kJacobiZero) {
#pragma unroll
    for (int q = 0; q < kRows2 + 2; ++q) {
      const size_t k = at(i, min(j0 - 1 + q, n), pitch);
      xv[q][0] = ld(x, k - 1);
      xv[q][1] = ld(x, k);
      xv[q][2] = ld(x, k + 1);
    }
  }
  const float xc = X[i], xe = X[s + i], xw = X[s + i - 1], xn = X[2 * s + i];
  const float xne = X[3 * s + i], xsw = X[3 * s + i - 1];
  const float w = MODE == kResidual ? 0.0f : cst[kCst * ib + kCstOmega];
#pragma unroll
  for (int q = 0; q < kRows2; ++q) {
    const int j = j0 + q;
    if (j < n) {
      const float cc = xc + Y[j];
      float out;
      if (MODE == kJacobiZero) {
        out = __fdividef(w, cc) * fv[q];
      } else {
        const float* r0 = xv[q];      // row j - 1
        const float* r1 = xv[q + 1];  // row j
        const float* r2 = xv[q + 2];  // row j + 1
        float v = cc * r1[1];
        v = fmaf(xe + Y[s + j], r1[2], v);
        v = fmaf(xw + Y[s + j], r1[0], v);
        v = fmaf(xn + Y[2 * s + j], r2[1], v);
        v = fmaf(xn + Y[2 * s + j - 1], r0[1], v);
        v = fmaf(xne + Y[3 * s + j], r2[2], v);
        v = fmaf(xsw + Y[3 * s + j - 1], r0[0], v);
        out = MODE == kResidual ? fv[q] - v : fmaf(__fdividef(w, cc), fv[q] - v, r1[1]);
      }
      st(y, at(i, j, pitch), out);
    }
  }
}

// four consecutive elements (FP32: 16 bytes, BF16: 8 bytes; the index a multiple of 4)
__device__ __forceinline__ void ld4v(const float* p, size_t k, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p + k);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld4v(const bf16* p, size_t k, float v[4]) {
  const uint2 t = *reinterpret_cast<const uint2*>(p + k);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&t.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&t.y);
  v[0] = __low2float(lo);
  v[1] = __high2float(lo);
  v[2] = __low2float(hi);
  v[3] = __high2float(hi);
}
__device__ __forceinline__ void st4v(float* p, size_t k, const float v[4]) {
  *reinterpret_cast<float4*>(p + k) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4v(bf16* p, size_t k, const float v[4]) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
  const __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 t;
  t.x = *reinterpret_cast<const uint32_t*>(&lo);
  t.y = *reinterpret_cast<const uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(p + k) = t;
}

// r_c = P^T r_f for coarse nodes 4Q .. 4Q + 3 of row J on one thread: fine columns
// 8Q - 4 .. 8Q + 7 of rows 2J - 1 .. 2J + 1 as three vector loads per row (inside the array:
// row 2J - 1 >= 1 starts past column 3, and rows have room past column nf + 3 or continue in
// the next row), the four results stored as one vector when all are interior.
template <typename S>
__global__ void k_restrict32_2d(int nc, int pc, int pf, size_t stc, size_t stf,
                                const S* __restrict__ rf, S* __restrict__ rc) {
  const int Q = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (4 * Q >= nc || J >= nc) return;
  const size_t k0 = blockIdx.z * stf + at(8 * Q - 4, 2 * J - 1, pf);
  float v[3][12];  // v[q][c]: fine row 2J - 1 + q, column 8Q - 4 + c
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) ld4v(rf, k0 + (size_t)q * pf + 4 * c, &v[q][4 * c]);
  float out[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {  // coarse node 4Q + d: fine centre column 8Q + 2d
    const int c = 4 + 2 * d;
    const float sum = ((v[1][c + 1] + v[1][c - 1]) + (v[2][c] + v[0][c])) +
                      (v[2][c + 1] + v[0][c - 1]);
    out[d] = fmaf(0.5f, sum, v[1][c]);
  }
  const size_t ko = blockIdx.z * stc + at(4 * Q, J, pc);
  if (Q > 0 && 4 * Q + 3 < nc) {
    st4v(rc, ko, out);
  } else {
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (4 * Q + d >= 1 && 4 * Q + d < nc) st(rc, ko + d, out[d]);
  }
}

// x_f += P e_c for fine columns 4P .. 4P + 3 of rows 2J and 2J + 1 (coarse cells 2P, 2P + 1
// of row J) on one thread: six coarse values (columns past nc clamped: their fine nodes are
// not written), two vector loads and stores of x; column 0 and row 0 are not written.
template <typename S>
__global__ void k_prolong32_2d(int nc, int pf, int pc, size_t st_, size_t stc,
                               const S* __restrict__ ec, S* __restrict__ xf) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int nf = 2 * nc;
  if (4 * P >= nf || J >= nc) return;
  const size_t kc = blockIdx.z * stc + at(0, J, pc);
  float e0[3], e1[3];  // coarse rows J, J + 1 at columns 2P, 2P + 1, 2P + 2
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int I = min(2 * P + c, nc);
    e0[c] = ld(ec, kc + I);
    e1[c] = ld(ec, kc + pc + I);
  }
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    if (b == 0 && J == 0) continue;
    const size_t k = blockIdx.z * st_ + at(4 * P, 2 * J + b, pf);
    float x[4];
    ld4v(xf, k, x);
#pragma unroll
    for (int a = 0; a < 4; ++a) {  // fine column 4P + a: cell 2P + (a >> 1), offset a & 1
      const int c = a >> 1, ai = a & 1;
      float e = e0[c];
      if (ai | b) e = 0.5f * (e + (b == 0 ? e0[c + 1] : (ai ? e1[c + 1] : e1[c])));
      x[a] = x[a] + e;
    }
    if (P > 0 && 4 * P + 3 < nf) {
      st4v(xf, k, x);
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a)
        if (4 * P + a >= 1 && 4 * P + a < nf) st(xf, k + a, x[a]);
    }
  }
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
  double v = fma(-c.a[0][k], x[k], f[k]);  // f - L x as one chain from f
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const long o = dir_off(d, pitch, plane);
    v = fma(-c.a[1 + d][k], x[k + o], v);
    v = fma(-c.a[1 + d][k - o], x[k - o], v);
  }
  st(r, k, d2f_rn(v));
}

// Coefficients of a 3D node p from the instance's tables T(ax, q)[c] = tab[(ax 5 + q) s + c]
// (s = n + 1) and constants cst = (C, axis, face, body), as in grid3d.cu:
//   C = cst0 + T(x,0) + T(y,0) + T(z,0);  axis d: cst1 + T(d,1) + sum_{ax != d} T(ax,2);
//   face with third axis o: cst2 + T(o,4) + sum_{ax != o} T(ax,3);  body: cst3 + sum T(ax,1).
// The coupling to p - o_d is the one of p - o_d to p.  q_of(d, ax) is the table a direction
// takes on an axis.  In FP32 the sum runs ((T(x) + T(y)) + T(z)) + constant: the constant
// (6h, -h) is much larger than the potential terms, and adding it last keeps each
// coefficient one rounding from its FP64 value (see CoefT in fmg_internal.h).
__device__ __forceinline__ constexpr int q_of(int d, int ax) {
  return d < 3 ? (ax == d ? 1 : 2) : (d < 6 ? (ax == 5 - d ? 4 : 3) : 1);
}
constexpr int kPlanes3 = 4;  // planes per thread

// A thread takes (i, j) and planes l0 .. l0 + kPlanes3 - 1 of instance ib, blockIdx.z =
// ib * chunks + (l0 - 1) / kPlanes3.  The x and y parts of its 15 coefficients (the centre and
// both ends of the 7 directions) are summed once; each plane adds its z-table entries and
// then the class constants.
template <typename S, int MODE>
__global__ void k_sweep32_3d(int n, int pitch, size_t st_, int chunks,
                             const float* __restrict__ tab, const float* __restrict__ cst,
                             const S* __restrict__ f, const S* __restrict__ x,
                             S* __restrict__ y) {
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int ib = blockIdx.z / chunks;
  const int l0 = 1 + ((int)blockIdx.z - ib * chunks) * kPlanes3;
  if (i >= n || j >= n) return;
  const int s = n + 1;
  const float* T = tab + (size_t)ib * 15 * s;
  const float* C = cst + kCst * ib;
  const long plane = (long)(n + 1) * pitch;
  const size_t base = (size_t)ib * st_;
  const size_t col = (size_t)j * pitch + i;  // (i, j) in plane 0
  f += base;
  x += base;
  y += base;
  float fv[kPlanes3];
#pragma unroll
  for (int q = 0; q < kPlanes3; ++q) fv[q] = ld(f, (size_t)min(l0 + q, n - 1) * plane + col);
  // x and y parts: cxy[0] the centre, cxy[1 + 2 d + e] direction d at p (e = 0) or p - o_d
  float cxy[15];
  cxy[0] = T[i] + T[5 * s + j];
#pragma unroll
  for (int d = 0; d < 7; ++d)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int ci = i - (e ? kDir[d][0] : 0), cj = j - (e ? kDir[d][1] : 0);
      cxy[1 + 2 * d + e] = T[q_of(d, 0) * s + ci] + T[(5 + q_of(d, 1)) * s + cj];
    }
  const float w = MODE == kResidual ? 0.0f : C[kCstOmega];
  const float* Tz = T + 10 * s;
  const float K0 = C[0], K1 = C[1], K2 = C[2], K3 = C[3];
#pragma unroll
  for (int q = 0; q < kPlanes3; ++q) {
    const int l = min(l0 + q, n - 1);  // planes past n - 1: computed on n - 1, not stored
    const size_t k = (size_t)l * plane + col;
    const float cc = (cxy[0] + Tz[l]) + K0;
    float out;
    if (MODE == kJacobiZero) {
      out = __fdividef(w, cc) * fv[q];
    } else {
      float v = cc * ld(x, k);
#pragma unroll
      for (int d = 0; d < 7; ++d) {
        const long o = dir_off(d, pitch, plane);
        const float K = d < 3 ? K1 : (d < 6 ? K2 : K3);
        const float a0 = (cxy[1 + 2 * d] + Tz[q_of(d, 2) * s + l]) + K;
        const float a1 = (cxy[2 + 2 * d] + Tz[q_of(d, 2) * s + l - kDir[d][2]]) + K;
        v = fmaf(a0, ld(x, k + o), v);
        v = fmaf(a1, ld(x, k - o), v);
      }
      out = MODE == kResidual ? fv[q] - v : fmaf(__fdividef(w, cc), fv[q] - v, ld(x, k));
    }
    if (l0 + q < n) st(y, k, out);
  }
}

// per-instance constants of the single-precision sweeps: omega and, in 3D, the constant parts
// of the coefficients (grid3d.cu's k_coef3d): C, axis, face, body; wl = 0 drops W (the
// paper-literal form)
__device__ __forceinline__ void put_split(float* c, int hi, int lo, double v) {
  const float f = __double2float_rn(v);
  c[hi] = f;
  c[lo] = __double2float_rn(v - (double)f);
}

__global__ void k_consts(int dim, int nb, double h, const PotentialParams* __restrict__ pp,
                         float* __restrict__ cst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const PotentialParams p = pp[b];
  float* c = cst + kCst * b;
  put_split(c, kCstOmega, kCstOmegaLo, p.omega);
  if (dim == 3) {
    const double wl = p.operator_form == FMG_W_LEFT ? 1.0 : 0.0;
    const double h3w = wl * h * h * h * p.w0;
    put_split(c, 0, kCstLo + 0, 6.0 * h + 0.4 * h3w);
    put_split(c, 1, kCstLo + 1, -h + h3w * (1.0 / 20.0));
    put_split(c, 2, kCstLo + 2, h3w * (1.0 / 30.0));
    put_split(c, 3, kCstLo + 3, h3w * (1.0 / 20.0));
  }
}

// r_c = P^T r_f for coarse nodes 4Q .. 4Q + 3 of row (J, L) on one thread: each of the seven
// fine rows they touch (rows 2J + dy of planes 2L + dz) read as vectors over columns
// 8Q - 4 .. 8Q + 7 (inside the array, as in the 2D kernel); per node the sums run in
// direction order as in a node-by-node evaluation.
template <typename S>
__global__ void k_restrict32_3d(int nc, int pc, int pf, size_t stc, size_t stf,
                                const S* __restrict__ rf, S* __restrict__ rc) {
  const int Q = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int ib = blockIdx.z / (nc - 1);
  const int L = 1 + (int)blockIdx.z - ib * (nc - 1);
  if (4 * Q >= nc || J >= nc) return;
  const long planef = (long)(2 * nc + 1) * pf;
  const size_t base = ib * stf + (size_t)(2 * L) * planef + (size_t)(2 * J) * pf + 8 * Q - 4;
  constexpr int kRow[7][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}, {-1, 0}, {0, -1}, {-1, -1}};
  constexpr int kPlus[7] = {0, 1, 2, 1, 2, 3, 3};
  constexpr int kMinus[7] = {0, 4, 5, 4, 5, 6, 6};
  constexpr int kDx[7] = {1, 0, 0, 1, 1, 0, 1};
  float v[7][12];  // v[r][c]: fine row kRow[r] at column 8Q - 4 + c
#pragma unroll
  for (int r = 0; r < 7; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      ld4v(rf, base + (long)kRow[r][0] * pf + (long)kRow[r][1] * planef + 4 * c, &v[r][4 * c]);
  float out[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {  // coarse node 4Q + d: fine centre column 8Q + 2d
    const int c = 4 + 2 * d;
    float sum = 0.0f;
#pragma unroll
    for (int q = 0; q < 7; ++q) sum += v[kPlus[q]][c + kDx[q]] + v[kMinus[q]][c - kDx[q]];
    out[d] = fmaf(0.5f, sum, v[0][c]);
  }
  const size_t ko = ib * stc + ((size_t)L * (nc + 1) + J) * pc + 4 * Q;
  if (Q > 0 && 4 * Q + 3 < nc) {
    st4v(rc, ko, out);
  } else {
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (4 * Q + d >= 1 && 4 * Q + d < nc) st(rc, ko + d, out[d]);
  }
}

// x_f += P e_c for fine columns 4P .. 4P + 3 of the four fine rows (2J + aj, 2L + al) of coarse
// cells (2P, J, L), (2P + 1, J, L) on one thread: twelve coarse values (columns past nc
// clamped: their fine nodes are not written), vector loads and stores of x; column, row and
// plane 0 are not written.
template <typename S>
__global__ void k_prolong32_3d(int nc, int pf, int pc, size_t st_, size_t stc,
                               const S* __restrict__ ec, S* __restrict__ xf) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int ib = blockIdx.z / nc;
  const int L = (int)blockIdx.z - ib * nc;
  const int nf = 2 * nc;
  if (4 * P >= nf || J >= nc) return;
  const long planec = (long)(nc + 1) * pc;
  const long planef = (long)(nf + 1) * pf;
  const size_t kc = ib * stc + (size_t)L * planec + (size_t)J * pc;
  float e[2][2][3];  // e[al][aj][c] = e_c(2P + c, J + aj, L + al)
#pragma unroll
  for (int al = 0; al < 2; ++al)
#pragma unroll
    for (int aj = 0; aj < 2; ++aj)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        e[al][aj][c] = ld(ec, kc + (size_t)al * planec + (size_t)aj * pc + min(2 * P + c, nc));
#pragma unroll
  for (int al = 0; al < 2; ++al)
#pragma unroll
    for (int aj = 0; aj < 2; ++aj) {
      if ((al == 0 && L == 0) || (aj == 0 && J == 0)) continue;
      const size_t k = ib * st_ + (size_t)(2 * L + al) * planef + (size_t)(2 * J + aj) * pf + 4 * P;
      float x[4];
      ld4v(xf, k, x);
#pragma unroll
      for (int a = 0; a < 4; ++a) {  // fine column 4P + a: cell 2P + (a >> 1), offset a & 1
        const int c = a >> 1, ai = a & 1;
        float v = e[0][0][c];
        if (ai | aj | al) v = 0.5f * (v + e[al][aj][c + ai]);
        x[a] = x[a] + v;
      }
      if (P > 0 && 4 * P + 3 < nf) {
        st4v(xf, k, x);
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (4 * P + a >= 1 && 4 * P + a < nf) st(xf, k + a, x[a]);
      }
    }
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

template <typename S, int MODE>
void sweep_t(const Grid& g, const CoefT& ct, const float* f, const float* x, float* y,
             cudaStream_t s) {
  const int m = g.n - 1;
  if (g.dim == 2) {
    k_sweep32_2d<S, MODE><<<grid2(g, m, (m + kRows2 - 1) / kRows2), blk(g), 0, s>>>(
        g.n, g.pitch, g.stride, ct.tab, ct.cst, sp<S>(f), sp<S>(x), sp<S>(y));
  } else {
    const int chunks = (m + kPlanes3 - 1) / kPlanes3;
    k_sweep32_3d<S, MODE><<<grid3(g, m, m, chunks), blk(g), 0, s>>>(
        g.n, g.pitch, g.stride, chunks, ct.tab, ct.cst, sp<S>(f), sp<S>(x), sp<S>(y));
  }
}

template <typename S>
void jacobi_t(const Grid& g, const CoefT& ct, const float* f, const float* x, float* xo,
              bool zero, cudaStream_t s) {
  if (zero) sweep_t<S, kJacobiZero>(g, ct, f, x, xo, s);
  else sweep_t<S, kJacobi>(g, ct, f, x, xo, s);
}

template <typename S>
void restrict_t(const Grid& fine, const Grid& coarse, const float* rf, float* rc, cudaStream_t s) {
  if (fine.dim == 2)
    k_restrict32_2d<S><<<dim3((coarse.n / 4 + 32) / 32, (coarse.n - 1 + 7) / 8, fine.nb),
                         dim3(32, 8), 0, s>>>(coarse.n, coarse.pitch, fine.pitch, coarse.stride,
                                              fine.stride, sp<S>(rf), sp<S>(rc));
  else
    k_restrict32_3d<S><<<dim3((coarse.n / 4 + 32) / 32, (coarse.n - 1 + 7) / 8,
                              (coarse.n - 1) * fine.nb),
                         dim3(32, 8), 0, s>>>(coarse.n, coarse.pitch, fine.pitch, coarse.stride,
                                              fine.stride, sp<S>(rf), sp<S>(rc));
}

template <typename S>
void prolong_t(const Grid& fine, const Grid& coarse, const float* ec, float* xf, cudaStream_t s) {
  if (fine.dim == 2)
    k_prolong32_2d<S><<<dim3(((fine.n + 3) / 4 + 31) / 32, (coarse.n + 7) / 8, fine.nb),
                        dim3(32, 8), 0, s>>>(coarse.n, fine.pitch, coarse.pitch, fine.stride,
                                             coarse.stride, sp<S>(ec), sp<S>(xf));
  else
    k_prolong32_3d<S><<<dim3(((fine.n + 3) / 4 + 31) / 32, (coarse.n + 7) / 8,
                             coarse.n * fine.nb),
                        dim3(32, 8), 0, s>>>(coarse.n, fine.pitch, coarse.pitch, fine.stride,
                                             coarse.stride, sp<S>(ec), sp<S>(xf));
}

}  // namespace

size_t mixed_elem_bytes(bool bf16_storage) { return bf16_storage ? sizeof(bf16) : sizeof(float); }

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

void tables_f32(const Grid& g, const Coef2D& c2, const Coef3D& c3,
                const PotentialParams* pp, const CoefT& ct, cudaStream_t s) {
  const size_t n = (size_t)(g.dim == 2 ? 8 : 15) * (g.n + 1) * g.nb;
  k_split_df<<<blocks_for(n), 256, 0, s>>>(n, g.dim == 2 ? c2.tab : c3.tab, ct.tab, ct.tablo);
  k_consts<<<(g.nb + 127) / 128, 128, 0, s>>>(g.dim, g.nb, g.h, pp, ct.cst);
}

void split_df(const double* u, float* hi, float* lo, size_t n, cudaStream_t s) {
  // n is a whole number of level vectors (rows of a multiple of 32 elements): even, and the
  // arrays are allocation-aligned
  k_split_u<<<blocks_for(n / 2), 256, 0, s>>>(n / 2, reinterpret_cast<const double2*>(u),
                                              reinterpret_cast<float2*>(hi),
                                              reinterpret_cast<float2*>(lo));
}

void jacobi32(const Grid& g, const CoefT& ct, const float* f, const float* x, float* xo,
              bool zero, cudaStream_t s, bool bf) {
  if (bf) jacobi_t<bf16>(g, ct, f, x, xo, zero, s);
  else jacobi_t<float>(g, ct, f, x, xo, zero, s);
}

void residual32(const Grid& g, const CoefT& ct, const float* f, const float* x, float* r,
                cudaStream_t s, bool bf) {
  if (bf) sweep_t<bf16, kResidual>(g, ct, f, x, r, s);
  else sweep_t<float, kResidual>(g, ct, f, x, r, s);
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
