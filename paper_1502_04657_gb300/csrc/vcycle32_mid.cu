// The levels of the single-precision 2D V-cycle (mixed modes) below the TMA-fed ones (at most
// kMid32MaxCells cells per side, level 2 and up) in two kernels per level instead of seven.
//
// A level of up to 256 cells per side costs its seven separate launches (the zero-start and
// second pre-smoothing sweeps, residual, restriction P^T, prolongation P, post-smoothing
// sweeps) in launch latency and memory round trips, not in work: single-precision arithmetic
// issues at 64x the FP64 rate.  Here a tile of 32 x 32 fine nodes does, in shared memory,
//   down: nu_pre damped Jacobi sweeps from zero, the residual and its restriction to the
//         coarse nodes 2I, 2J of the tile (writing the smoothed x and the coarse r), and
//   up:   x += P e_c and nu_post sweeps (writing x),
// loading its inputs with a halo wide enough for every step (2 + nu_pre nodes down, nu_post
// up) and recomputing the halo instead of exchanging it (temporal blocking).  The tiles are
// kept in the storage type S (FP32, or bfloat16 for the storage ablation) exactly where the
// separate kernels store and reload a vector, and every node is evaluated with the same FP32
// expressions in the same order as mixed.cu's k_sweep32_2d (coefficients from the per-axis
// tables: c = X[i] + Y[j]), k_restrict32_2d and k_prolong32_2d, so the results are
// bit-identical.  A tile's halo holds nodes other tiles own, so each leg reads x from one
// buffer and writes the other (the caller swaps them).
#include <cuda_bf16.h>

#include "fmg_internal.h"

namespace fmg {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kTile = 32;              // owned fine nodes per side
constexpr int kThreads = 256;
constexpr int kMaxNu = 4;              // sweeps per leg these kernels take
constexpr int kDownW = kTile + 2 * (kMaxNu + 2);
constexpr int kUpW = kTile + 2 * kMaxNu;

__device__ __forceinline__ float ldv(const float* p, size_t k) { return p[k]; }
__device__ __forceinline__ float ldv(const bf16* p, size_t k) { return __bfloat162float(p[k]); }
__device__ __forceinline__ void stv(float* p, size_t k, float v) { p[k] = v; }
__device__ __forceinline__ void stv(bf16* p, size_t k, float v) { p[k] = __float2bfloat16_rn(v); }

struct Lev32 {
  int n, pitch;
  size_t stride;
};

__device__ __forceinline__ size_t gidx(const Lev32& g, int ib, int i, int j) {
  return ib * g.stride + (size_t)j * g.pitch + i;
}

// One node of k_sweep32_2d (mode 0 residual, 1 Jacobi, 2 Jacobi from zero) at global (i, j)
// from the tile X (row length w, element e), with the instance's tables X, Y (s = n + 1
// entries each) and damping w0.
template <typename S, int MODE>
__device__ __forceinline__ float node32(const float* Xt, const float* Yt, int s, int i, int j,
                                        float w0, float fv, const S* X, int e, int w) {
  const float cc = Xt[i] + Yt[j];
  if (MODE == 2) return __fdividef(w0, cc) * fv;
  const float xe = Xt[s + i], xw = Xt[s + i - 1], xn = Xt[2 * s + i];
  const float xne = Xt[3 * s + i], xsw = Xt[3 * s + i - 1];
  const float c1 = ldv(X, e);
  float v = cc * c1;
  v = fmaf(xe + Yt[s + j], ldv(X, e + 1), v);
  v = fmaf(xw + Yt[s + j], ldv(X, e - 1), v);
  v = fmaf(xn + Yt[2 * s + j], ldv(X, e + w), v);
  v = fmaf(xn + Yt[2 * s + j - 1], ldv(X, e - w), v);
  v = fmaf(xne + Yt[3 * s + j], ldv(X, e + w + 1), v);
  v = fmaf(xsw + Yt[3 * s + j - 1], ldv(X, e - w - 1), v);
  return MODE == 0 ? fv - v : fmaf(__fdividef(w0, cc), fv - v, c1);
}

// nu Jacobi sweeps on the w x w tile whose element 0 is global (i0, j0) (zero: the first
// sweep starts from x = 0); after sweep s (from 1) the elements at distance >= s from the
// border hold the new iterate; nodes outside the domain interior stay zero.  X, XT alternate;
// returns the buffer holding the result.
template <typename S>
__device__ S* sweeps32(const Lev32& g, const float* Xt, const float* Yt, float w0, int i0, int j0,
                       int w, int nu, bool zero, S* X, S* XT, const S* F) {
  const int s = g.n + 1;
  for (int it = 0; it < nu; ++it) {
    const int b = it + 1, m = w - 2 * b;
    for (int q = threadIdx.x; q < m * m; q += kThreads) {
      const int ei = b + q % m, ej = b + q / m;
      const int i = i0 + ei, j = j0 + ej;
      const int e = ej * w + ei;
      float out = 0.0f;
      if (i >= 1 && j >= 1 && i < g.n && j < g.n) {
        const float fv = ldv(F, e);
        out = zero ? node32<S, 2>(Xt, Yt, s, i, j, w0, fv, X, e, w)
                   : node32<S, 1>(Xt, Yt, s, i, j, w0, fv, X, e, w);
      }
      stv(XT, e, out);
    }
    __syncthreads();
    S* t = X;
    X = XT;
    XT = t;
    zero = false;
  }
  return X;
}

// Down leg of level g (coarse level gc), from x = 0: xo = nu sweeps, rc = P^T (f - L xo).
template <typename S>
__global__ void __launch_bounds__(kThreads)
    k_v32down2d(Lev32 g, Lev32 gc, const float* __restrict__ tab, const float* __restrict__ cst,
                const S* __restrict__ f, S* __restrict__ xo, S* __restrict__ rc, int nu) {
  __shared__ S sX[kDownW * kDownW], sXT[kDownW * kDownW], sF[kDownW * kDownW];
  const int ib = blockIdx.z;
  const int s = g.n + 1;
  const float* Xt = tab + (size_t)ib * 8 * s;
  const float* Yt = Xt + 4 * s;
  const float w0 = cst[kCst * ib + kCstOmega];
  const int w = kTile + 2 * (nu + 2);
  const int i0 = 1 + kTile * blockIdx.x - (nu + 2), j0 = 1 + kTile * blockIdx.y - (nu + 2);
  for (int q = threadIdx.x; q < w * w; q += kThreads) {
    const int i = i0 + q % w, j = j0 + q / w;
    const bool in = i >= 1 && j >= 1 && i < g.n && j < g.n;
    sF[q] = in ? f[gidx(g, ib, i, j)] : S(0.0f);
    sX[q] = S(0.0f);
  }
  __syncthreads();
  S* X = sweeps32<S>(g, Xt, Yt, w0, i0, j0, w, nu, true, sX, sXT, sF);
  S* R = X == sX ? sXT : sX;  // the free buffer takes the residual
  {
    const int b = nu + 1, m = w - 2 * b;
    for (int q = threadIdx.x; q < m * m; q += kThreads) {
      const int ei = b + q % m, ej = b + q / m;
      const int i = i0 + ei, j = j0 + ej;
      const int e = ej * w + ei;
      float out = 0.0f;
      if (i >= 1 && j >= 1 && i < g.n && j < g.n)
        out = node32<S, 0>(Xt, Yt, s, i, j, w0, ldv(sF, e), X, e, w);
      stv(R, e, out);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kTile * kTile; q += kThreads) {
    const int i = 1 + kTile * blockIdx.x + q % kTile, j = 1 + kTile * blockIdx.y + q / kTile;
    if (i >= g.n || j >= g.n) continue;
    xo[gidx(g, ib, i, j)] = X[(j - j0) * w + (i - i0)];
  }
  constexpr int kC = kTile / 2;
  for (int q = threadIdx.x; q < kC * kC; q += kThreads) {  // k_restrict32_2d
    const int I = 1 + kC * blockIdx.x + q % kC, J = 1 + kC * blockIdx.y + q / kC;
    if (I >= gc.n || J >= gc.n) continue;
    const int kf = (2 * J - j0) * w + (2 * I - i0);
    const float sm = ((ldv(R, kf + 1) + ldv(R, kf - 1)) + (ldv(R, kf + w) + ldv(R, kf - w))) +
                     (ldv(R, kf + w + 1) + ldv(R, kf - w - 1));
    stv(rc, gidx(gc, ib, I, J), fmaf(0.5f, sm, ldv(R, kf)));
  }
}

// Up leg: xo = nu sweeps from x + P e_c.
template <typename S>
__global__ void __launch_bounds__(kThreads)
    k_v32up2d(Lev32 g, Lev32 gc, const float* __restrict__ tab, const float* __restrict__ cst,
              const S* __restrict__ f, const S* __restrict__ x, S* __restrict__ xo,
              const S* __restrict__ ec, int nu) {
  __shared__ S sX[kUpW * kUpW], sXT[kUpW * kUpW], sF[kUpW * kUpW];
  const int ib = blockIdx.z;
  const int s = g.n + 1;
  const float* Xt = tab + (size_t)ib * 8 * s;
  const float* Yt = Xt + 4 * s;
  const float w0 = cst[kCst * ib + kCstOmega];
  const int w = kTile + 2 * nu;
  const int i0 = 1 + kTile * blockIdx.x - nu, j0 = 1 + kTile * blockIdx.y - nu;
  for (int q = threadIdx.x; q < w * w; q += kThreads) {
    const int i = i0 + q % w, j = j0 + q / w;
    const bool in = i >= 1 && j >= 1 && i < g.n && j < g.n;
    S xv = S(0.0f), fv = S(0.0f);
    if (in) {
      const size_t k = gidx(g, ib, i, j);
      fv = f[k];
      // k_prolong32_2d
      const int ai = i & 1, aj = j & 1;
      const size_t kc = gidx(gc, ib, i >> 1, j >> 1);
      float e = ldv(ec, kc);
      if (ai | aj) e = 0.5f * (e + ldv(ec, kc + ai + (size_t)aj * gc.pitch));
      S t;
      stv(&t, 0, ldv(x, k) + e);
      xv = t;
    }
    sF[q] = fv;
    sX[q] = xv;
  }
  __syncthreads();
  const S* X = sweeps32<S>(g, Xt, Yt, w0, i0, j0, w, nu, false, sX, sXT, sF);
  for (int q = threadIdx.x; q < kTile * kTile; q += kThreads) {
    const int i = 1 + kTile * blockIdx.x + q % kTile, j = 1 + kTile * blockIdx.y + q / kTile;
    if (i >= g.n || j >= g.n) continue;
    xo[gidx(g, ib, i, j)] = X[(j - j0) * w + (i - i0)];
  }
}

Lev32 lev_of(const Grid& g) { return Lev32{g.n, g.pitch, g.stride}; }

dim3 tiles_of(const Grid& g) {
  const int m = g.n - 1;
  return dim3((m + kTile - 1) / kTile, (m + kTile - 1) / kTile, g.nb);
}

}  // namespace

bool vcycle32_mid_applies(const Grid& g, int nu_pre, int nu_post) {
  return g.dim == 2 && g.n <= kMid32MaxCells && nu_pre <= kMaxNu &&
         nu_post <= kMaxNu;
}

void vcycle32_down2d(const Grid& g, const CoefT& ct, const Grid& gc, const float* f, float* xo,
                     float* rc, int nu_pre, cudaStream_t s, bool bf) {
  if (bf)
    k_v32down2d<bf16><<<tiles_of(g), kThreads, 0, s>>>(
        lev_of(g), lev_of(gc), ct.tab, ct.cst, reinterpret_cast<const bf16*>(f),
        reinterpret_cast<bf16*>(xo), reinterpret_cast<bf16*>(rc), nu_pre);
  else
    k_v32down2d<float><<<tiles_of(g), kThreads, 0, s>>>(lev_of(g), lev_of(gc), ct.tab, ct.cst, f,
                                                       xo, rc, nu_pre);
}

void vcycle32_up2d(const Grid& g, const CoefT& ct, const Grid& gc, const float* f,
                   const float* x, float* xo, const float* ec, int nu_post, cudaStream_t s,
                   bool bf) {
  if (bf)
    k_v32up2d<bf16><<<tiles_of(g), kThreads, 0, s>>>(
        lev_of(g), lev_of(gc), ct.tab, ct.cst, reinterpret_cast<const bf16*>(f),
        reinterpret_cast<const bf16*>(x), reinterpret_cast<bf16*>(xo),
        reinterpret_cast<const bf16*>(ec), nu_post);
  else
    k_v32up2d<float><<<tiles_of(g), kThreads, 0, s>>>(lev_of(g), lev_of(gc), ct.tab, ct.cst, f, x,
                                                     xo, ec, nu_post);
}

}  // namespace fmg
