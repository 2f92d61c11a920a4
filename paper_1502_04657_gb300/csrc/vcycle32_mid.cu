// The levels of the single-precision V-cycle (mixed modes) below the TMA-fed ones (2D: at most
// kMid32MaxCells cells per side, 3D: kMid32MaxCells3; level 2 and up) in two kernels per level
// instead of seven.  The 2D kernels come first; the 3D ones follow the same plan on 8^3 tiles.
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

// The tile elements lo .. lo + m - 1 along one axis (tile origin o, width w) that are at
// distance >= b from the tile border and hold interior nodes 1 .. n - 1: the nodes a step
// evaluates.  Elements outside the interior are zero in every tile buffer and stay so.
__device__ __forceinline__ void span(int b, int w, int o, int n, int& lo, int& m) {
  lo = max(b, 1 - o);
  m = max(min(w - 1 - b, n - 1 - o) - lo + 1, 0);
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
// sweep starts from x = 0); after sweep s (from 1) the interior elements at distance >= s
// from the border hold the new iterate; elements outside the domain interior are zero in both
// buffers and are not written.  X, XT alternate; returns the buffer holding the result.
template <typename S>
__device__ S* sweeps32(const Lev32& g, const float* Xt, const float* Yt, float w0, int i0, int j0,
                       int w, int nu, bool zero, S* X, S* XT, const S* F) {
  const int s = g.n + 1;
  for (int it = 0; it < nu; ++it) {
    int lx, mx, ly, my;
    span(it + 1, w, i0, g.n, lx, mx);
    span(it + 1, w, j0, g.n, ly, my);
    for (int q = threadIdx.x; q < mx * my; q += kThreads) {
      const int ei = lx + q % mx, ej = ly + q / mx;
      const int i = i0 + ei, j = j0 + ej;
      const int e = ej * w + ei;
      const float fv = ldv(F, e);
      stv(XT, e, zero ? node32<S, 2>(Xt, Yt, s, i, j, w0, fv, X, e, w)
                      : node32<S, 1>(Xt, Yt, s, i, j, w0, fv, X, e, w));
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
    sXT[q] = S(0.0f);
  }
  __syncthreads();
  S* X = sweeps32<S>(g, Xt, Yt, w0, i0, j0, w, nu, true, sX, sXT, sF);
  S* R = X == sX ? sXT : sX;  // the free buffer takes the residual
  {
    int lx, mx, ly, my;
    span(nu + 1, w, i0, g.n, lx, mx);
    span(nu + 1, w, j0, g.n, ly, my);
    for (int q = threadIdx.x; q < mx * my; q += kThreads) {
      const int ei = lx + q % mx, ej = ly + q / mx;
      const int e = ej * w + ei;
      stv(R, e, node32<S, 0>(Xt, Yt, s, i0 + ei, j0 + ej, w0, ldv(sF, e), X, e, w));
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
    sXT[q] = S(0.0f);
  }
  __syncthreads();
  const S* X = sweeps32<S>(g, Xt, Yt, w0, i0, j0, w, nu, false, sX, sXT, sF);
  for (int q = threadIdx.x; q < kTile * kTile; q += kThreads) {
    const int i = 1 + kTile * blockIdx.x + q % kTile, j = 1 + kTile * blockIdx.y + q / kTile;
    if (i >= g.n || j >= g.n) continue;
    xo[gidx(g, ib, i, j)] = X[(j - j0) * w + (i - i0)];
  }
}

// ---- 3D: tiles of 8 x 8 x 8 owned nodes, at most 2 + 2 sweeps --------------------------
// The same two legs on the 3D Kuhn mesh, bit-identical to mixed.cu's k_sweep32_3d,
// k_restrict32_3d and k_prolong32_3d.  Per tile the x and y parts of the 15 coefficients of
// every column and the z tables of every plane are formed once in shared memory (the sums
// k_sweep32_3d forms per thread); a node then adds its plane's z entry and the class
// constant in the same order.
constexpr int kTile3 = 8;
constexpr int kMaxNu3 = 2;
constexpr int kW3Max = kTile3 + 2 * (kMaxNu3 + 2);  // the down leg's tile width at nu = 2

__device__ constexpr int kDir3[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                                        {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
__device__ __forceinline__ constexpr int q_of3(int d, int ax) {
  return d < 3 ? (ax == d ? 1 : 2) : (d < 6 ? (ax == 5 - d ? 4 : 3) : 1);
}

__device__ __forceinline__ size_t gidx3(const Lev32& g, int ib, int i, int j, int l) {
  return ib * g.stride + ((size_t)l * (g.n + 1) + j) * g.pitch + i;
}

template <typename S>
constexpr size_t smem3(int w) {  // x, its copy and f as S, then the coefficient tables
  return ((3 * (size_t)w * w * w * sizeof(S) + 15) / 16) * 16 +
         (15 * (size_t)w * w + 5 * (size_t)w) * sizeof(float);
}

// cxy[c * w^2 + col]: x and y parts of coefficient c of column col = ej w + ei (global i0 + ei,
// j0 + ej), c = 0 the centre, 1 + 2 d + e direction d at p (e = 0) or p - o_d (e = 1);
// tz[t * w + ez]: z table t at plane l0 + ez.  Indices outside the grid are clamped (their
// nodes are never evaluated).
__device__ void tables3(const Lev32& g, const float* __restrict__ T, int w, int i0, int j0,
                        int l0, float* cxy, float* tz) {
  const int s = g.n + 1, ww = w * w;
  auto cl = [&](int v) { return min(max(v, 0), g.n); };
  for (int q = threadIdx.x; q < ww; q += blockDim.x) {
    const int i = i0 + q % w, j = j0 + q / w;
    cxy[q] = T[cl(i)] + T[5 * s + cl(j)];
#pragma unroll
    for (int d = 0; d < 7; ++d)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int ci = cl(i - (e ? kDir3[d][0] : 0)), cj = cl(j - (e ? kDir3[d][1] : 0));
        cxy[(1 + 2 * d + e) * ww + q] = T[q_of3(d, 0) * s + ci] + T[(5 + q_of3(d, 1)) * s + cj];
      }
  }
  for (int q = threadIdx.x; q < 5 * w; q += blockDim.x) tz[q] = T[(10 + q / w) * s + cl(l0 + q % w)];
}

// One node of k_sweep32_3d at tile element e (column col, plane ez), constants K of the
// instance's classes (centre, axes, face diagonals, body diagonal) and damping w0.
template <typename S, int MODE>
__device__ __forceinline__ float node3(const float* cxy, const float* tz, int w, int col, int ez,
                                       const float (&K)[4], float w0, float fv, const S* X,
                                       int e) {
  const int ww = w * w;
  const float cc = (cxy[col] + tz[ez]) + K[0];
  if (MODE == 2) return __fdividef(w0, cc) * fv;
  const float xc = ldv(X, e);
  float v = cc * xc;
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const int o = kDir3[d][0] + kDir3[d][1] * w + kDir3[d][2] * ww;
    const float Kd = d < 3 ? K[1] : (d < 6 ? K[2] : K[3]);
    const int t = q_of3(d, 2);
    const float a0 = (cxy[(1 + 2 * d) * ww + col] + tz[t * w + ez]) + Kd;
    const float a1 = (cxy[(2 + 2 * d) * ww + col] + tz[t * w + ez - kDir3[d][2]]) + Kd;
    v = fmaf(a0, ldv(X, e + o), v);
    v = fmaf(a1, ldv(X, e - o), v);
  }
  return MODE == 0 ? fv - v : fmaf(__fdividef(w0, cc), fv - v, xc);
}

// The interior tile elements at distance >= b from the border of the w^3 tile at (i0, j0, l0).
struct Box3 {
  int lx, mx, ly, my, lz, mz;
  __device__ Box3(const Lev32& g, int b, int w, int i0, int j0, int l0) {
    span(b, w, i0, g.n, lx, mx);
    span(b, w, j0, g.n, ly, my);
    span(b, w, l0, g.n, lz, mz);
  }
  __device__ int count() const { return mx * my * mz; }
  __device__ void at(int q, int& ei, int& ej, int& ez) const {
    ei = lx + q % mx;
    ej = ly + (q / mx) % my;
    ez = lz + q / (mx * my);
  }
};

// nu Jacobi sweeps on the w^3 tile whose element 0 is global (i0, j0, l0), as sweeps32 in 2D.
template <typename S>
__device__ S* sweeps3(const Lev32& g, const float* cxy, const float* tz, const float (&K)[4],
                      float w0, int w, int i0, int j0, int l0, int nu, bool zero, S* X, S* XT,
                      const S* F) {
  for (int it = 0; it < nu; ++it) {
    const Box3 bx(g, it + 1, w, i0, j0, l0);
    for (int q = threadIdx.x; q < bx.count(); q += kThreads) {
      int ei, ej, ez;
      bx.at(q, ei, ej, ez);
      const int e = (ez * w + ej) * w + ei, col = ej * w + ei;
      const float fv = ldv(F, e);
      stv(XT, e, zero ? node3<S, 2>(cxy, tz, w, col, ez, K, w0, fv, X, e)
                      : node3<S, 1>(cxy, tz, w, col, ez, K, w0, fv, X, e));
    }
    __syncthreads();
    S* t = X;
    X = XT;
    XT = t;
    zero = false;
  }
  return X;
}

// Down leg (from x = 0): xo = nu sweeps, rc = P^T (f - L xo).  Block (tx, ty, ib * tiles + tz).
template <typename S>
__global__ void __launch_bounds__(kThreads)
    k_v32down3d(Lev32 g, Lev32 gc, const float* __restrict__ tab, const float* __restrict__ cst,
                const S* __restrict__ f, S* __restrict__ xo, S* __restrict__ rc, int nu,
                int tiles) {
  extern __shared__ __align__(16) unsigned char sm3[];
  const int w = kTile3 + 2 * (nu + 2), ww = w * w, www = ww * w;
  S* sX = reinterpret_cast<S*>(sm3);
  S* sXT = sX + www;
  S* sF = sXT + www;
  float* cxy = reinterpret_cast<float*>(sm3 + ((3 * (size_t)www * sizeof(S) + 15) / 16) * 16);
  float* tz = cxy + 15 * ww;
  const int ib = blockIdx.z / tiles, tzi = blockIdx.z - ib * tiles;
  const int s = g.n + 1;
  const float* C = cst + kCst * ib;
  const float K[4] = {C[0], C[1], C[2], C[3]};
  const float w0 = C[kCstOmega];
  const int hw = nu + 2;
  const int i0 = 1 + kTile3 * blockIdx.x - hw, j0 = 1 + kTile3 * blockIdx.y - hw,
            l0 = 1 + kTile3 * tzi - hw;
  tables3(g, tab + (size_t)ib * 15 * s, w, i0, j0, l0, cxy, tz);
  for (int q = threadIdx.x; q < www; q += kThreads) {
    const int i = i0 + q % w, j = j0 + (q / w) % w, l = l0 + q / ww;
    const bool in = i >= 1 && j >= 1 && l >= 1 && i < g.n && j < g.n && l < g.n;
    sF[q] = in ? f[gidx3(g, ib, i, j, l)] : S(0.0f);
    sX[q] = S(0.0f);
    sXT[q] = S(0.0f);
  }
  __syncthreads();
  S* X = sweeps3<S>(g, cxy, tz, K, w0, w, i0, j0, l0, nu, true, sX, sXT, sF);
  S* R = X == sX ? sXT : sX;
  {
    const Box3 bx(g, nu + 1, w, i0, j0, l0);
    for (int q = threadIdx.x; q < bx.count(); q += kThreads) {
      int ei, ej, ez;
      bx.at(q, ei, ej, ez);
      const int e = (ez * w + ej) * w + ei;
      stv(R, e, node3<S, 0>(cxy, tz, w, ej * w + ei, ez, K, w0, ldv(sF, e), X, e));
    }
  }
  __syncthreads();
  constexpr int kO = kTile3 * kTile3 * kTile3;
  for (int q = threadIdx.x; q < kO; q += kThreads) {
    const int i = 1 + kTile3 * blockIdx.x + q % kTile3;
    const int j = 1 + kTile3 * blockIdx.y + (q / kTile3) % kTile3;
    const int l = 1 + kTile3 * tzi + q / (kTile3 * kTile3);
    if (i >= g.n || j >= g.n || l >= g.n) continue;
    xo[gidx3(g, ib, i, j, l)] = X[((l - l0) * w + (j - j0)) * w + (i - i0)];
  }
  constexpr int kC = kTile3 / 2;
  for (int q = threadIdx.x; q < kC * kC * kC; q += kThreads) {  // k_restrict32_3d
    const int I = 1 + kC * blockIdx.x + q % kC, J = 1 + kC * blockIdx.y + (q / kC) % kC;
    const int L = 1 + kC * tzi + q / (kC * kC);
    if (I >= gc.n || J >= gc.n || L >= gc.n) continue;
    const int e = ((2 * L - l0) * w + (2 * J - j0)) * w + (2 * I - i0);
    float sum = 0.0f;
#pragma unroll
    for (int d = 0; d < 7; ++d) {
      const int o = kDir3[d][0] + kDir3[d][1] * w + kDir3[d][2] * ww;
      sum += ldv(R, e + o) + ldv(R, e - o);
    }
    stv(rc, gidx3(gc, ib, I, J, L), fmaf(0.5f, sum, ldv(R, e)));
  }
}

// Up leg: xo = nu sweeps from x + P e_c.
template <typename S>
__global__ void __launch_bounds__(kThreads)
    k_v32up3d(Lev32 g, Lev32 gc, const float* __restrict__ tab, const float* __restrict__ cst,
              const S* __restrict__ f, const S* __restrict__ x, S* __restrict__ xo,
              const S* __restrict__ ec, int nu, int tiles) {
  extern __shared__ __align__(16) unsigned char sm3[];
  const int w = kTile3 + 2 * nu, ww = w * w, www = ww * w;
  S* sX = reinterpret_cast<S*>(sm3);
  S* sXT = sX + www;
  S* sF = sXT + www;
  float* cxy = reinterpret_cast<float*>(sm3 + ((3 * (size_t)www * sizeof(S) + 15) / 16) * 16);
  float* tz = cxy + 15 * ww;
  const int ib = blockIdx.z / tiles, tzi = blockIdx.z - ib * tiles;
  const int s = g.n + 1;
  const float* C = cst + kCst * ib;
  const float K[4] = {C[0], C[1], C[2], C[3]};
  const float w0 = C[kCstOmega];
  const int i0 = 1 + kTile3 * blockIdx.x - nu, j0 = 1 + kTile3 * blockIdx.y - nu,
            l0 = 1 + kTile3 * tzi - nu;
  tables3(g, tab + (size_t)ib * 15 * s, w, i0, j0, l0, cxy, tz);
  const size_t planec = (size_t)(gc.n + 1) * gc.pitch;
  for (int q = threadIdx.x; q < www; q += kThreads) {
    const int i = i0 + q % w, j = j0 + (q / w) % w, l = l0 + q / ww;
    S xv = S(0.0f), fv = S(0.0f);
    if (i >= 1 && j >= 1 && l >= 1 && i < g.n && j < g.n && l < g.n) {
      const size_t k = gidx3(g, ib, i, j, l);
      fv = f[k];
      // k_prolong32_3d
      const int ai = i & 1, aj = j & 1, al = l & 1;
      const size_t kc = gidx3(gc, ib, i >> 1, j >> 1, l >> 1);
      float e = ldv(ec, kc);
      if (ai | aj | al) e = 0.5f * (e + ldv(ec, kc + ai + (size_t)aj * gc.pitch + al * planec));
      S t;
      stv(&t, 0, ldv(x, k) + e);
      xv = t;
    }
    sF[q] = fv;
    sX[q] = xv;
    sXT[q] = S(0.0f);
  }
  __syncthreads();
  const S* X = sweeps3<S>(g, cxy, tz, K, w0, w, i0, j0, l0, nu, false, sX, sXT, sF);
  constexpr int kO = kTile3 * kTile3 * kTile3;
  for (int q = threadIdx.x; q < kO; q += kThreads) {
    const int i = 1 + kTile3 * blockIdx.x + q % kTile3;
    const int j = 1 + kTile3 * blockIdx.y + (q / kTile3) % kTile3;
    const int l = 1 + kTile3 * tzi + q / (kTile3 * kTile3);
    if (i >= g.n || j >= g.n || l >= g.n) continue;
    xo[gidx3(g, ib, i, j, l)] = X[((l - l0) * w + (j - j0)) * w + (i - i0)];
  }
}

Lev32 lev_of(const Grid& g) { return Lev32{g.n, g.pitch, g.stride}; }

dim3 tiles_of(const Grid& g) {
  const int m = g.n - 1;
  return dim3((m + kTile - 1) / kTile, (m + kTile - 1) / kTile, g.nb);
}

}  // namespace

bool vcycle32_mid_applies(const Grid& g, int nu_pre, int nu_post) {
  if (g.dim == 3)  // one block row of tiles per instance and z tile: grid z = tiles * nb
    return g.n <= kMid32MaxCells3 && nu_pre <= kMaxNu3 && nu_post <= kMaxNu3 &&
           (size_t)((g.n - 2) / kTile3 + 1) * g.nb <= 65535;
  return g.dim == 2 && g.n <= kMid32MaxCells && nu_pre <= kMaxNu && nu_post <= kMaxNu;
}

void vcycle32_down(const Grid& g, const CoefT& ct, const Grid& gc, const float* f, float* xo,
                   float* rc, int nu_pre, cudaStream_t s, bool bf) {
  if (g.dim == 3) {
    const int tiles = (g.n - 1 + kTile3 - 1) / kTile3, w = kTile3 + 2 * (nu_pre + 2);
    const dim3 grid(tiles, tiles, tiles * g.nb);
    if (bf) {
      static const cudaError_t attr = cudaFuncSetAttribute(
          k_v32down3d<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3<bf16>(kW3Max));
      (void)attr;
      k_v32down3d<bf16><<<grid, kThreads, smem3<bf16>(w), s>>>(
          lev_of(g), lev_of(gc), ct.tab, ct.cst, reinterpret_cast<const bf16*>(f),
          reinterpret_cast<bf16*>(xo), reinterpret_cast<bf16*>(rc), nu_pre, tiles);
    } else {
      static const cudaError_t attr = cudaFuncSetAttribute(
          k_v32down3d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3<float>(kW3Max));
      (void)attr;
      k_v32down3d<float><<<grid, kThreads, smem3<float>(w), s>>>(
          lev_of(g), lev_of(gc), ct.tab, ct.cst, f, xo, rc, nu_pre, tiles);
    }
    return;
  }
  if (bf)
    k_v32down2d<bf16><<<tiles_of(g), kThreads, 0, s>>>(
        lev_of(g), lev_of(gc), ct.tab, ct.cst, reinterpret_cast<const bf16*>(f),
        reinterpret_cast<bf16*>(xo), reinterpret_cast<bf16*>(rc), nu_pre);
  else
    k_v32down2d<float><<<tiles_of(g), kThreads, 0, s>>>(lev_of(g), lev_of(gc), ct.tab, ct.cst, f,
                                                       xo, rc, nu_pre);
}

void vcycle32_up(const Grid& g, const CoefT& ct, const Grid& gc, const float* f,
                 const float* x, float* xo, const float* ec, int nu_post, cudaStream_t s,
                 bool bf) {
  if (g.dim == 3) {
    const int tiles = (g.n - 1 + kTile3 - 1) / kTile3, w = kTile3 + 2 * nu_post;
    const dim3 grid(tiles, tiles, tiles * g.nb);
    if (bf) {
      static const cudaError_t attr = cudaFuncSetAttribute(
          k_v32up3d<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3<bf16>(kW3Max));
      (void)attr;
      k_v32up3d<bf16><<<grid, kThreads, smem3<bf16>(w), s>>>(
          lev_of(g), lev_of(gc), ct.tab, ct.cst, reinterpret_cast<const bf16*>(f),
          reinterpret_cast<const bf16*>(x), reinterpret_cast<bf16*>(xo),
          reinterpret_cast<const bf16*>(ec), nu_post, tiles);
    } else {
      static const cudaError_t attr = cudaFuncSetAttribute(
          k_v32up3d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3<float>(kW3Max));
      (void)attr;
      k_v32up3d<float><<<grid, kThreads, smem3<float>(w), s>>>(
          lev_of(g), lev_of(gc), ct.tab, ct.cst, f, x, xo, ec, nu_post, tiles);
    }
    return;
  }
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
