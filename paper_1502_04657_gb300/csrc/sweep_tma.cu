// Single-precision Jacobi sweeps and residuals of the mixed-precision V-cycle on the large
// levels, fed by the Tensor Memory Accelerator.
//
// The register-blocked sweeps of mixed.cu keep only a few loads per thread in flight, which
// leaves a 12-byte-per-node stream at about a third of the HBM bandwidth.  Here each CTA is
// persistent over tiles of 128 x 16 nodes and keeps a ring of kStages tiles in shared memory:
// one thread asks the TMA for the x tile (with its one-node halo) and the f tile of the tile
// kStages ahead, and an mbarrier per stage counts the bytes in.  The bytes in flight then no
// longer depend on registers or occupancy.  The arithmetic is that of k_sweep32_2d node for
// node (coefficients rebuilt from the FP32 tables), so the two paths give the same values.
// 3D: tiles of 64 x 4 x 8 nodes, 4D tensor maps (columns, rows, planes, instances).
//
// Tensor maps (cuTensorMapEncodeTiled, from the driver through the runtime's entry-point
// query) describe a level vector as a 3D array: columns 0..n (x, innermost), rows 0..n,
// instances.  2D tile t_x covers node columns 128 t_x .. 128 t_x + 127 (so that a thread's
// four result columns are one aligned vector store).  Its f box starts at column 128 t_x; its
// x box starts 4 (FP32) or 8 (BF16) columns further left, so that every box starts on a
// 16-byte boundary as the TMA requires, and is 136 or 144 columns wide (a multiple of 16
// bytes).  Columns before 0 and columns and rows past n are zero-filled and never used.
//
// Every wait on an mbarrier is bounded.  If a wait runs out, the CTA records it in the
// launch's status word (wait_fail[instance] = 1, which the host reports as FMG_ETIMEOUT),
// writes NaN over its current tile (so no stale value passes for a result), waits a bounded
// time for its own loads still in flight and returns.  With `expire` set (a test hook) the
// tile waits give up at once, which exercises that path without any fault; the final waits
// for loads in flight always use the full bound.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "fmg_internal.h"

namespace fmg {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kTX = 128, kTY = 16;  // tile: columns x rows of nodes (wide rows: long TMA rows)
constexpr int kStages = 3;
constexpr int kThreads = 256;       // 2D: 32 groups of 4 columns x 8 pairs of rows
constexpr long kSpinLimit = 1L << 22;  // try_wait rounds before a wait counts as lost

__device__ __forceinline__ float ld(const float* p, int k) { return p[k]; }
__device__ __forceinline__ float ld(const bf16* p, int k) { return __bfloat162float(p[k]); }
__device__ __forceinline__ void st(float* p, size_t k, float v) { p[k] = v; }
__device__ __forceinline__ void st(bf16* p, size_t k, float v) { p[k] = __float2bfloat16_rn(v); }

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with parity `parity` to complete; false if it did not within
// `limit` try_wait rounds
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long limit = kSpinLimit) {
  for (long it = 0; it < limit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                         int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
      : "memory");
}

enum SweepMode { kResidual = 0, kJacobi = 1, kJacobiZero = 2 };

constexpr int round128(int b) { return (b + 127) / 128 * 128; }
// The x box of a 2D tile starts box_off columns left of the tile's first column, so that its
// start is 16-byte aligned (4 FP32 or 8 BF16 elements), and is box_w columns wide: the tile,
// the one-column halo on either side, rounded up to 16 bytes.  The f box is the tile itself.
template <typename S>
constexpr int box_off() {
  return 16 / (int)sizeof(S);
}
template <typename S>
constexpr int box_w() {
  return kTX + 2 * box_off<S>();
}
template <typename S>
constexpr int x_bytes() {  // the x box; the f box starts at the next 128-byte boundary
  return (kTY + 2) * box_w<S>() * (int)sizeof(S);
}
template <typename S>
constexpr int f_bytes() {
  return kTY * kTX * (int)sizeof(S);
}
template <typename S>
constexpr int stage_bytes() {
  return round128(x_bytes<S>()) + round128(f_bytes<S>());
}
template <typename S>
constexpr int smem_bytes() {  // the ring, the tile coordinates of each stage, one mbarrier each
  return kStages * stage_bytes<S>() + 16 * kStages + 8 * kStages;
}

// four consecutive elements from shared memory (16-byte aligned for FP32, 8 for BF16)
__device__ __forceinline__ void ld4(const float* p, int k, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p + k);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld4(const bf16* p, int k, float v[4]) {
  const uint2 t = *reinterpret_cast<const uint2*>(p + k);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&t.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&t.y);
  v[0] = __low2float(lo);
  v[1] = __high2float(lo);
  v[2] = __low2float(hi);
  v[3] = __high2float(hi);
}
// four consecutive nodes to global memory (k a multiple of 4, the vector 16-byte aligned)
__device__ __forceinline__ void st4(float* p, size_t k, const float v[4]) {
  *reinterpret_cast<float4*>(p + k) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(bf16* p, size_t k, const float v[4]) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 t;
  t.x = *reinterpret_cast<const uint32_t*>(&lo);
  t.y = *reinterpret_cast<const uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(p + k) = t;
}

// One CTA per (up to) three on an SM, persistent over the tiles blockIdx.x + k gridDim.x.
// Thread (cg, rg) = (tid % 32, tid / 32) takes tile columns 4 cg .. 4 cg + 3 (node columns
// i0 .. i0 + 3, i0 = 128 tx + 4 cg) and tile rows 2 rg, 2 rg + 1 (node rows j0, j0 + 1,
// j0 = 1 + 16 ty + 2 rg): each x row it needs is three vector loads of shared memory, its
// results two vector stores.  Node columns 0 and >= n and rows >= n are computed from clamped
// table entries and never stored.  Thread 0 issues the loads of a tile and writes its
// coordinates beside the ring, where the other threads read them before the tile's wait.
template <typename S, int MODE>
__global__ void __launch_bounds__(kThreads, 3)
    k_sweep32_tma_2d(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mf,
                     int n, int pitch, size_t st_, int tiles_x, int tiles_y, int ntiles,
                     const float* __restrict__ tab, const float* __restrict__ cst,
                     S* __restrict__ y, int* __restrict__ wait_fail, int expire) {
  constexpr int W = box_w<S>(), OFF = box_off<S>();
  extern __shared__ __align__(128) unsigned char smem[];
  int4* tinfo = reinterpret_cast<int4*>(smem + kStages * stage_bytes<S>());
  uint64_t* bar = reinterpret_cast<uint64_t*>(tinfo + kStages);
  const long limit = expire ? 0 : kSpinLimit;
  const int tid = threadIdx.x;
  const uint32_t tx_bytes = (MODE == kJacobiZero ? 0 : x_bytes<S>()) + f_bytes<S>();
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(&bar[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto issue = [&](int it) {  // thread 0: loads of the block's it-th tile into stage it % kStages
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= ntiles) return;
    const int tx = tile % tiles_x;
    const int r = tile / tiles_x;
    const int ty = r % tiles_y;
    const int ib = r / tiles_y;
    const int stage = it % kStages;
    tinfo[stage] = make_int4(tx, ty, ib, 0);
    unsigned char* base = smem + (size_t)stage * stage_bytes<S>();
    uint64_t* b = &bar[stage];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(b, tx_bytes);
    if (MODE != kJacobiZero) tma_load(base, &mx, b, tx * kTX - OFF, ty * kTY, ib);
    tma_load(base + round128(x_bytes<S>()), &mf, b, tx * kTX, 1 + ty * kTY, ib);
  };
  if (tid == 0)
    for (int it = 0; it < kStages; ++it) issue(it);
  // Orders the first stages' coordinates before their readers; later ones are written after
  // the barrier that ends an iteration and read at least one such barrier later.
  __syncthreads();

  const int c0 = 4 * (tid & 31);  // first tile column of this thread
  const int r0 = 2 * (tid >> 5);  // first tile row
  const int s = n + 1;
  int it = 0;
  for (;; ++it) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= ntiles) break;
    const int stage = it % kStages;
    const int4 ti = tinfo[stage];
    const int ib = ti.z;
    const int i0 = ti.x * kTX + c0;
    const int j0 = 1 + ti.y * kTY + r0;
    const float* X = tab + (size_t)ib * 8 * s;
    const float* Y = X + 4 * s;
    S* yb = y + (size_t)ib * st_;
    // Table entries, loaded before the wait for the tile so that their latency overlaps it:
    // xE[e], xNE[e] (E and NE x tables) belong to column i0 - 1 + e, xC[e], xN[e] to column
    // i0 + e; yN[q], yNE[q] to row j0 - 1 + q, yC[q], yE[q] to row j0 + q.
    float xC[4], xN[4], xE[5], xNE[5], yC[2], yE[2], yN[3], yNE[3];
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      const int ii = min(max(i0 - 1 + e, 0), n);
      xE[e] = X[s + ii];
      xNE[e] = X[3 * s + ii];
      if (e > 0) {
        xC[e - 1] = X[ii];
        xN[e - 1] = X[2 * s + ii];
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int jj = min(j0 - 1 + q, n);
      yN[q] = Y[2 * s + jj];
      yNE[q] = Y[3 * s + jj];
      if (q > 0) {
        yC[q - 1] = Y[jj];
        yE[q - 1] = Y[s + jj];
      }
    }
    const float w = MODE == kResidual ? 0.0f : cst[kCst * ib + kCstOmega];
    const bool ok = mbar_wait(&bar[stage], (uint32_t)((it / kStages) & 1), limit);
    const bool lost = __syncthreads_or(!ok);
    const S* xs = reinterpret_cast<const S*>(smem + (size_t)stage * stage_bytes<S>());
    const S* fs = reinterpret_cast<const S*>(smem + (size_t)stage * stage_bytes<S>() +
                                             round128(x_bytes<S>()));
    float out[2][4];
    if (lost) {
      if (tid == 0) atomicExch(&wait_fail[ib], 1);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) out[q][e] = __int_as_float(0x7fc00000);
    } else {
      float fv[2][4];
      ld4(fs, r0 * kTX + c0, fv[0]);
      ld4(fs, (r0 + 1) * kTX + c0, fv[1]);
      if (MODE == kJacobiZero) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int e = 0; e < 4; ++e) out[q][e] = __fdividef(w, xC[e] + yC[q]) * fv[q][e];
      } else {
        // x row arrays: element k is node column i0 - 1 + k (shared-memory column
        // c0 + OFF - 1 + k); tile row r0 + q + 1 is node row j0 + q
        auto row = [&](int r, float v[6]) {
          float a[4], b[4], c[4];
          ld4(xs, r * W + c0 + OFF - 4, a);
          ld4(xs, r * W + c0 + OFF, b);
          ld4(xs, r * W + c0 + OFF + 4, c);
          v[0] = a[3];
#pragma unroll
          for (int e = 0; e < 4; ++e) v[e + 1] = b[e];
          v[5] = c[0];
        };
        float rs[6], rc[6], rn[6];  // rows j - 1, j, j + 1
        row(r0, rs);
        row(r0 + 1, rc);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          row(r0 + q + 2, rn);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float cc = xC[e] + yC[q];
            float v = cc * rc[e + 1];
            v = fmaf(xE[e + 1] + yE[q], rc[e + 2], v);
            v = fmaf(xE[e] + yE[q], rc[e], v);
            v = fmaf(xN[e] + yN[q + 1], rn[e + 1], v);
            v = fmaf(xN[e] + yN[q], rs[e + 1], v);
            v = fmaf(xNE[e + 1] + yNE[q + 1], rn[e + 2], v);
            v = fmaf(xNE[e] + yNE[q], rs[e], v);
            out[q][e] = MODE == kResidual ? fv[q][e] - v
                                          : fmaf(__fdividef(w, cc), fv[q][e] - v, rc[e + 1]);
          }
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            rs[e] = rc[e];
            rc[e] = rn[e];
          }
        }
      }
    }
    // a lost wait writes NaN over the thread's nodes, so no stale value passes for a result
    const bool full = i0 >= 1 && i0 + 3 < n;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = j0 + q;
      if (j >= n) continue;
      const size_t k = (size_t)j * pitch + i0;
      if (full) {
        st4(yb, k, out[q]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (i0 + e >= 1 && i0 + e < n) st(yb, k + e, out[q][e]);
      }
    }
    if (lost) break;
    __syncthreads();  // every thread is done with this stage before it is refilled
    if (tid == 0) issue(it + kStages);
  }
  // loads still in flight (only after a lost wait, whose own tile may still be arriving):
  // wait for them a bounded time
  if (tid == 0) {
    for (int k = it; k < it + kStages; ++k) {
      const int tile = blockIdx.x + k * gridDim.x;
      if (tile >= ntiles) break;
      mbar_wait(&bar[k % kStages], (uint32_t)((k / kStages) & 1));
    }
  }
}

// ---- 3D ---------------------------------------------------------------------------------
// Tiles of 64 x 4 x 8 nodes; a thread takes (i, j) and walks the tile's 8 planes, reading the
// 15-point neighbourhood from the shared-memory tile.  Coefficients as in k_sweep32_3d: the x
// and y parts of the 15 couplings once per thread, the z table per plane.
constexpr int kTX3 = 64, kTY3 = 4, kTZ3 = 8;
constexpr int kBoxW3 = kTX3 + 8;  // 72 columns: halo + a 16-byte multiple for FP32 and BF16
constexpr int kStages3 = 3;

template <typename S>
constexpr int x_bytes3() {
  return (kTZ3 + 2) * (kTY3 + 2) * kBoxW3 * (int)sizeof(S);
}
template <typename S>
constexpr int f_bytes3() {
  return kTZ3 * kTY3 * kBoxW3 * (int)sizeof(S);
}
template <typename S>
constexpr int stage_bytes3() {
  return round128(x_bytes3<S>()) + round128(f_bytes3<S>());
}
template <typename S>
constexpr int smem_bytes3() {
  return kStages3 * stage_bytes3<S>() + 8 * kStages3;
}

__device__ constexpr int kDir3[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                                        {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
__device__ __forceinline__ constexpr int q_of3(int d, int ax) {
  return d < 3 ? (ax == d ? 1 : 2) : (d < 6 ? (ax == 5 - d ? 4 : 3) : 1);
}

__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                          int y, int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(saddr(bar))
      : "memory");
}

template <typename S, int MODE>
__global__ void __launch_bounds__(kThreads)
    k_sweep32_tma_3d(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mf,
                     int n, int pitch, size_t st_, int tiles_x, int tiles_y, int tiles_z,
                     int ntiles, const float* __restrict__ tab, const float* __restrict__ cst,
                     S* __restrict__ y, int* __restrict__ wait_fail, int expire) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kStages3 * stage_bytes3<S>());
  const long limit = expire ? 0 : kSpinLimit;
  __shared__ float sTz[5][kTZ3 + 1];  // z tables at the tile's planes l0 - 1 + p
  const int tid = threadIdx.x;
  const uint32_t tx_bytes = (MODE == kJacobiZero ? 0 : x_bytes3<S>()) + f_bytes3<S>();
  if (tid == 0) {
    for (int q = 0; q < kStages3; ++q) mbar_init(&bar[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto decode = [&](int tile, int& tx, int& ty, int& tz, int& ib) {
    tx = tile % tiles_x;
    int r = tile / tiles_x;
    ty = r % tiles_y;
    r /= tiles_y;
    tz = r % tiles_z;
    ib = r / tiles_z;
  };
  auto issue = [&](int it) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= ntiles) return;
    int tx, ty, tz, ib;
    decode(tile, tx, ty, tz, ib);
    unsigned char* base = smem + (size_t)(it % kStages3) * stage_bytes3<S>();
    uint64_t* b = &bar[it % kStages3];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(b, tx_bytes);
    if (MODE != kJacobiZero) tma_load4(base, &mx, b, tx * kTX3, ty * kTY3, tz * kTZ3, ib);
    tma_load4(base + round128(x_bytes3<S>()), &mf, b, tx * kTX3, 1 + ty * kTY3, 1 + tz * kTZ3, ib);
  };
  if (tid == 0)
    for (int it = 0; it < kStages3; ++it) issue(it);

  const int c = tid % kTX3, r = tid / kTX3;  // tile column and row of this thread
  const int s = n + 1;
  const long plane = (long)(n + 1) * pitch;
  constexpr int RW = kBoxW3, PL = (kTY3 + 2) * kBoxW3;  // x tile row and plane strides
  int it = 0;
  for (;; ++it) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= ntiles) break;
    int tx, ty, tz, ib;
    decode(tile, tx, ty, tz, ib);
    const int stage = it % kStages3;
    const int i = 1 + tx * kTX3 + c, j = 1 + ty * kTY3 + r, l0 = 1 + tz * kTZ3;
    S* yb = y + (size_t)ib * st_ + (size_t)j * pitch + i;
    const bool act = i < n && j < n;
    const float* T = tab + (size_t)ib * 15 * s;
    const float* C = cst + (size_t)kCst * ib;
    // before the wait for the tile: the z tables of its planes l0 - 1 .. l0 + kTZ3 - 1 into
    // shared memory (clamped to n) and the x and y parts of the thread's 15 coefficients
    if (tid < 5 * (kTZ3 + 1)) {
      const int q = tid / (kTZ3 + 1), p = tid % (kTZ3 + 1);
      sTz[q][p] = T[(10 + q) * s + min(l0 - 1 + p, n)];
    }
    float cxy[15];
    float w = 0.0f;
    if (act) {
      cxy[0] = T[i] + T[5 * s + j];
#pragma unroll
      for (int d = 0; d < 7; ++d)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int ci = i - (e ? kDir3[d][0] : 0), cj = j - (e ? kDir3[d][1] : 0);
          cxy[1 + 2 * d + e] = T[q_of3(d, 0) * s + ci] + T[(5 + q_of3(d, 1)) * s + cj];
        }
      w = MODE == kResidual ? 0.0f : C[kCstOmega];
    }
    const float K0 = C[0], K1 = C[1], K2 = C[2], K3 = C[3];
    const bool ok = mbar_wait(&bar[stage], (uint32_t)((it / kStages3) & 1), limit);
    const bool lost = __syncthreads_or(!ok);  // also publishes sTz
    const S* xs = reinterpret_cast<const S*>(smem + (size_t)stage * stage_bytes3<S>());
    const S* fs = reinterpret_cast<const S*>(smem + (size_t)stage * stage_bytes3<S>() +
                                             round128(x_bytes3<S>()));
    if (lost) {
      if (tid == 0) atomicExch(&wait_fail[ib], 1);
      for (int q = 0; q < kTZ3; ++q)
        if (act && l0 + q < n) st(yb, (size_t)(l0 + q) * plane, __int_as_float(0x7fc00000));
      break;
    }
    if (act) {
      const int lc = c + 1, lr = r + 1;  // the node's column and row in the x tile
#pragma unroll 2
      for (int q = 0; q < kTZ3; ++q) {
        const int l = l0 + q;
        if (l >= n) break;
        const float fv = ld(fs, (q * kTY3 + r) * kBoxW3 + lc);
        const float cc = (cxy[0] + sTz[0][q + 1]) + K0;
        float out;
        if (MODE == kJacobiZero) {
          out = __fdividef(w, cc) * fv;
        } else {
          const int k0 = (q + 1) * PL + lr * RW + lc;  // the node in the x tile
          const float xc = ld(xs, k0);
          float v = cc * xc;
#pragma unroll
          for (int d = 0; d < 7; ++d) {
            const int o = kDir3[d][0] + kDir3[d][1] * RW + kDir3[d][2] * PL;
            const float K = d < 3 ? K1 : (d < 6 ? K2 : K3);
            const float a0 = (cxy[1 + 2 * d] + sTz[q_of3(d, 2)][q + 1]) + K;
            const float a1 = (cxy[2 + 2 * d] + sTz[q_of3(d, 2)][q + 1 - kDir3[d][2]]) + K;
            v = fmaf(a0, ld(xs, k0 + o), v);
            v = fmaf(a1, ld(xs, k0 - o), v);
          }
          out = MODE == kResidual ? fv - v : fmaf(__fdividef(w, cc), fv - v, xc);
        }
        st(yb, (size_t)l * plane, out);
      }
    }
    __syncthreads();
    if (tid == 0) issue(it + kStages3);
  }
  if (tid == 0) {  // loads still in flight after a lost wait (see the 2D kernel)
    for (int k = it; k < it + kStages3; ++k) {
      const int tile = blockIdx.x + k * gridDim.x;
      if (tile >= ntiles) break;
      mbar_wait(&bar[k % kStages3], (uint32_t)((k / kStages3) & 1));
    }
  }
}

// ---- host ------------------------------------------------------------------------------
// cuTensorMapEncodeTiled (driver API, version 12.0 signature), looked up through the runtime
// so the library needs no link against the driver library
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;

EncodeTiledFn encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    else
      cudaGetLastError();
  });
  return g_encode;
}

int g_sms = 0;  // multiprocessors of the device (the persistent grids are a multiple)

int sms() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return g_sms;
}

template <typename S, int MODE>
void launch(const Grid& g, const CoefT& ct, const TMAMap& mx, const TMAMap& mf, float* y,
            int* wait_fail, int expire, cudaStream_t s) {
  const CUtensorMap& tx = *reinterpret_cast<const CUtensorMap*>(mx.bytes);
  const CUtensorMap& tf = *reinterpret_cast<const CUtensorMap*>(mf.bytes);
  const int m = g.n - 1;
  if (g.dim == 2) {
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_sweep32_tma_2d<S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<S>());
    (void)attr;
    // tile columns start at node column 0 (aligned vector stores); node columns 1 .. n - 1
    const int tiles_x = (g.n - 1) / kTX + 1, tiles_y = (m + kTY - 1) / kTY;
    const int ntiles = tiles_x * tiles_y * g.nb;
    const int cap = 3 * sms();  // 3 CTAs of 54 KB shared memory per SM
    k_sweep32_tma_2d<S, MODE><<<ntiles < cap ? ntiles : cap, kThreads, smem_bytes<S>(), s>>>(
        tx, tf, g.n, g.pitch, g.stride, tiles_x, tiles_y, ntiles, ct.tab, ct.cst,
        reinterpret_cast<S*>(y), wait_fail, expire);
  } else {
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_sweep32_tma_3d<S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes3<S>());
    (void)attr;
    const int tiles_x = (m + kTX3 - 1) / kTX3, tiles_y = (m + kTY3 - 1) / kTY3;
    const int tiles_z = (m + kTZ3 - 1) / kTZ3;
    const int ntiles = tiles_x * tiles_y * tiles_z * g.nb;
    const int cap = 2 * sms();  // 2 CTAs of 80 KB shared memory per SM
    k_sweep32_tma_3d<S, MODE><<<ntiles < cap ? ntiles : cap, kThreads, smem_bytes3<S>(), s>>>(
        tx, tf, g.n, g.pitch, g.stride, tiles_x, tiles_y, tiles_z, ntiles, ct.tab, ct.cst,
        reinterpret_cast<S*>(y), wait_fail, expire);
  }
}

}  // namespace

bool tma_sweep_applies(const Grid& g) {
  return g.n >= (g.dim == 2 ? kTMAMinCells2 : kTMAMinCells3);
}

bool encode_level_map(const Grid& g, int cap, const float* base, bool bf, bool halo,
                      TMAMap* out) {
  EncodeTiledFn enc = encoder();
  if (!enc) return false;
  static_assert(sizeof(TMAMap) == sizeof(CUtensorMap), "tensor map storage");
  const cuuint64_t es = bf ? 2 : 4;
  const cuuint64_t n1 = (cuuint64_t)g.n + 1;
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r;
  if (g.dim == 2) {
    const cuuint64_t dims[3] = {n1, n1, (cuuint64_t)cap};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.stride * es};
    const int bw = halo ? (bf ? box_w<bf16>() : box_w<float>()) : kTX;
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)(halo ? kTY + 2 : kTY), 1};
    r = enc(reinterpret_cast<CUtensorMap*>(out->bytes),
            bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
            const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[4] = {n1, n1, n1, (cuuint64_t)cap};
    const cuuint64_t strides[3] = {(cuuint64_t)g.pitch * es, n1 * g.pitch * es,
                                   (cuuint64_t)g.stride * es};
    const cuuint32_t box[4] = {(cuuint32_t)kBoxW3, (cuuint32_t)(halo ? kTY3 + 2 : kTY3),
                               (cuuint32_t)(halo ? kTZ3 + 2 : kTZ3), 1};
    r = enc(reinterpret_cast<CUtensorMap*>(out->bytes),
            bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
            const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS;
}

void sweep32_tma(const Grid& g, const CoefT& ct, const TMAMap& mx, const TMAMap& mf, float* y,
                 int mode, int* wait_fail, bool expire, cudaStream_t s, bool bf) {
  const int e = expire ? 1 : 0;
  if (bf) {
    if (mode == 0) launch<bf16, kResidual>(g, ct, mx, mf, y, wait_fail, e, s);
    else if (mode == 1) launch<bf16, kJacobi>(g, ct, mx, mf, y, wait_fail, e, s);
    else launch<bf16, kJacobiZero>(g, ct, mx, mf, y, wait_fail, e, s);
  } else {
    if (mode == 0) launch<float, kResidual>(g, ct, mx, mf, y, wait_fail, e, s);
    else if (mode == 1) launch<float, kJacobi>(g, ct, mx, mf, y, wait_fail, e, s);
    else launch<float, kJacobiZero>(g, ct, mx, mf, y, wait_fail, e, s);
  }
}

}  // namespace fmg
