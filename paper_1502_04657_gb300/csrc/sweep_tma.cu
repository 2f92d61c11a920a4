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
// instances.  A tile's boxes start at column 128 t_x, a multiple of 16 bytes for FP32 and
// BF16 as the TMA requires, and are 136 columns wide (a multiple of 16 bytes for both);
// columns and rows past n are zero-filled and never used.
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
constexpr int kBoxW = kTX + 8;      // box width in elements (halo + 16-byte multiple)
constexpr int kStages = 3;
constexpr int kThreads = 256;       // 128 columns x 2 row groups of 8 rows
constexpr int kRowsPerThread = kTY / (kThreads / kTX);
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
template <typename S>
constexpr int x_bytes() {  // the x box; the f box starts at the next 128-byte boundary
  return (kTY + 2) * kBoxW * (int)sizeof(S);
}
template <typename S>
constexpr int f_bytes() {
  return kTY * kBoxW * (int)sizeof(S);
}
template <typename S>
constexpr int stage_bytes() {
  return round128(x_bytes<S>()) + round128(f_bytes<S>());
}
template <typename S>
constexpr int smem_bytes() {  // the ring, then one mbarrier per stage
  return kStages * stage_bytes<S>() + 8 * kStages;
}

template <typename S, int MODE>
__global__ void __launch_bounds__(kThreads)
    k_sweep32_tma_2d(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mf,
                     int n, int pitch, size_t st_, int tiles_x, int tiles_y, int ntiles,
                     const float* __restrict__ tab, const float* __restrict__ cst,
                     S* __restrict__ y, int* __restrict__ wait_fail, int expire) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kStages * stage_bytes<S>());
  const long limit = expire ? 0 : kSpinLimit;
  const int tid = threadIdx.x;
  const uint32_t tx_bytes = (MODE == kJacobiZero ? 0 : x_bytes<S>()) + f_bytes<S>();
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(&bar[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // tile -> (column tile, row tile, instance)
  auto decode = [&](int tile, int& tx, int& ty, int& ib) {
    tx = tile % tiles_x;
    const int r = tile / tiles_x;
    ty = r % tiles_y;
    ib = r / tiles_y;
  };
  auto issue = [&](int it) {  // thread 0: loads of the block's it-th tile into stage it % kStages
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= ntiles) return;
    int tx, ty, ib;
    decode(tile, tx, ty, ib);
    unsigned char* base = smem + (size_t)(it % kStages) * stage_bytes<S>();
    uint64_t* b = &bar[it % kStages];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(b, tx_bytes);
    if (MODE != kJacobiZero) tma_load(base, &mx, b, tx * kTX, ty * kTY, ib);
    tma_load(base + round128(x_bytes<S>()), &mf, b, tx * kTX, 1 + ty * kTY, ib);
  };
  if (tid == 0)
    for (int it = 0; it < kStages; ++it) issue(it);

  const int c = tid % kTX;                   // tile column of this thread
  const int r0 = (tid / kTX) * kRowsPerThread;  // first tile row of this thread
  const int s = n + 1;
  int it = 0;
  for (;; ++it) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= ntiles) break;
    int tx, ty, ib;
    decode(tile, tx, ty, ib);
    const int stage = it % kStages;
    const int i = 1 + tx * kTX + c;
    const float* X = tab + (size_t)ib * 8 * s;
    const float* Y = X + 4 * s;
    S* yb = y + (size_t)ib * st_;
    const bool act = i < n;
    // The table entries of the thread's nodes are loaded before the wait for the tile, so
    // their latency overlaps it (rows past n - 1 clamped: loaded, never stored).  yN / yNE
    // at index q + 1 belong to row j0 + q; index 0 is the row below the first (S, SW).
    const int j0 = 1 + ty * kTY + r0;
    float xc = 0, xe = 0, xw = 0, xn = 0, xne = 0, xsw = 0, w = 0;
    float yC[kRowsPerThread], yE[kRowsPerThread], yN[kRowsPerThread + 1],
        yNE[kRowsPerThread + 1];
    if (act) {
      xc = X[i];
      xe = X[s + i];
      xw = X[s + i - 1];
      xn = X[2 * s + i];
      xne = X[3 * s + i];
      xsw = X[3 * s + i - 1];
      w = MODE == kResidual ? 0.0f : cst[kCst * ib + kCstOmega];
      yN[0] = Y[2 * s + j0 - 1];
      yNE[0] = Y[3 * s + j0 - 1];
#pragma unroll
      for (int q = 0; q < kRowsPerThread; ++q) {
        const int jj = min(j0 + q, n - 1);
        yC[q] = Y[jj];
        yE[q] = Y[s + jj];
        yN[q + 1] = Y[2 * s + jj];
        yNE[q + 1] = Y[3 * s + jj];
      }
    }
    const bool ok = mbar_wait(&bar[stage], (uint32_t)((it / kStages) & 1), limit);
    const bool lost = __syncthreads_or(!ok);
    const S* xs = reinterpret_cast<const S*>(smem + (size_t)stage * stage_bytes<S>());
    const S* fs = reinterpret_cast<const S*>(smem + (size_t)stage * stage_bytes<S>() +
                                             round128(x_bytes<S>()));
    if (lost) {
      if (tid == 0) atomicExch(&wait_fail[ib], 1);
      for (int q = 0; q < kRowsPerThread; ++q) {
        const int j = j0 + q;
        if (act && j < n) st(yb, (size_t)j * pitch + i, __int_as_float(0x7fc00000));
      }
      break;
    }
    if (act) {
      // x rows r0 .. r0 + kRowsPerThread + 1 of the tile are node rows j - 1 .. j + 1
      float rw[3], rc[3];  // rows j - 1 and j at columns c, c + 1, c + 2 (tile columns)
      if (MODE != kJacobiZero) {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          rw[e] = ld(xs, r0 * kBoxW + c + e);
          rc[e] = ld(xs, (r0 + 1) * kBoxW + c + e);
        }
      }
#pragma unroll
      for (int q = 0; q < kRowsPerThread; ++q) {
        const int j = j0 + q;
        const float fv = ld(fs, (r0 + q) * kBoxW + c + 1);
        const float cc = xc + yC[q];
        float out;
        if (MODE == kJacobiZero) {
          out = __fdividef(w, cc) * fv;
        } else {
          float rn[3];  // row j + 1
#pragma unroll
          for (int e = 0; e < 3; ++e) rn[e] = ld(xs, (r0 + q + 2) * kBoxW + c + e);
          float v = cc * rc[1];
          v = fmaf(xe + yE[q], rc[2], v);
          v = fmaf(xw + yE[q], rc[0], v);
          v = fmaf(xn + yN[q + 1], rn[1], v);
          v = fmaf(xn + yN[q], rw[1], v);
          v = fmaf(xne + yNE[q + 1], rn[2], v);
          v = fmaf(xsw + yNE[q], rw[0], v);
          out = MODE == kResidual ? fv - v : fmaf(__fdividef(w, cc), fv - v, rc[1]);
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            rw[e] = rc[e];
            rc[e] = rn[e];
          }
        }
        if (j < n) st(yb, (size_t)j * pitch + i, out);
      }
    }
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
    const int tiles_x = (m + kTX - 1) / kTX, tiles_y = (m + kTY - 1) / kTY;
    const int ntiles = tiles_x * tiles_y * g.nb;
    const int cap = 3 * sms();  // 3 CTAs of 56 KB shared memory per SM
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
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)(halo ? kTY + 2 : kTY), 1};
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
