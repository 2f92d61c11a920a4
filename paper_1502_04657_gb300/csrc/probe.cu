// Arithmetic-throughput probe: the FP64 (and FP32) fused multiply-add rate this GPU sustains,
// the denominator of the roofline of the FP64-bound kernels.
//
// Every thread runs C independent multiply-add chains a <- a * b + c in registers (b just
// below 1, so the values settle near c / (1 - b) and stay normal), `iters` rounds of all
// chains, on ctas_per_sm x SMs blocks of kThreads threads; the result reaches memory only
// through a store that a value test never takes, so the compiler keeps every operation and
// the probe needs no buffer.  One multiply-add counts 2 flops.  The form is the one that
// measured fastest on GB300: FP64 multiply-adds (and adds and multiplies alike) peak with 4
// chains per thread, each with its own multiplier and addend registers (1.91 of the nominal 2
// lanes per clock per SM; 8 chains reached 1.67, 16 chains 1.58, whatever the occupancy);
// FP32 with 8 chains sharing their operands (78 TFLOP/s; own operands measured 54).
#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr int kThreads = 256;
constexpr int kChains64 = 4;
constexpr int kChains32 = 8;

__device__ double g_probe_sink;

template <typename T, int C, bool OWN>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T b, T c) {
  T a[C], bk[C], ck[C];  // OWN: every chain has its own multiplier and addend
#pragma unroll
  for (int k = 0; k < C; ++k) {
    a[k] = (T)(threadIdx.x + k);
    bk[k] = OWN ? b - (T)k * (T)1e-9 : b;
    ck[k] = OWN ? c + (T)k * (T)1e-9 : c;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < C; ++k) a[k] = fma(a[k], bk[k], ck[k]);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < C; ++k) s += a[k];
  if (s == (T)-1) g_probe_sink = (double)s;  // never true: keeps the chains alive
}

}  // namespace
}  // namespace fmg

using namespace fmg;

extern "C" int fmg_eig_probe_fma(int32_t fp64, int32_t ctas_per_sm, int32_t iters, void* stream,
                                 double* ms_out, double* flops_out) {
  if (ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 || !ms_out || !flops_out)
    return FMG_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return FMG_ECUDA;
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = ctas_per_sm * sms;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return FMG_ECUDA;
  }
  auto launch = [&]() {
    if (fp64) k_fma_probe<double, kChains64, true><<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-6);
    else k_fma_probe<float, kChains32, false><<<blocks, kThreads, 0, s>>>(iters, 0.999f, 1e-3f);
  };
  launch();  // warm-up (module load, clocks)
  cudaEventRecord(e0, s);
  launch();
  cudaEventRecord(e1, s);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) {
    cudaGetLastError();
    return FMG_ECUDA;
  }
  *ms_out = ms;
  *flops_out = 2.0 * (fp64 ? kChains64 : kChains32) * (double)iters * kThreads * (double)blocks;
  return FMG_OK;
}
