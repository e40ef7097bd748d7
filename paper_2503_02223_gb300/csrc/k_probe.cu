// Throughput probes of the two arithmetic pipes the blend kernels are bound by: FP32
// fused multiply-add and the special-function unit's 2^x.  They give the measured peaks
// the blend kernels' FP32 roofline fractions are quoted against (no vendor figure is
// assumed).  Each thread runs kChains independent dependency chains, so with every SM
// full (2048 threads) neither the pipe's latency nor issue order limits the rate.
#include "dqo_internal.cuh"

namespace dqo {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

// a <- a * m + c on kProbeChains chains, kProbeUnroll steps per iteration; m < 1 keeps
// every chain bounded.  The sum is stored only if it equals a value it cannot reach, so
// the work stays live without a store per thread.
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, float seed, float* __restrict__ sink) {
  float a[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) a[i] = seed + 1e-3f * (float)(threadIdx.x + i);
  const float m = 0.9999f, c = 1e-4f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k)
#pragma unroll
      for (int i = 0; i < kProbeChains; ++i) a[i] = __fmaf_rn(a[i], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += a[i];
  if (s == -1.f) sink[0] = s;
}

// a <- 2^(-a): for a > 0 the chain stays in (0, 1).
__global__ void __launch_bounds__(kProbeThreads) k_ex2_probe(int iters, float seed, float* __restrict__ sink) {
  float a[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) a[i] = seed + 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k)
#pragma unroll
      for (int i = 0; i < kProbeChains; ++i) a[i] = ex2_approx(-a[i]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += a[i];
  if (s == -1.f) sink[0] = s;
}

}  // namespace

cudaError_t launch_alu_probe(int kind, int iters, float* sink, double* ops, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)(sms * kProbeBlocksPerSm)), block(kProbeThreads);
  const double per_thread = (double)iters * kProbeUnroll * kProbeChains;
  const double threads = (double)grid.x * kProbeThreads;
  if (kind == 0) {
    k_fma_probe<<<grid, block, 0, s>>>(iters, 0.5f, sink);
    *ops = 2.0 * per_thread * threads;   // an FMA is two flops
  } else {
    k_ex2_probe<<<grid, block, 0, s>>>(iters, 0.5f, sink);
    *ops = per_thread * threads;
  }
  return cudaGetLastError();
}

}  // namespace dqo

extern "C" dqo_status dqo_alu_probe(int32_t kind, int32_t iters, float* sink, double* ops, dqo_stream stream) {
  if ((kind != 0 && kind != 1) || iters < 1 || !sink || !ops) return DQO_EINVAL;
  return dqo::launch_alu_probe(kind, iters, sink, ops, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? DQO_OK
             : DQO_ECUDA;
}
