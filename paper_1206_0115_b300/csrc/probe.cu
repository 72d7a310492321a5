// probe.cu -- FP32 arithmetic-rate microbenchmark (fmm_measure_fp32_rate).
//
// The P2P roofline is the FP32 pipe's rate, which no vendor figure on this
// part states for the clocks it actually runs at.  This kernel measures it:
// every thread runs independent FMA chains (8 scalar chains, or 4 chains of
// packed fma.rn.f32x2 pairs) long enough that launch overhead is noise, on
// 8 blocks of 256 threads per SM, so each of the SM's four schedulers has
// more independent FMAs in flight than the pipe's latency.  The chains
// x <- a x + b with 0 < a < 1 stay bounded; the result is stored only under a
// condition the compiler cannot decide, so no chain is removed.
#include <algorithm>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_fma_rate(int iters, float a, float b, float* sink) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == -1.f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_fma2_rate(int iters, float a, float b, float* sink) {
  uint64_t x[4];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  const uint64_t av = *(const uint64_t*)&a2, bv = *(const uint64_t*)&b2;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 v = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)(threadIdx.x + 4 + j) * 1e-3f);
    x[j] = *(const uint64_t*)&v;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(av), "l"(bv));
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 v = *(const float2*)&x[j];
    s += v.x + v.y;
  }
  if (s == -1.f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_measure_fp32_rate(double* out) {
  if (!out) return FMM_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* sink = nullptr;
  fmm_status st = FMM_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess ||
      pool_alloc(dev, s, (void**)&sink, sizeof(float) * (size_t)sms * PROBE_BLOCKS_PER_SM) != cudaSuccess)
    st = FMM_ERR_CUDA;
  const int blocks = sms * PROBE_BLOCKS_PER_SM;
  // about 10 ms per timed launch at the nominal rate (2 flop per FMA, 128 lanes x 2 GHz per SM)
  const int iters = 1 << 17;
  double best[2] = {0.0, 0.0};
  for (int packed = 0; packed < 2 && st == FMM_OK; ++packed) {
    for (int rep = 0; rep < 4 && st == FMM_OK; ++rep) {
      // rep 0 warms up (clocks, instruction cache)
      if (cudaEventRecord(e0, s) != cudaSuccess) st = FMM_ERR_CUDA;
      if (packed)
        k_fma2_rate<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999f, 1e-4f, sink);
      else
        k_fma_rate<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999f, 1e-4f, sink);
      float ms = 0.f;
      if (st != FMM_OK || cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = FMM_ERR_CUDA;
        break;
      }
      // scalar: 8 FMAs per iteration and thread; packed: 4 instructions of two FMAs each
      const double flop = 2.0 * 8.0 * (double)iters * PROBE_THREADS * blocks;
      if (rep > 0 && ms > 0.f) best[packed] = std::max(best[packed], flop / (ms * 1e-3));
    }
  }
  if (sink) cudaFreeAsync(sink, s);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  if (st != FMM_OK) return st;
  out[0] = best[0];
  out[1] = best[1];
  out[2] = (double)sms;
  out[3] = 0.0;
  return FMM_OK;
}
