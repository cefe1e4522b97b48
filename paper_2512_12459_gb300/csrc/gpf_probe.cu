// gpf_measure_alu_peak: the throughput this GPU reaches on the two pipes the
// pair loops are bound by, measured rather than taken from a data sheet: the
// FP32 fused multiply-add pipe (flop/s, an FMA counted as 2 flops) and the
// special-function unit's 2^x (ex2.approx.ftz.f32, results/s), which every
// included pair of the forward and backward evaluates once.
//
// Each thread runs kChains independent dependency chains, so the issue of
// one chain's next operation never waits for its previous result; the grid
// holds kBlocksPerSM blocks of kThreads threads on every SM. The chains start
// from a value the host passes in and end in one store that depends on all of
// them (taken only when the result equals a value it cannot reach), so the
// compiler can neither fold nor drop the work.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 8;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ float g_probe_sink;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float seed, int iters) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  const float b = 0.999999f, d = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], b, d);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.0f) g_probe_sink = s;
}

__global__ void __launch_bounds__(kProbeThreads) ex2_probe_kernel(float seed, int iters) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed * (float)(c + 1) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        // x -> 2^-x maps [0, 1] into [0.5, 1]: bounded, never denormal
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-a[c]));
        a[c] = y;
      }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.0f) g_probe_sink = s;
}

}  // namespace

cudaError_t measure_alu_peak(int which, int iters, double* per_second, double* seconds) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(sms * kProbeBlocksPerSM);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    // one untimed launch (clocks up, code loaded), then the timed one
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      if (rep == 1) e = cudaEventRecord(e0, st);
      if (which == 0) fma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(1.0f, iters);
      else ex2_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(0.5f, iters);
      note_launches(1);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
      const double ops = (double)blocks * kProbeThreads * (double)iters * kUnroll * kChains;
      *seconds = ms * 1e-3;
      *per_second = (which == 0 ? 2.0 : 1.0) * ops / (ms * 1e-3);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return e;
}

}  // namespace gpf
