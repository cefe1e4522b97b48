// gpf_mse_loss_grad_noalloc: the MSE loss and its gradient for callers that
// cannot give the library any device memory of their own.
//
// gpf_mse_loss_grad needs a small scratch buffer (one partial sum and one
// count per block of 4096 hit points) and asks the caller for it. Some callers
// cannot provide one: code that runs where allocating is not permitted or not
// possible (inside a framework that owns every device allocation and offers no
// hook, or a loop that must not touch the allocator), or a C host that links
// this library without any CUDA memory management of its own. This entry
// point keeps that scratch in a fixed array in the library's own device
// memory instead, so the caller passes only its inputs and outputs.
//
// The array lives for as long as the library stays loaded, on every GPU that
// loads it (kNoAllocMaxBlocks partial sums and counts, 128 KiB in all). Every
// call shares it: two calls whose kernels overlap on the GPU (different
// streams, or devices sharing nothing) race on it, so callers must order them.
// Each call overwrites all the slots it reads, so nothing has to be cleared
// between calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPerBlock = 4096;                 // hit points per partial sum
constexpr int64_t kNoAllocMaxBlocks = 16384;           // 2^26 hit points at most

// The scratch: partial sums, partial counts and the gradient scale.
struct NoAllocScratch {
  float psum[kNoAllocMaxBlocks];
  uint32_t pcnt[kNoAllocMaxBlocks];
  float scale;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__global__ void noalloc_partial_kernel(int64_t m, int channels, const float* __restrict__ out,
                                       const float* __restrict__ target,
                                       const uint8_t* __restrict__ valid,
                                       NoAllocScratch* __restrict__ sc) {
  __shared__ float ssum[kNoAllocThreads];
  __shared__ uint32_t scnt[kNoAllocThreads];
  const int64_t base = (int64_t)blockIdx.x * kNoAllocPerBlock;
  float s = 0.0f;
  uint32_t cnt = 0;
  for (int i = threadIdx.x; i < kNoAllocPerBlock; i += kNoAllocThreads) {
    const int64_t q = base + i;
    if (q >= m) break;
    if (valid && !valid[q]) continue;
    ++cnt;
    for (int c = 0; c < channels; ++c) {
      const float d = out[(int64_t)c * m + q] - target[(int64_t)c * m + q];
      s = fmaf(d, d, s);
    }
  }
  ssum[threadIdx.x] = s;
  scnt[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = kNoAllocThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ssum[threadIdx.x] += ssum[threadIdx.x + o];
      scnt[threadIdx.x] += scnt[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sc->psum[blockIdx.x] = ssum[0];
    sc->pcnt[blockIdx.x] = scnt[0];
  }
}

// Sums the nb partials in block order (the order gpf_mse_loss_grad uses).
__global__ void noalloc_final_kernel(int64_t nb, NoAllocScratch* __restrict__ sc,
                                     float* __restrict__ loss) {
  double s = 0.0;
  uint64_t c = 0;
  for (int64_t b = 0; b < nb; ++b) {
    s += sc->psum[b];
    c += sc->pcnt[b];
  }
  *loss = c ? (float)(s / (double)c) : 0.0f;
  sc->scale = c ? (float)(2.0 / (double)c) : 0.0f;
}

__global__ void noalloc_grad_kernel(int64_t m, int channels, const float* __restrict__ out,
                                    const float* __restrict__ target,
                                    const uint8_t* __restrict__ valid,
                                    const NoAllocScratch* __restrict__ sc,
                                    float* __restrict__ grad) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  const bool ok = valid == nullptr || valid[q] != 0;
  const float sc_ = sc->scale;
  for (int c = 0; c < channels; ++c) {
    const int64_t i = (int64_t)c * m + q;
    grad[i] = ok ? (out[i] - target[i]) * sc_ : 0.0f;
  }
}

// Device address of the scratch array, looked up once per device. In host
// code the name g_noalloc_scratch only stands for the array; the address the
// kernels need comes from cudaGetSymbolAddress with the device current.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoAllocScratch* g_noalloc_ptr[kMaxDevices] = {};

cudaError_t noalloc_scratch(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

int64_t noalloc_max_points() { return kNoAllocMaxBlocks * kNoAllocPerBlock; }

cudaError_t launch_mse_noalloc(int64_t m, int channels, const float* out, const float* target,
                               const uint8_t* valid, float* loss, float* grad,
                               cudaStream_t stream) {
  NoAllocScratch* sc = nullptr;
  cudaError_t e = noalloc_scratch(&sc);
  if (e != cudaSuccess) return e;
  const int64_t nb = (m + kNoAllocPerBlock - 1) / kNoAllocPerBlock;
  if (nb > 0) {
    noalloc_partial_kernel<<<(unsigned)nb, kNoAllocThreads, 0, stream>>>(m, channels, out, target,
                                                                         valid, sc);
    note_launches(1);
  }
  noalloc_final_kernel<<<1, 1, 0, stream>>>(nb, sc, loss);
  note_launches(1);
  if (m > 0) {
    noalloc_grad_kernel<<<(unsigned)((m + 255) / 256), 256, 0, stream>>>(m, channels, out, target,
                                                                         valid, sc, grad);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace gpf
