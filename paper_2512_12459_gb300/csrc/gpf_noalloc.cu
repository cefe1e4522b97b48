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

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kNoAllocPerBlock = 4096;                 // = mse_points_per_partial()
constexpr int64_t kNoAllocMaxBlocks = 16384;           // 2^26 hit points at most

// The scratch: partial sums, partial counts and the gradient scale.
struct NoAllocScratch {
  float psum[kNoAllocMaxBlocks];
  uint32_t pcnt[kNoAllocMaxBlocks];
  float scale;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the scratch array on the current device. In host code the
// name g_noalloc_scratch only stands for the array; the address the kernels
// need comes from cudaGetSymbolAddress with the device current. It is looked
// up on every call and never cached: after cudaDeviceReset (or any other end
// of the device's context) the library's device code is loaded again and the
// array can sit at another address, so a cached pointer would go stale. Once
// the code is loaded the lookup is a host-side table search; the first call
// on a device (or in a new context) also loads the code there.
cudaError_t noalloc_scratch(NoAllocScratch** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<NoAllocScratch*>(p);
  return cudaSuccess;
}

}  // namespace

int64_t noalloc_max_points() { return kNoAllocMaxBlocks * kNoAllocPerBlock; }

cudaError_t launch_mse_noalloc(int64_t m, int channels, const float* out, const float* target,
                               const uint8_t* valid, float* loss, float* grad,
                               cudaStream_t stream) {
  if (mse_points_per_partial() != kNoAllocPerBlock) return cudaErrorInvalidConfiguration;
  NoAllocScratch* sc = nullptr;
  cudaError_t e = noalloc_scratch(&sc);
  if (e != cudaSuccess) return e;
  // the kernels of gpf_mse_loss_grad on the library's own scratch: the same
  // partial sums in the same order, so the results are equal bit for bit
  return launch_mse_parts(m, channels, out, target, valid, loss, grad, sc->psum, sc->pcnt,
                          &sc->scale, stream);
}

}  // namespace gpf
