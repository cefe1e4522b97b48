// MSE loss and its gradient (Sec. 4.3) and the Adam update (Sec. A.2).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kMseThreads = 512;
constexpr int kMsePerBlock = 4096;  // hit points per partial sum
constexpr int kMsePerThread = kMsePerBlock / kMseThreads;
constexpr int kMseFinalThreads = 256;

// Per block of kMsePerBlock hit points: the sum of squared differences over
// its valid points (float32; every thread's points in order, then a fixed
// reduction tree) and their count. The points' loads are all issued before
// the arithmetic.
__global__ void __launch_bounds__(kMseThreads)
mse_partial_kernel(int64_t m, int channels, const float* __restrict__ out,
                   const float* __restrict__ target, const uint8_t* __restrict__ valid,
                   float* __restrict__ psum, uint32_t* __restrict__ pcnt) {
  __shared__ float wsum[kMseThreads / kWarp];
  __shared__ uint32_t wcnt[kMseThreads / kWarp];
  const int64_t base = (int64_t)blockIdx.x * kMsePerBlock + threadIdx.x;
  bool ok[kMsePerThread];
#pragma unroll
  for (int r = 0; r < kMsePerThread; ++r) {
    const int64_t q = base + (int64_t)r * kMseThreads;
    ok[r] = q < m && (valid == nullptr || valid[q] != 0);
  }
  float s = 0.0f;
  uint32_t cnt = 0;
  for (int c = 0; c < channels; ++c) {
    float d[kMsePerThread];
#pragma unroll
    for (int r = 0; r < kMsePerThread; ++r) {
      const int64_t i = (int64_t)c * m + base + (int64_t)r * kMseThreads;
      d[r] = ok[r] ? out[i] - target[i] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < kMsePerThread; ++r) s = fmaf(d[r], d[r], s);
  }
#pragma unroll
  for (int r = 0; r < kMsePerThread; ++r) cnt += ok[r] ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(kFullMask, s, o);
    cnt += __shfl_xor_sync(kFullMask, cnt, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    wsum[warp] = s;
    wcnt[warp] = cnt;
  }
  __syncthreads();
  if (warp == 0) {
    s = lane < kMseThreads / kWarp ? wsum[lane] : 0.0f;
    cnt = lane < kMseThreads / kWarp ? wcnt[lane] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(kFullMask, s, o);
      cnt += __shfl_xor_sync(kFullMask, cnt, o);
    }
    if (lane == 0) {
      psum[blockIdx.x] = s;
      pcnt[blockIdx.x] = cnt;
    }
  }
}

// The partials summed in float64 in a fixed order (thread t takes partials
// t, t + 256, ..., then a fixed tree): loss = sum / count, scale = 2 / count.
__global__ void __launch_bounds__(kMseFinalThreads)
mse_final_kernel(int64_t nb, const float* __restrict__ psum, const uint32_t* __restrict__ pcnt,
                 float* __restrict__ loss, float* __restrict__ scale) {
  __shared__ double ss[kMseFinalThreads];
  __shared__ unsigned long long sc[kMseFinalThreads];
  double s = 0.0;
  unsigned long long c = 0;
  for (int64_t b = threadIdx.x; b < nb; b += kMseFinalThreads) {
    s += psum[b];
    c += pcnt[b];
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = kMseFinalThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *loss = sc[0] ? (float)(ss[0] / (double)sc[0]) : 0.0f;
    *scale = sc[0] ? (float)(2.0 / (double)sc[0]) : 0.0f;
  }
}

__global__ void mse_grad_kernel(int64_t m, int channels, const float* __restrict__ out,
                                const float* __restrict__ target,
                                const uint8_t* __restrict__ valid,
                                const float* __restrict__ scale, float* __restrict__ grad) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  const bool ok = valid == nullptr || valid[q] != 0;
  const float sc = *scale;
  for (int c = 0; c < channels; ++c) {
    const int64_t i = (int64_t)c * m + q;
    grad[i] = ok ? (out[i] - target[i]) * sc : 0.0f;
  }
}

// The four parameter tensors as one index space: element i belongs to tensor
// k with end[k-1] <= i < end[k] (in units of 4 floats when vectorised).
struct AdamArgs {
  float* p[4];
  const float* g[4];
  float* m[4];
  float* v[4];
  int64_t end[4];
  float lr[4];
  float b1, b2, eps;
  int64_t t_host;            // update index when counter is null
  const int64_t* counter;    // device count of updates applied, or null
  const DeviceHeader* guard; // an index whose flags cancel the update, or null
};

// torch.optim.Adam's update order: m += (1-b1)(g-m); v = b2 v + (1-b2) g^2;
// p -= step_size * m / (sqrt(v)/sqrt(1-b2^t) + eps)
__device__ __forceinline__ float adam_one(float g, float& m, float& v, float p, float b1, float b2,
                                          float eps, float step_size, float inv_bc2_sqrt) {
  m = fmaf(1.0f - b1, g - m, m);
  v = fmaf(1.0f - b2, g * g, b2 * v);
  const float denom = sqrtf(v) * inv_bc2_sqrt + eps;
  return p - step_size * (m / denom);
}

template <bool VEC>
__global__ void adam_kernel(AdamArgs a) {
  __shared__ float s_step[4];
  __shared__ float s_inv_bc2_sqrt;
  // gradients from an unusable build were never written: no update
  if (a.guard && index_unusable(a.guard)) return;
  if (threadIdx.x == 0) {
    const int64_t t = a.counter ? *a.counter + 1 : a.t_host;
    const double bc1 = 1.0 - pow((double)a.b1, (double)t);
    const double bc2 = 1.0 - pow((double)a.b2, (double)t);
    for (int k = 0; k < 4; ++k) s_step[k] = (float)((double)a.lr[k] / bc1);
    s_inv_bc2_sqrt = (float)(1.0 / sqrt(bc2));
  }
  __syncthreads();
  const float ib = s_inv_bc2_sqrt;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.end[3]; i += stride) {
    const int k = (i >= a.end[0]) + (i >= a.end[1]) + (i >= a.end[2]);
    const int64_t j = i - (k ? a.end[k - 1] : 0);
    const float ss = s_step[k];
    if (VEC) {
      const float4 g = reinterpret_cast<const float4*>(a.g[k])[j];
      float4 m = reinterpret_cast<float4*>(a.m[k])[j];
      float4 v = reinterpret_cast<float4*>(a.v[k])[j];
      float4 p = reinterpret_cast<float4*>(a.p[k])[j];
      p.x = adam_one(g.x, m.x, v.x, p.x, a.b1, a.b2, a.eps, ss, ib);
      p.y = adam_one(g.y, m.y, v.y, p.y, a.b1, a.b2, a.eps, ss, ib);
      p.z = adam_one(g.z, m.z, v.z, p.z, a.b1, a.b2, a.eps, ss, ib);
      p.w = adam_one(g.w, m.w, v.w, p.w, a.b1, a.b2, a.eps, ss, ib);
      reinterpret_cast<float4*>(a.p[k])[j] = p;
      reinterpret_cast<float4*>(a.m[k])[j] = m;
      reinterpret_cast<float4*>(a.v[k])[j] = v;
    } else {
      float m = a.m[k][j], v = a.v[k][j];
      a.p[k][j] = adam_one(a.g[k][j], m, v, a.p[k][j], a.b1, a.b2, a.eps, ss, ib);
      a.m[k][j] = m;
      a.v[k][j] = v;
    }
  }
}

__global__ void adam_count_kernel(int64_t* counter, const DeviceHeader* guard) {
  if (guard && index_unusable(guard)) return;
  *counter += 1;
}

}  // namespace

size_t mse_workspace_bytes(int64_t m) {
  const int64_t nb = (m + kMsePerBlock - 1) / kMsePerBlock;
  return align_up(sizeof(float) * (nb + 1)) + align_up(sizeof(uint32_t) * (nb + 1)) + 256;
}

cudaError_t launch_mse(int64_t m, int channels, const float* out, const float* target,
                       const uint8_t* valid, float* loss, float* grad, void* ws,
                       cudaStream_t stream) {
  const int64_t nb = (m + kMsePerBlock - 1) / kMsePerBlock;
  char* p = static_cast<char*>(ws);
  float* psum = reinterpret_cast<float*>(p);
  p += align_up(sizeof(float) * (nb + 1));
  uint32_t* pcnt = reinterpret_cast<uint32_t*>(p);
  p += align_up(sizeof(uint32_t) * (nb + 1));
  float* scale = reinterpret_cast<float*>(p);
  return launch_mse_parts(m, channels, out, target, valid, loss, grad, psum, pcnt, scale, stream);
}

int64_t mse_points_per_partial() { return kMsePerBlock; }

cudaError_t launch_mse_parts(int64_t m, int channels, const float* out, const float* target,
                             const uint8_t* valid, float* loss, float* grad, float* psum,
                             uint32_t* pcnt, float* scale, cudaStream_t stream) {
  const int64_t nb = (m + kMsePerBlock - 1) / kMsePerBlock;
  if (nb > 0) {
    mse_partial_kernel<<<(unsigned)nb, kMseThreads, 0, stream>>>(m, channels, out, target, valid,
                                                                 psum, pcnt);
    note_launches(1);
  }
  mse_final_kernel<<<1, kMseFinalThreads, 0, stream>>>(nb, psum, pcnt, loss, scale);
  note_launches(1);
  if (m > 0) {
    mse_grad_kernel<<<(unsigned)((m + 255) / 256), 256, 0, stream>>>(m, channels, out, target,
                                                                     valid, scale, grad);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_adam(const gpf_field& params, const gpf_field_grad& g, const gpf_field_grad& m,
                        const gpf_field_grad& v, const gpf_adam_hparams& hp,
                        const DeviceHeader* guard, cudaStream_t stream) {
  const int64_t n = params.n;
  if (n == 0) return cudaSuccess;
  AdamArgs a;
  float* P[4] = {static_cast<float*>(const_cast<void*>(params.mean)),
                 static_cast<float*>(const_cast<void*>(params.quat)),
                 static_cast<float*>(const_cast<void*>(params.logscale)),
                 static_cast<float*>(const_cast<void*>(params.spectrum))};
  const float* G[4] = {g.mean, g.quat, g.logscale, g.spectrum};
  float* Mm[4] = {m.mean, m.quat, m.logscale, m.spectrum};
  float* Vv[4] = {v.mean, v.quat, v.logscale, v.spectrum};
  const int64_t rows[4] = {3, 4, 3, params.channels};
  // float4 when every tensor holds a multiple of 4 floats on 16-byte boundaries
  bool vec = n % 4 == 0;
  for (int k = 0; k < 4; ++k)
    vec = vec && ((uintptr_t)P[k] | (uintptr_t)G[k] | (uintptr_t)Mm[k] | (uintptr_t)Vv[k]) % 16 == 0;
  const int64_t unit = vec ? 4 : 1;
  int64_t acc = 0;
  for (int k = 0; k < 4; ++k) {
    a.p[k] = P[k];
    a.g[k] = G[k];
    a.m[k] = Mm[k];
    a.v[k] = Vv[k];
    a.lr[k] = hp.lr[k];
    acc += rows[k] * n / unit;
    a.end[k] = acc;
  }
  a.b1 = hp.beta1;
  a.b2 = hp.beta2;
  a.eps = hp.eps;
  a.t_host = hp.step;
  a.counter = hp.step_counter;
  a.guard = guard;
  const int64_t blocks = std::min<int64_t>((acc + 255) / 256, 152 * 8);
  if (vec) adam_kernel<true><<<(unsigned)blocks, 256, 0, stream>>>(a);
  else adam_kernel<false><<<(unsigned)blocks, 256, 0, stream>>>(a);
  note_launches(1);
  if (hp.step_counter) {
    adam_count_kernel<<<1, 1, 0, stream>>>(hp.step_counter, guard);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace gpf
