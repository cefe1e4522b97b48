// MSE loss and its gradient (Sec. 4.3) and the Adam update (Sec. A.2).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kMseThreads = 256;
constexpr int kMsePerBlock = 4096;  // hit points per partial sum

__global__ void mse_partial_kernel(int64_t m, int channels, const float* __restrict__ out,
                                   const float* __restrict__ target,
                                   const uint8_t* __restrict__ valid, float* __restrict__ psum,
                                   uint32_t* __restrict__ pcnt) {
  __shared__ float ssum[kMseThreads];
  __shared__ uint32_t scnt[kMseThreads];
  const int64_t base = (int64_t)blockIdx.x * kMsePerBlock;
  float s = 0.0f;
  uint32_t cnt = 0;
  for (int i = threadIdx.x; i < kMsePerBlock; i += kMseThreads) {
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
  for (int o = kMseThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ssum[threadIdx.x] += ssum[threadIdx.x + o];
      scnt[threadIdx.x] += scnt[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    psum[blockIdx.x] = ssum[0];
    pcnt[blockIdx.x] = scnt[0];
  }
}

// One thread sums the partials in block order (fixed order, float64).
__global__ void mse_final_kernel(int64_t nb, const float* __restrict__ psum,
                                 const uint32_t* __restrict__ pcnt, float* __restrict__ loss,
                                 float* __restrict__ scale) {
  double s = 0.0;
  uint64_t c = 0;
  for (int64_t b = 0; b < nb; ++b) {
    s += psum[b];
    c += pcnt[b];
  }
  *loss = c ? (float)(s / (double)c) : 0.0f;
  *scale = c ? (float)(2.0 / (double)c) : 0.0f;
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

struct AdamGroup {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t count;
  float step_size;   // lr / (1 - b1^t)
};

// torch.optim.Adam's update order: m += (1-b1)(g-m); v = b2 v + (1-b2) g^2;
// p -= step_size * m / (sqrt(v)/sqrt(1-b2^t) + eps)
__global__ void adam_kernel(AdamGroup grp, float b1, float b2, float eps, float inv_bc2_sqrt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < grp.count; i += stride) {
    const float g = grp.g[i];
    float m = grp.m[i];
    float v = grp.v[i];
    m = fmaf(1.0f - b1, g - m, m);
    v = fmaf(1.0f - b2, g * g, b2 * v);
    const float denom = sqrtf(v) * inv_bc2_sqrt + eps;
    grp.p[i] = grp.p[i] - grp.step_size * (m / denom);
    grp.m[i] = m;
    grp.v[i] = v;
  }
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
  if (nb > 0) {
    mse_partial_kernel<<<(unsigned)nb, kMseThreads, 0, stream>>>(m, channels, out, target, valid,
                                                                 psum, pcnt);
    note_launches(1);
  }
  mse_final_kernel<<<1, 1, 0, stream>>>(nb, psum, pcnt, loss, scale);
  note_launches(1);
  if (m > 0) {
    mse_grad_kernel<<<(unsigned)((m + 255) / 256), 256, 0, stream>>>(m, channels, out, target,
                                                                     valid, scale, grad);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_adam(const gpf_field& params, const gpf_field_grad& g, const gpf_field_grad& m,
                        const gpf_field_grad& v, const gpf_adam_hparams& hp, cudaStream_t stream) {
  const int64_t n = params.n;
  if (n == 0) return cudaSuccess;
  const double bc1 = 1.0 - pow((double)hp.beta1, (double)hp.step);
  const double bc2 = 1.0 - pow((double)hp.beta2, (double)hp.step);
  const float inv_bc2_sqrt = (float)(1.0 / sqrt(bc2));
  float* P[4] = {const_cast<float*>(params.mean), const_cast<float*>(params.quat),
                 const_cast<float*>(params.logscale), const_cast<float*>(params.spectrum)};
  const float* G[4] = {g.mean, g.quat, g.logscale, g.spectrum};
  float* Mm[4] = {m.mean, m.quat, m.logscale, m.spectrum};
  float* Vv[4] = {v.mean, v.quat, v.logscale, v.spectrum};
  const int64_t rows[4] = {3, 4, 3, params.channels};
  for (int k = 0; k < 4; ++k) {
    AdamGroup grp{P[k], G[k], Mm[k], Vv[k], rows[k] * n, (float)(hp.lr[k] / bc1)};
    const int64_t blocks = std::min<int64_t>((grp.count + 255) / 256, 152 * 16);
    adam_kernel<<<(unsigned)blocks, 256, 0, stream>>>(grp, hp.beta1, hp.beta2, hp.eps,
                                                      inv_bc2_sqrt);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace gpf
