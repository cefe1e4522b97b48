// gpf_radiance_bwd: gradient of the hit-point radiance with respect to every
// Gaussian parameter (Sec. 4.2, Differentiable Accumulation).
//
// Chain rule for a pair (Gaussian i, hit point x) with w = exp(-Q/2) psi:
//   d loss / d w   = beta = zeta (sum_c gamma_c Phi_c - kappa)
//       gamma_c = g_c rho_c;  SUM: zeta = 1, kappa = 0;
//       NORMALIZED: zeta = 1/Z, kappa = sum_c g_c O_c (zeta = 1/eps, kappa = 0 when Z <= eps)
//   d loss / d Phi_c += gamma_c zeta w
//   dw/dl_j = w u_j^2, dw/dR_kj = -w u_j d_k / s_j, dw/dmu = w M^T u + w 6t/(r' |d|) d
// Per Gaussian the warp accumulates
//   A = sum beta w u u^T (6 floats), B = sum beta w u, D = sum beta w 6t/(r'|d|) d, dPhi
// and the epilogue turns them into gradients, using d = R S u:
//   d mu = M^T B + D,  d l_j = A_jj,  dR_kj = -(1/s_j) sum_m R_km s_m A_jm,
//   dq from dR through R(qhat) and qhat = q/|q|.
// Traversal is Gaussian-major: one warp per Gaussian, Gaussians in the order
// of the query-level cell of their mean (neighbouring warps share hit points
// in cache). The warp visits the hit points of every query-level cell that
// the Gaussian's k-sigma bounds overlap, so each pair is seen exactly once,
// and the sums are reduced inside the warp: no global atomics, bitwise
// reproducible.
// The sums have a type T: float in the product path; double in the
// gradient-check build (gpf_query_params.f64_sums), where the same float32
// pair terms are accumulated, reduced and turned into gradients in float64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kBwdWarps = 4;
constexpr int64_t kGrab = 4;            // work units per atomic of the persistent loop
constexpr int64_t kFineLarge = 4096;    // largest non-split Gaussians taken one per atomic
constexpr int kBwdThreads = kBwdWarps * kWarp;

struct BwdArgs {
  Grid grid;
  const DeviceHeader* header;
  const uint32_t* qval;
  const uint32_t* qstart;
  const float* x;
  const float* albedo;
  const float* grad_out;
  const float* out;
  const float* z;
  int64_t m;
  float* qrec;
  void* gacc;             // [N * NS] per-Gaussian sums (type T), by Gaussian id
  const uint8_t* glive;   // [N] 1 if the pair loop visits the Gaussian
  const uint2* qbox;      // [N] query-level cell bounds (pack_qbox), from the build
  void* bpart;            // [kSplitMax * kSplitWays * NS] split Gaussians' partials (T)
  const float* rec;
  const uint4* box;
  const uint32_t* order;  // Gaussian ids in mean-cell order
  const uint2* nbrange;   // hybrid neighbourhood: [start, end) of each Gaussian's pairs
  const uint32_t* nbval;  // hybrid neighbourhood: the pairs' hit point positions
  int64_t n;
  const float* quat;
  const float* logscale;
  int mode;
  float r, r2, inv_rr, eps, cut, cut2;
  double rd, r2d, inv_rrd;  // the falloff parameters in float64 (gradient-check build)
  int f64;                  // 1: the gradient-check build (float64 pair arithmetic)
  gpf_field_grad g;
  unsigned long long* next_work;  // work counter, zero at launch
};

template <int C>
__global__ void pack_qrec_kernel(BwdArgs a) {
  constexpr int QS = qrec_stride(C);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (index_unusable(a.header) || k >= (int64_t)a.header->n_active) return;
  const uint32_t q = a.qval[k];
  float gam[C];
  float kappa = 0.0f, zeta = 1.0f;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const float g = a.grad_out[(int64_t)c * a.m + q];
    gam[c] = g * (a.albedo ? a.albedo[(int64_t)c * a.m + q] : 1.0f);
  }
  if (a.mode == GPF_NORMALIZED) {
    const float Z = a.z[q];
    if (Z > a.eps) {
      if (a.f64) {
        // the check build rounds each to float32 once
        double k = 0.0;
#pragma unroll
        for (int c = 0; c < C; ++c)
          k = fma((double)a.grad_out[(int64_t)c * a.m + q], (double)a.out[(int64_t)c * a.m + q], k);
        kappa = (float)k;
        zeta = (float)(1.0 / (double)Z);
      } else {
        zeta = 1.0f / Z;
#pragma unroll
        for (int c = 0; c < C; ++c) kappa = fmaf(a.grad_out[(int64_t)c * a.m + q], a.out[(int64_t)c * a.m + q], kappa);
      }
    } else {
      zeta = 1.0f / a.eps;
    }
  }
  float* r = a.qrec + k * QS;
  r[0] = a.x[q];
  r[1] = a.x[a.m + q];
  r[2] = a.x[2 * a.m + q];
  r[3] = zeta;
  r[4] = kappa;
#pragma unroll
  for (int c = 0; c < C; ++c) r[5 + c] = gam[c];
#pragma unroll
  for (int c = 5 + C; c < QS; ++c) r[c] = 0.0f;
}

// acc += a * b and acc += a for float32 terms a, b into sums of type T:
// one fused multiply-add in float32, or the exact float64 product and sum.
template <typename T>
__device__ __forceinline__ void mac(T& acc, float a, float b) {
  if constexpr (sizeof(T) == 4) acc = fmaf(a, b, acc);
  else acc = fma((double)a, (double)b, acc);
}
template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c) {
  if constexpr (sizeof(T) == 4) return fmaf(a, b, c);
  else return fma(a, b, c);
}

template <int C, typename T>
struct Acc {
  T A00, A01, A02, A11, A12, A22;
  T B0, B1, B2;
  T D0, D1, D2;
  T P[C];
  __device__ void zero() {
    A00 = A01 = A02 = A11 = A12 = A22 = T(0);
    B0 = B1 = B2 = T(0);
    D0 = D1 = D2 = T(0);
#pragma unroll
    for (int c = 0; c < C; ++c) P[c] = T(0);
  }
  // The sums as an array of NS slots (zero padded): 16 for C <= 4, else 32.
  static constexpr int NV = 12 + C;
  static constexpr int NS = NV <= 16 ? 16 : 32;
  __device__ void to_array(T (&v)[NS]) const {
    v[0] = A00; v[1] = A01; v[2] = A02; v[3] = A11; v[4] = A12; v[5] = A22;
    v[6] = B0; v[7] = B1; v[8] = B2; v[9] = D0; v[10] = D1; v[11] = D2;
#pragma unroll
    for (int c = 0; c < C; ++c) v[12 + c] = P[c];
#pragma unroll
    for (int i = NV; i < NS; ++i) v[i] = T(0);
  }
  __device__ void from_array(const T* v) {
    A00 = v[0]; A01 = v[1]; A02 = v[2]; A11 = v[3]; A12 = v[4]; A22 = v[5];
    B0 = v[6]; B1 = v[7]; B2 = v[8]; D0 = v[9]; D1 = v[10]; D2 = v[11];
#pragma unroll
    for (int c = 0; c < C; ++c) P[c] = v[12 + c];
  }
};

// Sum NS values over the 32 lanes of a warp, scattered: each halving
// exchange (lane offsets 16, 8, ...) sends half of the values a lane still
// holds and keeps the other half, so NS - 1 shuffles leave every lane with
// one complete sum (for NS = 16 lanes l and l ^ 1 hold the same one). The
// slot a lane ends with is returned in *slot.
template <int NS, typename T>
__device__ __forceinline__ T reduce_scatter(T (&v)[NS], int lane, int* slot) {
  constexpr int kStages = NS == 16 ? 4 : 5;
  int idx = 0;
#pragma unroll
  for (int st = 0; st < kStages; ++st) {
    const int o = 16 >> st, h = NS >> (st + 1);
    const bool up = (lane & o) != 0;
    if (up) idx += h;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(kFullMask, send, o);
    }
  }
  if (NS == 16) v[0] += __shfl_xor_sync(kFullMask, v[0], 1);
  *slot = idx;
  return v[0];
}

struct GaussianRegs {
  float mx, my, mz;
  float M[9];
};

// A Gaussian as a pair loop holds it: its float32 record (mean, M = S^-1 R^T,
// Phi; the cull reads it too) and, for float64 sums, the same quantities in
// float64 computed from the raw parameters (R(q / |q|) and s = exp(l) in
// float64), so that the gradient-check build rounds nothing below float64.
template <int C, typename T>
struct PairG {
  GaussianRegs G;
  float phi[C];
};
template <int C>
struct PairG<C, double> {
  GaussianRegs G;
  float phi[C];
  double mx, my, mz, M[9], phid[C];
};

// A packed hit point, all of it (one 32-byte sector for C <= 3): the loads
// of a pair are issued together, before its arithmetic.
template <int C>
__device__ __forceinline__ void load_qrec(const float* __restrict__ qr,
                                          float (&q)[qrec_stride(C)]) {
#pragma unroll
  for (int v = 0; v < qrec_stride(C) / 4; ++v) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(qr) + v);
    q[4 * v] = t.x; q[4 * v + 1] = t.y; q[4 * v + 2] = t.z; q[4 * v + 3] = t.w;
  }
}

// One (Gaussian, hit point) pair of the backward in float64 (the
// gradient-check build): the steps of the float32 pair below, in float64.
template <int C, bool PSI>
__device__ __forceinline__ void bwd_pair_q64(const PairG<C, double>& P,
                                             const float (&q)[qrec_stride(C)], const BwdArgs& a,
                                             Acc<C, double>& acc) {
  const double dx = (double)q[0] - P.mx, dy = (double)q[1] - P.my, dz = (double)q[2] - P.mz;
  const double u0 = fma(P.M[0], dx, fma(P.M[1], dy, P.M[2] * dz));
  const double u1 = fma(P.M[3], dx, fma(P.M[4], dy, P.M[5] * dz));
  const double u2 = fma(P.M[6], dx, fma(P.M[7], dy, P.M[8] * dz));
  const double Q = fma(u0, u0, fma(u1, u1, u2 * u2));
  if (!(Q <= (double)a.cut2)) return;
  const float* qv = q + 4;
  double e = -0.5 * Q;
  double pcoef = 0.0;
  if (PSI) {
    const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
    if (d2 > a.r2d) {
      const double dist = sqrt(d2);
      const double t = (dist - a.rd) * a.inv_rrd;
      e = fma(-3.0 * t, t, e);
      pcoef = 6.0 * t * a.inv_rrd / dist;
    }
  }
  const double w = exp(e);
  const double zeta = q[3], kappa = qv[0];
  double gp = 0.0;
#pragma unroll
  for (int c = 0; c < C; ++c) gp = fma((double)qv[1 + c], P.phid[c], gp);
  const double bw = zeta * (gp - kappa) * w;
  const double b0 = bw * u0, b1 = bw * u1, b2 = bw * u2;
  acc.A00 = fma(b0, u0, acc.A00);
  acc.A01 = fma(b0, u1, acc.A01);
  acc.A02 = fma(b0, u2, acc.A02);
  acc.A11 = fma(b1, u1, acc.A11);
  acc.A12 = fma(b1, u2, acc.A12);
  acc.A22 = fma(b2, u2, acc.A22);
  acc.B0 += b0;
  acc.B1 += b1;
  acc.B2 += b2;
  if (PSI) {
    const double pc = bw * pcoef;
    acc.D0 = fma(pc, dx, acc.D0);
    acc.D1 = fma(pc, dy, acc.D1);
    acc.D2 = fma(pc, dz, acc.D2);
  }
  const double wz = w * zeta;
#pragma unroll
  for (int c = 0; c < C; ++c) acc.P[c] = fma((double)qv[1 + c], wz, acc.P[c]);
}

// One (Gaussian, hit point) pair of the backward, the hit point in q.
template <int C, bool PSI, typename T>
__device__ __forceinline__ void bwd_pair_q(const PairG<C, T>& P,
                                           const float (&q)[qrec_stride(C)], const BwdArgs& a,
                                           Acc<C, T>& acc) {
  if constexpr (sizeof(T) == 8) {
    bwd_pair_q64<C, PSI>(P, q, a, acc);
    return;
  } else {
  const GaussianRegs& G = P.G;
  const float (&phi)[C] = P.phi;
  const float dx = q[0] - G.mx, dy = q[1] - G.my, dz = q[2] - G.mz;
  const float u0 = fmaf(G.M[0], dx, fmaf(G.M[1], dy, G.M[2] * dz));
  const float u1 = fmaf(G.M[3], dx, fmaf(G.M[4], dy, G.M[5] * dz));
  const float u2 = fmaf(G.M[6], dx, fmaf(G.M[7], dy, G.M[8] * dz));
  const float Q = fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
  if (!(Q <= a.cut2)) return;
  const float* qv = q + 4;
  float e = -0.5f * Q;
  float pcoef = 0.0f;  // 6 t / (r' |d|), the falloff's share of dw/dmu per unit w
  if (PSI) {
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (d2 > a.r2) {
      // |d| and 1/|d| from one reciprocal square root (d2 > r^2 > 0)
      const float inv_d = rsqrtf(d2);
      const float dist = d2 * inv_d;
      const float t = (dist - a.r) * a.inv_rr;
      e = fmaf(-3.0f * t, t, e);
      pcoef = 6.0f * t * a.inv_rr * inv_d;
    }
  }
  const float w = ex2_approx(e * kLog2e);
  const float zeta = q[3], kappa = qv[0];
  float gp = 0.0f;
#pragma unroll
  for (int c = 0; c < C; ++c) gp = fmaf(qv[1 + c], phi[c], gp);
  const float bw = zeta * (gp - kappa) * w;
  const float b0 = bw * u0, b1 = bw * u1, b2 = bw * u2;
  mac(acc.A00, b0, u0);
  mac(acc.A01, b0, u1);
  mac(acc.A02, b0, u2);
  mac(acc.A11, b1, u1);
  mac(acc.A12, b1, u2);
  mac(acc.A22, b2, u2);
  acc.B0 += (T)b0;
  acc.B1 += (T)b1;
  acc.B2 += (T)b2;
  if (PSI) {
    const float pc = bw * pcoef;
    mac(acc.D0, pc, dx);
    mac(acc.D1, pc, dy);
    mac(acc.D2, pc, dz);
  }
  const float wz = w * zeta;
#pragma unroll
  for (int c = 0; c < C; ++c) mac(acc.P[c], qv[1 + c], wz);
  }
}

template <int C, bool PSI, typename T>
__device__ __forceinline__ void bwd_pair(const PairG<C, T>& P, const float* __restrict__ qr,
                                         const BwdArgs& a, Acc<C, T>& acc) {
  float q[qrec_stride(C)];
  load_qrec<C>(qr, q);
  bwd_pair_q<C, PSI, T>(P, q, a, acc);
}

// Gradients of one Gaussian from its reduced sums (runs on one lane), in
// the sums' type T.
template <int C, typename T>
__device__ void bwd_epilogue(const BwdArgs& a, int64_t gi, const Frame& fr, const Acc<C, T>& acc) {
  const int64_t n = a.n;
  T R[3][3], s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s[k] = (T)fr.s[k];
#pragma unroll
    for (int j = 0; j < 3; ++j) R[k][j] = (T)fr.R[k][j];
  }
  const T qw = fr.qhat[0], qx = fr.qhat[1], qy = fr.qhat[2], qz = fr.qhat[3];
  const T iq = fr.inv_qn;
  const T A[3][3] = {{acc.A00, acc.A01, acc.A02}, {acc.A01, acc.A11, acc.A12},
                     {acc.A02, acc.A12, acc.A22}};
  const T B[3] = {acc.B0, acc.B1, acc.B2};
  const T D[3] = {acc.D0, acc.D1, acc.D2};
  T dmu[3], dl[3], dR[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dmu[k] = D[k];
#pragma unroll
    for (int j = 0; j < 3; ++j) dmu[k] = fmaT<T>(R[k][j] / s[j], B[j], dmu[k]);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) dl[j] = A[j][j];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T t = T(0);
#pragma unroll
      for (int mm = 0; mm < 3; ++mm) t = fmaT<T>(R[k][mm] * s[mm], A[j][mm], t);
      dR[k][j] = -t / s[j];
    }
  // d loss / d qhat through the entries of R(qhat)
  const T gw = T(2) * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] -
                       qy * dR[2][0] + qx * dR[2][1]);
  const T gx = T(2) * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - T(2) * qx * dR[1][1] -
                       qw * dR[1][2] + qz * dR[2][0] + qw * dR[2][1] - T(2) * qx * dR[2][2]);
  const T gy = T(2) * (-T(2) * qy * dR[0][0] + qx * dR[0][1] + qw * dR[0][2] + qx * dR[1][0] +
                       qz * dR[1][2] - qw * dR[2][0] + qz * dR[2][1] - T(2) * qy * dR[2][2]);
  const T gz = T(2) * (-T(2) * qz * dR[0][0] - qw * dR[0][1] + qx * dR[0][2] + qw * dR[1][0] -
                       T(2) * qz * dR[1][1] + qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
  // through qhat = q / |q|
  const T dot = qw * gw + qx * gx + qy * gy + qz * gz;
  const T dq[4] = {(gw - qw * dot) * iq, (gx - qx * dot) * iq, (gy - qy * dot) * iq,
                   (gz - qz * dot) * iq};
  const bool accu = a.g.accumulate != 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float* p = a.g.mean + k * n + gi;
    *p = accu ? (float)((T)*p + dmu[k]) : (float)dmu[k];
    float* pl = a.g.logscale + k * n + gi;
    *pl = accu ? (float)((T)*pl + dl[k]) : (float)dl[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float* p = a.g.quat + k * n + gi;
    *p = accu ? (float)((T)*p + dq[k]) : (float)dq[k];
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float* p = a.g.spectrum + (int64_t)c * n + gi;
    *p = accu ? (float)((T)*p + acc.P[c]) : (float)acc.P[c];
  }
}

template <int C>
__device__ __forceinline__ void load_gaussian(const BwdArgs& a, int64_t gi, GaussianRegs& G,
                                              float (&phi)[C]) {
  constexpr int RS = rec_stride(C);
  const float* r = a.rec + gi * RS;
  const float4 r0 = *reinterpret_cast<const float4*>(r);
  const float4 r1 = *reinterpret_cast<const float4*>(r + 4);
  const float4 r2 = *reinterpret_cast<const float4*>(r + 8);
  G.mx = r0.x; G.my = r0.y; G.mz = r0.z;
  G.M[0] = r1.x; G.M[1] = r1.y; G.M[2] = r1.z; G.M[3] = r1.w;
  G.M[4] = r2.x; G.M[5] = r2.y; G.M[6] = r2.z; G.M[7] = r2.w;
  G.M[8] = r[12];
#pragma unroll
  for (int c = 0; c < C; ++c) phi[c] = r[13 + c];
}

template <int C, typename T>
__device__ __forceinline__ void load_pair_gaussian(const BwdArgs& a, int64_t gi, PairG<C, T>& P) {
  load_gaussian<C>(a, gi, P.G, P.phi);
  if constexpr (sizeof(T) == 8) {
    const int64_t n = a.n;
    double qw = a.quat[gi], qx = a.quat[n + gi], qy = a.quat[2 * n + gi], qz = a.quat[3 * n + gi];
    const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    const double iq = qn > 0.0 ? 1.0 / qn : 0.0;
    qw *= iq; qx *= iq; qy *= iq; qz *= iq;
    const double R[3][3] = {
        {1.0 - 2.0 * (qy * qy + qz * qz), 2.0 * (qx * qy - qw * qz), 2.0 * (qx * qz + qw * qy)},
        {2.0 * (qx * qy + qw * qz), 1.0 - 2.0 * (qx * qx + qz * qz), 2.0 * (qy * qz - qw * qx)},
        {2.0 * (qx * qz - qw * qy), 2.0 * (qy * qz + qw * qx), 1.0 - 2.0 * (qx * qx + qy * qy)}};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double inv_s = exp(-(double)a.logscale[j * n + gi]);
#pragma unroll
      for (int k = 0; k < 3; ++k) P.M[3 * j + k] = R[k][j] * inv_s;
    }
    P.mx = P.G.mx; P.my = P.G.my; P.mz = P.G.mz;
#pragma unroll
    for (int c = 0; c < C; ++c) P.phid[c] = P.phi[c];
  }
}

// Stores NS sums of type T (16-byte vectors).
template <int NS, typename T>
__device__ __forceinline__ void store_sums(T* dst, const T (&v)[NS]) {
  if constexpr (sizeof(T) == 4) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < NS / 4; ++i)
      d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int i = 0; i < NS / 2; ++i) d2[i] = make_double2(v[2 * i], v[2 * i + 1]);
  }
}

// One lane runs one small Gaussian (bounds within 2 x 2 x 2 query-level
// cells) alone: no reduction across lanes, the epilogues run side by side.
template <int C, bool PSI, typename T>
__device__ void bwd_lane_gaussian(const BwdArgs& a, int64_t gi) {
  constexpr int QS = qrec_stride(C);
  constexpr int NS = Acc<C, T>::NS;
  const Grid& Gd = a.grid;
  PairG<C, T> P;
  load_pair_gaussian<C, T>(a, gi, P);
  uint32_t lo[3], hi[3];
  unpack_qbox(a.qbox[gi], lo, hi);
  const uint32_t lx = lo[0], hx = hi[0], ly = lo[1], hy = hi[1], lz = lo[2], hz = hi[2];
  Acc<C, T> acc;
  acc.zero();
  for (uint32_t iz = lz; iz <= hz; ++iz)
    for (uint32_t iy = ly; iy <= hy; ++iy) {
      const uint32_t key = qkey_of(Gd, lx, iy, iz);
      const uint32_t e = a.qstart[key + (hx - lx) + 1];
      for (uint32_t k = a.qstart[key]; k < e; ++k)
        bwd_pair<C, PSI, T>(P, a.qrec + (int64_t)k * QS, a, acc);
    }
  T v[NS];
  acc.to_array(v);
  store_sums<NS, T>(static_cast<T*>(a.gacc) + gi * NS, v);
}

// Grid path. The Gaussians come in (class, size, mean-cell) order, the small
// ones first and the large ones largest first; the largest (up to kSplitMax)
// are split into kSplitWays work units, each over every kSplitWays-th block
// of 32 rows, whose partial sums bwd_split_combine_kernel adds in part order:
// the first ceil(n_small / 32) warps give each lane one small Gaussian; every
// later warp runs one large Gaussian over the hit points of every
// query-level cell its k-sigma bounds overlap. Gaussians whose level box
// holds no hit point come last and are skipped (zero gradient).
// float32 sums: 9 resident blocks per SM (56 registers); the float64 sums
// of the gradient-check build need more registers and run at fewer.
template <int C, bool PSI, typename T>
__global__ void __launch_bounds__(kBwdThreads, sizeof(T) == 4 ? 9 : 2)
bwd_grid_kernel(BwdArgs a) {
  constexpr int QS = qrec_stride(C);
  constexpr int NS = Acc<C, T>::NS;
  // per warp: first hit point minus flattened start of each non-empty row
  __shared__ uint32_t s_base[kBwdWarps][kWarp];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (index_unusable(a.header)) return;
  const int64_t n_small = a.header->n_small, n_live = a.header->n_live;
  const int64_t small_warps = (n_small + kWarp - 1) / kWarp;
  const int64_t n_split = min((int64_t)a.header->n_huge, kSplitMax);
  const int64_t units = small_warps + n_split * kSplitWays + (n_live - n_small - n_split);
  // persistent: every warp takes the next work units (each 32 small
  // Gaussians, one of the kSplitWays parts of a huge Gaussian, or one large
  // Gaussian) until none is left: kGrab at a time, so that one atomic on the
  // work counter (a single address) serves several units, except over the
  // split parts and the kFineLarge largest other Gaussians, which are taken
  // one by one so that no warp holds several heavy units
  const int64_t fine_begin = small_warps;
  const int64_t fine_end =
      small_warps + n_split * kSplitWays + min(n_live - n_small - n_split, kFineLarge);
  for (;;) {
  unsigned long long w_u = 0, g_u = 0;
  if (lane == 0) {
    const int64_t seen = (int64_t)*(volatile unsigned long long*)a.next_work;
    g_u = (seen + kGrab > fine_begin && seen < fine_end) ? 1ull : (unsigned long long)kGrab;
    w_u = atomicAdd(a.next_work, g_u);
  }
  const int64_t w0 = (int64_t)__shfl_sync(kFullMask, w_u, 0);
  const int64_t grab = (int64_t)__shfl_sync(kFullMask, g_u, 0);
  if (w0 >= units) break;
  const int64_t w_end = min(w0 + grab, units);
  for (int64_t w = w0; w < w_end; ++w) {
  if (w < small_warps) {
    const int64_t idx = w * kWarp + lane;
    if (idx < n_small) bwd_lane_gaussian<C, PSI, T>(a, a.order[idx]);
    __syncwarp();
    continue;
  }
  const int64_t u = w - small_warps;
  const bool split = u < n_split * kSplitWays;
  const int64_t j = split ? n_small + u / kSplitWays : n_small + n_split + (u - n_split * kSplitWays);
  const int part = split ? (int)(u % kSplitWays) : 0;       // this unit's share of the rows
  const int row_step = split ? kSplitWays * kWarp : kWarp;
  const Grid& Gd = a.grid;
  const int64_t gi = a.order[j];
  PairG<C, T> P;
  load_pair_gaussian<C, T>(a, gi, P);
  const GaussianRegs& G = P.G;
  uint32_t lo[3], hi[3];
  unpack_qbox(a.qbox[gi], lo, hi);
  const int K = Gd.qlevel;
  const int lx = (int)lo[0], ly = (int)lo[1], lz = (int)lo[2];
  const int nx = (int)hi[0] - lx + 1, ny = (int)hi[1] - ly + 1, nz = (int)hi[2] - lz + 1;
  const float cut_keep = a.cut * 1.0001f;
  const float cellK = Gd.cell0 * (float)(1u << K);
  const float half = 0.5f * cellK * 1.001f;
  // the cells lx..hx of one (iy, iz) row have consecutive keys, so the row's
  // hit points are one contiguous range of the sorted order
  const int rows = ny * nz;
  const bool xborder = lx == 0 || lx + nx - 1 == Gd.dx - 1;
  const float rcx = Gd.ox + (lx + 0.5f * nx) * cellK, rhx = 0.5f * nx * cellK * 1.001f;
  Acc<C, T> acc;
  acc.zero();
  for (int rb = part * kWarp; rb < rows; rb += row_step) {
    const int ri = rb + lane;
    uint32_t qs = 0, cnt = 0;
    if (ri < rows) {
      const int iy = ly + ri % ny, iz = lz + ri / ny;
      const uint32_t key = qkey_of(Gd, lx, iy, iz);
      qs = a.qstart[key];
      cnt = a.qstart[key + nx] - qs;
      // border cells also hold the clamped points outside the grid: no cull
      const bool border = xborder || iy == 0 || iz == 0 || iy == Gd.dy - 1 || iz == Gd.dz - 1;
      if (cnt > 0 && !border) {
        const float ccy = Gd.oy + (iy + 0.5f) * cellK;
        const float ccz = Gd.oz + (iz + 0.5f) * cellK;
        const float lb = mahalanobis_lower_bound(G.M, G.mx, G.my, G.mz, rcx, ccy, ccz, rhx,
                                                 half, half);
        if (lb > cut_keep) cnt = 0;
      }
    }
    // flatten the hit points of these (up to 32) cells over the lanes
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t tot = __shfl_sync(kFullMask, incl, 31);
    const uint32_t excl = incl - cnt;
    // item f of the flattened rows belongs to the non-empty row with the
    // largest start excl <= f. The non-empty rows, ranked in lane order, keep
    // (first hit point - start) in shared memory; a chunk's owner ranks come
    // from the starts that fall inside it (a bit per start, OR-reduced over
    // the warp) counted up to each lane, on top of the rank of the row that
    // holds the chunk's first item.
    const bool ne = cnt > 0;
    const uint32_t ne_mask = __ballot_sync(kFullMask, ne);
    if (ne) s_base[wib][__popc(ne_mask & lanemask_lt())] = qs - excl;
    __syncwarp();
    const uint32_t le = lanemask_lt() | (1u << lane);
    for (uint32_t f0 = 0; f0 < tot; f0 += kWarp) {
      const uint32_t f = f0 + lane;
      const uint32_t starts =
          __reduce_or_sync(kFullMask, ne && excl > f0 && excl < f0 + kWarp ? 1u << (excl - f0) : 0u);
      const int r0 = __popc(__ballot_sync(kFullMask, ne && excl <= f0)) - 1;
      if (f < tot) {
        const int r = r0 + __popc(starts & le);
        const uint32_t k = s_base[wib][r] + f;     // modulo 2^32: qs - excl may wrap
        bwd_pair<C, PSI, T>(P, a.qrec + (int64_t)k * QS, a, acc);
      }
    }
    __syncwarp();
  }
  T v[NS];
  acc.to_array(v);
  int slot;
  const T sum = reduce_scatter<NS, T>(v, lane, &slot);
  T* dst = split ? static_cast<T*>(a.bpart) + ((j - n_small) * kSplitWays + part) * NS
                 : static_cast<T*>(a.gacc) + gi * NS;
  if (NS == 32 || (lane & 1) == 0) dst[slot] = sum;
  }
  }  // work loop
}

// Brute-force path (no cell lists): one warp per Gaussian over all active hit points.
template <int C, bool PSI, typename T>
__global__ void __launch_bounds__(kBwdThreads)
bwd_brute_kernel(BwdArgs a) {
  constexpr int QS = qrec_stride(C);
  constexpr int NS = Acc<C, T>::NS;
  const int lane = threadIdx.x & 31;
  const int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gi >= a.n || index_unusable(a.header)) return;
  const int64_t n_act = a.header->n_active;
  PairG<C, T> P;
  load_pair_gaussian<C, T>(a, gi, P);
  Acc<C, T> acc;
  acc.zero();
  for (int64_t k = lane; k < n_act; k += kWarp) bwd_pair<C, PSI, T>(P, a.qrec + k * QS, a, acc);
  T v[NS];
  acc.to_array(v);
  int slot;
  const T sum = reduce_scatter<NS, T>(v, lane, &slot);
  if (NS == 32 || (lane & 1) == 0) static_cast<T*>(a.gacc)[gi * NS + slot] = sum;
}

// The paper's hybrid neighbourhood (GPF_NB_BALL_KNN): one warp per Gaussian
// over its selected hit points (the sorted pairs of launch_hybrid_pairs),
// lanes striding the run; the weights are untruncated (cut2 = +INF) and the
// selection is what makes a pair count. Persistent over Gaussian ids.
template <int C, bool PSI, typename T>
__global__ void __launch_bounds__(kBwdThreads)
bwd_hybrid_kernel(BwdArgs a) {
  constexpr int QS = qrec_stride(C);
  constexpr int NS = Acc<C, T>::NS;
  const int lane = threadIdx.x & 31;
  if (index_unusable(a.header)) return;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < a.n;
       gi += warps) {
    const uint2 rg = a.nbrange[gi];
    T* dst = static_cast<T*>(a.gacc) + gi * NS;
    if (rg.y <= rg.x) {
      if (lane < NS) dst[lane] = T(0);
      continue;
    }
    PairG<C, T> P;
    load_pair_gaussian<C, T>(a, gi, P);
    Acc<C, T> acc;
    acc.zero();
    for (uint32_t i = rg.x + lane; i < rg.y; i += kWarp)
      bwd_pair<C, PSI, T>(P, a.qrec + (int64_t)a.nbval[i] * QS, a, acc);
    T v[NS];
    acc.to_array(v);
    int slot;
    const T sum = reduce_scatter<NS, T>(v, lane, &slot);
    if (NS == 32 || (lane & 1) == 0) dst[slot] = sum;
  }
}

// The split Gaussians' sums: their kSplitWays parts added in part order,
// into gacc at the Gaussian's id (one thread per split Gaussian).
template <int C, typename T>
__global__ void bwd_split_combine_kernel(BwdArgs a) {
  constexpr int NS = Acc<C, T>::NS;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (index_unusable(a.header)) return;
  const int64_t n_split = min((int64_t)a.header->n_huge, kSplitMax);
  if (s >= n_split) return;
  const int64_t gi = a.order[(int64_t)a.header->n_small + s];
  T v[NS];
  const T* p = static_cast<const T*>(a.bpart) + s * kSplitWays * NS;
#pragma unroll
  for (int i = 0; i < NS; ++i) v[i] = p[i];
  for (int b = 1; b < kSplitWays; ++b)
#pragma unroll
    for (int i = 0; i < NS; ++i) v[i] += p[b * NS + i];
  store_sums<NS, T>(static_cast<T*>(a.gacc) + gi * NS, v);
}

// Gradients of every Gaussian from its sums, one thread per Gaussian id (so
// that every read and write is coalesced). Gaussians the pair loop did not
// visit (no hit point in reach) get zero gradients. With no hit points at
// all (sums_ready = false) every Gaussian gets zero gradients.
template <int C, typename T>
__global__ void bwd_epilogue_kernel(BwdArgs a, bool sums_ready, bool all_live) {
  constexpr int NS = Acc<C, T>::NS;
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.n || index_unusable(a.header)) return;
  Acc<C, T> acc;
  if (sums_ready && (all_live || a.glive[gi])) {
    T v[NS];
    const T* src = static_cast<const T*>(a.gacc) + gi * NS;
    if constexpr (sizeof(T) == 4) {
      const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
      for (int i = 0; i < NS / 4; ++i) {
        const float4 t = s4[i];
        v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
      }
    } else {
      const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
      for (int i = 0; i < NS / 2; ++i) {
        const double2 t = s2[i];
        v[2 * i] = t.x; v[2 * i + 1] = t.y;
      }
    }
    acc.from_array(v);
  } else {
    acc.zero();
  }
  const Frame fr = gaussian_frame(a.quat, a.logscale, a.n, gi);
  bwd_epilogue<C, T>(a, gi, fr, acc);
}

template <int C, typename T>
cudaError_t launch_ct(const BwdArgs& a, const IndexDims& d, bool psi, const KernelEvents& ev,
                      cudaStream_t stream) {
  if (a.n == 0) return cudaSuccess;
  const unsigned eblocks = (unsigned)((a.n + 255) / 256);
  if (a.m == 0) {
    // no hit points: every gradient is zero (written by the epilogue, which
    // leaves them untouched when the build set a flag)
    bwd_epilogue_kernel<C, T><<<eblocks, 256, 0, stream>>>(a, false, false);
    note_launches(1);
    return cudaGetLastError();
  }
  const unsigned pblocks = (unsigned)((a.m + 255) / 256);
  pack_qrec_kernel<C><<<pblocks, 256, 0, stream>>>(a);
  note_launches(1);
  cudaError_t e;
  if (a.nbrange) {
    // the hybrid neighbourhood: a warp per Gaussian over its selected pairs
    const int64_t want = (a.n * kWarp + kBwdThreads - 1) / kBwdThreads;
    const void* kfn = psi ? reinterpret_cast<const void*>(&bwd_hybrid_kernel<C, true, T>)
                          : reinterpret_cast<const void*>(&bwd_hybrid_kernel<C, false, T>);
    const unsigned hblocks = (unsigned)persistent_blocks(kfn, kBwdThreads, want);
    if (ev.start && (e = cudaEventRecord(ev.start, stream)) != cudaSuccess) return e;
    if (psi) bwd_hybrid_kernel<C, true, T><<<hblocks, kBwdThreads, 0, stream>>>(a);
    else bwd_hybrid_kernel<C, false, T><<<hblocks, kBwdThreads, 0, stream>>>(a);
    if (ev.stop && (e = cudaEventRecord(ev.stop, stream)) != cudaSuccess) return e;
    bwd_epilogue_kernel<C, T><<<eblocks, 256, 0, stream>>>(a, true, true);
    note_launches(2);
    return cudaGetLastError();
  }
  // brute force: a warp per Gaussian; grid: up to n / 32 lane warps + n warps
  const int64_t warps = d.brute ? a.n : a.n + (a.n + kWarp - 1) / kWarp;
  const unsigned blocks = (unsigned)((warps + kBwdWarps - 1) / kBwdWarps);
  if (!d.brute &&
      (e = cudaMemsetAsync(a.next_work, 0, sizeof(unsigned long long), stream)) != cudaSuccess)
    return e;
  if (ev.start && (e = cudaEventRecord(ev.start, stream)) != cudaSuccess) return e;
  if (d.brute) {
    if (psi) bwd_brute_kernel<C, true, T><<<blocks, kBwdThreads, 0, stream>>>(a);
    else bwd_brute_kernel<C, false, T><<<blocks, kBwdThreads, 0, stream>>>(a);
  } else {
    // persistent: as many blocks as can be resident at once
    const void* kfn = psi ? reinterpret_cast<const void*>(&bwd_grid_kernel<C, true, T>)
                          : reinterpret_cast<const void*>(&bwd_grid_kernel<C, false, T>);
    const unsigned gblocks = (unsigned)persistent_blocks(kfn, kBwdThreads, blocks);
    if (psi) bwd_grid_kernel<C, true, T><<<gblocks, kBwdThreads, 0, stream>>>(a);
    else bwd_grid_kernel<C, false, T><<<gblocks, kBwdThreads, 0, stream>>>(a);
  }
  if (ev.stop && (e = cudaEventRecord(ev.stop, stream)) != cudaSuccess) return e;
  if (!d.brute) {
    const int64_t max_split = std::min<int64_t>(a.n, kSplitMax);
    bwd_split_combine_kernel<C, T><<<(unsigned)((max_split + 127) / 128), 128, 0, stream>>>(a);
    note_launches(1);
  }
  bwd_epilogue_kernel<C, T><<<eblocks, 256, 0, stream>>>(a, true, false);
  note_launches(2);
  return cudaGetLastError();
}

template <int C>
cudaError_t launch_c(const BwdArgs& a, const IndexDims& d, bool psi, bool f64,
                     const KernelEvents& ev, cudaStream_t stream) {
  return f64 ? launch_ct<C, double>(a, d, psi, ev, stream)
             : launch_ct<C, float>(a, d, psi, ev, stream);
}

}  // namespace

cudaError_t launch_backward(const IndexDims& d, const IndexBuffers& b, const gpf_field& f,
                            const gpf_queries& q, const gpf_query_params& p,
                            const float* grad_out, const float* out, const float* z,
                            const gpf_field_grad& g, bool hyb_counted, const KernelEvents& ev,
                            cudaStream_t stream) {
  // every gradient is written by the epilogue kernel (zeros for Gaussians
  // out of reach), which leaves them untouched when the build set a flag
  const int64_t n = f.n;
  if (n == 0) return cudaSuccess;
  BwdArgs a;
  a.grid = d.grid;
  a.header = b.header;
  a.qval = b.qval[b.qsorted];
  a.qstart = b.qstart;
  a.x = q.x;
  a.albedo = q.albedo;
  a.grad_out = grad_out;
  a.out = out;
  a.z = z;
  a.m = q.m;
  a.qrec = b.qrec;
  a.gacc = b.gacc;
  a.glive = b.glive;
  a.qbox = b.qbox;
  a.bpart = b.bpart;
  a.rec = b.rec;
  a.box = b.box;
  a.order = b.oval[b.osorted];
  a.nbrange = nullptr;
  a.nbval = nullptr;
  a.n = n;
  a.quat = static_cast<const float*>(f.quat);
  a.logscale = static_cast<const float*>(f.logscale);
  a.mode = p.mode;
  const bool psi = isfinite(p.r_max);
  a.r = psi ? p.r_max : 0.0f;
  a.r2 = psi ? p.r_max * p.r_max : 0.0f;
  a.inv_rr = psi ? 1.0f / fmaxf(p.r_max, 1e-6f) : 0.0f;
  a.eps = p.eps;
  a.cut = d.cutoff;
  a.cut2 = isinf(d.cutoff) ? INFINITY : d.cutoff * d.cutoff;
  if (p.neighbourhood == GPF_NB_BALL_KNN) {
    // the selected pairs, sorted by Gaussian; no truncation of the weights
    const cudaError_t e = launch_hybrid_pairs(d, b, q, p, n, hyb_counted, stream);
    if (e != cudaSuccess) return e;
    a.nbrange = b.nbrange;
    a.nbval = b.nbval[b.nbsorted];
    a.cut2 = INFINITY;
  }
  a.rd = psi ? (double)p.r_max : 0.0;
  a.r2d = a.rd * a.rd;
  a.inv_rrd = psi ? 1.0 / fmax((double)p.r_max, 1e-6) : 0.0;
  const bool f64 = p.f64_sums != 0;
  a.f64 = f64 ? 1 : 0;
  a.g = g;
  a.next_work = &b.header->next_work;
  switch (d.channels) {
    case 1: return launch_c<1>(a, d, psi, f64, ev, stream);
    case 2: return launch_c<2>(a, d, psi, f64, ev, stream);
    case 3: return launch_c<3>(a, d, psi, f64, ev, stream);
    case 4: return launch_c<4>(a, d, psi, f64, ev, stream);
    case 5: return launch_c<5>(a, d, psi, f64, ev, stream);
    case 6: return launch_c<6>(a, d, psi, f64, ev, stream);
    case 7: return launch_c<7>(a, d, psi, f64, ev, stream);
    case 8: return launch_c<8>(a, d, psi, f64, ev, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gpf
