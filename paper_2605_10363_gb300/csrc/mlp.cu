// Learned functional: a 2 -> 64 -> 64 -> 2 MLP surrogate of the per-point
// PBE-form GGA (the evaluation between the density product and the V product,
// Sec. III-F; Eq. exc_quadrature).  The paper has no learned part; this file
// is the project's addition, in four kernels:
//
//  k_mlp_prepare    training inputs z = ((ln rho, ln sigma) - centre) / half
//                   and targets F* = f / e0, G* = v_rho / v0 of the analytic
//                   functional (FP64, stored FP32), valid = rho >= rho_min and
//                   inside the training box;
//  k_mlp_partials   forward + hand-written backward of the squared error over
//                   128 points per CTA (one thread per point, weights as FP32
//                   copies of their FP16 values in shared memory, FP32
//                   arithmetic); per-CTA partial gradients, loss and count;
//  k_mlp_reduce     fixed-order sum of the partials, divided by the count;
//  k_adam           Adam with bias correction on the FP32 master weights,
//                   refreshing their FP16 copies;
// and the inference kernels k_mlp_eval (per-point f, v_rho, v_sigma) and
// k_xc_mlp (the functional stage of the quadrature: the network replaces the
// analytic functional inside the box, the analytic form is the fallback).
//
// v_sigma is the exact derivative of the network's energy density: the
// forward pass carries the tangent d/dz2 through both layers.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "xc.cuh"
#include "xc_point.cuh"

namespace kldi {
namespace {

constexpr int kH = 64;
constexpr int kNP = KLDI_MLP_NPARAMS;
constexpr int O_W1 = 0;
constexpr int O_B1 = O_W1 + kH * 2;
constexpr int O_W2 = O_B1 + kH;
constexpr int O_B2 = O_W2 + kH * kH;
constexpr int O_W3 = O_B2 + kH;
constexpr int O_B3 = O_W3 + 2 * kH;
static_assert(O_B3 + 2 == kNP, "parameter layout");
static_assert(O_W2 % 4 == 0, "W2 rows are read as float4");
constexpr double kSigmaFloor = 1e-30;
constexpr int kPts = 128;          // points per CTA of the training kernel
constexpr int kLd = kPts + 1;      // padded row of the per-point activation tables
constexpr int kWPad = (kNP + 3) / 4 * 4;

// Training box as the kernels use it: z = (u - c) / s.
struct MlpMap {
  double c1, s1, c2, s2;
};

MlpMap map_of(const double* box) {
  return {0.5 * (box[0] + box[1]), 0.5 * (box[1] - box[0]), 0.5 * (box[2] + box[3]), 0.5 * (box[3] - box[2])};
}

__device__ __forceinline__ void load_weights(const __half* __restrict__ hw, float* W) {
  for (int k = threadIdx.x; k < kNP; k += blockDim.x) W[k] = __half2float(hw[k]);
}

// Inputs of one point: returns false outside the box.
__device__ __forceinline__ bool map_point(const MlpMap& M, double rho, double sigma, float& z1, float& z2) {
  const double a = (log(rho) - M.c1) / M.s1;
  const double b = (log(fmax(sigma, kSigmaFloor)) - M.c2) / M.s2;
  z1 = (float)a;
  z2 = (float)b;
  return fabs(a) <= 1.0 && fabs(b) <= 1.0;
}

// o = W3 tanh(W2 tanh(W1 z + b1) + b2) + b3 and d = d o1 / d z2.
__device__ __forceinline__ void mlp_forward(const float* __restrict__ W, float z1, float z2, float& o1, float& o2,
                                            float& d) {
  float h1[kH], t1[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) {
    const float a = fmaf(W[O_W1 + 2 * k], z1, fmaf(W[O_W1 + 2 * k + 1], z2, W[O_B1 + k]));
    const float h = tanhf(a);
    h1[k] = h;
    t1[k] = (1.f - h * h) * W[O_W1 + 2 * k + 1];      // d h1_k / d z2
  }
  float r1 = W[O_B3], r2 = W[O_B3 + 1], dd = 0.f;
#pragma unroll 2
  for (int j = 0; j < kH; ++j) {
    const float4* w4 = reinterpret_cast<const float4*>(W + O_W2 + j * kH);
    float a = W[O_B2 + j], t = 0.f;
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 w = w4[q];
      a = fmaf(w.x, h1[4 * q], a);
      a = fmaf(w.y, h1[4 * q + 1], a);
      a = fmaf(w.z, h1[4 * q + 2], a);
      a = fmaf(w.w, h1[4 * q + 3], a);
      t = fmaf(w.x, t1[4 * q], t);
      t = fmaf(w.y, t1[4 * q + 1], t);
      t = fmaf(w.z, t1[4 * q + 2], t);
      t = fmaf(w.w, t1[4 * q + 3], t);
    }
    const float h = tanhf(a);
    r1 = fmaf(W[O_W3 + j], h, r1);
    r2 = fmaf(W[O_W3 + kH + j], h, r2);
    dd = fmaf(W[O_W3 + j] * (1.f - h * h), t, dd);
  }
  o1 = r1;
  o2 = r2;
  d = dd;
}

// f, v_rho, v_sigma of one point: network inside the box, analytic outside,
// nothing below rho_min.
__device__ __forceinline__ XcOut mlp_point(const float* W, const MlpMap& M, double rho, double sigma,
                                           double rho_min, int& used) {
  XcOut o{0.0, 0.0, 0.0};
  used = 0;
  if (!(rho >= rho_min)) return o;
  float z1, z2;
  if (!map_point(M, rho, sigma, z1, z2)) return xc_pbe(rho, sigma);
  used = 1;
  float o1, o2, d;
  mlp_forward(W, z1, z2, o1, o2, d);
  const XcOut s = xc_lda_x(rho);
  o.f = s.f * (double)o1;
  o.vr = s.vr * (double)o2;
  o.vs = s.f * (double)d / (M.s2 * fmax(sigma, kSigmaFloor));
  return o;
}

__global__ void __launch_bounds__(128) k_mlp_eval(const __half* __restrict__ hw, MlpMap M, const double* rho,
                                                  const double* sigma, int64_t n, double rho_min, double* f,
                                                  double* vr, double* vs, int32_t* used) {
  __shared__ __align__(16) float W[kWPad];
  load_weights(hw, W);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int u;
  const XcOut o = mlp_point(W, M, rho[i], sigma[i], rho_min, u);
  f[i] = o.f;
  vr[i] = o.vr;
  vs[i] = o.vs;
  if (used) used[i] = u;
}

// Functional stage of the quadrature with the learned functional: one CTA of
// 128 threads per grid block, the same outputs as the analytic stage.
__global__ void __launch_bounds__(128) k_xc_mlp(GridView G, int64_t g0, double rho_min, MlpMap M,
                                                const __half* __restrict__ hw, const double* rho,
                                                const double* grad, double* xcoef, float4* xdf, double* eblk,
                                                float* pscale) {
  __shared__ __align__(16) float W[kWPad];
  __shared__ double red[4];
  load_weights(hw, W);
  __syncthreads();
  const int64_t g = g0 + blockIdx.x;
  const int64_t pt = g * kBlockPts + threadIdx.x;
  const double r = rho[pt];
  const double w = G.w[pt];
  const double gx = grad[pt * 3], gy = grad[pt * 3 + 1], gz = grad[pt * 3 + 2];
  int used;
  const XcOut o = mlp_point(W, M, r, gx * gx + gy * gy + gz * gz, rho_min, used);
  const double c = 2.0 * w * o.vs;
  xc_point_tail(g, pt, w * o.f, 0.5 * w * o.vr, c * gx, c * gy, c * gz, xcoef, xdf, eblk, pscale, red);
}

// ---------------------------------------------------------------------------
// Training.
__global__ void k_mlp_prepare(MlpMap M, const double* rho, const double* sigma, int64_t n, double rho_min,
                              float4* data, uint8_t* valid) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rho[i], s = sigma[i];
  float z1 = 0.f, z2 = 0.f, F = 0.f, Gt = 0.f;
  bool ok = r >= rho_min && map_point(M, r, s, z1, z2);
  if (ok) {
    const XcOut a = xc_pbe(r, s);
    const XcOut l = xc_lda_x(r);
    F = (float)(a.f / l.f);
    Gt = (float)(a.vr / l.vr);
  } else {
    z1 = z2 = 0.f;
  }
  data[i] = make_float4(z1, z2, F, Gt);
  valid[i] = ok ? 1 : 0;
}

// Batch element j in [j0, j0 + count) is training point (A j + C) mod n
// (A = 0: point j).  Shared memory: weights, then H1, H2 (later A1), D2 as
// [64][kLd] tables, then z and d loss / d o as [2][128].
constexpr int kTrainSmemFloats = kWPad + 3 * kH * kLd + 4 * kPts + 8;

__global__ void __launch_bounds__(kPts) k_mlp_partials(const float4* __restrict__ data,
                                                       const uint8_t* __restrict__ valid, int64_t n, int64_t A,
                                                       int64_t C, int64_t j0, int64_t count,
                                                       const __half* __restrict__ hw, float* part) {
  extern __shared__ __align__(16) float sm[];
  float* W = sm;
  float* H1 = W + kWPad;
  float* H2 = H1 + kH * kLd;      // reused for A1 = d loss / d (W1 z + b1)
  float* D2 = H2 + kH * kLd;      // d loss / d (W2 h1 + b2)
  float* Z = D2 + kH * kLd;       // [2][kPts]
  float* DO = Z + 2 * kPts;       // [2][kPts]
  float* red = DO + 2 * kPts;     // [8]
  load_weights(hw, W);
  __syncthreads();
  const int i = threadIdx.x;
  const int64_t j = j0 + (int64_t)blockIdx.x * kPts + i;
  float m = 0.f;
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
  if (j < j0 + count) {
    const int64_t idx = A ? (int64_t)(((unsigned long long)A * (unsigned long long)j + (unsigned long long)C) %
                                      (unsigned long long)n)
                          : j;
    if (valid[idx]) {
      m = 1.f;
      x = data[idx];
    }
  }
  // forward
  float h1[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) {
    const float a = fmaf(W[O_W1 + 2 * k], x.x, fmaf(W[O_W1 + 2 * k + 1], x.y, W[O_B1 + k]));
    h1[k] = tanhf(a);
    H1[k * kLd + i] = h1[k];
  }
  float o1 = W[O_B3], o2 = W[O_B3 + 1];
#pragma unroll 2
  for (int jj = 0; jj < kH; ++jj) {
    const float4* w4 = reinterpret_cast<const float4*>(W + O_W2 + jj * kH);
    float a = W[O_B2 + jj];
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 w = w4[q];
      a = fmaf(w.x, h1[4 * q], a);
      a = fmaf(w.y, h1[4 * q + 1], a);
      a = fmaf(w.z, h1[4 * q + 2], a);
      a = fmaf(w.w, h1[4 * q + 3], a);
    }
    const float h = tanhf(a);
    H2[jj * kLd + i] = h;
    o1 = fmaf(W[O_W3 + jj], h, o1);
    o2 = fmaf(W[O_W3 + kH + jj], h, o2);
  }
  // loss and its derivative with respect to the outputs (unnormalised sums)
  const float r1 = o1 - x.z, r2 = o2 - x.w;
  const float loss = m * (r1 * r1 + r2 * r2);
  const float do1 = 2.f * m * r1, do2 = 2.f * m * r2;
  Z[i] = x.x;
  Z[kPts + i] = x.y;
  DO[i] = do1;
  DO[kPts + i] = do2;
  // backward through layer 2 and the hidden layer
  float dh1[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) dh1[k] = 0.f;
#pragma unroll 2
  for (int jj = 0; jj < kH; ++jj) {
    const float h = H2[jj * kLd + i];
    const float da2 = (W[O_W3 + jj] * do1 + W[O_W3 + kH + jj] * do2) * (1.f - h * h);
    D2[jj * kLd + i] = da2;
    const float4* w4 = reinterpret_cast<const float4*>(W + O_W2 + jj * kH);
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 w = w4[q];
      dh1[4 * q] = fmaf(w.x, da2, dh1[4 * q]);
      dh1[4 * q + 1] = fmaf(w.y, da2, dh1[4 * q + 1]);
      dh1[4 * q + 2] = fmaf(w.z, da2, dh1[4 * q + 2]);
      dh1[4 * q + 3] = fmaf(w.w, da2, dh1[4 * q + 3]);
    }
  }
  __syncthreads();
  float* out = part + (int64_t)blockIdx.x * (kNP + 2);
  // dW3, db3 (from H2 and DO), db2 (from D2)
  for (int q = i; q < 2 * kH + 2; q += kPts) {
    float s = 0.f;
    if (q < 2 * kH) {
      const int c = q / kH, jj = q % kH;
      for (int p = 0; p < kPts; ++p) s = fmaf(DO[c * kPts + p], H2[jj * kLd + p], s);
      out[O_W3 + q] = s;
    } else {
      const int c = q - 2 * kH;
      for (int p = 0; p < kPts; ++p) s += DO[c * kPts + p];
      out[O_B3 + c] = s;
    }
  }
  if (i < kH) {
    float s = 0.f;
    for (int p = 0; p < kPts; ++p) s += D2[i * kLd + p];
    out[O_B2 + i] = s;
  }
  __syncthreads();
  float* A1 = H2;
#pragma unroll
  for (int k = 0; k < kH; ++k) A1[k * kLd + i] = dh1[k] * (1.f - h1[k] * h1[k]);
  __syncthreads();
  // dW2: a 4 x 8 tile per thread
  {
    const int jb = (i >> 3) * 4, kb = (i & 7) * 8;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    for (int p = 0; p < kPts; ++p) {
      float dv[4], hv[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) dv[a] = D2[(jb + a) * kLd + p];
#pragma unroll
      for (int b = 0; b < 8; ++b) hv[b] = H1[(kb + b) * kLd + p];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(dv[a], hv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) out[O_W2 + (jb + a) * kH + kb + b] = acc[a][b];
  }
  // dW1, db1 (from A1 and Z)
  for (int q = i; q < 3 * kH; q += kPts) {
    float s = 0.f;
    if (q < 2 * kH) {
      const int k = q >> 1, c = q & 1;
      for (int p = 0; p < kPts; ++p) s = fmaf(A1[k * kLd + p], Z[c * kPts + p], s);
      out[O_W1 + q] = s;
    } else {
      const int k = q - 2 * kH;
      for (int p = 0; p < kPts; ++p) s += A1[k * kLd + p];
      out[O_B1 + k] = s;
    }
  }
  // loss and count
  float l = loss, c = m;
  for (int o = 16; o > 0; o >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((i & 31) == 0) {
    red[i >> 5] = l;
    red[4 + (i >> 5)] = c;
  }
  __syncthreads();
  if (i == 0) {
    out[kNP] = (red[0] + red[1]) + (red[2] + red[3]);
    out[kNP + 1] = (red[4] + red[5]) + (red[6] + red[7]);
  }
}

// grad = sum of the partials / count, in a fixed order; loss likewise.
__global__ void k_mlp_reduce(const float* __restrict__ part, int64_t nctas, float* grad, float* loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kNP) return;
  double cnt = 0.0, s = 0.0;
  for (int64_t c = 0; c < nctas; ++c) {
    cnt += part[c * (kNP + 2) + kNP + 1];
    s += part[c * (kNP + 2) + k];
  }
  const double v = cnt > 0.0 ? s / cnt : 0.0;
  if (k < kNP) grad[k] = (float)v;
  else if (loss) *loss = (float)v;
}

// omb1 = 1 - beta1 and omb2 = 1 - beta2 come from the host in FP64 (1 - 0.999f
// in FP32 is 5e-5 off 1e-3).
__global__ void k_adam(float* p, __half* ph, float* m, float* v, const float* __restrict__ g, float lr, float b1,
                       float omb1, float b2, float omb2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNP) return;
  const float gk = g[k];
  const float mk = fmaf(b1, m[k], omb1 * gk);
  const float vk = fmaf(b2, v[k], omb2 * gk * gk);
  m[k] = mk;
  v[k] = vk;
  const float pk = p[k] - lr * (mk * c1) / (sqrtf(vk * c2) + eps);
  p[k] = pk;
  ph[k] = __float2half_rn(pk);
}

__global__ void k_to_half(const float* p, __half* ph) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kNP) ph[k] = __float2half_rn(p[k]);
}

// Device buffer released at scope exit.
template <class T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  kldi_status alloc(size_t n) {
    if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error("device allocation of %zu bytes failed", sizeof(T) * n);
      return KLDI_ENOMEM;
    }
    return KLDI_OK;
  }
};

// rho / sigma on the device (copied when they are host arrays).
kldi_status device_inputs(const double* rho, const double* sigma, int64_t n, DevBuf<double>& tmp,
                          const double*& drho, const double*& dsig, cudaStream_t s) {
  drho = rho;
  dsig = sigma;
  const bool hr = !is_device_ptr(rho), hs = !is_device_ptr(sigma);
  if (hr || hs) {
    KLDI_TRY(tmp.alloc(2 * (size_t)n));
    if (hr) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(tmp.p, rho, 8 * n, cudaMemcpyHostToDevice, s));
      drho = tmp.p;
    }
    if (hs) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(tmp.p + n, sigma, 8 * n, cudaMemcpyHostToDevice, s));
      dsig = tmp.p + n;
    }
  }
  return KLDI_OK;
}

kldi_status ensure_parts(kldi_mlp* M, int64_t nctas) {
  if (M->part_cap >= nctas) return KLDI_OK;
  if (M->d_part) cudaFree(M->d_part);
  M->d_part = nullptr;
  M->part_cap = 0;
  if (cudaMalloc(&M->d_part, sizeof(float) * (kNP + 2) * nctas) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of the partial gradients failed");
    return KLDI_ENOMEM;
  }
  M->part_cap = nctas;
  return KLDI_OK;
}

kldi_status set_train_smem() {
  return once_per_device([]() -> kldi_status {
    KLDI_TRY_CUDA(cudaFuncSetAttribute(k_mlp_partials, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kTrainSmemFloats * (int)sizeof(float)));
    return KLDI_OK;
  });
}

kldi_status launch_partials(kldi_mlp* M, const float4* data, const uint8_t* valid, int64_t n, int64_t A, int64_t C,
                            int64_t j0, int64_t count, float* loss_out, cudaStream_t s) {
  const int64_t nctas = (count + kPts - 1) / kPts;
  KLDI_TRY(ensure_parts(M, nctas));
  KLDI_TRY(set_train_smem());
  k_mlp_partials<<<(unsigned)nctas, kPts, kTrainSmemFloats * sizeof(float), s>>>(data, valid, n, A, C, j0, count,
                                                                                   M->d_half, M->d_part);
  KLDI_TRY_CUDA(cudaGetLastError());
  k_mlp_reduce<<<(kNP + 1 + 255) / 256, 256, 0, s>>>(M->d_part, nctas, M->d_grad, loss_out);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

kldi_status launch_adam(kldi_mlp* M, const float* grad, double lr, double b1, double b2, double eps,
                        cudaStream_t s) {
  M->step += 1;
  const double c1 = 1.0 / (1.0 - std::pow(b1, (double)M->step));
  const double c2 = 1.0 / (1.0 - std::pow(b2, (double)M->step));
  k_adam<<<(kNP + 255) / 256, 256, 0, s>>>(M->d_param, M->d_half, M->d_m, M->d_v, grad, (float)lr, (float)b1,
                                            (float)(1.0 - b1), (float)b2, (float)(1.0 - b2), (float)eps, (float)c1,
                                            (float)c2);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

kldi_status launch_xc_mlp(const kldi_plan* P, const Batch& b, const double* rho, const double* grad,
                          cudaStream_t s) {
  const int64_t n = b.g1 - b.g0;
  if (n == 0) return KLDI_OK;
  k_xc_mlp<<<(unsigned)n, kBlockPts, 0, s>>>(P->grid_view(), b.g0, P->opt.rho_min, map_of(P->mlp->box),
                                             P->mlp->d_half, rho, grad, P->d_xcoef,
                                             P->prec == KLDI_BF16X10 ? P->d_xdf : nullptr, P->d_eblk,
                                             P->prec == KLDI_FP64 ? nullptr : P->d_pscale);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

}  // namespace kldi

using namespace kldi;

extern "C" kldi_status kldi_mlp_create(const float* params, const double* box, kldi_mlp** out) {
  return kldi::guarded("kldi_mlp_create", [&]() -> kldi_status {
    if (!params || !box || !out) {
      set_error("kldi_mlp_create: null argument");
      return KLDI_EINVAL;
    }
    *out = nullptr;
    if (!(box[1] > box[0]) || !(box[3] > box[2]) || !std::isfinite(box[0]) || !std::isfinite(box[1]) ||
        !std::isfinite(box[2]) || !std::isfinite(box[3])) {
      set_error("kldi_mlp_create: the box needs lo < hi for both inputs");
      return KLDI_EINVAL;
    }
    kldi_mlp* M = new kldi_mlp();
    auto fail = [&](kldi_status st) {
      kldi_mlp_free(M);
      return st;
    };
    cudaGetDevice(&M->device);
    std::memcpy(M->box, box, sizeof(M->box));
    const size_t nb = sizeof(float) * kNP;
    if (cudaMalloc(&M->d_param, nb) != cudaSuccess || cudaMalloc(&M->d_half, sizeof(__half) * kNP) != cudaSuccess ||
        cudaMalloc(&M->d_m, nb) != cudaSuccess || cudaMalloc(&M->d_v, nb) != cudaSuccess ||
        cudaMalloc(&M->d_grad, nb) != cudaSuccess || cudaMalloc(&M->d_loss, sizeof(float) * 2) != cudaSuccess) {
      cudaGetLastError();
      set_error("kldi_mlp_create: device allocation failed");
      return fail(KLDI_ENOMEM);
    }
    if (cudaMemcpy(M->d_param, params, nb, is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(M->d_m, 0, nb) != cudaSuccess || cudaMemset(M->d_v, 0, nb) != cudaSuccess) {
      set_error("kldi_mlp_create: %s", cudaGetErrorString(cudaGetLastError()));
      return fail(KLDI_ECUDA);
    }
    k_to_half<<<(kNP + 255) / 256, 256>>>(M->d_param, M->d_half);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      set_error("kldi_mlp_create: %s", cudaGetErrorString(cudaGetLastError()));
      return fail(KLDI_ECUDA);
    }
    *out = M;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_mlp_get_params(const kldi_mlp* M, float* params) {
  return kldi::guarded("kldi_mlp_get_params", [&]() -> kldi_status {
    if (!M || !params) {
      set_error("kldi_mlp_get_params: null argument");
      return KLDI_EINVAL;
    }
    KLDI_TRY_CUDA(cudaDeviceSynchronize());
    KLDI_TRY_CUDA(cudaMemcpy(params, M->d_param, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_mlp_get_state(const kldi_mlp* M, float* state, int64_t* step) {
  return kldi::guarded("kldi_mlp_get_state", [&]() -> kldi_status {
    if (!M || !state || !step) {
      set_error("kldi_mlp_get_state: null argument");
      return KLDI_EINVAL;
    }
    KLDI_TRY_CUDA(cudaDeviceSynchronize());
    KLDI_TRY_CUDA(cudaMemcpy(state, M->d_param, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
    KLDI_TRY_CUDA(cudaMemcpy(state + kNP, M->d_m, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
    KLDI_TRY_CUDA(cudaMemcpy(state + 2 * kNP, M->d_v, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
    *step = M->step;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_mlp_set_state(kldi_mlp* M, const float* state, int64_t step) {
  return kldi::guarded("kldi_mlp_set_state", [&]() -> kldi_status {
    if (!M || !state || step < 0) {
      set_error("kldi_mlp_set_state: null argument or negative step");
      return KLDI_EINVAL;
    }
    KLDI_TRY_CUDA(cudaDeviceSynchronize());
    KLDI_TRY_CUDA(cudaMemcpy(M->d_param, state, sizeof(float) * kNP, cudaMemcpyHostToDevice));
    KLDI_TRY_CUDA(cudaMemcpy(M->d_m, state + kNP, sizeof(float) * kNP, cudaMemcpyHostToDevice));
    KLDI_TRY_CUDA(cudaMemcpy(M->d_v, state + 2 * kNP, sizeof(float) * kNP, cudaMemcpyHostToDevice));
    k_to_half<<<(kNP + 255) / 256, 256>>>(M->d_param, M->d_half);
    KLDI_TRY_CUDA(cudaGetLastError());
    KLDI_TRY_CUDA(cudaDeviceSynchronize());
    M->step = step;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_mlp_loss_grad(kldi_mlp* M, const double* rho, const double* sigma, int64_t n,
                                          double rho_min, float* grad, float* loss) {
  return kldi::guarded("kldi_mlp_loss_grad", [&]() -> kldi_status {
    if (!M || !rho || !sigma || !grad || !loss || n <= 0 || n >= (int64_t(1) << 31)) {
      set_error("kldi_mlp_loss_grad: null argument or n out of range");
      return KLDI_EINVAL;
    }
    cudaStream_t s = nullptr;
    DevBuf<double> tmp;
    const double *drho, *dsig;
    KLDI_TRY(device_inputs(rho, sigma, n, tmp, drho, dsig, s));
    DevBuf<float4> data;
    DevBuf<uint8_t> valid;
    KLDI_TRY(data.alloc(n));
    KLDI_TRY(valid.alloc(n));
    k_mlp_prepare<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(map_of(M->box), drho, dsig, n, rho_min, data.p,
                                                               valid.p);
    KLDI_TRY_CUDA(cudaGetLastError());
    KLDI_TRY(launch_partials(M, data.p, valid.p, n, 0, 0, 0, n, M->d_loss, s));
    KLDI_TRY_CUDA(cudaMemcpyAsync(grad, M->d_grad, sizeof(float) * kNP, cudaMemcpyDeviceToHost, s));
    KLDI_TRY_CUDA(cudaMemcpyAsync(loss, M->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    KLDI_TRY_CUDA(cudaStreamSynchronize(s));
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_mlp_adam_step(kldi_mlp* M, const float* grad, double lr, double beta1, double beta2,
                                          double eps) {
  return kldi::guarded("kldi_mlp_adam_step", [&]() -> kldi_status {
    if (!M || !grad || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
        !(eps >= 0.0)) {
      set_error("kldi_mlp_adam_step: invalid argument");
      return KLDI_EINVAL;
    }
    const float* g = grad;
    if (!is_device_ptr(grad)) {
      KLDI_TRY_CUDA(cudaMemcpy(M->d_grad, grad, sizeof(float) * kNP, cudaMemcpyHostToDevice));
      g = M->d_grad;
    }
    KLDI_TRY(launch_adam(M, g, lr, beta1, beta2, eps, nullptr));
    KLDI_TRY_CUDA(cudaDeviceSynchronize());
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_mlp_train(kldi_mlp* M, const double* rho, const double* sigma, int64_t n,
                                      const kldi_train_options* opt, float* loss_per_epoch) {
  return kldi::guarded("kldi_mlp_train", [&]() -> kldi_status {
    if (!M || !rho || !sigma || !opt || n <= 0 || n >= (int64_t(1) << 31) || opt->epochs < 1 || opt->batch < 1 ||
        opt->batch > 65536 || !(opt->lr0 >= 0.0) || !(opt->lr1 >= 0.0) || !(opt->beta1 >= 0.0 && opt->beta1 < 1.0) ||
        !(opt->beta2 >= 0.0 && opt->beta2 < 1.0) || !(opt->eps >= 0.0)) {
      set_error("kldi_mlp_train: invalid argument");
      return KLDI_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(opt->stream);
    DevBuf<double> tmp;
    const double *drho, *dsig;
    KLDI_TRY(device_inputs(rho, sigma, n, tmp, drho, dsig, s));
    DevBuf<float4> data;
    DevBuf<uint8_t> valid;
    KLDI_TRY(data.alloc(n));
    KLDI_TRY(valid.alloc(n));
    k_mlp_prepare<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(map_of(M->box), drho, dsig, n, opt->rho_min, data.p,
                                                               valid.p);
    KLDI_TRY_CUDA(cudaGetLastError());
    const int64_t per_epoch = (n + opt->batch - 1) / opt->batch;
    const int64_t total = per_epoch * opt->epochs;
    DevBuf<float> hist;
    KLDI_TRY(hist.alloc(total));
    // multiplier of the affine permutation: coprime with n
    uint64_t A = (0x9E3779B97F4A7C15ull % (uint64_t)n) | 1ull;
    if (n == 1) A = 1;
    while (gcd_u64(A, (uint64_t)n) != 1) A += 1;
    const double kPi = 3.14159265358979323846;
    int64_t step = 0;
    for (int e = 0; e < opt->epochs; ++e) {
      const uint64_t C = (uint64_t)(((unsigned __int128)(uint64_t)(e + 1) * 0xD1B54A32D192ED03ull) % (uint64_t)n);
      for (int64_t b = 0; b < per_epoch; ++b, ++step) {
        const int64_t j0 = b * opt->batch;
        const int64_t cnt = std::min<int64_t>(opt->batch, n - j0);
        KLDI_TRY(launch_partials(M, data.p, valid.p, n, (int64_t)A, (int64_t)C, j0, cnt, hist.p + step, s));
        const double lr = total <= 1 ? opt->lr0
                                     : opt->lr1 + 0.5 * (opt->lr0 - opt->lr1) *
                                                      (1.0 + std::cos(kPi * (double)step / (double)(total - 1)));
        KLDI_TRY(launch_adam(M, M->d_grad, lr, opt->beta1, opt->beta2, opt->eps, s));
      }
    }
    std::vector<float> h(total);
    KLDI_TRY_CUDA(cudaMemcpyAsync(h.data(), hist.p, sizeof(float) * total, cudaMemcpyDeviceToHost, s));
    KLDI_TRY_CUDA(cudaStreamSynchronize(s));
    if (loss_per_epoch)
      for (int e = 0; e < opt->epochs; ++e) {
        double acc = 0.0;
        for (int64_t b = 0; b < per_epoch; ++b) acc += h[e * per_epoch + b];
        loss_per_epoch[e] = (float)(acc / (double)per_epoch);
      }
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_mlp_eval(const kldi_mlp* M, const double* rho, const double* sigma, int64_t n,
                                     double rho_min, double* f, double* vrho, double* vsigma, int32_t* used) {
  return kldi::guarded("kldi_mlp_eval", [&]() -> kldi_status {
    if (!M || !rho || !sigma || !f || !vrho || !vsigma || n <= 0) {
      set_error("kldi_mlp_eval: null argument or n <= 0");
      return KLDI_EINVAL;
    }
    const bool host_out = !is_device_ptr(f);
    if (is_device_ptr(vrho) == host_out || is_device_ptr(vsigma) == host_out ||
        (used && is_device_ptr(used) == host_out)) {
      set_error("kldi_mlp_eval: f, vrho, vsigma and used must be all host or all device memory");
      return KLDI_EINVAL;
    }
    cudaStream_t s = nullptr;
    DevBuf<double> tmp;
    const double *drho, *dsig;
    KLDI_TRY(device_inputs(rho, sigma, n, tmp, drho, dsig, s));
    DevBuf<double> out;
    DevBuf<int32_t> dused;
    double *df = f, *dvr = vrho, *dvs = vsigma;
    int32_t* du = used;
    if (host_out) {
      KLDI_TRY(out.alloc(3 * (size_t)n));
      df = out.p;
      dvr = out.p + n;
      dvs = out.p + 2 * n;
      if (used) {
        KLDI_TRY(dused.alloc(n));
        du = dused.p;
      }
    }
    k_mlp_eval<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(M->d_half, map_of(M->box), drho, dsig, n, rho_min, df,
                                                            dvr, dvs, du);
    KLDI_TRY_CUDA(cudaGetLastError());
    if (host_out) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(f, df, 8 * n, cudaMemcpyDeviceToHost, s));
      KLDI_TRY_CUDA(cudaMemcpyAsync(vrho, dvr, 8 * n, cudaMemcpyDeviceToHost, s));
      KLDI_TRY_CUDA(cudaMemcpyAsync(vsigma, dvs, 8 * n, cudaMemcpyDeviceToHost, s));
      if (used) KLDI_TRY_CUDA(cudaMemcpyAsync(used, du, 4 * n, cudaMemcpyDeviceToHost, s));
      KLDI_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_set_mlp(kldi_plan* P, const kldi_mlp* M) {
  return kldi::guarded("kldi_plan_set_mlp", [&]() -> kldi_status {
    if (!P) {
      set_error("kldi_plan_set_mlp: null plan");
      return KLDI_EINVAL;
    }
    if (M && !P->gga) {
      set_error("kldi_plan_set_mlp: the learned functional is a GGA; screen the plan with KLDI_XC_PBE");
      return KLDI_EINVAL;
    }
    if (M && M->device != P->device) {
      set_error("kldi_plan_set_mlp: network and plan live on different devices");
      return KLDI_EINVAL;
    }
    P->mlp = M;
    return KLDI_OK;
  });
}

extern "C" void kldi_mlp_free(kldi_mlp* M) {
  if (!M) return;
  cudaFree(M->d_param);
  cudaFree(M->d_half);
  cudaFree(M->d_m);
  cudaFree(M->d_v);
  cudaFree(M->d_grad);
  cudaFree(M->d_part);
  cudaFree(M->d_loss);
  delete M;
}
