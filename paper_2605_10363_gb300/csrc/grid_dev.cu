// Becke partition weights of the molecular grid on the GPU (preprocessing,
// App. A "Numerical integration grids"): one thread per point, the same cell
// functions, multiplication order and 1e-40 cut-off as the host loop in
// grid.cpp.  FP64.
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace kldi {
namespace {

constexpr int kCache = 32;   // distances to the first atoms of the owner's neighbour order, per thread

__device__ __forceinline__ double becke_s_dev(double mu) {
  double p = mu;
  for (int k = 0; k < 3; ++k) p = 1.5 * p - 0.5 * p * p * p;
  return 0.5 * (1.0 - p);
}

__device__ __forceinline__ double dist_to(const double* __restrict__ A, int b, double x, double y, double z) {
  const double dx = x - A[3 * b], dy = y - A[3 * b + 1], dz = z - A[3 * b + 2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

__global__ void __launch_bounds__(128) k_becke(const double* __restrict__ xyz, const int32_t* __restrict__ owner,
                                               int64_t n, const double* __restrict__ A,
                                               const double* __restrict__ R, const int32_t* __restrict__ nbr,
                                               const double* __restrict__ raw_w, int natm, double* w) {
  __shared__ double dc[kCache][128];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  const int own = owner[i];
  const int32_t* order = nbr + (int64_t)own * natm;
  const int nc = natm < kCache ? natm : kCache;
  for (int k = 0; k < nc; ++k) dc[k][threadIdx.x] = dist_to(A, order[k], x, y, z);
  double sum = 0.0, pown = 0.0;
  for (int ib = 0; ib < natm; ++ib) {
    const int b = order[ib];
    const double db = ib < kCache ? dc[ib][threadIdx.x] : dist_to(A, b, x, y, z);
    const double* Rb = R + (int64_t)b * natm;
    double P = 1.0;
    for (int ic = 0; ic < natm; ++ic) {
      const int c = order[ic];
      if (c == b) continue;
      const double dcv = ic < kCache ? dc[ic][threadIdx.x] : dist_to(A, c, x, y, z);
      P *= becke_s_dev((db - dcv) / Rb[c]);
      if (P < 1e-40) {
        P = 0.0;
        break;
      }
    }
    sum += P;
    if (b == own) pown = P;
  }
  w[i] = raw_w[i] * (pown / sum);
}

template <class T>
struct Buf {
  T* p = nullptr;
  ~Buf() {
    if (p) cudaFree(p);
  }
};

template <class T>
kldi_status put(Buf<T>& b, const T* h, size_t n) {
  KLDI_TRY_CUDA(cudaMalloc(&b.p, sizeof(T) * (n ? n : 1)));
  if (n) KLDI_TRY_CUDA(cudaMemcpy(b.p, h, sizeof(T) * n, cudaMemcpyHostToDevice));
  return KLDI_OK;
}

}  // namespace

// w[k] = raw_w[k] P_owner / sum_b P_b for the nreal points (host arrays).
kldi_status becke_weights_device(int natm, const double* atom_xyz, const double* R, const int32_t* nbr,
                                 const double* xyz, const int32_t* owner, const double* raw_w, int64_t nreal,
                                 double* w) {
  if (nreal == 0) return KLDI_OK;
  Buf<double> dA, dR, dxyz, draw, dw;
  Buf<int32_t> dnbr, down;
  KLDI_TRY(put(dA, atom_xyz, (size_t)natm * 3));
  KLDI_TRY(put(dR, R, (size_t)natm * natm));
  KLDI_TRY(put(dnbr, nbr, (size_t)natm * natm));
  KLDI_TRY(put(dxyz, xyz, (size_t)nreal * 3));
  KLDI_TRY(put(down, owner, (size_t)nreal));
  KLDI_TRY(put(draw, raw_w, (size_t)nreal));
  KLDI_TRY_CUDA(cudaMalloc(&dw.p, sizeof(double) * nreal));
  k_becke<<<(unsigned)((nreal + 127) / 128), 128>>>(dxyz.p, down.p, nreal, dA.p, dR.p, dnbr.p, draw.p, natm, dw.p);
  KLDI_TRY_CUDA(cudaGetLastError());
  KLDI_TRY_CUDA(cudaMemcpy(w, dw.p, sizeof(double) * nreal, cudaMemcpyDeviceToHost));
  return KLDI_OK;
}

}  // namespace kldi
