// kldi_exc_energy_noalloc: E_xc = sum_i w_i f(rho_i, sigma_i) from a density
// the caller already holds on the device, without allocating any memory.
//
// It is the energy half of the functional kernel and its fixed-order
// reduction, with the per-block partial sums kept in a file-scope device
// array instead of plan-owned scratch.  Some callers may not allocate:
// code that runs while a stream is being captured into a CUDA graph (an
// allocation is not a capturable operation), hosts that reserve all device
// memory up front and forbid later cudaMalloc calls, and allocator or
// memory-pool callbacks that must not re-enter the allocator.  They can still
// obtain the exchange-correlation energy of a density through this call.
//
// The array g_partials (kMaxPartials doubles, 512 KiB) exists on every GPU
// that loads the library, until the process exits; each GPU has its own copy.
// The first call on a device looks up the array's device address with that
// device current (cudaGetSymbolAddress); make that first call outside any
// stream capture.  Every call overwrites the slots it uses before reading
// them, so nothing needs clearing; the array keeps the last call's partial
// sums.  All calls on one GPU share the array: calls whose GPU work overlaps
// (for example on two streams) race on it and must be ordered by the caller.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "internal.h"
#include "xc.cuh"

namespace kldi {
namespace {

constexpr int kMaxPartials = 65536;               // grid blocks of 128 points: at most 8,388,608 points
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_partials[kMaxPartials];

// Device address of g_partials, looked up once per device with that device
// current.  In host code the symbol name is only a host-side stand-in.  The
// slots are atomics: a call may read a slot while another thread's first call
// on the same device writes it (under g_setup_mutex).
std::atomic<double*> g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA of 128 threads per block of 128 points: w f summed in the same
// order as the plan path (warp sums, then (w0 + w1) + (w2 + w3)).
__global__ void k_energy_partials(const double* __restrict__ rho, const double* __restrict__ grad,
                                  const double* __restrict__ w, int64_t n, int xc, double rho_min, double* part) {
  __shared__ double red[4];
  const int64_t pt = (int64_t)blockIdx.x * kBlockPts + threadIdx.x;
  double e = 0.0;
  if (pt < n) {
    const double r = rho[pt];
    if (r >= rho_min) {
      if (xc == KLDI_XC_LDA_X) {
        e = w[pt] * xc_lda_x(r).f;
      } else {
        const double gx = grad[pt * 3], gy = grad[pt * 3 + 1], gz = grad[pt * 3 + 2];
        e = w[pt] * xc_pbe(r, gx * gx + gy * gy + gz * gz).f;
      }
    }
  }
  e = warp_sum_d(e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) part[blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
}

__global__ void k_energy_sum(const double* __restrict__ part, int64_t nb, double* exc) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < nb; k += blockDim.x) s += part[k];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum_d(v);
    if (threadIdx.x == 0) exc[0] = v;
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace kldi

extern "C" kldi_status kldi_exc_energy_noalloc(int xc, int64_t npoints, const double* rho, const double* grad,
                                               const double* w, double rho_min, double* Exc, void* stream) {
  return kldi::guarded("kldi_exc_energy_noalloc", [&]() -> kldi_status {
    using namespace kldi;
    if (xc != KLDI_XC_LDA_X && xc != KLDI_XC_PBE) {
      set_error("kldi_exc_energy_noalloc: functional must be KLDI_XC_LDA_X or KLDI_XC_PBE");
      return KLDI_EINVAL;
    }
    if (npoints <= 0 || !rho || !w || !Exc || (xc == KLDI_XC_PBE && !grad)) {
      set_error("kldi_exc_energy_noalloc: null pointer or npoints <= 0");
      return KLDI_EINVAL;
    }
    const int64_t nb = (npoints + kBlockPts - 1) / kBlockPts;
    if (nb > kMaxPartials) {
      set_error("kldi_exc_energy_noalloc: %lld points exceed the fixed maximum of %lld (%d blocks of %d)",
                (long long)npoints, (long long)kMaxPartials * kBlockPts, kMaxPartials, kBlockPts);
      return KLDI_EINVAL;
    }
    if (!on_device(rho) || !on_device(w) || !on_device(Exc) || (grad && !on_device(grad))) {
      set_error("kldi_exc_energy_noalloc: rho, grad, w and Exc must be device memory (host data would need a staging allocation)");
      return KLDI_EINVAL;
    }
    int dev = 0;
    KLDI_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
      set_error("kldi_exc_energy_noalloc: device ordinal %d out of range", dev);
      return KLDI_EUNSUPPORTED;
    }
    double* part = g_partials_addr[dev].load(std::memory_order_acquire);
    if (!part) {
      // first call on this device: resolve the device address of the array
      std::lock_guard<std::mutex> lk(g_setup_mutex);
      part = g_partials_addr[dev].load(std::memory_order_relaxed);
      if (!part) {
        void* p = nullptr;
        KLDI_TRY_CUDA(cudaGetSymbolAddress(&p, g_partials));
        part = static_cast<double*>(p);
        g_partials_addr[dev].store(part, std::memory_order_release);
      }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_energy_partials<<<(unsigned)nb, kBlockPts, 0, s>>>(rho, grad, w, npoints, xc, rho_min, part);
    KLDI_TRY_CUDA(cudaGetLastError());
    k_energy_sum<<<1, 1024, 0, s>>>(part, nb, Exc);
    KLDI_TRY_CUDA(cudaGetLastError());
    return KLDI_OK;
  });
}
