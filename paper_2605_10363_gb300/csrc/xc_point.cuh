// Per-point tail of the functional stage, shared by the analytic and the
// learned functional kernels: the X coefficients (a, b) = (w v_rho / 2,
// 2 w v_sigma grad rho), in FP64 and as FP32 hi / lo pairs (so that the
// double-float X kernel needs no FP64 arithmetic), the V-product balance c_i
// and the grid block's E_xc partial sum (one CTA of 128 threads per grid
// block).
#pragma once

#include "internal.h"

namespace kldi {

__device__ __forceinline__ double xc_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void xc_point_tail(int64_t g, int64_t pt, double e, double a, double bx, double by,
                                              double bz, double* xcoef, float4* xdf, double* eblk, float* pscale,
                                              double* red) {
  xcoef[pt * 4 + 0] = a;
  xcoef[pt * 4 + 1] = bx;
  xcoef[pt * 4 + 2] = by;
  xcoef[pt * 4 + 3] = bz;
  if (xdf) {
    const float ah = (float)a, bxh = (float)bx, byh = (float)by, bzh = (float)bz;
    xdf[pt * 2] = make_float4(ah, bxh, byh, bzh);
    xdf[pt * 2 + 1] = make_float4((float)(a - (double)ah), (float)(bx - (double)bxh), (float)(by - (double)byh),
                                  (float)(bz - (double)bzh));
  }
  if (pscale) {
    // balance c_i = 2^round(log2(|a| + |b|) / 2): the V product uses Phi c and X / c,
    // whose magnitudes are then alike at every point (X ~ (|a| + |b|) Phi).  A point
    // with X = 0 (zero weight, rho below rho_min) adds nothing to Phi^T X: c_i = 0
    // drops its Phi row too, so it cannot inflate a function's column maximum.
    const double m = fabs(a) + sqrt(bx * bx + by * by + bz * bz);
    float c = 0.f;
    if (m > 0.0) c = ldexpf(1.f, (int)lrint(0.5 * log2(m)));
    pscale[pt] = c;
  }
  // E_xc of the block: warp sums, then (w0 + w1) + (w2 + w3)
  e = xc_warp_sum(e);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = e;
  __syncthreads();
  if (threadIdx.x == 0) eblk[g] = (red[0] + red[1]) + (red[2] + red[3]);
}

}  // namespace kldi
