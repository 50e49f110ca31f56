// Contracted Cartesian Gaussian values and gradients on the device.
//
// chi_mu(r) = P(x, y, z) * sum_k c_k exp(-a_k |r - A|^2)       (App. A, "Gaussian basis functions")
// with P = f_comp x^i y^j z^k, f_comp = 1/sqrt((2i-1)!!(2j-1)!!(2k-1)!!), and
// d chi / dx = (dP/dx) g - 2 x P sum_k c_k a_k exp(-a_k r^2).
#pragma once

#include "internal.h"

namespace kldi {

// exp for the FP32 basis values.  A library exp can carry a small systematic
// bias (a few hundredths of an ulp), which a quadrature of ~1e6 points turns
// into a visible energy error, so the FP32 path uses its own: Cody-Waite
// reduction x = n ln2 + r with ln2 = L_hi + L_lo (L_hi has 16 significant bits,
// so n L_hi is exact for |n| < 256), |r| <= ln2 / 2, then the Taylor series of
// e^r to degree 8 (remainder below 2e-10 relative) by Horner's rule, times 2^n.
// The last Horner step rounds to nearest, so the error is close to a single
// round-to-nearest and symmetric.  Results below 2^-125 are flushed to zero.
__device__ __forceinline__ float exp_rn(float x) {
  const float n = rintf(x * 1.4426950216293335f);
  float r = fmaf(-n, 0.693145751953125f, x);
  r = fmaf(-n, 1.428606765330187e-06f, r);
  float p = 2.4801587642286904e-05f;        // 1/8!
  p = fmaf(p, r, 0.00019841270113829523f);  // 1/7!
  p = fmaf(p, r, 0.0013888889225199819f);   // 1/6!
  p = fmaf(p, r, 0.008333333767950535f);    // 1/5!
  p = fmaf(p, r, 0.0416666679084301f);      // 1/4!
  p = fmaf(p, r, 0.1666666716337204f);      // 1/3!
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  if (n < -125.f) return 0.f;
  return p * __int_as_float(((int)n + 127) << 23);
}

// 1/sqrt(3) for the xx, yy, zz components: one FP64 constant, or an FP32
// hi/lo pair so the FP32 path does not inherit a fixed rounding of it.
__device__ __forceinline__ double mul_s3(double v) { return v * 0.57735026918962576451; }
__device__ __forceinline__ float mul_s3(float v) { return fmaf(v, 0.5773502588272095f, v * 1.0362416702491828e-08f); }

// Calls f(local_index, value, dx, dy, dz) for every basis function of basis
// block p (functions [32 p, 32 p + 32) that exist) at point (px, py, pz).
// Gradients are zero when GRAD is false.
// Point coordinates: FP64 absolute coordinates for T = double; for T = float
// coordinates relative to the grid block's anchor atom `anchor`, with shell
// centres taken from the anchor-relative hi/lo table, so that no fixed
// rounding of a centre enters the FP32 values.
template <typename T, bool GRAD, typename F>
__device__ __forceinline__ void for_block_functions(const BasisView& B, int p, T px, T py, T pz, F&& f,
                                                    int anchor = 0) {
  const int lo = p * kBasisBlk;
  const int hi = lo + kBasisBlk;
  const int sb = B.bb_shell_begin[p];
  const int se = B.bb_shell_end[p];
  for (int s = sb; s < se; ++s) {
    T dx, dy, dz;
    int l, fn_off;
    T g = T(0), gd = T(0);
    if constexpr (sizeof(T) == 8) {
      const DevShell sh = B.shells[s];
      l = sh.l;
      fn_off = sh.fn_off;
      dx = px - sh.cx;
      dy = py - sh.cy;
      dz = pz - sh.cz;
      const T r2 = dx * dx + dy * dy + dz * dz;
      for (int k = 0; k < sh.nprim; ++k) {
        const double a = B.alpha[sh.prim_off + k];
        const double e = B.coef[sh.prim_off + k] * exp(-a * r2);
        g += e;
        if (GRAD) gd += a * e;
      }
    } else {
      // packed shell record, anchor-relative centre (hi, lo), primitives as
      // FP32 hi/lo pairs of the exponent, coefficient and their product
      const int4 sh = B.shell_f[s];
      l = sh.x & 255;
      fn_off = sh.z;
      const float4* r = reinterpret_cast<const float4*>(B.relatom + ((size_t)anchor * B.natm + sh.w) * 8);
      const float4 r0 = r[0], r1 = r[1];
      dx = (px - r0.x) - r0.w;
      dy = (py - r0.y) - r1.x;
      dz = (pz - r0.z) - r1.y;
      const T r2 = dx * dx + dy * dy + dz * dz;
      const int np = sh.x >> 8;
      for (int k = 0; k < np; ++k) {
        const float4 pr = B.prim_f[sh.y + k];
        const float e = exp_rn(fmaf(-pr.x, r2, -pr.y * r2));
        g = fmaf(pr.z, e, fmaf(pr.w, e, g));
        if (GRAD) {
          const float2 ac = B.prim_ac[sh.y + k];
          gd = fmaf(ac.x, e, fmaf(ac.y, e, gd));
        }
      }
    }
    const T m2gd = T(-2) * gd;
    auto emit = [&](int mu, T P, T px_, T py_, T pz_) {
      if (mu >= lo && mu < hi) {
        if (GRAD)
          f(mu - lo, P * g, px_ * g + dx * m2gd * P, py_ * g + dy * m2gd * P, pz_ * g + dz * m2gd * P);
        else
          f(mu - lo, P * g, T(0), T(0), T(0));
      }
    };
    const int b = fn_off;
    if (l == 0) {
      emit(b, T(1), T(0), T(0), T(0));
    } else if (l == 1) {
      emit(b + 0, dx, T(1), T(0), T(0));
      emit(b + 1, dy, T(0), T(1), T(0));
      emit(b + 2, dz, T(0), T(0), T(1));
    } else {
      emit(b + 0, mul_s3(dx * dx), mul_s3(T(2) * dx), T(0), T(0));
      emit(b + 1, dx * dy, dy, dx, T(0));
      emit(b + 2, dx * dz, dz, T(0), dx);
      emit(b + 3, mul_s3(dy * dy), T(0), mul_s3(T(2) * dy), T(0));
      emit(b + 4, dy * dz, T(0), dz, dy);
      emit(b + 5, mul_s3(dz * dz), T(0), T(0), mul_s3(T(2) * dz));
    }
  }
}

}  // namespace kldi
