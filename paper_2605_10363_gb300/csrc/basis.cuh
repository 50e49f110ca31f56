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
// n = rint(x log2 e) as (y + 1.5 x 2^23) - 1.5 x 2^23 with y = x log2 e rounded
// (exact for |y| < 2^22, ties to even); the bits of y + 1.5 x 2^23 hold n.
__device__ __forceinline__ float exp_rn(float x) {
  const float t = __fadd_rn(__fmul_rn(x, 1.4426950216293335f), 12582912.f);
  const float n = __fsub_rn(t, 12582912.f);
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
  return p * __int_as_float((__float_as_int(t) - 0x4B400000 + 127) << 23);
}

// 1/sqrt(3) for the xx, yy, zz components: one FP64 constant, or an FP32
// hi/lo pair so the FP32 path does not inherit a fixed rounding of it.
__device__ __forceinline__ double mul_s3(double v) { return v * 0.57735026918962576451; }
__device__ __forceinline__ float mul_s3(float v) { return fmaf(v, 0.5773502588272095f, v * 1.0362416702491828e-08f); }

// Calls f(local index, value, dx, dy, dz) for the functions of one shell
// whose index relative to the basis block, first + c, lies in [0, 32):
// chi = P g, d chi / dr_a = (d_a P) g - 2 r_a P gd with gd = sum_k c_k a_k e^{-a_k r^2}.
template <typename T, bool GRAD, typename F>
__device__ __forceinline__ void emit_shell(int l, int first, T dx, T dy, T dz, T g, T gd, F&& f) {
  const T m2gd = T(-2) * gd;
  auto emit = [&](int c, T P, T px_, T py_, T pz_) {
    const int mu = first + c;
    if (mu >= 0 && mu < kBasisBlk) {
      if (GRAD)
        f(mu, P * g, px_ * g + dx * m2gd * P, py_ * g + dy * m2gd * P, pz_ * g + dz * m2gd * P);
      else
        f(mu, P * g, T(0), T(0), T(0));
    }
  };
  if (l == 0) {
    emit(0, T(1), T(0), T(0), T(0));
  } else if (l == 1) {
    emit(0, dx, T(1), T(0), T(0));
    emit(1, dy, T(0), T(1), T(0));
    emit(2, dz, T(0), T(0), T(1));
  } else {
    emit(0, mul_s3(dx * dx), mul_s3(T(2) * dx), T(0), T(0));
    emit(1, dx * dy, dy, dx, T(0));
    emit(2, dx * dz, dz, T(0), dx);
    emit(3, mul_s3(dy * dy), T(0), mul_s3(T(2) * dy), T(0));
    emit(4, dy * dz, T(0), dz, dy);
    emit(5, mul_s3(dz * dz), T(0), T(0), mul_s3(T(2) * dz));
  }
}

// Contracted radial factor of the FP32 path: g = sum_k c_k e^{-a_k r^2} and
// gd = sum_k c_k a_k e^{-a_k r^2} from hi/lo pairs of a, c and a c.
template <bool GRAD>
__device__ __forceinline__ void radial_f(const float4* pf, const float2* pac, int np, float r2, float& g,
                                         float& gd) {
  g = 0.f;
  gd = 0.f;
  for (int k = 0; k < np; ++k) {
    const float4 pr = pf[k];
    const float e = exp_rn(fmaf(-pr.x, r2, -pr.y * r2));
    g = fmaf(pr.z, e, fmaf(pr.w, e, g));
    if (GRAD) {
      const float2 ac = pac[k];
      gd = fmaf(ac.x, e, fmaf(ac.y, e, gd));
    }
  }
}

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
  const int sb = B.bb_shell_begin[p];
  const int se = B.bb_shell_end[p];
  for (int s = sb; s < se; ++s) {
    if constexpr (sizeof(T) == 8) {
      const DevShell sh = B.shells[s];
      const T dx = px - sh.cx, dy = py - sh.cy, dz = pz - sh.cz;
      const T r2 = dx * dx + dy * dy + dz * dz;
      T g = T(0), gd = T(0);
      for (int k = 0; k < sh.nprim; ++k) {
        const double a = B.alpha[sh.prim_off + k];
        const double e = B.coef[sh.prim_off + k] * exp(-a * r2);
        g += e;
        if (GRAD) gd += a * e;
      }
      emit_shell<T, GRAD>(sh.l, sh.fn_off - lo, dx, dy, dz, g, gd, f);
    } else {
      // packed shell record, anchor-relative centre (hi, lo), primitives as
      // FP32 hi/lo pairs of the exponent, coefficient and their product
      const int4 sh = B.shell_f[s];
      const float4* r = reinterpret_cast<const float4*>(B.relatom + ((size_t)anchor * B.natm + sh.w) * 8);
      const float4 r0 = r[0], r1 = r[1];
      const float dx = (px - r0.x) - r0.w, dy = (py - r0.y) - r1.x, dz = (pz - r0.z) - r1.y;
      const float r2 = dx * dx + dy * dy + dz * dz;
      float g, gd;
      radial_f<GRAD>(B.prim_f + sh.y, B.prim_ac + sh.y, sh.x >> 8, r2, g, gd);
      emit_shell<float, GRAD>(sh.x & 255, sh.z - lo, dx, dy, dz, g, gd, f);
    }
  }
}

// Shared-memory copy of one basis block's shells, for the FP32 evaluation at
// the points of one grid block: shell centres relative to the grid block's
// anchor atom (hi, lo), a packed header and the primitives.  Every thread of
// the evaluation reads the same record, so the reads are broadcasts, and no
// load depends on another (the global tables chain shell -> centre and
// shell -> primitives).  Blocks with more shells or primitives than the
// record holds are evaluated from the global tables; both give the same bits.
constexpr int kRecShells = 40;
constexpr int kRecPrims = 80;
struct BlockRec {
  float4 c0[kRecShells];   // x hi, y hi, z hi, x lo of A_atom - A_anchor
  float4 c1[kRecShells];   // y lo, z lo, header (l | nprim << 8 | (first + 64) << 16), first primitive
  float4 pf[kRecPrims];    // alpha hi, alpha lo, coef hi, coef lo
  float2 pac[kRecPrims];   // alpha coef hi, lo
  float ds[kBasisBlk];     // per-function factor, filled by the caller where needed
  int atom[kRecShells];    // atom of each shell
  int nshell;
  int split;               // first shell of the second half (about half of the functions each)
  int pad[2];
};

// True when basis block p fits a BlockRec (the same answer on every thread).
__device__ __forceinline__ bool block_rec_fits(const BasisView& B, int p) {
  const int sb = B.bb_shell_begin[p], se = B.bb_shell_end[p];
  if (se - sb > kRecShells) return false;
  if (se == sb) return true;
  const int4 a = B.shell_f[sb], z = B.shell_f[se - 1];
  return (z.y + (z.x >> 8)) - a.y <= kRecPrims;
}

// Fills rec for basis block p at anchor atom `anchor`, cooperatively over
// threads t = 0 .. nthr - 1 (the caller synchronises before the reads).
__device__ __forceinline__ void stage_block_rec(const BasisView& B, int p, int anchor, BlockRec* rec, int t,
                                                int nthr) {
  const int sb = B.bb_shell_begin[p], se = B.bb_shell_end[p];
  if (t == 0) {
    rec->nshell = se - sb;
    rec->split = B.bb_split[p];
  }
  if (se == sb) return;
  const int pbase = B.shell_f[sb].y;
  const int4 z = B.shell_f[se - 1];
  const int np = z.y + (z.x >> 8) - pbase;
  const int lo = p * kBasisBlk;
  for (int s = t; s < se - sb; s += nthr) {
    const int4 sh = B.shell_f[sb + s];
    const float4* r = reinterpret_cast<const float4*>(B.relatom + ((size_t)anchor * B.natm + sh.w) * 8);
    const float4 r0 = r[0], r1 = r[1];
    const int hdr = (sh.x & 0xffff) | ((sh.z - lo + 64) << 16);
    rec->c0[s] = r0;
    rec->c1[s] = make_float4(r1.x, r1.y, __int_as_float(hdr), __int_as_float(sh.y - pbase));
    rec->atom[s] = sh.w;
  }
  for (int k = t; k < np; k += nthr) {
    rec->pf[k] = B.prim_f[pbase + k];
    rec->pac[k] = B.prim_ac[pbase + k];
  }
}

// for_block_functions<float> from a staged record (same arithmetic, same bits).
// Shells s0, s0 + sstep, ... (all by default).
template <bool GRAD, typename F>
__device__ __forceinline__ void for_rec_functions(const BlockRec* rec, float px, float py, float pz, F&& f,
                                                  int s0 = 0, int sstep = 1) {
  const int ns = rec->nshell;
  for (int s = s0; s < ns; s += sstep) {
    const float4 c0 = rec->c0[s], c1 = rec->c1[s];
    const int hdr = __float_as_int(c1.z), pi = __float_as_int(c1.w);
    const float dx = (px - c0.x) - c0.w, dy = (py - c0.y) - c1.x, dz = (pz - c0.z) - c1.y;
    const float r2 = dx * dx + dy * dy + dz * dz;
    float g, gd;
    radial_f<GRAD>(rec->pf + pi, rec->pac + pi, (hdr >> 8) & 255, r2, g, gd);
    emit_shell<float, GRAD>(hdr & 255, (hdr >> 16) - 64, dx, dy, dz, g, gd, f);
  }
}

// First and second derivatives of the functions of a staged block, FP32, for
// the nuclear gradient (accuracy ~1e-7 relative; no hi/lo compensation).
// With chi = P g(r^2), g = sum c e^{-a r^2}, g1 = sum c a e, g2 = sum c a^2 e:
//   d_a chi = (d_a P) g - 2 r_a P g1
//   d_a d_b chi = (d_a d_b P) g - 2 (d_a P r_b + d_b P r_a) g1 + P (4 r_a r_b g2 - 2 delta_ab g1)
// Calls f(atom, nu, d[3], h[6]) with h = (xx, xy, xz, yy, yz, zz) (zero when
// HESS is false).
template <bool HESS, typename F>
__device__ __forceinline__ void for_rec_derivatives(const BlockRec* rec, float px, float py, float pz, F&& f) {
  const int ns = rec->nshell;
  for (int s = 0; s < ns; ++s) {
    const float4 c0 = rec->c0[s], c1 = rec->c1[s];
    const int hdr = __float_as_int(c1.z), pi = __float_as_int(c1.w);
    const int l = hdr & 255, np = (hdr >> 8) & 255, first = (hdr >> 16) - 64;
    const int atom = rec->atom[s];
    const float r[3] = {(px - c0.x) - c0.w, (py - c0.y) - c1.x, (pz - c0.z) - c1.y};
    const float r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    float g = 0.f, g1 = 0.f, g2 = 0.f;
    for (int k = 0; k < np; ++k) {
      const float4 pr = rec->pf[pi + k];
      const float2 ac = rec->pac[pi + k];
      const float e = exp_rn(fmaf(-pr.x, r2, -pr.y * r2));
      g = fmaf(pr.z, e, fmaf(pr.w, e, g));
      const float ace = (ac.x + ac.y) * e;
      g1 += ace;
      if (HESS) g2 = fmaf(pr.x + pr.y, ace, g2);
    }
    const int ncomp = (l + 1) * (l + 2) / 2;
    for (int c = 0; c < ncomp; ++c) {
      const int nu = first + c;
      if (nu < 0 || nu >= kBasisBlk) continue;
      // exponents of x, y, z and the normalisation of this component
      int e[3];
      float fc = 1.f;
      if (l == 0) {
        e[0] = e[1] = e[2] = 0;
      } else if (l == 1) {
        e[0] = c == 0; e[1] = c == 1; e[2] = c == 2;
      } else {
        e[0] = (c == 0) * 2 + (c == 1) + (c == 2);
        e[1] = (c == 3) * 2 + (c == 1) + (c == 4);
        e[2] = (c == 5) * 2 + (c == 2) + (c == 4);
        if (c == 0 || c == 3 || c == 5) fc = 0.57735026918962576f;
      }
      float p0[3], p1[3], p2[3];   // per axis: r^e, d/dr, d2/dr2
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        p0[a] = e[a] == 0 ? 1.f : (e[a] == 1 ? r[a] : r[a] * r[a]);
        p1[a] = e[a] == 0 ? 0.f : (e[a] == 1 ? 1.f : 2.f * r[a]);
        p2[a] = e[a] == 2 ? 2.f : 0.f;
      }
      const float P = fc * p0[0] * p0[1] * p0[2];
      float dP[3];
      dP[0] = fc * p1[0] * p0[1] * p0[2];
      dP[1] = fc * p0[0] * p1[1] * p0[2];
      dP[2] = fc * p0[0] * p0[1] * p1[2];
      float d[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) d[a] = dP[a] * g - 2.f * r[a] * P * g1;
      float h[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (HESS) {
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int a = ia[k], b = ib[k];
          float ddP;
          if (a == b)
            ddP = fc * (a == 0 ? p2[0] * p0[1] * p0[2] : a == 1 ? p0[0] * p2[1] * p0[2] : p0[0] * p0[1] * p2[2]);
          else
            ddP = fc * (3 - a - b == 2 ? p1[0] * p1[1] * p0[2] : 3 - a - b == 1 ? p1[0] * p0[1] * p1[2]
                                                                               : p0[0] * p1[1] * p1[2]);
          h[k] = ddP * g - 2.f * (dP[a] * r[b] + dP[b] * r[a]) * g1 +
                 P * (4.f * r[a] * r[b] * g2 - (a == b ? 2.f * g1 : 0.f));
        }
      }
      f(atom, nu, d, h);
    }
  }
}

}  // namespace kldi
