// Double-float (FP32 hi + lo) basis values for the BF16X10 mode.
//
// The tensor-core sums of the BF16X10 mode resolve 2^-32 of an operand's
// scale, so the operands themselves (basis values, X, the row-dot) must be
// accurate to that level: an FP32 value carries 2^-24, and in a quadrature of
// ~1e7 points its rounding (and the rounding of the exponent argument, which
// an FP32 exp amplifies by the argument's size) adds up to more than the
// 1e-6 Ha target.  Here every quantity is a pair (h, l) with value h + l:
//   offsets    r = (p_hi - c_hi) + (p_lo - c_lo) from hi / lo point and
//              centre coordinates relative to the grid block's anchor atom;
//   r^2, a r^2 error-free products (two_prod via fma) and sums;
//   exp(x)     x = k ln2/256 + r: 2^(k>>8) * T[k&255] * e^r with the table
//              T[j] = 2^(j/256) as hi / lo pairs and e^r = 1 + r + q,
//              q = r^2 (1/2 + r/6 + r^2/24) in FP32 (|r| <= ln2/512, so the
//              dropped r^5/120 is below 4e-17 and q's rounding below 2^-44);
//              the reduction subtracts k ln2/256 in three parts (the first
//              with 9 significant bits, so k times it is exact for |k| < 2^15);
//   contraction g = sum_k c_k e^{-a_k r^2} and gd = sum_k a_k c_k e^{-a_k r^2}
//              with hi / lo coefficients;
//   components chi = P g with the Cartesian polynomial P in hi / lo.
// The relative error of a value is ~2^-44 unless its sum cancels; the
// gradients d chi / dr_a = (d_a P) g - 2 r_a P gd are formed the same way.
#pragma once

#include "basis.cuh"

namespace kldi {

struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
  const f2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ f2 df_sub(f2 a, f2 b) { return df_add(a, f2{-b.h, -b.l}); }
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  const f2 p = two_prod(a.h, b.h);
  return fast_two_sum(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}
__device__ __forceinline__ f2 df_mulf(f2 a, float b) {   // b an FP32 number
  const f2 p = two_prod(a.h, b);
  return fast_two_sum(p.h, fmaf(a.l, b, p.l));
}
__device__ __forceinline__ f2 df_scale(f2 a, float s) { return {a.h * s, a.l * s}; }   // s a power of two
// Unnormalised forms for short chains (a product or sum feeding the next):
// the low part may exceed half an ulp of the high part, which the products
// below still take into account; dropped terms are ~2^-44 of the result.
__device__ __forceinline__ f2 df_mul_u(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  return {p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)))};
}
__device__ __forceinline__ f2 df_add_u(f2 a, f2 b) {
  const f2 s = two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ f2 df_sub_u(f2 a, f2 b) {
  const f2 s = two_sum(a.h, -b.h);
  return {s.h, __fadd_rn(s.l, __fsub_rn(a.l, b.l))};
}
__device__ __forceinline__ f2 df_neg(f2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ double df_to_double(f2 a) { return (double)a.h + (double)a.l; }

// ln 2 / 256 in three parts: kC1 has 9 significant bits and kC1 <= ln2/256,
// kC2 and kC3 the next 24 bits each.
constexpr float kLn2_256_1 = 0.0027008056640625f;
constexpr float kLn2_256_2 = 6.80051016388461e-06f;
constexpr float kLn2_256_3 = -1.6409833561437104e-13f;
constexpr float kInvLn2_256 = 369.329930467f;   // 256 / ln 2 (only used to pick k)

// e^x for x = (xh, xl) <= 0 with the table T[j] = 2^(j/256) (hi, lo).
// Returns 0 below x = -87 (the value is then below 2^-125 of any operand
// scale and contributes nothing).
__device__ __forceinline__ f2 exp_df(f2 x, const float2* __restrict__ tab) {
  if (x.h < -87.f) return {0.f, 0.f};
  // k = rint(x 256 / ln 2), by adding and subtracting 1.5 x 2^23
  const float t = __fadd_rn(__fmul_rn(x.h, kInvLn2_256), 12582912.f);
  const float kf = __fsub_rn(t, 12582912.f);
  const int k = __float_as_int(t) - 0x4B400000;
  // r = x - k ln2/256: the first part exactly (Sterbenz), then error-free
  // products and sums for the second, the third and x's low part rounded
  const float r1 = __fsub_rn(x.h, __fmul_rn(kf, kLn2_256_1));
  const f2 p2 = two_prod(kf, kLn2_256_2);
  const f2 s = two_sum(r1, -p2.h);
  const float rl = __fadd_rn(__fsub_rn(__fsub_rn(s.l, p2.l), __fmul_rn(kf, kLn2_256_3)), x.l);
  const float rh = s.h;
  // e^r - 1 = rh + (rl + q)
  const float q = __fmul_rn(__fmul_rn(rh, rh), fmaf(rh, fmaf(rh, 0.041666666666666664f, 0.16666666666666666f), 0.5f));
  const float pl = __fadd_rn(rl, q);
  const int j = k & 255, m = k >> 8;
  const float2 T = tab[j];
  // T (1 + rh + pl) = T.x + T.x rh + [T.y + T.x pl + T.y rh]
  const f2 a = two_prod(T.x, rh);
  const f2 hi = fast_two_sum(T.x, a.h);
  const float lo = __fadd_rn(hi.l, __fadd_rn(a.l, fmaf(T.x, pl, fmaf(T.y, rh, T.y))));
  const f2 v = fast_two_sum(hi.h, lo);
  const float sc = __int_as_float((m + 127) << 23);   // 2^m, m >= -126 here
  return {v.h * sc, v.l * sc};
}

// 1/sqrt(3) as hi / lo
constexpr float kS3h = 0.5773502588272095f, kS3l = 1.0362416702491828e-08f;

// Radial factors of one shell at offset (dx, dy, dz): r^2, g = sum c e^{-a r^2}
// and (GRAD) gd = sum a c e^{-a r^2}, primitives from a staged record.  The
// exponent argument and the sums of at most a few terms use the unnormalised
// products and sums (their consumers take both parts into account).
template <bool GRAD>
__device__ __forceinline__ void radial_df(const float4* pf, const float2* pac, int np, f2 r2, const float2* tab,
                                          f2& g, f2& gd) {
  g = {0.f, 0.f};
  gd = {0.f, 0.f};
  for (int k = 0; k < np; ++k) {
    const float4 pr = pf[k];
    const f2 e = exp_df(df_neg(df_mul_u(f2{pr.x, pr.y}, r2)), tab);
    g = df_add_u(g, df_mul_u(f2{pr.z, pr.w}, e));
    if (GRAD) {
      const float2 ac = pac[k];
      gd = df_add_u(gd, df_mul_u(f2{ac.x, ac.y}, e));
    }
  }
}

// Offsets of a point from a staged shell centre and r^2, hi / lo (r^2
// unnormalised, a sum of three error-free squares).
__device__ __forceinline__ void offsets_df(const float4& c0, const float4& c1, f2 px, f2 py, f2 pz, f2& dx, f2& dy,
                                           f2& dz, f2& r2) {
  dx = df_sub(px, f2{c0.x, c0.w});
  dy = df_sub(py, f2{c0.y, c1.x});
  dz = df_sub(pz, f2{c0.z, c1.y});
  r2 = df_add_u(df_add_u(df_mul_u(dx, dx), df_mul_u(dy, dy)), df_mul_u(dz, dz));
}

// Offsets of a point from a staged shell centre, hi / lo (no r^2).
__device__ __forceinline__ void offsets3_df(const float4& c0, const float4& c1, f2 px, f2 py, f2 pz, f2& dx, f2& dy,
                                            f2& dz) {
  dx = df_sub_u(px, f2{c0.x, c0.w});
  dy = df_sub_u(py, f2{c0.y, c1.x});
  dz = df_sub_u(pz, f2{c0.z, c1.y});
}

// Cartesian component c of a shell of angular momentum l: P and dP/dr_a
// (normalisation 1/sqrt(3) on xx, yy, zz), hi / lo.
__device__ __forceinline__ void cart_df(int l, int c, f2 dx, f2 dy, f2 dz, f2& P, f2& Px, f2& Py, f2& Pz) {
  const f2 z{0.f, 0.f}, one{1.f, 0.f};
  const f2 s3{kS3h, kS3l};
  if (l == 0) {
    P = one; Px = Py = Pz = z;
  } else if (l == 1) {
    P = c == 0 ? dx : (c == 1 ? dy : dz);
    Px = c == 0 ? one : z;
    Py = c == 1 ? one : z;
    Pz = c == 2 ? one : z;
  } else {
    switch (c) {
      case 0: P = df_mul(df_mul(dx, dx), s3); Px = df_mul(df_scale(dx, 2.f), s3); Py = Pz = z; break;
      case 1: P = df_mul(dx, dy); Px = dy; Py = dx; Pz = z; break;
      case 2: P = df_mul(dx, dz); Px = dz; Py = z; Pz = dx; break;
      case 3: P = df_mul(df_mul(dy, dy), s3); Py = df_mul(df_scale(dy, 2.f), s3); Px = Pz = z; break;
      case 4: P = df_mul(dy, dz); Px = z; Py = dz; Pz = dy; break;
      default: P = df_mul(df_mul(dz, dz), s3); Pz = df_mul(df_scale(dz, 2.f), s3); Px = Py = z; break;
    }
  }
}

// Calls f(nu, value, d/dx, d/dy, d/dz) (hi / lo) for every function of a
// staged basis block at the point (px, py, pz) (hi / lo, anchor-relative).
template <bool GRAD, typename F>
__device__ __forceinline__ void for_rec_functions_df(const BlockRec* rec, const float2* tab, f2 px, f2 py, f2 pz,
                                                     F&& f) {
  const int ns = rec->nshell;
  for (int s = 0; s < ns; ++s) {
    const float4 c0 = rec->c0[s], c1 = rec->c1[s];
    const int hdr = __float_as_int(c1.z), pi = __float_as_int(c1.w);
    const int l = hdr & 255, np = (hdr >> 8) & 255, first = (hdr >> 16) - 64;
    f2 dx, dy, dz, r2, g, gd;
    offsets_df(c0, c1, px, py, pz, dx, dy, dz, r2);
    radial_df<GRAD>(rec->pf + pi, rec->pac + pi, np, r2, tab, g, gd);
    f2 ux{0.f, 0.f}, uy{0.f, 0.f}, uz{0.f, 0.f};   // -2 r_a gd
    if (GRAD) {
      const f2 m2 = df_scale(gd, -2.f);
      ux = df_mul(dx, m2);
      uy = df_mul(dy, m2);
      uz = df_mul(dz, m2);
    }
    const int ncomp = (l + 1) * (l + 2) / 2;
    for (int c = 0; c < ncomp; ++c) {
      const int nu = first + c;
      if (nu < 0 || nu >= kBasisBlk) continue;
      f2 P, Px, Py, Pz;
      cart_df(l, c, dx, dy, dz, P, Px, Py, Pz);
      const f2 v = df_mul(P, g);
      if (GRAD)
        f(nu, v, df_add(df_mul(Px, g), df_mul(P, ux)), df_add(df_mul(Py, g), df_mul(P, uy)),
          df_add(df_mul(Pz, g), df_mul(P, uz)));
      else
        f(nu, v, f2{0.f, 0.f}, f2{0.f, 0.f}, f2{0.f, 0.f});
    }
  }
}

// Calls f(nu, chi, X) (hi / lo) for every function of a staged basis block,
// with X = a chi + b . grad chi (the V product's operand; a, b per point).
// Per shell, with chi = P g and grad chi = (grad P) g + P u (u = -2 r gd):
//   X = a chi + (g b) . grad P + P (b . u),
// where grad P has one or two non-zero components, so each function costs a
// few double-float products.
// The radial factors come from the Phi kernel: rad[s * 128] = (g hi, g lo,
// gd hi, gd lo) of shell s of the block at this point.
// Shells sb .. se - 1 of the block; the offsets are formed once per run of
// shells on one atom.
template <bool GRAD, typename F>
__device__ __forceinline__ void for_rec_phix_df(const BlockRec* rec, const float4* rad, int sb, int se, f2 px,
                                                f2 py, f2 pz, f2 a, f2 bx, f2 by, f2 bz, F&& f) {
  const f2 s3{kS3h, kS3l};
  // radial factors loaded two shells ahead (the loads come from HBM / L2)
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 qa = sb < se ? rad[sb * kBlockPts] : z4;
  float4 qb = sb + 1 < se ? rad[(sb + 1) * kBlockPts] : z4;
  f2 dx, dy, dz, br{0.f, 0.f};   // br = b . r, once per run of shells on one atom
  for (int s = sb; s < se; ++s) {
    const float4 q = qa;
    qa = qb;
    qb = s + 2 < se ? rad[(s + 2) * kBlockPts] : z4;
    const float4 c0 = rec->c0[s], c1 = rec->c1[s];
    const int hdr = __float_as_int(c1.z);
    const int l = hdr & 255, first = (hdr >> 16) - 64;
    const f2 g{q.x, q.y}, gd{q.z, q.w};
    if (s == sb || rec->atom[s] != rec->atom[s - 1]) {
      offsets3_df(c0, c1, px, py, pz, dx, dy, dz);
      if (GRAD) br = df_add_u(df_add_u(df_mul_u(bx, dx), df_mul_u(by, dy)), df_mul_u(bz, dz));
    }
    f2 w{0.f, 0.f}, gbx{0.f, 0.f}, gby{0.f, 0.f}, gbz{0.f, 0.f};
    if (GRAD) {
      w = df_mul_u(df_scale(gd, -2.f), br);
      gbx = df_mul_u(g, bx);
      gby = df_mul_u(g, by);
      gbz = df_mul_u(g, bz);
    }
    auto emit = [&](int c, f2 P, f2 bdP) {   // bdP = (g b) . grad P
      const int nu = first + c;
      if (nu < 0 || nu >= kBasisBlk) return;
      const f2 v = df_mul_u(P, g);
      f2 x = df_mul_u(a, v);
      if (GRAD) x = df_add_u(x, df_add_u(bdP, df_mul_u(P, w)));
      // normalised for the slicing (which takes the top digits from hi alone)
      f(nu, two_sum(v.h, v.l), two_sum(x.h, x.l));
    };
    const f2 z{0.f, 0.f};
    if (l == 0) {
      emit(0, f2{1.f, 0.f}, z);
    } else if (l == 1) {
      emit(0, dx, gbx);
      emit(1, dy, gby);
      emit(2, dz, gbz);
    } else {
      const f2 sx = df_mul_u(dx, s3), sy = df_mul_u(dy, s3), sz = df_mul_u(dz, s3);
      emit(0, df_mul_u(dx, sx), GRAD ? df_scale(df_mul_u(gbx, sx), 2.f) : z);
      emit(1, df_mul_u(dx, dy), GRAD ? df_add_u(df_mul_u(gbx, dy), df_mul_u(gby, dx)) : z);
      emit(2, df_mul_u(dx, dz), GRAD ? df_add_u(df_mul_u(gbx, dz), df_mul_u(gbz, dx)) : z);
      emit(3, df_mul_u(dy, sy), GRAD ? df_scale(df_mul_u(gby, sy), 2.f) : z);
      emit(4, df_mul_u(dy, dz), GRAD ? df_add_u(df_mul_u(gby, dz), df_mul_u(gbz, dy)) : z);
      emit(5, df_mul_u(dz, sz), GRAD ? df_scale(df_mul_u(gbz, sz), 2.f) : z);
    }
  }
}

// Balanced digits of a = h + l (|a| <= 1) on the grids 2^-7, 2^-15, 2^-23,
// 2^-31: s0 and s1 from h exactly (as in slice<>), then t = (h - s0 - s1) + l
// rounded (|t| <= 2^-16, error <= 2^-41), s2 = rint(t 2^23) 2^-23 and
// s3 = rint((t - s2) 2^31) 2^-31 (t - s2 is exact).  Every digit is an integer
// of at most 8 bits times its grid step, exact in BF16.
__device__ __forceinline__ void slice4_df(float h, float l, float* s) {
  constexpr float C0 = 98304.f, C1 = 384.f, C2 = 1.5f, C3 = 0.005859375f;   // 1.5 x 2^16, 2^8, 2^0, 2^-8
  const float s0 = __fsub_rn(__fadd_rn(h, C0), C0);
  float r = __fsub_rn(h, s0);
  const float s1 = __fsub_rn(__fadd_rn(r, C1), C1);
  r = __fadd_rn(__fsub_rn(r, s1), l);
  const float s2 = __fsub_rn(__fadd_rn(r, C2), C2);
  r = __fsub_rn(r, s2);
  s[0] = s0;
  s[1] = s1;
  s[2] = s2;
  s[3] = __fsub_rn(__fadd_rn(r, C3), C3);
}

}  // namespace kldi
