// Split-precision tensor-core path (tcgen05, sm_103a) with exact accumulation.
//
// Slicing.  A row (or column) of an operand is scaled by a power of two s so
// that |a / s| <= 1, and a / s is cut into NS BF16 slices on fixed-point grids
//   a0 = rint(a/s * 2^7) 2^-7,  a1 = rint((a/s - a0) 2^15) 2^-15,
//   a2 = rint((a/s - a0 - a1) 2^23) 2^-23,
// every slice an integer of at most 8 bits times its grid step, hence exact in
// BF16.  The product sum over k of slice products is kept per "level"
// l = i + j (only levels l < NS are formed: 3 products for NS = 2, 6 for
// NS = 3).  All products of one level are multiples of 2^-(14 + 8 l) and at
// most (l + 1) 2^-8l in size, so a level's partial sum over at most 256 terms
// needs at most 24 significant bits: the FP32 tensor-memory accumulator
// represents every partial sum exactly and its own rounding never acts.
// Levels are combined, and K-segments summed, on CUDA cores with
// round-to-nearest.  The tensor cores therefore add no bias; the only error is
// the dropped tail of each slice expansion (2^-8 NS of the scale, unbiased).
//
// Kernels
//  k_dscale     power-of-two column scales f_nu >= max_mu |D_mu nu|.
//  k_dsplit     per 32 x 32 block pair (p, q): the density product's B operand
//               [32 n][32 k] = D[32p + k][32q + n] / f_n in NS BF16 planes,
//               64-byte swizzle.
//  k_phi_split  per grid block: point scales e_i >= max_mu |phi_mu(r_i)| from the
//               shell bound r^l sum_k |c_k| exp(-a_k r^2); then every retained
//               tile (g, p) of Phi (Eq. phi_def) sliced by point: the A operand
//               of the density product.
//  k_rho_tc     density product R = Phi_g D over the executed pairs of grid
//               block g (Eq. executed_block_output), warp-ballot pair screen
//               (Eq. block_pair_filter), bulk-copy pipeline, tcgen05.mma
//               M = 128 N = 128 per level, drains every <= 8 executed chunks
//               (256 K), fused row-dot rho = sum Phi . R, grad rho; with the
//               gradient epilogues, the Q = Z D and R = Phi D terms of the
//               nuclear gradient contracted with basis derivatives per atom.
//  k_z_split    the gradient's Z = 2 a phi + b . grad phi tiles, sliced by point.
//  k_x_split    X tile = w (v_rho / 2 phi + 2 v_sigma grad rho . grad phi);
//               Phi~ = c phi and X~ = X / c (per-point balance c), sliced per
//               function with one shared column scale; x_gq = max |X|.
//  k_v_tc       V = Phi^T X + X^T Phi, one pair P <= Q of 128-function
//               windows (4 consecutive basis blocks; each grid block's
//               retained blocks are covered by the fewest windows) over a
//               segment of its grid-block list; one grid block per exact
//               accumulation (K = 256: [Phi~ | X~] against [X~ ; Phi~]),
//               drained into compensated FP32 sums with the 32 x 32 block
//               pairs that are not executed for that grid block left out,
//               FP64 scatter-add; V = A + A^T afterwards.
//  BF16X10 (four slices): k_phi_split4 and k_x_split4 evaluate the basis in
//  double-float (basis_df.cuh) and cut hi + lo into four slices; k_rho_tc<4>
//  keeps four exact levels in N = 64 tiles (two TMEM buffers) and forms R and
//  the row-dot in double-float; k_v_tc<4> keeps levels 0 and 1 exact and
//  accumulates levels 2 and 3 together.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "basis.cuh"
#include "basis_df.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace kldi {

using namespace tc;

constexpr int kPlaneBytes = 8192;   // [128][32] BF16 plane of a tile
constexpr int kDPlane = 2048;       // [32][32] BF16 plane of a D block pair
constexpr int kMaxRet = 256;        // retained basis blocks per grid block the density kernel handles

__host__ __device__ constexpr int tile_bytes(int ns) { return ns * kPlaneBytes; }

// ---------------------------------------------------------------------------
// FP32 -> FP64, exactly, by integer operations on the bits (the conversion
// instruction runs on the FP64 pipe, which this GPU provides at a small
// fraction of the FP32 rate); an FP32 subnormal m 2^-149 is normalised with a
// leading-zero count.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  if (e == 0u) {
    if (m == 0u) return __longlong_as_double((long long)sign);
    const int sh = __clz((int)m) - 8;   // moves the leading one to bit 23
    m = (m << sh) & 0x7fffffu;
    e = 1u - (uint32_t)sh;               // may wrap below zero: the FP64 exponent below stays positive
  }
  const uint64_t d = sign | ((uint64_t)(uint32_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  return __longlong_as_double((long long)d);
}

// slicing helpers
__device__ __forceinline__ float pow2_ceil(float m) {
  // smallest power of two >= m (m > 0), 1 for m <= 0, at least 2^-100 so that
  // its reciprocal stays finite (values below 2^-124 then slice to zero)
  if (!(m > 0.f)) return 1.f;
  int e;
  const float f = frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  return ldexpf(1.f, max(f == 0.5f ? e - 1 : e, -100));
}

// Balanced digits of a on the grids 2^-7, 2^-15, 2^-23: s0 = rint(a 2^7) 2^-7,
// s1 = rint((a - s0) 2^15) 2^-15, s2 = rint((a - s0 - s1) 2^23) 2^-23.  Each
// rint is one addition and one subtraction of 1.5 x 2^(23 - e) (e = 7, 15,
// 23): the sum lies in [2^(23-e), 2^(24-e)), where the spacing of FP32 numbers
// is 2^-e, so the addition rounds to the grid (ties to even) and the
// subtraction is exact.  Valid for |a| <= 1 (the residuals are then below
// 2^-8 and 2^-16).
template <int NS>
__device__ __forceinline__ void slice(float a, float* s) {  // |a| <= 1
  constexpr float C0 = 98304.f, C1 = 384.f, C2 = 1.5f;   // 1.5 x 2^16, 1.5 x 2^8, 1.5
  const float s0 = __fsub_rn(__fadd_rn(a, C0), C0);
  float r = __fsub_rn(a, s0);
  s[0] = s0;
  if (NS >= 2) {
    const float s1 = __fsub_rn(__fadd_rn(r, C1), C1);
    r = __fsub_rn(r, s1);
    s[1] = s1;
  }
  if (NS >= 3) {
    const float s2 = __fsub_rn(__fadd_rn(r, C2), C2);
    r = __fsub_rn(r, s2);
    s[2] = s2;
  }
  if (NS >= 4) s[3] = __fsub_rn(__fadd_rn(r, 0.005859375f), 0.005859375f);   // grid 2^-31 (1.5 x 2^-8)
}

template <int NS>
__device__ __forceinline__ void slice_d(double a, float* s) {  // |a| <= 1, FP64 input
  const double s0 = rint(a * 128.0) / 128.0;
  double r = a - s0;
  s[0] = (float)s0;
  if (NS >= 2) {
    const double s1 = rint(r * 32768.0) / 32768.0;
    r = r - s1;
    s[1] = (float)s1;
  }
  if (NS >= 3) {
    const double s2 = rint(r * 8388608.0) / 8388608.0;
    r = r - s2;
    s[2] = (float)s2;
  }
  if (NS >= 4) s[3] = (float)(rint(r * 2147483648.0) / 2147483648.0);
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {   // a in the low half
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Row `row` of NS swizzled [rows][32] planes (plane stride `pstride` bytes)
// from 32 scaled values v[] (|v| <= 1).
template <int NS>
__device__ __forceinline__ void store_sliced_row(uint8_t* base, int pstride, int row, const float* v) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t w[NS][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s0[NS], s1[NS];
      slice<NS>(v[c * 8 + 2 * k], s0);
      slice<NS>(v[c * 8 + 2 * k + 1], s1);
#pragma unroll
      for (int l = 0; l < NS; ++l) w[l][k] = pack2(s0[l], s1[l]);
    }
    const uint32_t off = swz64_off(row, c * 8);
#pragma unroll
    for (int l = 0; l < NS; ++l)
      *reinterpret_cast<uint4*>(base + l * pstride + off) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
  }
}

// Row `row` of four swizzled planes from 32 double-float values (vh + vl,
// |v| <= 1): the digits of slice4_df.
template <int C0 = 0, int C1 = 4>   // the 16-byte chunks [C0, C1) of the row
__device__ __forceinline__ void store_sliced_row4(uint8_t* base, int pstride, int row, const float* vh,
                                                  const float* vl) {
#pragma unroll
  for (int c = C0; c < C1; ++c) {
    uint32_t w[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s0[4], s1[4];
      slice4_df(vh[c * 8 + 2 * k], vl[c * 8 + 2 * k], s0);
      slice4_df(vh[c * 8 + 2 * k + 1], vl[c * 8 + 2 * k + 1], s1);
#pragma unroll
      for (int l = 0; l < 4; ++l) w[l][k] = pack2(s0[l], s1[l]);
    }
    const uint32_t off = swz64_off(row, c * 8);
#pragma unroll
    for (int l = 0; l < 4; ++l)
      *reinterpret_cast<uint4*>(base + l * pstride + off) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
  }
}

// Row `row` of a chunk-major tile: rows 32 kc .. 32 kc + 31 of all NS planes
// are contiguous ([kc][plane][32 rows x 64 B], each 2 KB chunk swizzled as a
// plane), so one bulk copy of NS x 2 KB moves a K = 32 chunk of every plane.
template <int NS>
__device__ __forceinline__ void store_sliced_row_kc(uint8_t* base, int row, const float* v) {
  store_sliced_row<NS>(base + (row >> 5) * (NS * 2048) - (row & ~31) * 64, 2048, row, v);
}
template <int C0 = 0, int C1 = 4>
__device__ __forceinline__ void store_sliced_row4_kc(uint8_t* base, int row, const float* vh, const float* vl) {
  store_sliced_row4<C0, C1>(base + (row >> 5) * (4 * 2048) - (row & ~31) * 64, 2048, row, vh, vl);
}

// Slices per operand of a tensor-core precision mode.
inline int slices_of(int prec) { return prec == KLDI_BF16X10 ? 4 : (prec == KLDI_BF16X6 ? 3 : 2); }

// 2^(j/256), j = 0..255, as FP32 hi / lo pairs: the table of exp_df.  Filled
// once per device (prepare_tc_kernels); kernels copy it to shared memory.
__device__ float2 g_exp2_tab[256];

__device__ __forceinline__ void load_exp_tab(float2* dst, int t, int nthr) {
  for (int j = t; j < 256; j += nthr) dst[j] = g_exp2_tab[j];
}




// ---------------------------------------------------------------------------
// D column scales (D symmetric: the row maximum is the column maximum).
__global__ void k_dscale(const double* __restrict__ D, int nbf, int nbf_pad, float* dscale) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nbf_pad) return;
  double m = 0.0;
  if (row < nbf)
    for (int c = lane; c < nbf; c += 32) m = fmax(m, fabs(D[(int64_t)row * nbf + c]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) dscale[row] = pow2_ceil((float)(m * (1.0 + 1e-6)));
}

template <int NS>
__global__ void k_dsplit(const double* __restrict__ D, const float* __restrict__ dscale, int nbf, int nbb,
                         uint8_t* out) {
  __shared__ double Ds[kBasisBlk][kBasisBlk + 1];
  const int p = blockIdx.y, q = blockIdx.x;
  for (int e = threadIdx.x; e < kBasisBlk * kBasisBlk; e += blockDim.x) {
    const int k = e / kBasisBlk, n = e % kBasisBlk;
    const int r = p * kBasisBlk + k, c = q * kBasisBlk + n;
    Ds[k][n] = (r < nbf && c < nbf) ? D[(int64_t)r * nbf + c] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < kBasisBlk) {
    const int n = threadIdx.x;
    const double inv = 1.0 / (double)dscale[q * kBasisBlk + n];
    uint8_t* base = out + ((int64_t)p * nbb + q) * (NS * kDPlane);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t w[NS][4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float s0[NS], s1[NS];
        slice_d<NS>(Ds[c * 8 + 2 * k][n] * inv, s0);
        slice_d<NS>(Ds[c * 8 + 2 * k + 1][n] * inv, s1);
#pragma unroll
        for (int l = 0; l < NS; ++l) w[l][k] = pack2(s0[l], s1[l]);
      }
      const uint32_t off = swz64_off(n, c * 8);
#pragma unroll
      for (int l = 0; l < NS; ++l)
        *reinterpret_cast<uint4*>(base + l * kDPlane + off) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
    }
  }
}

template <int NS>
static kldi_status dsplit_ns(const kldi_plan* P, const double* D, cudaStream_t s) {
  k_dscale<<<(unsigned)((P->nbf_pad + 7) / 8), 256, 0, s>>>(D, (int)P->nbf, (int)P->nbf_pad, P->d_dscale);
  dim3 grid((unsigned)P->nbb, (unsigned)P->nbb);
  k_dsplit<NS><<<grid, 128, 0, s>>>(D, P->d_dscale, (int)P->nbf, (int)P->nbb,
                                    reinterpret_cast<uint8_t*>(P->d_dsplit));
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

kldi_status launch_dsplit(const kldi_plan* P, const double* D, cudaStream_t s) {
  switch (slices_of(P->prec)) {
    case 4: return dsplit_ns<4>(P, D, s);
    case 3: return dsplit_ns<3>(P, D, s);
    default: return dsplit_ns<2>(P, D, s);
  }
}

// ---------------------------------------------------------------------------
// Phi tiles: one CTA (128 threads = points) per grid block.
template <int NS>
__global__ void __launch_bounds__(128) k_phi_split(BasisView B, GridView G, ListView L, int64_t g0, int64_t t0,
                                                   uint8_t* out_row, float* rowscale) {
  __shared__ float st[kBasisBlk][kBlockPts + 1];
  __shared__ BlockRec rec[2];
  const int64_t g = g0 + blockIdx.x;
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  const float4 pr = G.prel[pt];
  const float px = pr.x, py = pr.y, pz = pr.z;
  const int anc = G.anchor[g];
  const int tb = L.blk_ptr[g], te = L.blk_ptr[g + 1];
  // pass 1: point scale from the shell bound r^l sum_k |c_k| exp(-a_k r^2) >= |phi_mu(r_i)|;
  // a bound needs no unbiased exp: the hardware exp's ~1e-6 relative error is
  // covered by the 1.001 margin below.  Shell records are staged in shared
  // memory per basis block (double-buffered: one barrier per block).
  auto shell_bound = [&](int l, int np, const float4* pf, float dx, float dy, float dz) {
    const float r2 = dx * dx + dy * dy + dz * dz;
    float sum = 0.f;
    for (int k = 0; k < np; ++k) sum += fabsf(pf[k].z) * __expf(-pf[k].x * r2);
    const float poly = l == 0 ? 1.f : (l == 1 ? sqrtf(r2) : r2);
    return poly * sum;
  };
  float M = 0.f;
  for (int j = tb; j < te; ++j) {
    const int p = L.blk_idx[j];
    BlockRec* rc = rec + ((j - tb) & 1);
    if (block_rec_fits(B, p)) {
      stage_block_rec(B, p, anc, rc, i, kBlockPts);
      __syncthreads();
      for (int s = 0; s < rc->nshell; ++s) {
        const float4 c0 = rc->c0[s], c1 = rc->c1[s];
        const int hdr = __float_as_int(c1.z);
        M = fmaxf(M, shell_bound(hdr & 255, (hdr >> 8) & 255, rc->pf + __float_as_int(c1.w), (px - c0.x) - c0.w,
                                 (py - c0.y) - c1.x, (pz - c0.z) - c1.y));
      }
    } else {
      __syncthreads();
      for (int s = B.bb_shell_begin[p]; s < B.bb_shell_end[p]; ++s) {
        const int4 sh = B.shell_f[s];
        const float4* ra = reinterpret_cast<const float4*>(B.relatom + ((size_t)anc * B.natm + sh.w) * 8);
        const float4 r0 = ra[0], r1 = ra[1];
        M = fmaxf(M, shell_bound(sh.x & 255, sh.x >> 8, B.prim_f + sh.y, (px - r0.x) - r0.w, (py - r0.y) - r1.x,
                                 (pz - r0.z) - r1.y));
      }
    }
  }
  const float rs = pow2_ceil(M * 1.001f);
  rowscale[pt] = rs;
  const float rinv = 1.f / rs;
  // pass 2: per-point slicing of every retained tile
  for (int j = tb; j < te; ++j) {
    const int p = L.blk_idx[j];
    BlockRec* rc = rec + ((j - tb + te - tb) & 1);
    const bool fits = block_rec_fits(B, p);
    if (fits) stage_block_rec(B, p, anc, rc, i, kBlockPts);
    __syncthreads();
    float v[kBasisBlk];
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) st[nu][i] = 0.f;
    auto put = [&](int nu, float x, float, float, float) { st[nu][i] = x; };
    if (fits)
      for_rec_functions<false>(rc, px, py, pz, put);
    else
      for_block_functions<float, false>(B, p, px, py, pz, put, anc);
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) v[nu] = st[nu][i] * rinv;
    store_sliced_row<NS>(out_row + (int64_t)(j - t0) * tile_bytes(NS), kPlaneBytes, i, v);
  }
}

// BF16X10 Phi tiles: the point scale as in k_phi_split, then the values in
// double-float (hi / lo staged in shared memory) cut into four slices.  Every
// basis block must fit a shared-memory shell record (checked on the host).
template <bool GRAD>
__global__ void __launch_bounds__(128) k_phi_split4(BasisView B, GridView G, ListView L, int64_t g0, int64_t t0,
                                                    uint8_t* out_row, float* rowscale, float4* __restrict__ rad,
                                                    const int64_t* __restrict__ rad_ptr) {
  __shared__ float sth[kBasisBlk][kBlockPts + 1];
  __shared__ float stl[kBasisBlk][kBlockPts + 1];
  __shared__ BlockRec rec[2];
  __shared__ float2 tab[256];
  const int64_t g = g0 + blockIdx.x;
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  load_exp_tab(tab, i, kBlockPts);
  const float4 pr = G.prel[pt], pl = G.prel_lo[pt];
  const f2 px{pr.x, pl.x}, py{pr.y, pl.y}, pz{pr.z, pl.z};
  const int anc = G.anchor[g];
  const int tb = L.blk_ptr[g], te = L.blk_ptr[g + 1], n = te - tb;
  // The shell records are staged one block ahead: step q (blocks of pass 1,
  // then of pass 2) reads buffer q & 1, staged during step q - 1, while it
  // stages step q + 1 into the other buffer (read last at step q - 1, which
  // every thread has left at the barrier of step q).
  auto stage_step = [&](int q) {
    if (q < 2 * n) stage_block_rec(B, L.blk_idx[tb + (q < n ? q : q - n)], anc, rec + (q & 1), i, kBlockPts);
  };
  stage_step(0);
  // pass 1: point scale from the shell bound r^l sum_k |c_k| exp(-a_k r^2) (FP32, 1.001 margin)
  float M = 0.f;
  for (int j = tb; j < te; ++j) {
    const int q = j - tb;
    const BlockRec* rc = rec + (q & 1);
    __syncthreads();
    stage_step(q + 1);
    for (int s = 0; s < rc->nshell; ++s) {
      const float4 c0 = rc->c0[s], c1 = rc->c1[s];
      const int hdr = __float_as_int(c1.z), l = hdr & 255, np = (hdr >> 8) & 255;
      const float4* pf = rc->pf + __float_as_int(c1.w);
      const float dx = (pr.x - c0.x) - c0.w, dy = (pr.y - c0.y) - c1.x, dz = (pr.z - c0.z) - c1.y;
      const float r2 = dx * dx + dy * dy + dz * dz;
      float sum = 0.f;
      for (int k = 0; k < np; ++k) sum += fabsf(pf[k].z) * __expf(-pf[k].x * r2);
      M = fmaxf(M, (l == 0 ? 1.f : (l == 1 ? sqrtf(r2) : r2)) * sum);
    }
  }
  const float rs = pow2_ceil(M * 1.001f);
  rowscale[pt] = rs;
  const float rinv = 1.f / rs;
  // pass 2: double-float values of every retained tile, four slices per point
  for (int j = tb; j < te; ++j) {
    const int q = n + j - tb;
    const BlockRec* rc = rec + (q & 1);
    if ((L.blk_idx[j] + 1) * kBasisBlk > B.nbf) {   // a partial last block: its padding columns are zero
#pragma unroll
      for (int nu = 0; nu < kBasisBlk; ++nu) sth[nu][i] = stl[nu][i] = 0.f;
    }
    __syncthreads();
    stage_step(q + 1);
    // per shell: the radial factors g (and gd) go to the radial buffer for the
    // row-dot and the X kernel, the values P g to the staging array
    float4* rtile = rad + (rad_ptr[j] - rad_ptr[t0]) * kBlockPts;
    f2 dx, dy, dz, r2;   // offsets of the point from the current shell's atom
    for (int s = 0; s < rc->nshell; ++s) {
      const float4 c0 = rc->c0[s], c1 = rc->c1[s];
      const int hdr = __float_as_int(c1.z), pi = __float_as_int(c1.w);
      const int l = hdr & 255, np = (hdr >> 8) & 255, first = (hdr >> 16) - 64;
      f2 g, gd;
      if (s == 0 || rc->atom[s] != rc->atom[s - 1]) offsets_df(c0, c1, px, py, pz, dx, dy, dz, r2);
      radial_df<GRAD>(rc->pf + pi, rc->pac + pi, np, r2, tab, g, gd);
      rtile[s * kBlockPts + i] = make_float4(g.h, g.l, gd.h, gd.l);
      const int ncomp = (l + 1) * (l + 2) / 2;
      for (int c = 0; c < ncomp; ++c) {
        const int nu = first + c;
        if (nu < 0 || nu >= kBasisBlk) continue;
        f2 P, Px, Py, Pz;
        cart_df(l, c, dx, dy, dz, P, Px, Py, Pz);
        const f2 v = df_mul(P, g);
        sth[nu][i] = v.h;
        stl[nu][i] = v.l;
      }
    }
    float vh[kBasisBlk], vl[kBasisBlk];
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) {
      vh[nu] = sth[nu][i] * rinv;
      vl[nu] = stl[nu][i] * rinv;
    }
    store_sliced_row4(out_row + (int64_t)(j - t0) * tile_bytes(4), kPlaneBytes, i, vh, vl);
  }
}

// Z tiles of the nuclear gradient: Z_nu,i = 2 a_i chi_nu(r_i) + b_i . grad chi_nu(r_i)
// (a = w v_rho / 2, b = 2 w v_sigma grad rho), sliced per point like the Phi
// tiles, so that Q = Z D runs through the density product.  Point scale from
// the shell bounds |chi| <= r^l S0 and |d_a chi| <= l r^(l-1) S0 + 2 r^(l+1) S1
// (S0 = sum |c| e^{-a r^2}, S1 = sum |c| a e^{-a r^2}; |P| <= r^l and
// |d_a P| <= l r^(l-1) for the Cartesian components):
// |Z| <= 2 |a| r^l S0 + (|b_x| + |b_y| + |b_z|) (l r^(l-1) S0 + 2 r^(l+1) S1).
template <int NS>
__global__ void __launch_bounds__(128) k_z_split(BasisView B, GridView G, ListView L, int64_t g0, int64_t t0,
                                                 const double* __restrict__ xcoef, uint8_t* out_row,
                                                 float* zscale) {
  __shared__ float st[kBasisBlk][kBlockPts + 1];
  __shared__ BlockRec rec[2];
  const int64_t g = g0 + blockIdx.x;
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  const float4 pr = G.prel[pt];
  const float px = pr.x, py = pr.y, pz = pr.z;
  const int anc = G.anchor[g];
  const int tb = L.blk_ptr[g], te = L.blk_ptr[g + 1];
  const float a2 = 2.f * (float)xcoef[pt * 4];
  const float bx = (float)xcoef[pt * 4 + 1], by = (float)xcoef[pt * 4 + 2], bz = (float)xcoef[pt * 4 + 3];
  const float bsum = fabsf(bx) + fabsf(by) + fabsf(bz);
  float M = 0.f;
  for (int j = tb; j < te; ++j) {
    const int p = L.blk_idx[j];
    BlockRec* rc = rec + ((j - tb) & 1);
    stage_block_rec(B, p, anc, rc, i, kBlockPts);   // every block fits (checked on the host)
    __syncthreads();
    for (int s = 0; s < rc->nshell; ++s) {
      const float4 c0 = rc->c0[s], c1 = rc->c1[s];
      const int hdr = __float_as_int(c1.z), pi = __float_as_int(c1.w);
      const int l = hdr & 255, np = (hdr >> 8) & 255;
      const float dx = (px - c0.x) - c0.w, dy = (py - c0.y) - c1.x, dz = (pz - c0.z) - c1.y;
      const float r2 = dx * dx + dy * dy + dz * dz, r = sqrtf(r2);
      float s0 = 0.f, s1 = 0.f;
      for (int k = 0; k < np; ++k) {
        const float4 q = rc->pf[pi + k];
        const float e = fabsf(q.z) * __expf(-q.x * r2);
        s0 += e;
        s1 += q.x * e;
      }
      const float rl = l == 0 ? 1.f : (l == 1 ? r : r2);                 // r^l
      const float dl = l == 0 ? 0.f : (l == 1 ? 1.f : 2.f * r);          // l r^(l-1)
      M = fmaxf(M, fabsf(a2) * rl * s0 + bsum * (dl * s0 + 2.f * r * rl * s1));
    }
  }
  const float zs = pow2_ceil(M * 1.001f);
  zscale[pt] = zs;
  const float rinv = 1.f / zs;
  for (int j = tb; j < te; ++j) {
    const int p = L.blk_idx[j];
    BlockRec* rc = rec + ((j - tb + te - tb) & 1);
    stage_block_rec(B, p, anc, rc, i, kBlockPts);
    __syncthreads();
    float v[kBasisBlk];
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) st[nu][i] = 0.f;
    for_rec_functions<true>(rc, px, py, pz, [&](int nu, float x, float gx, float gy, float gz) {
      st[nu][i] = fmaf(bx, gx, fmaf(by, gy, fmaf(bz, gz, a2 * x)));
    });
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) v[nu] = st[nu][i] * rinv;
    store_sliced_row<NS>(out_row + (int64_t)(j - t0) * tile_bytes(NS), kPlaneBytes, i, v);
  }
}

template <int NS>
static kldi_status phi_ns(const kldi_plan* P, const Batch& b, cudaStream_t s) {
  const int64_t n = b.g1 - b.g0;
  if (n == 0) return KLDI_OK;
  k_phi_split<NS><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                    reinterpret_cast<uint8_t*>(P->d_phi_s), P->d_rowscale);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

kldi_status launch_phi_split(const kldi_plan* P, const Batch& b, cudaStream_t s) {
  switch (slices_of(P->prec)) {
    case 4: {
      const int64_t n = b.g1 - b.g0;
      if (n == 0) return KLDI_OK;
      KLDI_TRY(prepare_tc_kernels());   // the exp table
      if (P->gga)
        k_phi_split4<true><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                             b.t0, reinterpret_cast<uint8_t*>(P->d_phi_s),
                                                             P->d_rowscale, P->d_rad, P->d_rad_ptr);
      else
        k_phi_split4<false><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                              b.t0, reinterpret_cast<uint8_t*>(P->d_phi_s),
                                                              P->d_rowscale, P->d_rad, P->d_rad_ptr);
      KLDI_TRY_CUDA(cudaGetLastError());
      return KLDI_OK;
    }
    case 3: return phi_ns<3>(P, b, s);
    default: return phi_ns<2>(P, b, s);
  }
}

// ---------------------------------------------------------------------------
// Column maxima of a [32][128 + 1] staging array -> power-of-two scales.
__device__ __forceinline__ void column_scales(float (*st)[kBlockPts + 1], float* out, float* raw) {
  const int i = threadIdx.x;
  const int col = i >> 2, part = i & 3;
  float m = 0.f;
  for (int r = part * 32; r < part * 32 + 32; ++r) m = fmaxf(m, fabsf(st[col][r]));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
  if (part == 0) {
    out[col] = pow2_ceil(m * 1.000001f);
    if (raw) raw[col] = m;
  }
}

// V-product operands of tile (g, p): Phi~ = c_i Phi and X~ = X / c_i with
// X = w (v_rho / 2 phi + 2 v_sigma grad rho . grad phi), both sliced per
// function with the larger of their two column maxima.
template <int NS, bool GRAD>
__global__ void __launch_bounds__(128) k_x_split(BasisView B, GridView G, ListView L, int64_t g0, int64_t t0,
                                                 const double* __restrict__ xcoef, const float* __restrict__ pscale,
                                                 uint8_t* out_phi, float* phi_scale, uint8_t* out_x, float* x_scale,
                                                 double* xmax, float* xmaxf) {
  __shared__ float sp[kBasisBlk][kBlockPts + 1];
  __shared__ float sx[kBasisBlk][kBlockPts + 1];
  __shared__ float cp[kBasisBlk], cx[kBasisBlk], rawx[kBasisBlk];
  __shared__ BlockRec rec;
  const int64_t t = t0 + blockIdx.x;
  const int64_t g = L.tile_g[t];
  const int p = L.blk_idx[t];
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  const float c = pscale[pt], cinv = c > 0.f ? 1.f / c : 0.f;   // c = 0: X = 0 at this point
  const float a = (float)xcoef[pt * 4], bx = (float)xcoef[pt * 4 + 1], by = (float)xcoef[pt * 4 + 2],
              bz = (float)xcoef[pt * 4 + 3];
#pragma unroll
  for (int nu = 0; nu < kBasisBlk; ++nu) sp[nu][i] = sx[nu][i] = 0.f;
  const float4 pr = G.prel[pt];
  const bool fits = block_rec_fits(B, p);
  if (fits) stage_block_rec(B, p, G.anchor[g], &rec, i, kBlockPts);
  __syncthreads();
  auto put = [&](int nu, float v, float dx, float dy, float dz) {
    float x = a * v;
    if (GRAD) x = fmaf(bx, dx, fmaf(by, dy, fmaf(bz, dz, x)));
    sp[nu][i] = v * c;
    sx[nu][i] = x * cinv;
  };
  if (fits)
    for_rec_functions<GRAD>(&rec, pr.x, pr.y, pr.z, put);
  else
    for_block_functions<float, GRAD>(B, p, pr.x, pr.y, pr.z, put, G.anchor[g]);
  __syncthreads();
  column_scales(sp, cp, nullptr);
  column_scales(sx, cx, rawx);
  __syncthreads();
  // one scale per function for Phi~ and X~: they meet in one exact chain
  // (A = [Phi~ | X~], B = [X~ ; Phi~]); balancing keeps the two maxima alike
  if (i < kBasisBlk) {
    cp[i] = fmaxf(cp[i], cx[i]);
    cx[i] = 1.f / cp[i];            // exact: the scales are powers of two
  }
  __syncthreads();
  float v[kBasisBlk];
#pragma unroll
  for (int nu = 0; nu < kBasisBlk; ++nu) v[nu] = sp[nu][i] * cx[nu];
  store_sliced_row_kc<NS>(out_phi + (t - t0) * tile_bytes(NS), i, v);
#pragma unroll
  for (int nu = 0; nu < kBasisBlk; ++nu) v[nu] = sx[nu][i] * cx[nu];
  store_sliced_row_kc<NS>(out_x + (t - t0) * tile_bytes(NS), i, v);
  if (i < kBasisBlk) {
    phi_scale[(t - t0) * kBasisBlk + i] = cp[i];
    x_scale[(t - t0) * kBasisBlk + i] = cp[i];
  }
  // x_gq = max |X| over the tile, with X = X~ c_i
  float mx = 0.f;
#pragma unroll
  for (int nu = 0; nu < kBasisBlk; ++nu) mx = fmaxf(mx, fabsf(sx[nu][i]) * c);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if ((i & 31) == 0) rawx[i >> 5] = mx;
  __syncthreads();
  if (i == 0) {
    const float m = fmaxf(fmaxf(rawx[0], rawx[1]), fmaxf(rawx[2], rawx[3]));
    xmax[t] = (double)m;
    xmaxf[t] = m;
  }
}

// BF16X10 V-product operands: as k_x_split, with Phi and X in double-float
// (hi / lo staged in dynamic shared memory, four [32][129] arrays) and four
// slices per function.  256 threads: point i = t % 128, and the shells of the
// block split between the two halves t / 128 (even, odd), which also split
// each row's 16-byte chunks when slicing.  The radial factors come from the
// Phi kernel.
constexpr int kX4Smem = 4 * kBasisBlk * (kBlockPts + 1) * 4;
constexpr int kX4Threads = 256;

template <bool GRAD>
__global__ void __launch_bounds__(kX4Threads, 3) k_x_split4(BasisView B, GridView G, ListView L, int64_t g0,
                                                         int64_t t0, const float4* __restrict__ xdf,
                                                         const float* __restrict__ pscale, uint8_t* out_phi,
                                                         float* phi_scale, uint8_t* out_x, float* x_scale,
                                                         double* xmax, float* xmaxf, const float4* __restrict__ rad,
                                                         const int64_t* __restrict__ rad_ptr, int64_t t1,
                                                         int64_t ahead) {
  extern __shared__ float xsm[];
  float(*sph)[kBlockPts + 1] = reinterpret_cast<float(*)[kBlockPts + 1]>(xsm);
  float(*spl)[kBlockPts + 1] = sph + kBasisBlk;
  float(*sxh)[kBlockPts + 1] = spl + kBasisBlk;
  float(*sxl)[kBlockPts + 1] = sxh + kBasisBlk;
  __shared__ float cp[kBasisBlk], cx[kBasisBlk], rawx[kBasisBlk];
  __shared__ unsigned colmax[kBasisBlk];   // per function: max |Phi~|, |X~| (hi parts) as FP32 bits
  __shared__ BlockRec rec;
  const int64_t t = t0 + blockIdx.x;
  const int64_t g = L.tile_g[t];
  const int p = L.blk_idx[t];
  const int i = threadIdx.x & (kBlockPts - 1), half = threadIdx.x >> 7;
  const int64_t pt = g * kBlockPts + i;
  const float c = pscale[pt], cinv = c > 0.f ? 1.f / c : 0.f;   // c = 0: X = 0 at this point
  const float4 xh = xdf[pt * 2], xl = xdf[pt * 2 + 1];   // (a, b) hi / lo
  if (threadIdx.x < kBasisBlk) colmax[threadIdx.x] = 0u;
  const f2 a{xh.x, xl.x}, bx{xh.y, xl.y}, by{xh.z, xl.z}, bz{xh.w, xl.w};
  if ((p + 1) * kBasisBlk > B.nbf) {   // a partial last block: its padding columns are zero
#pragma unroll
    for (int k = 0; k < kBasisBlk / 2; ++k) {
      const int nu = half * (kBasisBlk / 2) + k;
      sph[nu][i] = spl[nu][i] = sxh[nu][i] = sxl[nu][i] = 0.f;
    }
  }
  const float4 pr = G.prel[pt], pl = G.prel_lo[pt];
  if (threadIdx.x == 0 && t + ahead < t1) {
    // the radial factors of the tile that runs about `ahead` tiles later
    // (the CTAs resident on the GPU take tiles in order), moved into L2 now
    const int64_t ra = rad_ptr[t + ahead], rb = rad_ptr[t + ahead + 1];
    if (rb > ra) prefetch_l2(rad + (ra - rad_ptr[t0]) * kBlockPts, (uint32_t)((rb - ra) * kBlockPts * 16));
  }
  stage_block_rec(B, p, G.anchor[g], &rec, threadIdx.x, kX4Threads);
  __syncthreads();
  const int mid = rec.split;   // the two halves take consecutive shell ranges of about equal functions
  for_rec_phix_df<GRAD>(&rec, rad + (rad_ptr[t] - rad_ptr[t0]) * kBlockPts + i, half == 0 ? 0 : mid,
                        half == 0 ? mid : rec.nshell, f2{pr.x, pl.x},
                        f2{pr.y, pl.y}, f2{pr.z, pl.z}, a, bx, by, bz, [&](int nu, f2 v, f2 x) {
                          const float ph = v.h * c, xhh = x.h * cinv;
                          sph[nu][i] = ph;
                          spl[nu][i] = v.l * c;
                          sxh[nu][i] = xhh;
                          sxl[nu][i] = x.l * cinv;
                          // the function's column maximum: a warp reduction
                          // (every lane evaluates the same function), then
                          // one shared-memory maximum per warp; non-negative
                          // FP32 values order like their bit patterns
                          const unsigned m = __reduce_max_sync(
                              0xffffffffu, __float_as_uint(fmaxf(fabsf(ph), fabsf(xhh))));
                          if ((threadIdx.x & 31) == 0) atomicMax(&colmax[nu], m);
                        });
  __syncthreads();
  // one scale per function for Phi~ and X~ (they meet in one exact chain):
  // the power of two above the larger of their column maxima
  if (threadIdx.x < kBasisBlk) {
    cp[threadIdx.x] = pow2_ceil(__uint_as_float(colmax[threadIdx.x]) * 1.000001f);
    cx[threadIdx.x] = 1.f / cp[threadIdx.x];   // exact: the scales are powers of two
  }
  __syncthreads();
  float vh[kBasisBlk], vl[kBasisBlk];
#pragma unroll
  for (int nu = 0; nu < kBasisBlk; ++nu) {
    vh[nu] = sph[nu][i] * cx[nu];
    vl[nu] = spl[nu][i] * cx[nu];
  }
  if (half == 0)
    store_sliced_row4_kc<0, 2>(out_phi + (t - t0) * tile_bytes(4), i, vh, vl);
  else
    store_sliced_row4_kc<2, 4>(out_phi + (t - t0) * tile_bytes(4), i, vh, vl);
#pragma unroll
  for (int nu = 0; nu < kBasisBlk; ++nu) {
    vh[nu] = sxh[nu][i] * cx[nu];
    vl[nu] = sxl[nu][i] * cx[nu];
  }
  if (half == 0)
    store_sliced_row4_kc<0, 2>(out_x + (t - t0) * tile_bytes(4), i, vh, vl);
  else
    store_sliced_row4_kc<2, 4>(out_x + (t - t0) * tile_bytes(4), i, vh, vl);
  if (threadIdx.x < kBasisBlk) {
    phi_scale[(t - t0) * kBasisBlk + threadIdx.x] = cp[threadIdx.x];
    x_scale[(t - t0) * kBasisBlk + threadIdx.x] = cp[threadIdx.x];
  }
  // x_gq = max |X| over the tile, with X = X~ c_i
  float mx = 0.f;
  if (half == 0) {
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) mx = fmaxf(mx, fabsf(sxh[nu][i]) * c);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (half == 0 && (i & 31) == 0) rawx[i >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    const float m = fmaxf(fmaxf(rawx[0], rawx[1]), fmaxf(rawx[2], rawx[3]));
    xmax[t] = (double)m;
    xmaxf[t] = m;
  }
}

template <int NS>
static kldi_status x_ns(const kldi_plan* P, const Batch& b, cudaStream_t s) {
  const int64_t n = b.t1 - b.t0;
  if (n == 0) return KLDI_OK;
  uint8_t* op = reinterpret_cast<uint8_t*>(P->d_phic_s);
  uint8_t* ox = reinterpret_cast<uint8_t*>(P->d_x_s);
  if (P->gga)
    k_x_split<NS, true><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                          b.t0, P->d_xcoef, P->d_pscale, op, P->d_phic_scale, ox,
                                                          P->d_x_scale, P->d_xmax, P->d_xmaxf);
  else
    k_x_split<NS, false><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                           b.t0, P->d_xcoef, P->d_pscale, op, P->d_phic_scale, ox,
                                                           P->d_x_scale, P->d_xmax, P->d_xmaxf);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

static kldi_status x_ns4(const kldi_plan* P, const Batch& b, cudaStream_t s) {
  const int64_t n = b.t1 - b.t0;
  if (n == 0) return KLDI_OK;
  KLDI_TRY(prepare_tc_kernels());
  uint8_t* op = reinterpret_cast<uint8_t*>(P->d_phic_s);
  uint8_t* ox = reinterpret_cast<uint8_t*>(P->d_x_s);
  if (P->gga)
    k_x_split4<true><<<(unsigned)n, kX4Threads, kX4Smem, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                             b.t0, P->d_xdf, P->d_pscale, op, P->d_phic_scale, ox,
                                                             P->d_x_scale, P->d_xmax, P->d_xmaxf, P->d_rad, P->d_rad_ptr, b.t1,
                                                             (int64_t)3 * P->num_sms);
  else
    k_x_split4<false><<<(unsigned)n, kX4Threads, kX4Smem, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                              b.t0, P->d_xdf, P->d_pscale, op, P->d_phic_scale, ox,
                                                              P->d_x_scale, P->d_xmax, P->d_xmaxf, P->d_rad, P->d_rad_ptr, b.t1,
                                                              (int64_t)3 * P->num_sms);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

kldi_status launch_x_split(const kldi_plan* P, const Batch& b, cudaStream_t s) {
  switch (slices_of(P->prec)) {
    case 4: return x_ns4(P, b, s);
    case 3: return x_ns<3>(P, b, s);
    default: return x_ns<2>(P, b, s);
  }
}

// ---------------------------------------------------------------------------
// MMA issue of one K = 16 step for all slice products of levels < NS.  Level
// l goes to accumulator min(l, NACC - 1): with NACC < NS the smallest levels
// share the last accumulator (BF16X10 V product: levels 2 and 3).
template <int NS, int NACC = NS>
__device__ __forceinline__ void issue_levels(uint32_t d0, uint32_t lstride, const uint64_t* a, const uint64_t* b,
                                             uint32_t idesc, uint32_t* started) {
#pragma unroll
  for (int l = 0; l < NS; ++l) {
    const int acc = l < NACC ? l : NACC - 1;
#pragma unroll
    for (int i = 0; i <= l; ++i) {
      mma_f16(d0 + acc * lstride, a[i], b[l - i], idesc, started[acc]);
      started[acc] = 1;
    }
  }
}

// Density product, persistent: one CTA per SM walks grid blocks g0 + c,
// g0 + c + G, ...  Warp 0 = producer (all lanes build the next block's
// retained list and executed-pair bit matrix with warp ballots into a
// double-buffered shared-memory record, then issue each chunk's bulk copies
// together), warp 1 = TMEM owner and MMA issuer, the remaining kEpi warps =
// epilogue (lane quarter = warp % 4; the warps of a quarter take one basis
// block of each N tile each; their partial rho and grad rho are summed in a
// fixed order).  BF16X6 / BF16X3: N tiles of 4 basis blocks, 16 epilogue
// warps; BF16X10: N tiles of 2 basis blocks so that two buffers of the four
// level accumulators fit TMEM (drains and row-dot overlap the next tile's
// products), 16 epilogue warps, two per (lane quarter, q block) draining half
// the columns each and sharing the row-dot's shells, R and the row-dot in
// double-float.
template <int NS, int NQ = (NS == 4 ? 2 : 4)>
struct RhoCfg {
  static constexpr int kNQ = NQ;                                  // q blocks per N tile (2 or 4)
  static constexpr int kHalves = NQ == 2 ? 2 : 1;                 // warps per (lane quarter, q block)
  static constexpr int kEpi = 4 * kNQ * kHalves;                  // epilogue warps (16)
  static constexpr int kGroups = kNQ * kHalves;                   // epilogue groups of 4 warps (one per quarter)
  static constexpr int kColsPerWarp = 32 / kHalves;               // TMEM columns a warp drains
  static constexpr int kLevelCols = 32 * kNQ;                     // TMEM columns of one level accumulator
  static constexpr int kBufCols = NS * kLevelCols;                // NS level accumulators
  static constexpr int kBufs = 2 * kBufCols <= 512 ? 2 : 1;
  static constexpr int kStageBytes = NS * kPlaneBytes + NS * kNQ * kDPlane;
  static constexpr int kStages = NS == 4 ? 2 : (NS == 2 || NQ == 2 ? 3 : 2);
  static constexpr int kRsElem = NS == 4 ? 8 : 4;                 // R staged as FP32, or hi / lo pairs
  static constexpr int kOffR = kStages * kStageBytes;             // [kNQ q blocks][32][128] R
  static constexpr int kOffRed = kOffR + kNQ * kBasisBlk * kBlockPts * kRsElem;   // [kGroups][4][128] double
  // per-block record: n, tb, the retained list, the executed-pair bit matrix,
  // and per N tile the number of p blocks with an executed pair
  static constexpr int kOffNexec = 4 + kMaxRet + kMaxRet * (kMaxRet / 32);
  static constexpr int kMetaWords = kOffNexec + kMaxRet / 2;
  static constexpr int kOffMeta = kOffRed + kGroups * 4 * kBlockPts * 8;
  static constexpr int kOffRec = kOffMeta + 2 * kMetaWords * 4;  // [kNQ q blocks][2] BlockRec
  static constexpr int kOffTab = kOffRec + 2 * kNQ * (int)sizeof(BlockRec);
  static constexpr int kOffBar = kOffTab;
  static constexpr int kSmem = kOffBar + 256 + 1024;
  static constexpr int kSegChunks = 8;                            // 8 x 32 = 256 K per exact accumulation
  static constexpr int kThreads = 64 + 32 * kEpi;
  static_assert(kSmem <= 232448, "shared memory");
  static_assert(kBufs * kBufCols <= 512, "TMEM");
  static_assert(NQ == 2 || NQ == 4, "N tile of 2 or 4 basis blocks");
};

// Row-dot of one basis block in double-float (BF16X10), over the shells
// sb .. se - 1: with R_nu (hi / lo, staged [32][128]) and the shell
// factorisation chi = P g,
// grad chi = (grad P) g + P u (u = -2 r gd),
//   sum_nu chi R = sum_s g S0,   sum_nu grad chi R = sum_s (g S1 + u S0),
// S0 = sum_c P_c R_c and S1 = sum_c (grad P_c) R_c over the shell's components.
// The shells of one atom share r, so their u S0 terms are gathered as
// -2 r T with T = sum_s gd S0 over the run of shells on that atom (the
// shells of a block are grouped by atom), and the offsets are formed once
// per run.  The radial factors g, gd of each shell at this point come from
// the Phi kernel (rad[s * 128]).
template <bool GRAD>
__device__ __forceinline__ void rowdot_df(const BlockRec* rec, const float4* rad, const float2* Rs, int i, int sb,
                                          int se, f2 px, f2 py, f2 pz, f2& pr, f2& gx, f2& gy, f2& gz) {
  const f2 s3{kS3h, kS3l};
  // radial factors loaded one shell ahead (the loads come from HBM / L2)
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 qa = sb < se ? rad[sb * kBlockPts] : z4;
  f2 dx{0.f, 0.f}, dy{0.f, 0.f}, dz{0.f, 0.f}, T{0.f, 0.f};
  auto flush = [&]() {   // the run's u S0 terms: -2 r T
    const f2 m2 = df_scale(T, -2.f);
    gx = df_add_u(gx, df_mul_u(dx, m2));
    gy = df_add_u(gy, df_mul_u(dy, m2));
    gz = df_add_u(gz, df_mul_u(dz, m2));
    T = f2{0.f, 0.f};
  };
  for (int s = sb; s < se; ++s) {
    const float4 q = qa;
    qa = s + 1 < se ? rad[(s + 1) * kBlockPts] : z4;
    const float4 c0 = rec->c0[s], c1 = rec->c1[s];
    const int hdr = __float_as_int(c1.z);
    const int l = hdr & 255, first = (hdr >> 16) - 64;
    const f2 g{q.x, q.y}, gd{q.z, q.w};
    if (s == sb || rec->atom[s] != rec->atom[s - 1]) {
      if (GRAD && s != sb) flush();
      offsets3_df(c0, c1, px, py, pz, dx, dy, dz);
    }
    auto Rv = [&](int c) -> f2 {
      const int nu = first + c;
      if (nu < 0 || nu >= kBasisBlk) return f2{0.f, 0.f};
      const float2 r = Rs[nu * kBlockPts + i];
      return f2{r.x, r.y};
    };
    // S0 = sum_c P_c R_c and S1 = sum_c (grad P_c) R_c, one component at a
    // time (few values live at once)
    f2 S0{0.f, 0.f}, S1x{0.f, 0.f}, S1y{0.f, 0.f}, S1z{0.f, 0.f};
    if (l == 0) {
      S0 = Rv(0);
    } else if (l == 1) {
      S1x = Rv(0);
      S1y = Rv(1);
      S1z = Rv(2);
      S0 = df_add_u(df_add_u(df_mul_u(dx, S1x), df_mul_u(dy, S1y)), df_mul_u(dz, S1z));
    } else {
      // xx, yy, zz (with 1/sqrt(3)): P = r_a^2 s3, d_a P = 2 r_a s3
      // xy, xz, yz: P = r_a r_b, d_a P = r_b, d_b P = r_a
      {
        const f2 t = df_mul_u(dx, df_mul_u(Rv(0), s3));
        S0 = df_mul_u(dx, t);
        S1x = df_scale(t, 2.f);
      }
      {
        const f2 r = Rv(1);
        const f2 t = df_mul_u(dy, r);
        S0 = df_add_u(S0, df_mul_u(dx, t));
        S1x = df_add_u(S1x, t);
        S1y = df_mul_u(dx, r);
      }
      {
        const f2 r = Rv(2);
        const f2 t = df_mul_u(dz, r);
        S0 = df_add_u(S0, df_mul_u(dx, t));
        S1x = df_add_u(S1x, t);
        S1z = df_mul_u(dx, r);
      }
      {
        const f2 t = df_mul_u(dy, df_mul_u(Rv(3), s3));
        S0 = df_add_u(S0, df_mul_u(dy, t));
        S1y = df_add_u(S1y, df_scale(t, 2.f));
      }
      {
        const f2 r = Rv(4);
        const f2 t = df_mul_u(dz, r);
        S0 = df_add_u(S0, df_mul_u(dy, t));
        S1y = df_add_u(S1y, t);
        S1z = df_add_u(S1z, df_mul_u(dy, r));
      }
      {
        const f2 t = df_mul_u(dz, df_mul_u(Rv(5), s3));
        S0 = df_add_u(S0, df_mul_u(dz, t));
        S1z = df_add_u(S1z, df_scale(t, 2.f));
      }
    }
    pr = df_add_u(pr, df_mul_u(g, S0));
    if (GRAD) {
      T = df_add_u(T, df_mul_u(gd, S0));
      if (l > 0) {
        gx = df_add_u(gx, df_mul_u(g, S1x));
        gy = df_add_u(gy, df_mul_u(g, S1y));
        gz = df_add_u(gz, df_mul_u(g, S1z));
      }
    }
  }
  if (GRAD && se > sb) flush();
}

// Epilogue of the density-product kernel: the row-dot (rho, grad rho), or
// one of the two terms of the nuclear gradient of E_xc on a fixed grid,
//   dE/dR_A = -2 sum_{mu on A} sum_i [ grad chi_mu Q_mu,i + (b_i . grad grad chi_mu) R_mu,i ]
// with R = Phi D and Q = Z D (Z = 2 a phi + b . grad phi) over the executed pairs:
// kGradQ takes the Z~ tiles as operand A and contracts Q with grad chi,
// kGradR takes the Phi~ tiles and contracts R with b . grad grad chi.
enum { kRowDot = 0, kGradR = 1, kGradQ = 2 };

template <int NS, bool GRAD, int MODE = kRowDot, int NQ = (NS == 4 ? 2 : 4)>
__global__ void __launch_bounds__(RhoCfg<NS, NQ>::kThreads, 1)
    k_rho_tc(BasisView B, GridView G, ListView L, int64_t g0, int64_t g1, int64_t t0,
             const uint8_t* __restrict__ phi, const uint8_t* __restrict__ dsplit, const uint8_t* __restrict__ zero,
             const double* __restrict__ dmax, const float* __restrict__ dscale, const float* __restrict__ rowscale,
             double t_b, double t_d, double* rho, double* grad, const double* __restrict__ xcoef, double* gout,
             int* err, uint64_t wait_ns, const float4* __restrict__ rad, const int64_t* __restrict__ rad_ptr) {
  using C = RhoCfg<NS, NQ>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  int32_t* meta_base = reinterpret_cast<int32_t*>(sm + C::kOffMeta);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::kOffBar);
  uint64_t* empty = full + C::kStages;
  uint64_t* tfull = empty + C::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* mfull = tempty + 2;
  uint64_t* mempty = mfull + 2;
  uint64_t* rfull = mempty + 2;       // partial sums of the four q-block groups written
  uint64_t* rempty = rfull + 1;       // ... and read by the combining warps
  uint64_t* mdone = rempty + 1;       // all products of the MMA thread completed (exit)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G_ = gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], C::kEpi);
      mbar_init(&mfull[b], 1);
      mbar_init(&mempty[b], 1 + C::kEpi);   // the MMA thread and the epilogue warps
    }
    mbar_init(rfull, C::kEpi);
    mbar_init(rempty, 4);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  // per-block record: [0] n, [1] tb, [4 .. 4+kMaxRet) plist, then the bit matrix
  auto meta = [&](int b) { return meta_base + b * C::kMetaWords; };
  auto tile_bits = [](const int32_t* m, int jp, int q0, int nq) -> uint32_t {
    const int nw = (m[0] + 31) >> 5;
    const uint32_t* mask = reinterpret_cast<const uint32_t*>(m + 4 + kMaxRet);
    return (mask[jp * nw + (q0 >> 5)] >> (q0 & 31)) & ((1u << nq) - 1u);
  };
  // exact segments of N tile nt (one empty segment when nothing is executed)
  auto nsegs = [&](const int32_t* m, int nt) -> int {
    const int c = m[C::kOffNexec + nt];
    return c == 0 ? 1 : (c + C::kSegChunks - 1) / C::kSegChunks;
  };

  if (warp == 0) {
    uint32_t it = 0;
    for (int64_t k = 0;; ++k) {
      const int64_t g = g0 + blockIdx.x + k * G_;
      if (g >= g1 || *abort_flag) break;
      const int b = (int)(k & 1);
      if (!mbar_wait_warp(&mempty[b], (uint32_t)(((k >> 1) & 1) ^ 1), abort_flag, err, 110, wait_ns)) break;
      int32_t* m = meta(b);
      const int tb = L.blk_ptr[g];
      int n = L.blk_ptr[g + 1] - tb;
      if (n > kMaxRet) {
        if (lane == 0) atomicCAS(err, 0, 101);
        n = 0;
      }
      const int nw = (n + 31) >> 5;
      int32_t* plist = m + 4;
      uint32_t* mask = reinterpret_cast<uint32_t*>(m + 4 + kMaxRet);
      for (int j = lane; j < n; j += 32) plist[j] = L.blk_idx[tb + j];
      __syncwarp();
      // executed pairs E1_g: one ballot per 32 (jp, jq) predicates; lane owns
      // column jq = 32 w + lane, the loads of eight rows are issued together
      for (int w = 0; w < nw; ++w) {
        const int jq = w * 32 + lane;
        const bool in = jq < n;
        const int qblk = in ? plist[jq] : 0;
        const double bq = in ? L.bmax[tb + jq] : 0.0;
        for (int jp0 = 0; jp0 < n; jp0 += 8) {
          double dm[8], bp[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int jp = jp0 + u;
            dm[u] = (in && jp < n) ? dmax[plist[jp] * L.nbb + qblk] : 0.0;
            bp[u] = jp < n ? L.bmax[tb + jp] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int jp = jp0 + u;
            const bool pred = in && jp < n && dm[u] >= t_b && bp[u] * dm[u] * bq >= t_d;
            const uint32_t word = __ballot_sync(0xffffffffu, pred);
            if (lane == 0 && jp < n) mask[jp * nw + w] = word;
          }
        }
      }
      if (lane == 0) {
        m[0] = n;
        m[1] = tb;
      }
      __syncwarp();
      for (int nt = lane; nt < (n + C::kNQ - 1) / C::kNQ; nt += 32) {
        const int q0 = nt * C::kNQ, nq = min(C::kNQ, n - q0);
        int c = 0;
        for (int jp = 0; jp < n; ++jp) c += tile_bits(m, jp, q0, nq) != 0;
        m[C::kOffNexec + nt] = c;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&mfull[b]);
      {
        // the warp issues each chunk's copies together: lane 31 the Phi~ tile
        // (its NS planes in one copy), lanes 0 .. NS nq - 1 one D plane each
        const int ntile = (n + C::kNQ - 1) / C::kNQ;
        bool ok = true;
        for (int nt = 0; nt < ntile && ok; ++nt) {
          const int q0 = nt * C::kNQ, nq = min(C::kNQ, n - q0);
          if constexpr (MODE == kRowDot && NS == 4) {
            // the radial factors the row-dot of this N tile reads, moved into
            // L2 while its products run
            if (lane < nq) {
              const int64_t tq = tb + q0 + lane, r0 = rad_ptr[tq], r1 = rad_ptr[tq + 1];
              if (r1 > r0) prefetch_l2(rad + (r0 - rad_ptr[t0]) * kBlockPts, (uint32_t)((r1 - r0) * kBlockPts * 16));
            }
          }
          for (int jp = 0; jp < n; ++jp) {
            const uint32_t bits = tile_bits(m, jp, q0, nq);
            if (!bits) continue;
            const int s = it % C::kStages;
            const uint32_t ph = (it / C::kStages) & 1;
            if (!mbar_wait_warp(&empty[s], ph ^ 1, abort_flag, err, 111, wait_ns)) { ok = false; break; }
            uint8_t* st = sm + s * C::kStageBytes;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], NS * kPlaneBytes + NS * nq * kDPlane);
            __syncwarp();
            if (lane == 31) {
              bulk_g2s(st, phi + (int64_t)(tb + jp - t0) * tile_bytes(NS), NS * kPlaneBytes, &full[s]);
            } else if (lane < NS * nq) {
              const int kq = lane / NS, l = lane % NS;
              const bool on = (bits >> kq) & 1u;
              const uint8_t* d = dsplit + ((int64_t)plist[jp] * L.nbb + plist[q0 + kq]) * (NS * kDPlane);
              bulk_g2s(st + NS * kPlaneBytes + l * (C::kNQ * kDPlane) + kq * kDPlane, on ? d + l * kDPlane : zero,
                       kDPlane, &full[s]);
            }
            ++it;
          }
        }
      }
      __syncwarp();
    }
    if (lane == 0)
      for (uint32_t k = (it > (uint32_t)C::kStages ? it - C::kStages : 0); k < it; ++k) {
        volatile int no_abort = 0;
        mbar_wait(&full[k % C::kStages], (k / C::kStages) & 1, &no_abort, nullptr, 0);
      }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0, job = 0;
      bool ok = true;
      for (int64_t k = 0; ok; ++k) {
        const int64_t g = g0 + blockIdx.x + k * G_;
        if (g >= g1 || *abort_flag) break;
        const int b = (int)(k & 1);
        if (!mbar_wait(&mfull[b], (uint32_t)((k >> 1) & 1), abort_flag, err, 115, wait_ns)) break;
        const int32_t* m = meta(b);
        const int n = m[0];
        const int ntile = (n + C::kNQ - 1) / C::kNQ;
        for (int nt = 0; nt < ntile && ok; ++nt) {
          const int q0 = nt * C::kNQ, nq = min(C::kNQ, n - q0);
          const uint32_t idesc = instr_desc(128, 32 * nq, 1, 0, 0);
          int jp = 0;
          const int ns = nsegs(m, nt);
          for (int sg = 0; sg < ns && ok; ++sg, ++job) {
            const int buf = job % C::kBufs;
            const uint32_t use = job / C::kBufs;
            if (!mbar_wait(&tempty[buf], (use & 1) ^ 1, abort_flag, err, 112, wait_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d0 = tbase + buf * C::kBufCols;
            uint32_t started[NS];
#pragma unroll
            for (int l = 0; l < NS; ++l) started[l] = 0;
            int taken = 0;
            for (; jp < n && taken < C::kSegChunks; ++jp) {
              if (!tile_bits(m, jp, q0, nq)) continue;
              const int s = it % C::kStages;
              const uint32_t ph = (it / C::kStages) & 1;
              if (!mbar_wait(&full[s], ph, abort_flag, err, 113, wait_ns)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a = smem_u32(sm + s * C::kStageBytes);
              const uint32_t bsm = a + NS * kPlaneBytes;
              if constexpr (NQ == 2) {
                // The NS planes of B lie one after another (64 rows each), and
                // so do the level accumulators (64 columns each): one product
                // of slice a_i with [b_0 | ... | b_{NS-1-i}] (N = 64 (NS - i))
                // adds a_i b_j to level i + j for every j at once, NS
                // products per K = 16 step instead of NS (NS + 1) / 2.  The
                // first one of a segment (i = 0) starts all NS levels.  A tile
                // of one q block leaves the second 32 columns of each level
                // undefined; the drain reads only the first 32.
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                  const uint64_t bd = smem_desc(bsm + kk * 32, 16, 512, kSwz64);
#pragma unroll
                  for (int i = 0; i < NS; ++i) {
                    const uint64_t ad = smem_desc(a + i * kPlaneBytes + kk * 32, 16, 512, kSwz64);
                    mma_f16(d0 + i * C::kLevelCols, ad, bd, instr_desc(128, 64 * (NS - i), 1, 0, 0),
                            i == 0 ? started[0] : 1u);
                  }
                  started[0] = 1;
                }
              } else {
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                  uint64_t ad[NS], bd[NS];
#pragma unroll
                  for (int l = 0; l < NS; ++l) {
                    ad[l] = smem_desc(a + l * kPlaneBytes + kk * 32, 16, 512, kSwz64);
                    bd[l] = smem_desc(bsm + l * (C::kNQ * kDPlane) + kk * 32, 16, 512, kSwz64);
                  }
                  issue_levels<NS>(d0, C::kLevelCols, ad, bd, idesc, started);
                }
              }
              mma_commit(&empty[s]);
              ++it;
              ++taken;
            }
            if (!ok) break;
            mma_commit(&tfull[buf]);
          }
        }
        mbar_arrive(&mempty[b]);
      }
      if (!ok) *abort_flag = 1;
      // every product this thread issued completes before the CTA frees its
      // tensor memory, also when a wait gave up in the middle of a stream
      mma_commit(mdone);
      volatile int no_abort = 0;
      mbar_wait(mdone, 0, &no_abort, nullptr, 0);
    }
  } else {
    // warp w: lane quarter w % 4 (its TMEM lanes), group grp = q block k4 of
    // every N tile and, for BF16X10, half: the half of the q block's columns it
    // drains and the parity of the shells whose row-dot terms it forms
    const int quarter = warp & 3;
    const int grp = (warp - 2) >> 2;
    const int k4 = grp % C::kNQ;
    const int half = grp / C::kNQ;
    const int i = quarter * 32 + lane;
    float* Rs = reinterpret_cast<float*>(sm + C::kOffR) + k4 * (kBasisBlk * kBlockPts);
    float2* Rs2 = reinterpret_cast<float2*>(sm + C::kOffR) + k4 * (kBasisBlk * kBlockPts);   // BF16X10
    // R_nu of this thread's point as FP32 (the gradient epilogues)
    auto rget = [&](int nu, int i_) -> float {
      if constexpr (NS == 4) return Rs2[nu * kBlockPts + i_].x;
      else return Rs[nu * kBlockPts + i_];
    };
    double* red = reinterpret_cast<double*>(sm + C::kOffRed);
    BlockRec* recs = reinterpret_cast<BlockRec*>(sm + C::kOffRec) + 2 * k4;
    uint32_t job = 0, ruse = 0;
    bool ok = true;
    for (int64_t k = 0; ok; ++k) {
      const int64_t g = g0 + blockIdx.x + k * G_;
      if (g >= g1 || *abort_flag) break;
      const int b = (int)(k & 1);
      if (!mbar_wait_warp(&mfull[b], (uint32_t)((k >> 1) & 1), abort_flag, err, 116, wait_ns)) break;
      const int32_t* m = meta(b);
      const int n = m[0];
      const int32_t* plist = m + 4;
      const int64_t pt = g * kBlockPts + i;
      const float4 prl = G.prel[pt];
      float4 prlo = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (NS == 4) prlo = G.prel_lo[pt];
      const int anc = G.anchor[g];
      const double rsc = (double)rowscale[pt];
      // the point's sums over its tiles in double-float (FP64 arithmetic is
      // slow on this GPU), scaled and converted once per grid block
      f2 ar{0.f, 0.f}, agx{0.f, 0.f}, agy{0.f, 0.f}, agz{0.f, 0.f};
      float bx = 0.f, by = 0.f, bz = 0.f;   // b_i of the gradient's Hessian term
      if constexpr (MODE == kGradR) {
        bx = (float)xcoef[pt * 4 + 1];
        by = (float)xcoef[pt * 4 + 2];
        bz = (float)xcoef[pt * 4 + 3];
      }
      const int ntile = (n + C::kNQ - 1) / C::kNQ;
      for (int nt = 0; nt < ntile && ok; ++nt) {
        const int q0 = nt * C::kNQ, nq = min(C::kNQ, n - q0);
        const int ns = nsegs(m, nt);
        const bool work = m[C::kOffNexec + nt] > 0;
        const bool mine = work && k4 < nq;
        // the four warps of this q block stage its shells (double-buffered
        // record, one named barrier per use) while the products run
        BlockRec* rec = recs + (ruse & 1);
        const int qb = mine ? plist[q0 + k4] : 0;
        const bool staged = mine && block_rec_fits(B, qb);
        if (staged) {
          stage_block_rec(B, qb, anc, rec, half * 128 + quarter * 32 + lane, 128 * C::kHalves);
          if (quarter == 0 && half == 0) rec->ds[lane] = dscale[qb * kBasisBlk + lane];
        }
        float R[32], Rl[32];   // Rl: low parts (BF16X10)
#pragma unroll
        for (int c = 0; c < 32; ++c) R[c] = Rl[c] = 0.f;
        for (int sg = 0; sg < ns; ++sg, ++job) {
          const int buf = job % C::kBufs;
          const uint32_t use = job / C::kBufs;
          if (!mbar_wait_warp(&tfull[buf], use & 1, abort_flag, err, 114, wait_ns)) { ok = false; break; }
          tc_fence_after();
          if (mine) {
            const uint32_t ta = tbase + ((uint32_t)(quarter * 32) << 16) + buf * C::kBufCols + k4 * 32 +
                                half * C::kColsPerWarp;
            constexpr uint32_t LC = C::kLevelCols;
            if constexpr (NS == 4) {
              // 8 columns of the four levels at a time (registers)
#pragma unroll
              for (int h = 0; h < C::kColsPerWarp / 8; ++h) {
                float t[32];
                tmem_ld8x4(ta + 3 * LC + h * 8, ta + 2 * LC + h * 8, ta + LC + h * 8, ta + h * 8, t);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                  // hi: the running sum plus L0, error-free; lo: its error plus
                  // L1 and the two small levels (rounded at ~2^-32 of the scale)
                  const f2 sg = two_sum(R[h * 8 + c], t[24 + c]);
                  R[h * 8 + c] = sg.h;
                  Rl[h * 8 + c] = __fadd_rn(Rl[h * 8 + c],
                                            __fadd_rn(__fadd_rn(sg.l, t[16 + c]), __fadd_rn(t[8 + c], t[c])));
                }
              }
            }
#pragma unroll
            for (int h = 0; h < (NS == 4 ? 0 : C::kColsPerWarp / 16); ++h) {
              // the NS levels of 16 columns, smallest first, one wait
              float t[16 * NS];
              if constexpr (NS == 3)
                tmem_ld16x3(ta + 2 * LC + h * 16, ta + LC + h * 16, ta + h * 16, t);
              else if constexpr (NS == 2)
                tmem_ld16x2(ta + LC + h * 16, ta + h * 16, t);
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                float acc = t[c];
#pragma unroll
                for (int l = 1; l < NS; ++l) acc += t[16 * l + c];
                R[h * 16 + c] += acc;
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (!ok) break;
        // row-dot with this warp's basis block: R_i,nu = e_i f_nu R[c]
        // (a tile without executed pairs has R = 0 and adds nothing)
        if (mine) {
          const int q = qb;
          named_bar_sync(1 + k4, 128 * C::kHalves);
          ++ruse;
          if constexpr (NS == 4) {
            // this warp's columns; the row-dot reads both halves' columns
#pragma unroll
            for (int c = 0; c < C::kColsPerWarp; ++c) {
              const int col = half * C::kColsPerWarp + c;
              const float f = staged ? rec->ds[col] : dscale[q * kBasisBlk + col];
              const f2 r = two_sum(R[c], Rl[c]);   // normalised: hi is R to FP32 (the gradient epilogues read hi)
              Rs2[col * kBlockPts + i] = make_float2(r.h * f, r.l * f);
            }
            named_bar_sync(1 + k4, 128 * C::kHalves);
          } else {
#pragma unroll
            for (int c = 0; c < C::kColsPerWarp; ++c) {
              const int col = half * C::kColsPerWarp + c;
              Rs[col * kBlockPts + i] = R[c] * (staged ? rec->ds[col] : dscale[q * kBasisBlk + col]);
            }
            if constexpr (C::kHalves > 1) named_bar_sync(1 + k4, 128 * C::kHalves);
          }
          if constexpr (MODE == kRowDot && NS == 4) {
            if (staged) {
              f2 pr{0.f, 0.f}, px_{0.f, 0.f}, py_{0.f, 0.f}, pz_{0.f, 0.f};
              const int64_t tq = m[1] + q0 + k4;   // tile (g, q block)
              const int nsh = rec->nshell, mid = rec->split;   // the halves take consecutive shells
              rowdot_df<GRAD>(rec, rad + (rad_ptr[tq] - rad_ptr[t0]) * kBlockPts + i, Rs2, i, half == 0 ? 0 : mid,
                              half == 0 ? mid : nsh, f2{prl.x, prlo.x}, f2{prl.y, prlo.y}, f2{prl.z, prlo.z}, pr,
                              px_, py_, pz_);
              ar = df_add(ar, pr);
              if (GRAD) {
                agx = df_add(agx, px_);
                agy = df_add(agy, py_);
                agz = df_add(agz, pz_);
              }
            } else if (lane == 0) {
              atomicCAS(err, 0, 102);   // the double-float row-dot needs staged shell records
            }
          } else if constexpr (MODE == kRowDot) {
            float pr = 0.f, px_ = 0.f, py_ = 0.f, pz_ = 0.f;
            auto acc = [&](int nu, float v, float dx, float dy, float dz) {
              const float rr = Rs[nu * kBlockPts + i];
              pr = fmaf(v, rr, pr);
              if (GRAD) {
                px_ = fmaf(dx, rr, px_);
                py_ = fmaf(dy, rr, py_);
                pz_ = fmaf(dz, rr, pz_);
              }
            };
            if (staged)
              for_rec_functions<GRAD>(rec, prl.x, prl.y, prl.z, acc, half, C::kHalves);
            else if (half == 0)
              for_block_functions<float, GRAD>(B, q, prl.x, prl.y, prl.z, acc, anc);
            ar = df_add(ar, f2{pr, 0.f});
            if (GRAD) {
              agx = df_add(agx, f2{px_, 0.f});
              agy = df_add(agy, f2{py_, 0.f});
              agz = df_add(agz, f2{pz_, 0.f});
            }
          } else if (staged && half == 0) {
            // per atom of the block's shells: the warp's sum over its 32
            // points, one FP64 atomic per atom and component (BF16X10: the
            // first half of the warps)
            int cur = -1;
            float tx = 0.f, ty = 0.f, tz = 0.f;
            auto flush = [&]() {
              const float rscf = (float)rsc;
              float v[3] = {tx * rscf, ty * rscf, tz * rscf};
#pragma unroll
              for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
              if (lane == 0)
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(&gout[cur * 3 + c], -2.0 * (double)v[c]);
            };
            for_rec_derivatives<MODE == kGradR>(rec, prl.x, prl.y, prl.z,
                                                [&](int atom, int nu, const float* d, const float* h) {
              if (atom != cur) {
                if (cur >= 0) flush();
                cur = atom;
                tx = ty = tz = 0.f;
              }
              const float rr = rget(nu, i);
              if constexpr (MODE == kGradQ) {
                tx = fmaf(d[0], rr, tx);
                ty = fmaf(d[1], rr, ty);
                tz = fmaf(d[2], rr, tz);
              } else {
                // (b . grad d_x chi) = b_x h_xx + b_y h_xy + b_z h_xz, ...
                tx = fmaf(fmaf(bx, h[0], fmaf(by, h[1], bz * h[2])), rr, tx);
                ty = fmaf(fmaf(bx, h[1], fmaf(by, h[3], bz * h[4])), rr, ty);
                tz = fmaf(fmaf(bx, h[2], fmaf(by, h[4], bz * h[5])), rr, tz);
              }
            });
            if (cur >= 0) flush();
          } else if (!staged && lane == 0) {
            atomicCAS(err, 0, 102);   // the gradient epilogue needs staged shell records
          }
        }
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(&mempty[b]);
      if constexpr (MODE != kRowDot) continue;
      const double r_i = rsc * df_to_double(ar);    // rsc: a power of two
      const double gx = 2.0 * rsc * df_to_double(agx);
      const double gy = 2.0 * rsc * df_to_double(agy);
      const double gz = 2.0 * rsc * df_to_double(agz);
      // combine the four q-block groups of each point in a fixed order
      if (!mbar_wait_warp(rempty, (uint32_t)(k & 1) ^ 1u, abort_flag, err, 117, wait_ns)) break;
      red[(grp * 4 + 0) * kBlockPts + i] = r_i;
      red[(grp * 4 + 1) * kBlockPts + i] = gx;
      red[(grp * 4 + 2) * kBlockPts + i] = gy;
      red[(grp * 4 + 3) * kBlockPts + i] = gz;
      __syncwarp();
      if (lane == 0) mbar_arrive(rfull);
      if (grp == 0) {
        if (!mbar_wait_warp(rfull, (uint32_t)(k & 1), abort_flag, err, 118, wait_ns)) break;
        double v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          v[c] = red[c * kBlockPts + i];
#pragma unroll
          for (int q = 1; q < C::kGroups; ++q) v[c] += red[(q * 4 + c) * kBlockPts + i];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(rempty);
        rho[pt] = v[0];
        if (GRAD) {
          grad[pt * 3] = v[1];
          grad[pt * 3 + 1] = v[2];
          grad[pt * 3 + 2] = v[3];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

kldi_status prepare_tc_kernels();   // defined after the kernels: shared-memory opt-in, register check

template <int NS, int NQ = (NS == 4 ? 2 : 4)>
static kldi_status rho_ns(const kldi_plan* P, const Batch& b, double* rho_out, double* grad_out, cudaStream_t s) {
  using C = RhoCfg<NS, NQ>;
  const int64_t n = b.g1 - b.g0;
  if (n == 0) return KLDI_OK;
  KLDI_TRY(prepare_tc_kernels());
  const unsigned grid = (unsigned)std::min<int64_t>(n, P->num_sms);
  const uint8_t* phi = reinterpret_cast<const uint8_t*>(P->d_phi_s);
  const uint8_t* ds = reinterpret_cast<const uint8_t*>(P->d_dsplit);
  const uint8_t* z = reinterpret_cast<const uint8_t*>(P->d_zero);
  if (P->gga)
    k_rho_tc<NS, true, kRowDot, NQ><<<grid, C::kThreads, C::kSmem, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                           b.g1, b.t0, phi, ds, z, P->d_dmax, P->d_dscale,
                                                           P->d_rowscale, P->opt.t_b, P->opt.t_d, rho_out, grad_out,
                                                           nullptr, nullptr, P->d_err, P->wait_ns, P->d_rad, P->d_rad_ptr);
  else
    k_rho_tc<NS, false, kRowDot, NQ><<<grid, C::kThreads, C::kSmem, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0,
                                                            b.g1, b.t0, phi, ds, z, P->d_dmax, P->d_dscale,
                                                            P->d_rowscale, P->opt.t_b, P->opt.t_d, rho_out, grad_out,
                                                            nullptr, nullptr, P->d_err, P->wait_ns, P->d_rad, P->d_rad_ptr);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// The density product's N tile: 2 basis blocks (64 functions, two TMEM
// buffers) or 4 (128 functions; one buffer for BF16X6): the plan's tuning,
// else the mode's default (BF16X10 only has the 64-function tile).
kldi_status launch_rho_tc(const kldi_plan* P, const Batch& b, double* rho_out, double* grad_out, cudaStream_t s) {
  const bool narrow = P->tune.rho_ntile == 64;
  switch (slices_of(P->prec)) {
    case 4: return rho_ns<4>(P, b, rho_out, grad_out, s);
    case 3: return narrow ? rho_ns<3, 2>(P, b, rho_out, grad_out, s) : rho_ns<3>(P, b, rho_out, grad_out, s);
    default: return narrow ? rho_ns<2, 2>(P, b, rho_out, grad_out, s) : rho_ns<2>(P, b, rho_out, grad_out, s);
  }
}

// Nuclear gradient of one batch (after its density and functional stages):
// Z tiles into the X-tile buffer, then the Q term (operand Z~) and, for a GGA
// functional, the R term (operand Phi~) of the density-product kernel.
template <int NS>
static kldi_status grad_ns(const kldi_plan* P, const Batch& b, bool gga_xc, double* G, cudaStream_t s) {
  using C = RhoCfg<NS>;
  const int64_t n = b.g1 - b.g0;
  if (n == 0) return KLDI_OK;
  KLDI_TRY(prepare_tc_kernels());
  uint8_t* zt = reinterpret_cast<uint8_t*>(P->d_x_s);
  k_z_split<NS><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                  P->d_xcoef, zt, P->d_zscale);
  KLDI_TRY_CUDA(cudaGetLastError());
  const unsigned grid = (unsigned)std::min<int64_t>(n, P->num_sms);
  const uint8_t* ds = reinterpret_cast<const uint8_t*>(P->d_dsplit);
  const uint8_t* z = reinterpret_cast<const uint8_t*>(P->d_zero);
  k_rho_tc<NS, false, kGradQ><<<grid, C::kThreads, C::kSmem, s>>>(
      P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.g1, b.t0, zt, ds, z, P->d_dmax, P->d_dscale,
      P->d_zscale, P->opt.t_b, P->opt.t_d, nullptr, nullptr, P->d_xcoef, G, P->d_err, P->wait_ns, P->d_rad, P->d_rad_ptr);
  KLDI_TRY_CUDA(cudaGetLastError());
  if (gga_xc) {
    k_rho_tc<NS, false, kGradR><<<grid, C::kThreads, C::kSmem, s>>>(
        P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.g1, b.t0,
        reinterpret_cast<const uint8_t*>(P->d_phi_s), ds, z, P->d_dmax, P->d_dscale, P->d_rowscale, P->opt.t_b,
        P->opt.t_d, nullptr, nullptr, P->d_xcoef, G, P->d_err, P->wait_ns, P->d_rad, P->d_rad_ptr);
    KLDI_TRY_CUDA(cudaGetLastError());
  }
  return KLDI_OK;
}

kldi_status launch_grad_tc(const kldi_plan* P, const Batch& b, bool gga_xc, double* G, cudaStream_t s) {
  switch (slices_of(P->prec)) {
    case 4: return grad_ns<4>(P, b, gga_xc, G, s);
    case 3: return grad_ns<3>(P, b, gga_xc, G, s);
    default: return grad_ns<2>(P, b, gga_xc, G, s);
  }
}

// ---------------------------------------------------------------------------
// V product, persistent over work items (pair P <= Q of 128-function windows
// of 4 consecutive basis blocks, segment of its grid-block list).  Per grid
// block one exact chain of K = 256: A = [Phi~_P | X~_P]^T, B = [X~_Q ; Phi~_Q]
// (MN-major operands), so the chain yields Phi^T X + X^T Phi of the window
// pair at once.  A diagonal pair (P = Q) runs the first half only (K = 128,
// S = Phi~_P^T X~_P).  The finish kernel forms V = A + A^T of the accumulated
// products A (off-diagonal pairs lie above the block diagonal).  384 threads in three
// warpgroups: warpgroup 0 = warp 0 producer (one lane per bulk copy), warp 1
// TMEM owner + MMA issue, warps 2-3 idle; warpgroups 1-2 = epilogue (lane
// quarter = warp % 4, column half = warpgroup - 1) with compensated FP32 sums
// per element (sums in registers, compensation terms in the TMEM columns after
// the level accumulators) and an FP64 scatter-add at the end of each work
// item.  Work items come from a global counter (a dynamic queue, so that CTAs
// running together take neighbouring items).  Registers move from warpgroup 0
// (kRegsLow) to the epilogue (kRegsHigh).
template <int NS>
struct VCfg {
  static constexpr int kChunk = 2048;                   // 32 points x 64 B of one plane of one tile
  static constexpr int kOp = 4 * kChunk;                // 4 tiles (128 functions) of one plane
  static constexpr int kStageBytes = 2 * NS * kOp;      // [side A, B][tile j][plane][32 points x 64 B]
  static constexpr int kStages = NS == 4 ? 3 : 4;
  // accumulators: one per level; BF16X10 keeps levels 0 and 1 exact and lets
  // levels 2 and 3 (2^-16 and 2^-24 of the scale) share a rounding one, whose
  // truncation then acts at ~2^-40 of the scale per step
  static constexpr int kAcc = NS == 4 ? 3 : NS;
  static constexpr int kBufCols = kAcc * 128;
  static constexpr int kCcCol = kAcc * 128;             // TMEM columns of the compensation terms
  static_assert(kCcCol + 128 <= 512, "levels and compensation terms exceed TMEM");
  static constexpr int kOffBar = kStages * kStageBytes;
  static constexpr int kSmem = kOffBar + 256 + 1024;
  static constexpr int kThreads = 384;
  static constexpr int kLaunchRegs = 168;               // per thread at launch (checked on the host)
  static constexpr uint32_t kRegsLow = 64, kRegsHigh = 200;
  static_assert(128 * kRegsLow + 256 * kRegsHigh <= kThreads * kLaunchRegs, "register budgets exceed the pool");
  // per SM sub-partition: one warp of warpgroup 0 and two epilogue warps
  static_assert(32 * kRegsLow + 2 * 32 * kRegsHigh <= 16384, "register file of an SM sub-partition");
  static_assert(8 * NS <= 32, "one producer lane per copy of a stage");
};

__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (x - bp);
  s = t;
  c += e;
}

template <int NS>
__global__ void __launch_bounds__(384, 1)
    k_v_tc(ListView L, const VWorkTC* __restrict__ work, int64_t nwork, const int32_t* __restrict__ glist,
           int64_t t0, const uint8_t* __restrict__ phic, const uint8_t* __restrict__ xs,
           const float* __restrict__ scale, const float* __restrict__ bmaxf, const float* __restrict__ xmaxf,
           const uint8_t* __restrict__ zero, int nbf, float t_bf, float t_df, double* V, int* next, int* err,
           uint64_t wait_ns, int withhold) {
  using C = VCfg<NS>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::kOffBar);
  uint64_t* empty = full + C::kStages;
  uint64_t* tfull = empty + C::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* ifull = tempty + 2;       // work-item ring: index published by the producer
  uint64_t* iempty = ifull + 4;       // ... and read by the MMA thread and the 8 epilogue warps
  uint64_t* mdone = iempty + 4;       // all products of the MMA thread completed (exit)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* ring = reinterpret_cast<volatile int*>(tmem_slot + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
    }
    for (int r = 0; r < 4; ++r) {
      mbar_init(&ifull[r], 1);
      mbar_init(&iempty[r], 9);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;

  if (warp < 4) {
    regs_dec<C::kRegsLow>();
    if (warp == 0) {
      // lane -> copy (side, tile j): lanes 0..7, one bulk copy of NS x 2 KB each per stage
      const int side = (lane >> 2) & 1, j = lane & 3;
      const bool copier = lane < 8;
      uint32_t it = 0;
      bool ok = true;
      for (uint32_t k = 0; ok; ++k) {
        // next work item from the global counter: CTAs take neighbouring items
        // and so share the tiles of the same grid-block range in L2
        const int slot = k & 3;
        if (!mbar_wait_warp(&iempty[slot], ((k >> 2) & 1) ^ 1, abort_flag, err, 125, wait_ns)) { ok = false; break; }
        int wi = 0;
        if (lane == 0) {
          const int x = atomicAdd(next, 1);
          wi = x < nwork ? x : -1;
          if (x == withhold) {
            wi = -2;   // test hook: item not handed out, the consumers' bounded wait runs out
          } else {
            ring[slot] = wi;
            mbar_arrive(&ifull[slot]);
          }
        }
        wi = __shfl_sync(0xffffffffu, wi, 0);
        if (wi < 0) break;
        const VWorkTC wk = work[wi];
        for (int e = 0; e < wk.end - wk.beg && ok; ++e) {
          const int64_t gb = glist[wk.beg + e];
          const int p = (side == 0 ? wk.P : wk.Q) + j;
          const uint8_t* sp = zero;   // Phi~ tile (gb, p), or zeros
          const uint8_t* sx = zero;   // X~ tile, or zeros (tile absent); pair screening in the epilogue
          if (p < L.nbb) {
            const int t = L.tile_of[gb * L.nbb + p];
            if (t >= 0) {
              const int64_t off = (int64_t)(t - t0) * tile_bytes(NS);
              sp = phic + off;
              sx = xs + off;
            }
          }
          // a diagonal pair (P == Q) runs only the first half of the chain,
          // S = Phi~_P^T X~_P (K = 128); the finish step adds S^T
          const int nchunk = wk.P == wk.Q ? 4 : 8;
          for (int c = 0; c < nchunk; ++c) {
            const int h = c >> 2, kc = c & 3;
            const int s = it % C::kStages;
            const uint32_t ph = (it / C::kStages) & 1;
            if (!mbar_wait_warp(&empty[s], ph ^ 1, abort_flag, err, 121, wait_ns)) { ok = false; break; }
            if (lane == 0) mbar_arrive_expect_tx(&full[s], C::kStageBytes);
            __syncwarp();
            if (copier) {
              // A = Phi~ then X~ along K; B = X~ then Phi~
              const bool use_x = (side == 0) == (h == 1);
              const uint8_t* src = use_x ? sx : sp;
              if (src != zero) src += kc * (NS * C::kChunk);
              bulk_g2s(sm + s * C::kStageBytes + (side * 4 + j) * (NS * C::kChunk), src, NS * C::kChunk, &full[s]);
            }
            ++it;
          }
        }
      }
      if (lane == 0)
        for (uint32_t k = (it > (uint32_t)C::kStages ? it - C::kStages : 0); k < it; ++k) {
          volatile int no_abort = 0;
          mbar_wait(&full[k % C::kStages], (k / C::kStages) & 1, &no_abort, nullptr, 0);
        }
    } else if (warp == 1) {
      if (lane == 0) {
        const uint32_t idesc = instr_desc(128, 128, 1, 1, 1);
        uint32_t it = 0, job = 0;
        bool ok = true;
        for (uint32_t k = 0; ok; ++k) {
          const int slot = k & 3;
          if (!mbar_wait(&ifull[slot], (k >> 2) & 1, abort_flag, err, 126, wait_ns)) { ok = false; break; }
          const int wi = ring[slot];
          mbar_arrive(&iempty[slot]);
          if (wi < 0) break;
          const VWorkTC wk = work[wi];
          for (int e = 0; e < wk.end - wk.beg && ok; ++e, ++job) {
            if (!mbar_wait(&tempty[0], (job & 1) ^ 1, abort_flag, err, 124, wait_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d0 = tbase;
            uint32_t started[C::kAcc];
#pragma unroll
            for (int l = 0; l < C::kAcc; ++l) started[l] = 0;
            const int nchunk = wk.P == wk.Q ? 4 : 8;
            for (int c = 0; c < nchunk; ++c) {
              const int s = it % C::kStages;
              const uint32_t ph = (it / C::kStages) & 1;
              if (!mbar_wait(&full[s], ph, abort_flag, err, 122, wait_ns)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a = smem_u32(sm + s * C::kStageBytes);
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                uint64_t ad[NS], bd[NS];
#pragma unroll
                for (int l = 0; l < NS; ++l) {
                  ad[l] = smem_desc(a + l * C::kChunk + k * 1024, NS * C::kChunk, 512, kSwz64);
                  bd[l] = smem_desc(a + 4 * NS * C::kChunk + l * C::kChunk + k * 1024, NS * C::kChunk, 512, kSwz64);
                }
                issue_levels<NS, C::kAcc>(d0, 128, ad, bd, idesc, started);
              }
              mma_commit(&empty[s]);
              ++it;
            }
            if (!ok) break;
            mma_commit(&tfull[0]);
          }
        }
        if (!ok) *abort_flag = 1;
        // every product this thread issued completes before the CTA frees its
        // tensor memory, also when a wait gave up in the middle of a stream
        mma_commit(mdone);
        volatile int no_abort = 0;
        mbar_wait(mdone, 0, &no_abort, nullptr, 0);
      }
    }
  } else {
    regs_inc<C::kRegsHigh>();
    const int quarter = warp & 3;
    const int half = (warp >> 2) - 1;
    const int m = quarter * 32 + lane;       // row inside the tile (function of P)
    const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16) + half * 64;
    uint32_t job = 0;
    bool ok = true;
    for (uint32_t k = 0; ok; ++k) {
      const int slot = k & 3;
      if (!mbar_wait_warp(&ifull[slot], (k >> 2) & 1, abort_flag, err, 127, wait_ns)) { ok = false; break; }
      const int wi = ring[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&iempty[slot]);
      if (wi < 0) break;
      const VWorkTC wk = work[wi];
      float S[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) S[c] = 0.f;
      {
        float z[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) z[c] = 0.f;
#pragma unroll
        for (int cq = 0; cq < 4; ++cq) tmem_st16(trow + C::kCcCol + cq * 16, z);
        tmem_st_wait();
      }
      for (int e = 0; e < wk.end - wk.beg; ++e, ++job) {
        const int64_t gb = glist[wk.beg + e];
        const int pr = wk.P + (m >> 5);
        float rsc = 0.f, bp = 0.f, xp = 0.f;
        if (pr < L.nbb) {
          const int t = L.tile_of[gb * L.nbb + pr];
          if (t >= 0) {
            rsc = scale[(int64_t)(t - t0) * kBasisBlk + (m & 31)];
            bp = bmaxf[t];
            xp = xmaxf[t];
          }
        }
        // column scales, zero where the block pair (p, q) of this grid block
        // is not executed: (p, q) or (q, p) in E2_g (x_gq >= t_b and
        // b_gp x_gq >= t_d, or the same with p and q exchanged)
        float csc[2];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int qb = wk.Q + half * 2 + cc;
          csc[cc] = 0.f;
          if (qb < L.nbb) {
            const int t = L.tile_of[gb * L.nbb + qb];
            if (t >= 0) {
              const float bq = bmaxf[t], xq = xmaxf[t];
              const bool on = (xq >= t_bf && bp * xq >= t_df) || (xp >= t_bf && bq * xp >= t_df);
              if (on) csc[cc] = scale[(int64_t)(t - t0) * kBasisBlk + lane];
            }
          }
        }
        if (!mbar_wait_warp(&tfull[0], job & 1, abort_flag, err, 123, wait_ns)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int cq = 0; cq < 4; ++cq) {            // 16 columns at a time
          const int cc = cq >> 1;
          // levels (smallest first) and the compensation terms, one wait
          float t[16 * (C::kAcc + 1)];
          if constexpr (C::kAcc == 3)
            tmem_ld16x4(trow + 2 * 128 + cq * 16, trow + 128 + cq * 16, trow + cq * 16, trow + C::kCcCol + cq * 16, t);
          else
            tmem_ld16x3(trow + 128 + cq * 16, trow + cq * 16, trow + C::kCcCol + cq * 16, t);
          float cmp[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            cmp[c] = t[16 * C::kAcc + c];
            const float sc = rsc * __shfl_sync(0xffffffffu, csc[cc], (cq & 1) * 16 + c);   // a power of two
            if constexpr (NS == 4) {
              // L0 + L1 error-free; the low part and the rounded L23 go to the compensation
              const f2 sg = two_sum(t[32 + c], t[16 + c]);
              two_sum_acc(S[cq * 16 + c], cmp[c], sg.h * sc);
              cmp[c] = __fadd_rn(cmp[c], __fadd_rn(sg.l, t[c]) * sc);
            } else {
              float acc = t[c];
#pragma unroll
              for (int l = 1; l < NS; ++l) acc += t[16 * l + c];
              two_sum_acc(S[cq * 16 + c], cmp[c], acc * sc);
            }
          }
          tmem_st16(trow + C::kCcCol + cq * 16, cmp);
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[0]);
      }
      if (!ok) break;
      const int r = wk.P * kBasisBlk + m;
#pragma unroll
      for (int cq = 0; cq < 4; ++cq) {
        float cmp[16];
        tmem_ld16(trow + C::kCcCol + cq * 16, cmp);
        if (r < nbf) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int col = wk.Q * kBasisBlk + half * 64 + cq * 16 + c;
            if (col < nbf) {
              // the sum and its compensation term, each widened to FP64 by
              // integer operations (no FP64 arithmetic), added by the atomics
              atomicAdd(&V[(int64_t)r * nbf + col], f32_to_f64(S[cq * 16 + c]));
              if (cmp[c] != 0.f) atomicAdd(&V[(int64_t)r * nbf + col], f32_to_f64(cmp[c]));
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

template <int NS>
static kldi_status v_ns(const kldi_plan* P, const Batch& b, double* V, cudaStream_t s) {
  using C = VCfg<NS>;
  if (b.n_vtc_work == 0) return KLDI_OK;
  KLDI_TRY(prepare_tc_kernels());
  const unsigned grid = (unsigned)std::min<int64_t>(b.n_vtc_work, P->num_sms);
  KLDI_TRY_CUDA(cudaMemsetAsync(P->d_vnext, 0, sizeof(int), s));
  k_v_tc<NS><<<grid, C::kThreads, C::kSmem, s>>>(
      P->list_view(), b.d_vtc_work, b.n_vtc_work, b.d_vtc_g, b.t0, reinterpret_cast<const uint8_t*>(P->d_phic_s),
      reinterpret_cast<const uint8_t*>(P->d_x_s), P->d_phic_scale, P->d_bmaxf, P->d_xmaxf,
      reinterpret_cast<const uint8_t*>(P->d_zero), (int)P->nbf, (float)P->opt.t_b, (float)P->opt.t_d, V, P->d_vnext,
      P->d_err, P->wait_ns,
      (int)P->withhold_item);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

template <int NS>
static kldi_status prepare_v_kernel() {
  using C = VCfg<NS>;
  // the register budgets of the warpgroups assume the launch allocation
  cudaFuncAttributes fa;
  KLDI_TRY_CUDA(cudaFuncGetAttributes(&fa, k_v_tc<NS>));
  if (fa.numRegs != C::kLaunchRegs) {
    set_error("k_v_tc: built with %d registers per thread, register budgets assume %d", fa.numRegs, C::kLaunchRegs);
    return KLDI_EUNSUPPORTED;
  }
  KLDI_TRY_CUDA(cudaFuncSetAttribute(k_v_tc<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
  return KLDI_OK;
}

template <int NS, int NQ>
static kldi_status prepare_rho_rowdot() {
  using C = RhoCfg<NS, NQ>;
  KLDI_TRY_CUDA(cudaFuncSetAttribute(k_rho_tc<NS, true, kRowDot, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     C::kSmem));
  KLDI_TRY_CUDA(cudaFuncSetAttribute(k_rho_tc<NS, false, kRowDot, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     C::kSmem));
  return KLDI_OK;
}

template <int NS>
static kldi_status prepare_rho_kernel() {
  using C = RhoCfg<NS>;
  if constexpr (NS < 4) KLDI_TRY((prepare_rho_rowdot<NS, 2>()));
  KLDI_TRY_CUDA(cudaFuncSetAttribute(k_rho_tc<NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
  KLDI_TRY_CUDA(cudaFuncSetAttribute(k_rho_tc<NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
  KLDI_TRY_CUDA(cudaFuncSetAttribute(k_rho_tc<NS, false, kGradQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     C::kSmem));
  KLDI_TRY_CUDA(cudaFuncSetAttribute(k_rho_tc<NS, false, kGradR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     C::kSmem));
  return KLDI_OK;
}

// Kernel attributes set once per process (outside any stream capture).
// Kernel attributes belong to a device: set once per device, under a lock so
// that plans created on several host threads do not race.
kldi_status prepare_tc_kernels() {
  static std::mutex mu;
  static std::map<int, kldi_status> done;
  int dev = 0;
  KLDI_TRY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(dev);
  if (it != done.end()) {
    if (it->second != KLDI_OK) set_error("tensor-core kernels could not be prepared on device %d", dev);
    return it->second;
  }
  kldi_status st = prepare_rho_kernel<2>();
  if (st == KLDI_OK) st = prepare_rho_kernel<3>();
  if (st == KLDI_OK) st = prepare_rho_kernel<4>();
  if (st == KLDI_OK) st = prepare_v_kernel<2>();
  if (st == KLDI_OK) st = prepare_v_kernel<3>();
  if (st == KLDI_OK) st = prepare_v_kernel<4>();
  if (st == KLDI_OK) {
    // the X kernel of BF16X10 stages hi / lo values in dynamic shared memory
    const cudaError_t e1 = cudaFuncSetAttribute(k_x_split4<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kX4Smem);
    const cudaError_t e2 = cudaFuncSetAttribute(k_x_split4<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kX4Smem);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      set_error("k_x_split4: shared-memory opt-in failed");
      st = KLDI_ECUDA;
    }
  }
  if (st == KLDI_OK) {
    // 2^(j/256) as hi / lo pairs for exp_df (from the host's double exp2)
    float2 tab[256];
    for (int j = 0; j < 256; ++j) {
      const double v = std::exp2((double)j / 256.0);
      tab[j].x = (float)v;
      tab[j].y = (float)(v - (double)tab[j].x);
    }
    if (cudaMemcpyToSymbol(g_exp2_tab, tab, sizeof(tab)) != cudaSuccess) {
      set_error("exp table upload failed");
      st = KLDI_ECUDA;
    }
  }
  done[dev] = st;
  return st;
}

// Self-test of the bounded wait: warp 0 waits (limit_ns) on an mbarrier of
// count 1 at which warp 1 arrives only when `arrive` is set.  Nothing else is
// in flight (no copies, no products, no tensor memory), so a wait that runs
// out leaves the CTA in a clean state.  out[0] = 1 when the wait completed,
// out[1] = the recorded code (0 or 901).
__global__ void k_selftest_wait(uint64_t limit_ns, int arrive, int* out) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  __shared__ int err;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    err = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x >> 5 == 1) {
    if (arrive && (threadIdx.x & 31) == 0) mbar_arrive(&bar);
  } else {
    const bool ok = mbar_wait_warp(&bar, 0, &abort_flag, &err, 901, limit_ns);
    if (threadIdx.x == 0) {
      out[0] = ok ? 1 : 0;
      out[1] = err;
    }
  }
}

kldi_status launch_v_tc(const kldi_plan* P, const Batch& b, double* V, cudaStream_t s) {
  switch (slices_of(P->prec)) {
    case 4: return v_ns<4>(P, b, V, s);
    case 3: return v_ns<3>(P, b, V, s);
    default: return v_ns<2>(P, b, V, s);
  }
}

}  // namespace kldi

extern "C" kldi_status kldi_selftest_wait(uint64_t limit_ns, int arrive, void* stream) {
  return kldi::guarded("kldi_selftest_wait", [&]() -> kldi_status {
    using namespace kldi;
    int* d = nullptr;
    KLDI_TRY_CUDA(cudaMalloc(&d, 2 * sizeof(int)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h[2] = {0, 0};
    k_selftest_wait<<<1, 64, 0, s>>>(limit_ns, arrive, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    KLDI_TRY_CUDA(e);
    if (h[0] == 1 && h[1] == 0) return KLDI_OK;
    set_error("kldi_selftest_wait: the bounded wait gave up (code %d)", h[1]);
    return KLDI_ETIMEOUT;
  });
}
