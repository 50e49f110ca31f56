// Kernels shared by every precision mode (block summaries, D block maxima,
// functional, E_xc reduction, V mirror) and the plain FP64 block form of the
// two block products.
//
// FP64 block form (the speedup denominator): the same block-filtered algorithm
// as the tensor-core path, on FP64 CUDA cores.
//   rho:  per grid block g, R_q = sum_{p:(p,q) in E1_g} Phi_p D_pq, then
//         rho_i = sum_q Phi_q . R_q and grad rho_i = 2 sum_q grad Phi_q . R_q
//         (Eq. executed_block_output; App. A density).
//   V:    per basis-block pair p <= q over its list of grid blocks,
//         V_pq += [E2(p,q) or E2(q,p)] (Phi_p^T X_q + X_p^T Phi_q).
#include <cfloat>

#include "basis.cuh"
#include "internal.h"
#include "xc.cuh"
#include "xc_point.cuh"

namespace kldi {

static __device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
static __device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 128-thread block reductions (4 warps).
static __device__ double block_max128(double v, double* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double r = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Block summaries b_gp = max |phi| (and |grad phi|) over grid block g and basis
// block p, FP64 (Eq. block_summary_A applied to Phi).  One CTA of 128 threads
// per candidate (g, p); thread i evaluates point i.
template <bool GRAD>
__global__ void k_block_max(BasisView B, GridView G, const int32_t* cand_g, const int32_t* cand_p,
                            double* out) {
  __shared__ double red[4];
  const int64_t c = blockIdx.x;
  const int64_t g = cand_g[c];
  const int p = cand_p[c];
  const int64_t pt = g * kBlockPts + threadIdx.x;
  const double px = G.xyz[pt * 3 + 0], py = G.xyz[pt * 3 + 1], pz = G.xyz[pt * 3 + 2];
  double m = 0.0;
  for_block_functions<double, GRAD>(B, p, px, py, pz, [&](int, double v, double gx, double gy, double gz) {
    m = fmax(m, fabs(v));
    if (GRAD) m = fmax(m, fmax(fabs(gx), fmax(fabs(gy), fabs(gz))));
  });
  m = block_max128(m, red);
  if (threadIdx.x == 0) out[c] = m;
}

kldi_status launch_block_max(const kldi_plan* P, const int32_t* d_cand_g, const int32_t* d_cand_p,
                             int64_t ncand, double* d_out, cudaStream_t s) {
  if (ncand == 0) return KLDI_OK;
  const int64_t chunk = 1 << 30;
  for (int64_t c0 = 0; c0 < ncand; c0 += chunk) {
    const int64_t n = ncand - c0 < chunk ? ncand - c0 : chunk;
    if (P->gga)
      k_block_max<true><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), d_cand_g + c0,
                                                          d_cand_p + c0, d_out + c0);
    else
      k_block_max<false><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), d_cand_g + c0,
                                                           d_cand_p + c0, d_out + c0);
  }
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// ---------------------------------------------------------------------------
// d_pq = max |D_pq| over 32 x 32 blocks (Eq. block_summary_A with A = D).
__global__ void k_dmax(const double* D, int nbf, int nbb, double* dmax) {
  __shared__ double red[8];
  const int p = blockIdx.y, q = blockIdx.x;
  double m = 0.0;
  for (int e = threadIdx.x; e < kBasisBlk * kBasisBlk; e += blockDim.x) {
    const int r = p * kBasisBlk + e / kBasisBlk, c = q * kBasisBlk + e % kBasisBlk;
    if (r < nbf && c < nbf) m = fmax(m, fabs(D[(int64_t)r * nbf + c]));
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    dmax[p * nbb + q] = r;
  }
}

kldi_status launch_dmax(const kldi_plan* P, const double* D, cudaStream_t s) {
  dim3 grid((unsigned)P->nbb, (unsigned)P->nbb);
  k_dmax<<<grid, 256, 0, s>>>(D, (int)P->nbf, (int)P->nbb, P->d_dmax);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// ---------------------------------------------------------------------------
// FP64 Phi tiles: tile t = (g, p) stored [32 functions][128 points].
__global__ void k_phi64(BasisView B, GridView G, ListView L, int64_t g0, int64_t t0, double* tiles) {
  const int64_t t = t0 + blockIdx.x;
  const int64_t g = L.tile_g[t];
  const int p = L.blk_idx[t];
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  double* out = tiles + (t - t0) * (kBasisBlk * kBlockPts);
  for (int nu = 0; nu < kBasisBlk; ++nu) out[nu * kBlockPts + i] = 0.0;
  for_block_functions<double, false>(B, p, G.xyz[pt * 3], G.xyz[pt * 3 + 1], G.xyz[pt * 3 + 2],
                                     [&](int nu, double v, double, double, double) { out[nu * kBlockPts + i] = v; });
}

kldi_status launch_phi64(const kldi_plan* P, const Batch& b, cudaStream_t s) {
  const int64_t n = b.t1 - b.t0;
  if (n == 0) return KLDI_OK;
  k_phi64<<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                            P->d_phi64);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// ---------------------------------------------------------------------------
// FP64 density: one CTA (128 threads, one point each) per grid block.
template <bool GRAD>
__global__ void __launch_bounds__(128) k_rho64(BasisView B, GridView G, ListView L, int64_t g0, int64_t t0,
                                               const double* __restrict__ phi, const double* __restrict__ D,
                                               const double* __restrict__ dmax, int nbf, double t_b, double t_d,
                                               double* rho, double* grad) {
  __shared__ double Dsm[kBasisBlk][kBasisBlk + 1];
  __shared__ double Rsm[kBasisBlk][kBlockPts];
  const int64_t g = g0 + blockIdx.x;
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  const double px = G.xyz[pt * 3], py = G.xyz[pt * 3 + 1], pz = G.xyz[pt * 3 + 2];
  const int tb = L.blk_ptr[g], te = L.blk_ptr[g + 1];
  double r_i = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  for (int jq = tb; jq < te; ++jq) {
    const int q = L.blk_idx[jq];
    const double bq = L.bmax[jq];
    double acc[kBasisBlk];
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) acc[nu] = 0.0;
    for (int jp = tb; jp < te; ++jp) {
      const int p = L.blk_idx[jp];
      const double dm = dmax[p * L.nbb + q];
      if (!(dm >= t_b && L.bmax[jp] * dm * bq >= t_d)) continue;  // (p, q) not in E1_g
      __syncthreads();
      for (int e = i; e < kBasisBlk * kBasisBlk; e += kBlockPts) {
        const int mu = e / kBasisBlk, nu = e % kBasisBlk;
        const int r = p * kBasisBlk + mu, c = q * kBasisBlk + nu;
        Dsm[mu][nu] = (r < nbf && c < nbf) ? D[(int64_t)r * nbf + c] : 0.0;
      }
      __syncthreads();
      const double* ph = phi + (int64_t)(jp - t0) * (kBasisBlk * kBlockPts);
#pragma unroll 4
      for (int mu = 0; mu < kBasisBlk; ++mu) {
        const double f = ph[mu * kBlockPts + i];
#pragma unroll
        for (int nu = 0; nu < kBasisBlk; ++nu) acc[nu] = fma(f, Dsm[mu][nu], acc[nu]);
      }
    }
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) Rsm[nu][i] = acc[nu];
    for_block_functions<double, GRAD>(B, q, px, py, pz, [&](int nu, double v, double dx, double dy, double dz) {
      const double r = Rsm[nu][i];
      r_i = fma(v, r, r_i);
      if (GRAD) {
        gx = fma(2.0 * dx, r, gx);
        gy = fma(2.0 * dy, r, gy);
        gz = fma(2.0 * dz, r, gz);
      }
    });
  }
  rho[pt] = r_i;
  if (GRAD) {
    grad[pt * 3 + 0] = gx;
    grad[pt * 3 + 1] = gy;
    grad[pt * 3 + 2] = gz;
  }
}

kldi_status launch_rho64(const kldi_plan* P, const Batch& b, const double* D, double* rho, double* grad,
                         cudaStream_t s) {
  const int64_t n = b.g1 - b.g0;
  if (n == 0) return KLDI_OK;
  if (P->gga)
    k_rho64<true><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                    P->d_phi64, D, P->d_dmax, (int)P->nbf, P->opt.t_b,
                                                    P->opt.t_d, rho, grad);
  else
    k_rho64<false><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                     P->d_phi64, D, P->d_dmax, (int)P->nbf, P->opt.t_b,
                                                     P->opt.t_d, rho, grad);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// ---------------------------------------------------------------------------
// Functional (FP64) per point, E_xc partial per grid block, and the X
// coefficients c = (w v_rho / 2, 2 w v_sigma grad rho).
__global__ void k_xc(GridView G, int64_t g0, int xc, double rho_min, const double* rho, const double* grad,
                     double* xcoef, float4* xdf, double* eblk, float* pscale) {
  __shared__ double red[4];
  const int64_t g = g0 + blockIdx.x;
  const int64_t pt = g * kBlockPts + threadIdx.x;
  const double r = rho[pt];
  const double w = G.w[pt];
  double e = 0.0, a = 0.0, bx = 0.0, by = 0.0, bz = 0.0;
  if (r >= rho_min) {
    if (xc == KLDI_XC_LDA_X) {
      const XcOut o = xc_lda_x(r);
      e = w * o.f;
      a = 0.5 * w * o.vr;
    } else {
      const double g0x = grad[pt * 3], g0y = grad[pt * 3 + 1], g0z = grad[pt * 3 + 2];
      const double sigma = g0x * g0x + g0y * g0y + g0z * g0z;
      const XcOut o = xc_pbe(r, sigma);
      e = w * o.f;
      a = 0.5 * w * o.vr;
      const double c = 2.0 * w * o.vs;
      bx = c * g0x;
      by = c * g0y;
      bz = c * g0z;
    }
  }
  xc_point_tail(g, pt, e, a, bx, by, bz, xcoef, xdf, eblk, pscale, red);
}

kldi_status launch_xc(const kldi_plan* P, const Batch& b, int xc, const double* rho, const double* grad,
                      cudaStream_t s) {
  if (xc == KLDI_XC_MLP) return launch_xc_mlp(P, b, rho, grad, s);
  const int64_t n = b.g1 - b.g0;
  if (n == 0) return KLDI_OK;
  k_xc<<<(unsigned)n, kBlockPts, 0, s>>>(P->grid_view(), b.g0, xc, P->opt.rho_min, rho, grad, P->d_xcoef,
                                         P->prec == KLDI_BF16X10 ? P->d_xdf : nullptr, P->d_eblk,
                                         P->prec == KLDI_FP64 ? nullptr : P->d_pscale);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// ---------------------------------------------------------------------------
// FP64 X tiles X_{i nu} = a_i phi_nu + b_i . grad phi_nu and x_gp = max |X|.
template <bool GRAD>
__global__ void k_x64(BasisView B, GridView G, ListView L, int64_t g0, int64_t t0, const double* xcoef,
                      double* xt, double* xmax) {
  __shared__ double red[4];
  const int64_t t = t0 + blockIdx.x;
  const int64_t g = L.tile_g[t];
  const int p = L.blk_idx[t];
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  const double a = xcoef[pt * 4], bx = xcoef[pt * 4 + 1], by = xcoef[pt * 4 + 2], bz = xcoef[pt * 4 + 3];
  double* out = xt + (t - t0) * (kBasisBlk * kBlockPts);
  for (int nu = 0; nu < kBasisBlk; ++nu) out[nu * kBlockPts + i] = 0.0;
  double m = 0.0;
  for_block_functions<double, GRAD>(B, p, G.xyz[pt * 3], G.xyz[pt * 3 + 1], G.xyz[pt * 3 + 2],
                                    [&](int nu, double v, double dx, double dy, double dz) {
                                      double x = a * v;
                                      if (GRAD) x += bx * dx + by * dy + bz * dz;
                                      out[nu * kBlockPts + i] = x;
                                      m = fmax(m, fabs(x));
                                    });
  m = block_max128(m, red);
  if (i == 0) xmax[t] = m;
}

kldi_status launch_x64(const kldi_plan* P, const Batch& b, cudaStream_t s) {
  const int64_t n = b.t1 - b.t0;
  if (n == 0) return KLDI_OK;
  if (P->gga)
    k_x64<true><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                  P->d_xcoef, P->d_x64, P->d_xmax);
  else
    k_x64<false><<<(unsigned)n, kBlockPts, 0, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                   P->d_xcoef, P->d_x64, P->d_xmax);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// ---------------------------------------------------------------------------
// FP64 V: one CTA (256 threads) per work item (p <= q, segment of its grid
// block list); tiles staged transposed in shared memory ([point][function]).
__global__ void __launch_bounds__(256) k_v64(ListView L, const VWork64* work, const int32_t* glist,
                                             const double* __restrict__ phi, const double* __restrict__ xt,
                                             const double* __restrict__ xmax, int64_t t0, int nbf, double t_b,
                                             double t_d, double* V) {
  extern __shared__ double sm[];
  double* Pp = sm;                                   // [128][33]
  double* Xq = Pp + kBlockPts * (kBasisBlk + 1);
  double* Xp = Xq + kBlockPts * (kBasisBlk + 1);
  double* Pq = Xp + kBlockPts * (kBasisBlk + 1);
  const VWork64 wk = work[blockIdx.x];
  const int tid = threadIdx.x;
  const int mu = tid >> 3;          // 0..31
  const int nu0 = (tid & 7) * 4;    // 0,4,..,28
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = wk.beg; e < wk.end; ++e) {
    const int64_t g = glist[e];
    const int tp = L.tile_of[g * L.nbb + wk.p];
    const int tq = L.tile_of[g * L.nbb + wk.q];
    const double xp = xmax[tp], xq = xmax[tq];
    const double bp = L.bmax[tp], bq = L.bmax[tq];
    // block (p, q) of Phi^T X + X^T Phi is computed, both terms, when (p, q)
    // or (q, p) is in E2_g (the pair rule applied to the unordered pair)
    const bool m1 = (xq >= t_b && bp * xq >= t_d) || (xp >= t_b && bq * xp >= t_d);
    const bool m2 = m1;
    if (!m1) continue;
    __syncthreads();
    const double* sp = phi + (int64_t)(tp - t0) * (kBasisBlk * kBlockPts);
    const double* sq = phi + (int64_t)(tq - t0) * (kBasisBlk * kBlockPts);
    const double* xpp = xt + (int64_t)(tp - t0) * (kBasisBlk * kBlockPts);
    const double* xqq = xt + (int64_t)(tq - t0) * (kBasisBlk * kBlockPts);
    for (int k = tid; k < kBasisBlk * kBlockPts; k += 256) {
      const int f = k / kBlockPts, i = k % kBlockPts;
      Pp[i * (kBasisBlk + 1) + f] = m1 ? sp[k] : 0.0;
      Xq[i * (kBasisBlk + 1) + f] = m1 ? xqq[k] : 0.0;
      Xp[i * (kBasisBlk + 1) + f] = m2 ? xpp[k] : 0.0;
      Pq[i * (kBasisBlk + 1) + f] = m2 ? sq[k] : 0.0;
    }
    __syncthreads();
    for (int i = 0; i < kBlockPts; ++i) {
      const double a1 = Pp[i * (kBasisBlk + 1) + mu];
      const double a2 = Xp[i * (kBasisBlk + 1) + mu];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        acc[k] = fma(a1, Xq[i * (kBasisBlk + 1) + nu0 + k], acc[k]);
        acc[k] = fma(a2, Pq[i * (kBasisBlk + 1) + nu0 + k], acc[k]);
      }
    }
  }
  const int r = wk.p * kBasisBlk + mu;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = wk.q * kBasisBlk + nu0 + k;
    if (r < nbf && c < nbf) atomicAdd(&V[(int64_t)r * nbf + c], acc[k]);
  }
}

kldi_status launch_v64(const kldi_plan* P, const Batch& b, double* V, cudaStream_t s) {
  if (b.n_v64_work == 0) return KLDI_OK;
  const size_t smem = 4 * kBlockPts * (kBasisBlk + 1) * sizeof(double);
  KLDI_TRY(once_per_device([&]() -> kldi_status {
    KLDI_TRY_CUDA(cudaFuncSetAttribute(k_v64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KLDI_OK;
  }));
  k_v64<<<(unsigned)b.n_v64_work, 256, smem, s>>>(P->list_view(), b.d_v64_work, b.d_v64_g, P->d_phi64, P->d_x64,
                                                   P->d_xmax, b.t0, (int)P->nbf, P->opt.t_b, P->opt.t_d, V);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

// ---------------------------------------------------------------------------
// E_xc = sum of the per-block partials (one CTA, fixed order), and the mirror
// V[nu][mu] = V[mu][nu] for mu < nu: only blocks p <= q are accumulated, and
// the copy also makes the diagonal blocks exactly symmetric.
__global__ void k_esum(const double* eblk, int64_t n, double* exc) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += eblk[k];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) exc[0] = v;
  }
}

__global__ void k_mirror(double* V, int nbf) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nbf * nbf) return;
  const int r = (int)(idx / nbf), c = (int)(idx % nbf);
  if (r > c) V[idx] = V[(int64_t)c * nbf + r];
}

// Tensor-core V: the products accumulated in A (off-diagonal window pairs
// above the block diagonal, diagonal windows S = Phi^T X with both triangles)
// give V = A + A^T.  One thread per pair r <= c.
__global__ void k_finish_tc(double* V, int nbf) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nbf * nbf) return;
  const int r = (int)(idx / nbf), c = (int)(idx % nbf);
  if (r > c) return;
  if (r == c) {
    V[idx] = 2.0 * V[idx];
  } else {
    const double v = V[idx] + V[(int64_t)c * nbf + r];
    V[idx] = v;
    V[(int64_t)c * nbf + r] = v;
  }
}

kldi_status launch_finish(const kldi_plan* P, double* V, double* exc, cudaStream_t s) {
  k_esum<<<1, 1024, 0, s>>>(P->d_eblk, P->nblocks, exc);
  KLDI_TRY_CUDA(cudaGetLastError());
  if (V) {
    const int64_t n = P->nbf * P->nbf;
    if (P->prec == KLDI_FP64)
      k_mirror<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, (int)P->nbf);
    else
      k_finish_tc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, (int)P->nbf);
    KLDI_TRY_CUDA(cudaGetLastError());
  }
  return KLDI_OK;
}

// Reordered plans: D into the internal function order, V back to the caller's.
__global__ void k_permute(const double* __restrict__ src, double* __restrict__ dst, const int32_t* __restrict__ fp,
                          int n, int gather) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  const int64_t o = (int64_t)fp[i] * n + fp[j];
  if (gather)
    dst[idx] = src[o];
  else
    dst[o] = src[idx];
}

kldi_status launch_permute(const kldi_plan* P, const double* src, double* dst, bool gather, cudaStream_t s) {
  const int64_t n2 = P->nbf * P->nbf;
  k_permute<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(src, dst, P->d_fnperm, (int)P->nbf, gather ? 1 : 0);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

}  // namespace kldi
