// Nuclear gradient of E_xc on a fixed grid (the paper's second workload,
// Sec. IV "energies and gradients"), FP64 block form:
//
//   dE/dR_A,x = -2 sum_{mu on A} sum_i [ d_x chi_mu Q_mu,i + (b_i . grad d_x chi_mu) R_mu,i ]
//   R = Phi D, Q = Z D over the executed pairs E1_g, Z = 2 a phi + b . grad phi
//   (a = w v_rho / 2, b = 2 w v_sigma grad rho: the X coefficients of the functional stage)
//
// One CTA of 128 threads (one point each) per grid block; per retained basis
// block q the CTA forms R and Q of q's functions from the FP64 Phi and X tiles
// of the batch (Z = X + a phi), evaluates grad chi and the Hessian of q's
// functions at its point, and accumulates the contributions per function in
// shared memory before one FP64 atomic per function and component into G.
#include <cuda_runtime.h>

#include "internal.h"

namespace kldi {
namespace {

// d^k x^e / dx^k at x (k <= e), e, k <= 2
__device__ __forceinline__ double dpow(double x, int e, int k) {
  if (k > e) return 0.0;
  double c = 1.0;
  for (int t = 0; t < k; ++t) c *= (double)(e - t);
  double v = 1.0;
  for (int t = 0; t < e - k; ++t) v *= x;
  return c * v;
}

// Calls f(local index, atom, value, grad[3], hess[3][3]) for the functions of
// basis block p at (px, py, pz), FP64.  chi = fc P g with g = sum c e^{-a r^2},
// G1 = sum c a e^{-a r^2}, G2 = sum c a^2 e^{-a r^2}:
//   d_a chi = fc [(d_a P) g - 2 r_a P G1]
//   d_a d_b chi = fc [(d_a d_b P) g - 2 (d_a P r_b + d_b P r_a) G1 + P (4 r_a r_b G2 - 2 delta_ab G1)]
// (fc = 1/sqrt 3 for the xx, yy, zz components).
template <typename F>
__device__ void for_block_functions_hess(const BasisView& B, int p, double px, double py, double pz, F&& f) {
  const int lo = p * kBasisBlk, hi = lo + kBasisBlk;
  for (int s = B.bb_shell_begin[p]; s < B.bb_shell_end[p]; ++s) {
    const DevShell sh = B.shells[s];
    const double d[3] = {px - sh.cx, py - sh.cy, pz - sh.cz};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double g = 0.0, g1 = 0.0, g2 = 0.0;
    for (int k = 0; k < sh.nprim; ++k) {
      const double a = B.alpha[sh.prim_off + k];
      const double e = B.coef[sh.prim_off + k] * exp(-a * r2);
      g += e;
      g1 += a * e;
      g2 += a * a * e;
    }
    const int ncomp = (sh.l + 1) * (sh.l + 2) / 2;
    for (int c = 0; c < ncomp; ++c) {
      const int mu = sh.fn_off + c;
      if (mu < lo || mu >= hi) continue;
      int ex[3];
      double fc = 1.0;
      if (sh.l == 0) {
        ex[0] = ex[1] = ex[2] = 0;
      } else if (sh.l == 1) {
        ex[0] = c == 0; ex[1] = c == 1; ex[2] = c == 2;
      } else {
        // xx, xy, xz, yy, yz, zz
        const int tab[6][3] = {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
        ex[0] = tab[c][0]; ex[1] = tab[c][1]; ex[2] = tab[c][2];
        if (c == 0 || c == 3 || c == 5) fc = 0.57735026918962576451;
      }
      double P0[3], P1[3], P2[3];   // per axis: x^e, d/dx, d2/dx2
      for (int a = 0; a < 3; ++a) {
        P0[a] = dpow(d[a], ex[a], 0);
        P1[a] = dpow(d[a], ex[a], 1);
        P2[a] = dpow(d[a], ex[a], 2);
      }
      const double P = P0[0] * P0[1] * P0[2];
      double dP[3], grad[3], hess[3][3];
      dP[0] = P1[0] * P0[1] * P0[2];
      dP[1] = P0[0] * P1[1] * P0[2];
      dP[2] = P0[0] * P0[1] * P1[2];
      for (int a = 0; a < 3; ++a) grad[a] = fc * (dP[a] * g - 2.0 * d[a] * P * g1);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double ddP;
          if (a == b) {
            ddP = (a == 0 ? P2[0] * P0[1] * P0[2] : a == 1 ? P0[0] * P2[1] * P0[2] : P0[0] * P0[1] * P2[2]);
          } else {
            const int o = 3 - a - b;
            double t[3];
            t[a] = P1[a];
            t[b] = P1[b];
            t[o] = P0[o];
            ddP = t[0] * t[1] * t[2];
          }
          hess[a][b] = fc * (ddP * g - 2.0 * (dP[a] * d[b] + dP[b] * d[a]) * g1 +
                             P * (4.0 * d[a] * d[b] * g2 - (a == b ? 2.0 * g1 : 0.0)));
        }
      f(mu - lo, sh.atom, fc * P * g, grad, hess);
    }
  }
}

template <bool GGA>
__global__ void __launch_bounds__(128) k_grad64(BasisView B, GridView Gv, ListView L, int64_t g0, int64_t t0,
                                                const double* __restrict__ phi, const double* __restrict__ xt,
                                                const double* __restrict__ xcoef, const double* __restrict__ D,
                                                const double* __restrict__ dmax, int nbf, double t_b, double t_d,
                                                double* G) {
  __shared__ double Dsm[kBasisBlk][kBasisBlk + 1];
  __shared__ double gsm[kBasisBlk][3];
  __shared__ int atm[kBasisBlk];
  // R and Q of the current basis block, [32][128] each (dynamic shared memory):
  // the basis callback indexes them with the function index
  extern __shared__ double dyn[];
  double (*Rs)[kBlockPts] = reinterpret_cast<double (*)[kBlockPts]>(dyn);
  double (*Qs)[kBlockPts] = reinterpret_cast<double (*)[kBlockPts]>(dyn + kBasisBlk * kBlockPts);
  const int64_t g = g0 + blockIdx.x;
  const int i = threadIdx.x;
  const int64_t pt = g * kBlockPts + i;
  const double px = Gv.xyz[pt * 3], py = Gv.xyz[pt * 3 + 1], pz = Gv.xyz[pt * 3 + 2];
  const double a_i = xcoef[pt * 4];
  const double b_i[3] = {xcoef[pt * 4 + 1], xcoef[pt * 4 + 2], xcoef[pt * 4 + 3]};
  const int tb = L.blk_ptr[g], te = L.blk_ptr[g + 1];
  for (int jq = tb; jq < te; ++jq) {
    const int q = L.blk_idx[jq];
    const double bq = L.bmax[jq];
    double accR[kBasisBlk], accQ[kBasisBlk];
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) accR[nu] = accQ[nu] = 0.0;
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
      const double* xx = xt + (int64_t)(jp - t0) * (kBasisBlk * kBlockPts);
#pragma unroll 2
      for (int mu = 0; mu < kBasisBlk; ++mu) {
        const double f = ph[mu * kBlockPts + i];
        const double z = fma(a_i, f, xx[mu * kBlockPts + i]);      // Z = X + a phi = 2 a phi + b . grad phi
#pragma unroll
        for (int nu = 0; nu < kBasisBlk; ++nu) {
          accR[nu] = fma(f, Dsm[mu][nu], accR[nu]);
          accQ[nu] = fma(z, Dsm[mu][nu], accQ[nu]);
        }
      }
    }
    __syncthreads();
    if (i < kBasisBlk) {
      gsm[i][0] = gsm[i][1] = gsm[i][2] = 0.0;
      atm[i] = -1;
    }
    __syncthreads();
#pragma unroll
    for (int nu = 0; nu < kBasisBlk; ++nu) {
      Rs[nu][i] = accR[nu];
      Qs[nu][i] = accQ[nu];
    }
    for_block_functions_hess(B, q, px, py, pz, [&](int nu, int atom, double, const double* gr, const double (*h)[3]) {
      const double R = Rs[nu][i], Q = Qs[nu][i];
      for (int x = 0; x < 3; ++x) {
        double t = gr[x] * Q;
        if (GGA) t = fma(b_i[0] * h[0][x] + b_i[1] * h[1][x] + b_i[2] * h[2][x], R, t);
        atomicAdd(&gsm[nu][x], t);
      }
      if (i == 0) atm[nu] = atom;
    });
    __syncthreads();
    if (i < 3 * kBasisBlk) {
      const int nu = i / 3, x = i % 3;
      if (atm[nu] >= 0) atomicAdd(&G[atm[nu] * 3 + x], -2.0 * gsm[nu][x]);
    }
  }
}

}  // namespace

kldi_status launch_grad64(const kldi_plan* P, const Batch& b, const double* D, double* G, cudaStream_t s) {
  const int64_t n = b.g1 - b.g0;
  if (n == 0) return KLDI_OK;
  constexpr int kDyn = 2 * kBasisBlk * kBlockPts * (int)sizeof(double);
  KLDI_TRY(once_per_device([&]() -> kldi_status {
    KLDI_TRY_CUDA(cudaFuncSetAttribute(k_grad64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn));
    KLDI_TRY_CUDA(cudaFuncSetAttribute(k_grad64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn));
    return KLDI_OK;
  }));
  if (P->gga)
    k_grad64<true><<<(unsigned)n, kBlockPts, kDyn, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                     P->d_phi64, P->d_x64, P->d_xcoef, D, P->d_dmax, (int)P->nbf,
                                                     P->opt.t_b, P->opt.t_d, G);
  else
    k_grad64<false><<<(unsigned)n, kBlockPts, kDyn, s>>>(P->basis_view(), P->grid_view(), P->list_view(), b.g0, b.t0,
                                                      P->d_phi64, P->d_x64, P->d_xcoef, D, P->d_dmax, (int)P->nbf,
                                                      P->opt.t_b, P->opt.t_d, G);
  KLDI_TRY_CUDA(cudaGetLastError());
  return KLDI_OK;
}

}  // namespace kldi
