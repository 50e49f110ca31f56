// kldi_screen and plan management: basis normalisation, geometric candidate
// search, FP64 block summaries on the GPU (Eq. block_summary_A applied to Phi),
// retained lists S_g (Eq. retained_blocks_A; a block-CSR list per grid block,
// the BCS(R) analogue of App. C), batching of grid blocks, the per-pair grid
// block lists of the V product (the BCS(C) analogue), and all work buffers.
#include <omp.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>

#include "internal.h"

using namespace kldi;

BasisView kldi_plan::basis_view() const {
  BasisView v;
  v.shells = d_shells;
  v.alpha = d_alpha;
  v.coef = d_coef;
  v.alpha_f = d_alpha_f;
  v.alpha_lo = d_alpha_f ? d_alpha_f + nprim_total : nullptr;
  v.coef_f = d_alpha_f ? d_alpha_f + 2 * nprim_total : nullptr;
  v.coef_lo = d_alpha_f ? d_alpha_f + 3 * nprim_total : nullptr;
  v.ac_f = d_coef_f;
  v.ac_lo = d_coef_f ? d_coef_f + nprim_total : nullptr;
  v.shell_f = d_shell_f;
  v.prim_f = d_prim_f;
  v.prim_ac = d_prim_ac;
  v.bb_shell_begin = d_bb_begin;
  v.bb_shell_end = d_bb_end;
  v.bb_split = d_bb_split;
  v.relatom = d_relatom;
  v.natm = natm;
  v.nbf = (int32_t)nbf;
  v.nbb = (int32_t)nbb;
  return v;
}

GridView kldi_plan::grid_view() const {
  GridView v;
  v.xyz = d_xyz;
  v.w = d_w;
  v.prel = d_prel;
  v.prel_lo = d_prel_lo;
  v.anchor = d_anchor;
  v.npoints = npoints;
  v.nblocks = nblocks;
  return v;
}

ListView kldi_plan::list_view() const {
  ListView v;
  v.blk_ptr = d_blk_ptr;
  v.blk_idx = d_blk_idx;
  v.bmax = d_bmax;
  v.tile_of = d_tile_of;
  v.tile_g = d_tile_g;
  v.nbb = (int32_t)nbb;
  return v;
}

namespace {

template <typename T>
kldi_status dalloc(kldi_plan* P, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return KLDI_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    *p = nullptr;
    return KLDI_ENOMEM;
  }
  P->workspace_bytes += (int64_t)(count * sizeof(T));
  return KLDI_OK;
}

template <typename T>
kldi_status upload(kldi_plan* P, T** p, const T* h, size_t count) {
  KLDI_TRY(dalloc(P, p, count));
  if (count) KLDI_TRY_CUDA(cudaMemcpy(*p, h, count * sizeof(T), cudaMemcpyHostToDevice));
  return KLDI_OK;
}

void free_plan_buffers(kldi_plan* P) {
  free_own_tile_buffers(P);
  void* ptrs[] = {P->d_xyz, P->d_w, P->d_prel, P->d_prel_lo, P->d_anchor, P->d_relatom, P->d_shells, P->d_alpha, P->d_coef, P->d_alpha_f, P->d_coef_f, P->d_shell_f, P->d_prim_f, P->d_prim_ac,
                  P->d_bb_begin, P->d_bb_end, P->d_bb_split, P->d_blk_ptr, P->d_blk_idx, P->d_bmax, P->d_tile_of, P->d_tile_g,
                  P->d_D, P->d_V, P->d_fnperm, P->d_Dint, P->d_Vint, P->d_dmax, P->d_rho, P->d_grad, P->d_xcoef, P->d_xdf, P->d_xmax, P->d_xmaxf, P->d_bmaxf, P->d_eblk,
                  P->d_exc, P->d_err, P->d_vnext, P->d_G, P->d_rowscale, P->d_pscale, P->d_zscale, P->d_dscale, P->d_dsplit, P->d_zero, P->d_rad_ptr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (P->d_rad && !P->ws) cudaFree(P->d_rad);   // else a view into the workspace
  P->d_rad = nullptr;
  for (auto& b : P->batches) {
    if (b.d_v64_g) cudaFree(b.d_v64_g);
    if (b.d_v64_work) cudaFree(b.d_v64_work);
    if (b.d_vtc_g) cudaFree(b.d_vtc_g);
    if (b.d_vtc_work) cudaFree(b.d_vtc_work);
  }
  P->batches.clear();
}

}  // namespace

namespace kldi {

void free_own_tile_buffers(kldi_plan* P) {
  if (!P->ws) {
    void* own[] = {P->d_phi64, P->d_x64, P->d_phi_s, P->d_phic_s, P->d_x_s, P->d_phic_scale, P->d_x_scale};
    for (void* p : own)
      if (p) cudaFree(p);
  }
  P->d_phi64 = P->d_x64 = nullptr;
  P->d_phi_s = P->d_phic_s = P->d_x_s = nullptr;
  P->d_phic_scale = P->d_x_scale = nullptr;
}

// Bytes of the per-tile buffers each precision mode needs.
int64_t tile_bytes_for(int prec) {
  if (prec == KLDI_FP64) return 2LL * kBasisBlk * kBlockPts * 8;        // Phi and X tiles, FP64
  return 3LL * 4 * kBasisBlk * kBlockPts * 2 + 2LL * kBasisBlk * 4;   // Phi (two slicings) and X, up to 4 planes
}

// Largest per-tile footprint of the precision modes (the shared workspace
// holds either layout).
int64_t tile_bytes_max() { return std::max(tile_bytes_for(KLDI_FP64), tile_bytes_for(KLDI_BF16X10)); }

void free_work_lists(kldi_plan* P) {
  for (auto& b : P->batches) {
    if (b.d_v64_g) cudaFree(b.d_v64_g);
    if (b.d_v64_work) cudaFree(b.d_v64_work);
    if (b.d_vtc_g) cudaFree(b.d_vtc_g);
    if (b.d_vtc_work) cudaFree(b.d_vtc_work);
  }
  P->batches.clear();
}

// Batches of grid blocks whose tiles fit `cap` tiles, and per batch the V
// work lists: FP64 per basis-block pair (p <= q), tensor cores per 128-tile
// pair (P <= Q), each cut into segments of grid blocks.
kldi_status build_work(kldi_plan* P, int64_t cap) {
  free_work_lists(P);
  P->vtile_work = 0;
  const int64_t nblk = P->nblocks, nbb = P->nbb;
  int64_t maxblk = 0;
  for (int64_t g = 0; g < nblk; ++g) maxblk = std::max<int64_t>(maxblk, P->blk_ptr[g + 1] - P->blk_ptr[g]);
  cap = std::max(cap, maxblk);
  cap = std::min<int64_t>(cap, std::max<int64_t>(P->ntiles, 1));
  P->tile_cap = cap;
  {
    // grid blocks of this plan's range (all by default)
    const int64_t gend = P->range_g1 >= 0 ? P->range_g1 : nblk;
    int64_t g0 = P->range_g0;
    while (g0 < gend) {
      int64_t g1 = g0;
      while (g1 < gend && P->blk_ptr[g1 + 1] - P->blk_ptr[g0] <= cap &&
             P->rad_ptr[P->blk_ptr[g1 + 1]] - P->rad_ptr[P->blk_ptr[g0]] <= P->rad_rows_cap)
        ++g1;
      if (g1 == g0) ++g1;   // one grid block always fits (checked when the workspace is set)
      Batch b;
      b.g0 = g0;
      b.g1 = g1;
      b.t0 = P->blk_ptr[g0];
      b.t1 = P->blk_ptr[g1];
      P->batches.push_back(b);
      g0 = g1;
    }
  }
  const int kSeg = 64;
  P->work_fp64 = P->prec == KLDI_FP64;
  for (auto& b : P->batches) {
    if (P->work_fp64) {
      std::map<int64_t, std::vector<int32_t>> pl;
      for (int64_t g = b.g0; g < b.g1; ++g)
        for (int32_t i = P->blk_ptr[g]; i < P->blk_ptr[g + 1]; ++i)
          for (int32_t j = i; j < P->blk_ptr[g + 1]; ++j)
            pl[(int64_t)P->blk_idx[i] * nbb + P->blk_idx[j]].push_back((int32_t)g);
      std::vector<int32_t> gl;
      std::vector<VWork64> wk;
      for (auto& kv : pl) {
        const int32_t p = (int32_t)(kv.first / nbb), q = (int32_t)(kv.first % nbb);
        const int32_t base = (int32_t)gl.size();
        gl.insert(gl.end(), kv.second.begin(), kv.second.end());
        for (int32_t s0 = 0; s0 < (int32_t)kv.second.size(); s0 += kSeg)
          wk.push_back(VWork64{p, q, base + s0, base + std::min<int32_t>(s0 + kSeg, (int32_t)kv.second.size())});
      }
      KLDI_TRY(upload(P, &b.d_v64_g, gl.data(), gl.size()));
      KLDI_TRY(upload(P, &b.d_v64_work, wk.data(), wk.size()));
      b.n_v64_work = (int64_t)wk.size();
      continue;
    }
    // Each grid block's retained basis blocks (ascending) are covered by
    // windows of 4 consecutive blocks, greedily: a window starts at the first
    // retained block not yet covered, rounded down to a multiple of the
    // alignment A (4: the fixed 128-function tiles; 1: the fewest windows
    // that cover the list, and so the fewest zero blocks the 128 x 128
    // products run over).  The windows of one grid block are disjoint (a
    // start lies past the previous window's last block for A <= 4); V = A + A^T
    // of the accumulated products A.
    std::map<int64_t, std::vector<int32_t>> tl;
    const int64_t nvt = nbb;   // window keys: first blocks P, Q
    const int32_t align = P->tune.v_align > 0 ? P->tune.v_align : 2;
    for (int64_t g = b.g0; g < b.g1; ++g) {
      std::vector<int32_t> vt;
      int32_t cov = -1;
      for (int32_t i = P->blk_ptr[g]; i < P->blk_ptr[g + 1]; ++i) {
        const int32_t p = P->blk_idx[i];
        if (p > cov) {
          const int32_t w = p - p % align;
          vt.push_back(w);
          cov = w + 3;
        }
      }
      for (size_t i = 0; i < vt.size(); ++i)
        for (size_t j = i; j < vt.size(); ++j) tl[(int64_t)vt[i] * nvt + vt[j]].push_back((int32_t)g);
    }
    std::vector<int32_t> tg;
    std::vector<VWorkTC> tw;
    // Work items are cut at grid-block ranges of `span` blocks and ordered
    // range-major: CTAs running at the same time then work on the same few
    // ranges, whose Phi~ / X~ tiles stay in L2 across the window pairs that
    // reuse them.  span: the tuned value, else 64 grid blocks.
    const int64_t span = P->tune.v_seg > 0 ? P->tune.v_seg : 64;
    struct PairList {
      int32_t Pt, Qt, base, n;
    };
    std::vector<PairList> pls;
    for (auto& kv : tl) {
      const int32_t base = (int32_t)tg.size();
      tg.insert(tg.end(), kv.second.begin(), kv.second.end());
      pls.push_back({(int32_t)(kv.first / nvt), (int32_t)(kv.first % nvt), base, (int32_t)kv.second.size()});
      P->vtile_work += (int64_t)kv.second.size();
    }
    std::vector<int32_t> pos(pls.size(), 0);   // next unassigned entry of each pair list
    for (int64_t r0 = b.g0; r0 < b.g1; r0 += span) {
      const int64_t r1 = std::min<int64_t>(r0 + span, b.g1);
      for (size_t k = 0; k < pls.size(); ++k) {
        const PairList& pl = pls[k];
        int32_t e = pos[k];
        while (e < pl.n && tg[pl.base + e] < r1) ++e;
        if (e > pos[k]) tw.push_back(VWorkTC{pl.Pt, pl.Qt, pl.base + pos[k], pl.base + e});
        pos[k] = e;
      }
    }
    KLDI_TRY(upload(P, &b.d_vtc_g, tg.data(), tg.size()));
    KLDI_TRY(upload(P, &b.d_vtc_work, tw.data(), tw.size()));
    b.n_vtc_work = (int64_t)tw.size();
  }
  return KLDI_OK;
}

kldi_status ensure_tile_buffers(kldi_plan* P, int prec) {
  if (prec == KLDI_TF32X3) {
    set_error("KLDI_TF32X3 is not provided: 11-bit slices cannot keep the tensor-core sums exact");
    return KLDI_EUNSUPPORTED;
  }
  if (P->ws) {
    // per-tile buffers are views into the shared workspace (either layout)
    uint8_t* base = static_cast<uint8_t*>(P->ws->base);
    const int64_t cap = P->tile_cap;
    P->d_phi64 = reinterpret_cast<double*>(base);
    P->d_x64 = P->d_phi64 + cap * kBasisBlk * kBlockPts;
    const size_t plane4 = (size_t)cap * 4 * kBasisBlk * kBlockPts;   // up to four planes per tile
    P->d_phi_s = reinterpret_cast<uint16_t*>(base);
    P->d_phic_s = P->d_phi_s + plane4;
    P->d_x_s = P->d_phic_s + plane4;
    P->d_phic_scale = reinterpret_cast<float*>(P->d_x_s + plane4);
    P->d_x_scale = P->d_phic_scale + cap * kBasisBlk;
  }
  if (prec == KLDI_FP64) {
    if (!P->d_phi64) KLDI_TRY(dalloc(P, &P->d_phi64, (size_t)P->tile_cap * kBasisBlk * kBlockPts));
    if (!P->d_x64) KLDI_TRY(dalloc(P, &P->d_x64, (size_t)P->tile_cap * kBasisBlk * kBlockPts));
    return KLDI_OK;
  }
  if (prec == KLDI_BF16X10 && !P->rec_fit_all) {
    set_error("KLDI_BF16X10: a basis block has more than 40 shells or 80 primitives");
    return KLDI_EUNSUPPORTED;
  }
  if (prec == KLDI_BF16X10 && P->ws) {
    // the radial rows follow the tile buffers in the workspace
    uint8_t* base = static_cast<uint8_t*>(P->ws->base);
    P->d_rad = reinterpret_cast<float4*>(base + P->tile_cap * tile_bytes_max());
    P->rad_cap = P->rad_rows_cap;
  } else if (prec == KLDI_BF16X10) {
    // radial factors of the largest batch (the batches change with the block range and tuning)
    int64_t need = 1;
    for (const Batch& b : P->batches) need = std::max(need, P->rad_ptr[b.t1] - P->rad_ptr[b.t0]);
    if (need > P->rad_cap) {
      if (P->d_rad) cudaFree(P->d_rad);
      P->d_rad = nullptr;
      P->rad_cap = 0;
      KLDI_TRY(dalloc(P, &P->d_rad, (size_t)need * kBlockPts));
      P->rad_cap = need;
    }
  }
  // 16-bit words per tile: four planes, the most any mode uses (so a plan can
  // switch modes without reallocating; the batch capacity assumes this size)
  const size_t per_tile = (size_t)4 * kBasisBlk * kBlockPts;
  if (!P->d_phi_s) KLDI_TRY(dalloc(P, &P->d_phi_s, (size_t)P->tile_cap * per_tile));
  if (!P->d_phic_s) KLDI_TRY(dalloc(P, &P->d_phic_s, (size_t)P->tile_cap * per_tile));
  if (!P->d_x_s) KLDI_TRY(dalloc(P, &P->d_x_s, (size_t)P->tile_cap * per_tile));
  if (!P->d_phic_scale) KLDI_TRY(dalloc(P, &P->d_phic_scale, (size_t)P->tile_cap * kBasisBlk));
  if (!P->d_x_scale) KLDI_TRY(dalloc(P, &P->d_x_scale, (size_t)P->tile_cap * kBasisBlk));
  if (!P->d_rowscale) KLDI_TRY(dalloc(P, &P->d_rowscale, (size_t)P->npoints));
  if (!P->d_pscale) KLDI_TRY(dalloc(P, &P->d_pscale, (size_t)P->npoints));
  if (!P->d_dscale) KLDI_TRY(dalloc(P, &P->d_dscale, (size_t)P->nbf_pad));
  if (!P->d_dsplit) KLDI_TRY(dalloc(P, &P->d_dsplit, (size_t)P->nbb * P->nbb * 4 * kBasisBlk * kBasisBlk));
  if (!P->d_zero) {
    KLDI_TRY(dalloc(P, &P->d_zero, (size_t)kBasisBlk * kBlockPts));
    KLDI_TRY_CUDA(cudaMemset(P->d_zero, 0, (size_t)kBasisBlk * kBlockPts * sizeof(uint16_t)));
  }
  return KLDI_OK;
}

}  // namespace kldi

extern "C" kldi_status kldi_screen(const kldi_grid* grid, const kldi_molecule* mol, const kldi_basis* basis,
                                   const kldi_options* opt, kldi_plan** out) {
  return kldi::guarded("kldi_screen", [&]() -> kldi_status {
    if (!grid || !mol || !basis || !opt || !out) {
      set_error("kldi_screen: null argument");
      return KLDI_EINVAL;
    }
    if (basis->nshell <= 0 || !basis->atom || !basis->l || !basis->nprim || !basis->exps || !basis->coefs) {
      set_error("kldi_screen: empty or incomplete basis");
      return KLDI_EINVAL;
    }
    if (opt->prec < KLDI_FP64 || opt->prec > KLDI_BF16X10 || opt->xc < KLDI_XC_LDA_X || opt->xc > KLDI_XC_MLP) {
      set_error("kldi_screen: bad precision or functional");
      return KLDI_EINVAL;
    }
    if (!(opt->t_b >= 0.0) || !(opt->t_d >= 0.0) || !(opt->rho_min >= 0.0)) {
      set_error("kldi_screen: thresholds must be >= 0");
      return KLDI_EINVAL;
    }
    if (opt->prec == KLDI_TF32X3) {
      set_error("KLDI_TF32X3 is not provided: 11-bit slices cannot keep the tensor-core sums exact");
      return KLDI_EUNSUPPORTED;
    }
    if (mol->natm <= 0 || !mol->xyz) {
      set_error("kldi_screen: molecule without atoms or coordinates");
      return KLDI_EINVAL;
    }
    for (int64_t k = 0; k < 3 * (int64_t)mol->natm; ++k)
      if (!std::isfinite(mol->xyz[k])) {
        set_error("kldi_screen: atom %lld has a non-finite coordinate", (long long)(k / 3));
        return KLDI_EINVAL;
      }
    // the grid's owning atoms index the molecule's coordinates here and the
    // per-atom-pair offsets on the device: a grid made for another molecule
    // must not get that far
    if (grid->nblocks <= 0 || grid->npoints != grid->nblocks * kBlockPts ||
        (int64_t)grid->atom.size() != grid->npoints) {
      set_error("kldi_screen: malformed grid");
      return KLDI_EINVAL;
    }
    for (int64_t k = 0; k < grid->npoints; ++k)
      if (grid->atom[k] < 0 || grid->atom[k] >= mol->natm) {
        set_error("kldi_screen: grid point %lld belongs to atom %d, the molecule has %d atoms", (long long)k,
                  grid->atom[k], mol->natm);
        return KLDI_EINVAL;
      }
    // optional shell order: the plan works on the permuted basis; fnperm maps an
    // internal function index to the caller's
    std::vector<int32_t> p_atom, p_l, p_nprim, fnperm;
    std::vector<double> p_exps, p_coefs;
    kldi_basis permuted;
    {
      // The plan's shell order: the caller's (shell_order) or the given one,
      // refined so that within each 32-function block the shells that lie
      // wholly inside it are grouped by atom (stable).  A block keeps its set
      // of functions, hence every screening decision; the kernels form the
      // point offsets once per run of shells on one atom.  fnperm maps an
      // internal function index to the caller's; without a caller's order and
      // with nothing to regroup (an atom-ordered basis) no permutation is made.
      const int ns0 = basis->nshell;
      std::vector<char> seen(ns0, 0);
      std::vector<int64_t> poff(ns0 + 1, 0), foff(ns0 + 1, 0);
      for (int s = 0; s < ns0; ++s) {
        const int l = basis->l[s];
        if (l < 0 || l > 2 || basis->nprim[s] <= 0 || basis->atom[s] < 0 || basis->atom[s] >= mol->natm) {
          set_error("kldi_screen: shell %d has l=%d nprim=%d atom=%d (supported: l <= 2; %d atoms)", s, l,
                    basis->nprim[s], basis->atom[s], mol->natm);
          return l > 2 ? KLDI_EUNSUPPORTED : KLDI_EINVAL;
        }
        poff[s + 1] = poff[s] + basis->nprim[s];
        foff[s + 1] = foff[s] + (l + 1) * (l + 2) / 2;
      }
      for (int64_t k = 0; k < poff[ns0]; ++k)
        if (!(basis->exps[k] > 0.0) || !std::isfinite(basis->exps[k]) || !std::isfinite(basis->coefs[k])) {
          set_error("kldi_screen: primitive %lld has exponent %g, coefficient %g (exponents must be positive, "
                    "both finite)", (long long)k, basis->exps[k], basis->coefs[k]);
          return KLDI_EINVAL;
        }
      std::vector<int> order(ns0);
      for (int k = 0; k < ns0; ++k) {
        const int s = opt->shell_order ? opt->shell_order[k] : k;
        if (s < 0 || s >= ns0 || seen[s]) {
          set_error("kldi_screen: shell_order is not a permutation of 0 .. %d", ns0 - 1);
          return KLDI_EINVAL;
        }
        seen[s] = 1;
        order[k] = s;
      }
      {
        int64_t f = 0;
        int k = 0;
        while (k < ns0) {
          const int l0 = basis->l[order[k]];
          const int64_t f1 = f + (l0 + 1) * (l0 + 2) / 2;
          if (f / kBasisBlk != (f1 - 1) / kBasisBlk) {   // straddles a block boundary: stays
            f = f1;
            ++k;
            continue;
          }
          const int64_t blk = f / kBasisBlk;
          int e = k;
          int64_t fe = f;
          while (e < ns0) {
            const int le = basis->l[order[e]];
            const int64_t fn1 = fe + (le + 1) * (le + 2) / 2;
            if (fe / kBasisBlk != blk || (fn1 - 1) / kBasisBlk != blk) break;
            fe = fn1;
            ++e;
          }
          std::stable_sort(order.begin() + k, order.begin() + e,
                           [&](int a, int b) { return basis->atom[a] < basis->atom[b]; });
          f = fe;
          k = e;
        }
      }
      bool identity = true;
      for (int k = 0; k < ns0 && identity; ++k) identity = order[k] == k;
      if (opt->shell_order || !identity) {
        for (int k = 0; k < ns0; ++k) {
          const int s = order[k];
          p_atom.push_back(basis->atom[s]);
          p_l.push_back(basis->l[s]);
          p_nprim.push_back(basis->nprim[s]);
          for (int64_t i = poff[s]; i < poff[s + 1]; ++i) {
            p_exps.push_back(basis->exps[i]);
            p_coefs.push_back(basis->coefs[i]);
          }
          for (int64_t f = foff[s]; f < foff[s + 1]; ++f) fnperm.push_back((int32_t)f);
        }
        permuted = kldi_basis{ns0, p_atom.data(), p_l.data(), p_nprim.data(), p_exps.data(), p_coefs.data()};
        basis = &permuted;
      }
    }
    kldi_plan* P = new (std::nothrow) kldi_plan;
    if (!P) { set_error("kldi_screen: out of host memory"); return KLDI_ENOMEM; }
    P->opt = *opt;
    P->opt.shell_order = nullptr;   // read here only
    P->gga = opt->xc != KLDI_XC_LDA_X;
    P->prec = opt->prec;
    P->stream = (cudaStream_t)opt->stream;
    cudaGetDevice(&P->device);
    cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    auto fail = [&](kldi_status s) {
      free_plan_buffers(P);
      delete P;
      return s;
    };

    // ---- basis: normalised coefficients, function offsets, block -> shell ranges
    const int ns = basis->nshell;
    std::vector<DevShell> shells(ns);
    std::vector<double> alpha, coef;
    int fn = 0, off = 0;
    for (int s = 0; s < ns; ++s) {
      const int l = basis->l[s], np = basis->nprim[s], a = basis->atom[s];
      if (l < 0 || l > 2 || np <= 0 || a < 0 || a >= mol->natm) {
        set_error("kldi_screen: shell %d has l=%d nprim=%d atom=%d (supported: l <= 2)", s, l, np, a);
        return fail(l > 2 ? KLDI_EUNSUPPORTED : KLDI_EINVAL);
      }
      const double* ex = basis->exps + off;
      const double* cc = basis->coefs + off;
      double so = 0.0;
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j)
          so += cc[i] * cc[j] * std::pow(2.0 * std::sqrt(ex[i] * ex[j]) / (ex[i] + ex[j]), l + 1.5);
      if (!(so > 0.0)) {
        set_error("kldi_screen: shell %d has zero norm", s);
        return fail(KLDI_EINVAL);
      }
      const double rescale = 1.0 / std::sqrt(so);
      for (int i = 0; i < np; ++i) {
        if (!(ex[i] > 0.0)) { set_error("kldi_screen: non-positive exponent"); return fail(KLDI_EINVAL); }
        alpha.push_back(ex[i]);
        coef.push_back(cc[i] * std::pow(2.0 * ex[i] / M_PI, 0.75) * std::pow(4.0 * ex[i], 0.5 * l) * rescale);
      }
      shells[s] = DevShell{mol->xyz[3 * a], mol->xyz[3 * a + 1], mol->xyz[3 * a + 2], l, np, off, fn, a, 0};
      fn += (l + 1) * (l + 2) / 2;
      off += np;
    }
    P->nbf = fn;
    P->nshell = ns;
    P->nbb = (fn + kBasisBlk - 1) / kBasisBlk;
    P->nbf_pad = P->nbb * kBasisBlk;
    P->npoints = grid->npoints;
    P->nblocks = grid->nblocks;
    const int64_t nbb = P->nbb, nblk = P->nblocks;
    std::vector<int32_t> bb_begin(nbb, ns), bb_end(nbb, 0);
    for (int s = 0; s < ns; ++s) {
      const int f0 = shells[s].fn_off, f1 = f0 + (shells[s].l + 1) * (shells[s].l + 2) / 2;
      for (int p = f0 / kBasisBlk; p <= (f1 - 1) / kBasisBlk; ++p) {
        bb_begin[p] = std::min(bb_begin[p], s);
        bb_end[p] = std::max(bb_end[p], s + 1);
      }
    }
    for (int64_t p = 0; p < nbb; ++p) {
      int npr_blk = 0;
      for (int s = bb_begin[p]; s < bb_end[p]; ++s) {
        npr_blk += shells[s].nprim;
        if (shells[s].nprim > 255) npr_blk += 1 << 20;
      }
      if (bb_end[p] - bb_begin[p] > 40 || npr_blk > 80) P->rec_fit_all = false;
    }
    // FP32 hi/lo pairs: hi = fp32(v), lo = fp32(v - hi)
    const size_t npr = alpha.size();
    P->nprim_total = (int64_t)npr;
    std::vector<float> alpha_f(4 * npr), coef_f(2 * npr);
    for (size_t k = 0; k < npr; ++k) {
      const double ac = alpha[k] * coef[k];
      alpha_f[k] = (float)alpha[k];
      alpha_f[npr + k] = (float)(alpha[k] - (double)alpha_f[k]);
      alpha_f[2 * npr + k] = (float)coef[k];
      alpha_f[3 * npr + k] = (float)(coef[k] - (double)alpha_f[2 * npr + k]);
      coef_f[k] = (float)ac;
      coef_f[npr + k] = (float)(ac - (double)coef_f[k]);
    }
    kldi_status st;
    if ((st = upload(P, &P->d_xyz, grid->xyz.data(), grid->xyz.size())) != KLDI_OK) return fail(st);
    {
      // anchors and relative FP32 coordinates for the FP32 basis kernels
      const int natm = mol->natm;
      P->natm = natm;
      std::vector<int32_t> anchor(grid->nblocks);
      std::vector<float4> prel(grid->npoints), prel_lo(grid->npoints);
      for (int64_t g = 0; g < grid->nblocks; ++g) {
        const int a = grid->atom[g * kBlockPts];
        anchor[g] = a;
        for (int i = 0; i < kBlockPts; ++i) {
          const int64_t k = g * kBlockPts + i;
          double d[3];
          float h[3];
          for (int c = 0; c < 3; ++c) {
            d[c] = grid->xyz[k * 3 + c] - mol->xyz[3 * a + c];
            h[c] = (float)d[c];
          }
          prel[k] = make_float4(h[0], h[1], h[2], 0.f);
          // low parts for the double-float (BF16X10) basis values
          prel_lo[k] = make_float4((float)(d[0] - (double)h[0]), (float)(d[1] - (double)h[1]),
                                   (float)(d[2] - (double)h[2]), 0.f);
        }
      }
      std::vector<float> rel((size_t)natm * natm * 8, 0.f);
      for (int a = 0; a < natm; ++a)
        for (int b = 0; b < natm; ++b) {
          float* r = &rel[((size_t)a * natm + b) * 8];
          for (int c = 0; c < 3; ++c) {
            const double d = mol->xyz[3 * b + c] - mol->xyz[3 * a + c];
            r[c] = (float)d;
            r[3 + c] = (float)(d - (double)r[c]);
          }
        }
      if ((st = upload(P, &P->d_anchor, anchor.data(), anchor.size())) != KLDI_OK) return fail(st);
      if ((st = upload(P, &P->d_prel, prel.data(), prel.size())) != KLDI_OK) return fail(st);
      if ((st = upload(P, &P->d_prel_lo, prel_lo.data(), prel_lo.size())) != KLDI_OK) return fail(st);
      if ((st = upload(P, &P->d_relatom, rel.data(), rel.size())) != KLDI_OK) return fail(st);
    }
    if ((st = upload(P, &P->d_w, grid->w.data(), grid->w.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_shells, shells.data(), shells.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_alpha, alpha.data(), alpha.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_coef, coef.data(), coef.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_alpha_f, alpha_f.data(), alpha_f.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_coef_f, coef_f.data(), coef_f.size())) != KLDI_OK) return fail(st);
    {
      // packed copies for the FP32 kernels (one vector load per shell / primitive)
      std::vector<int4> shf(ns);
      for (int s2 = 0; s2 < ns; ++s2)
        shf[s2] = make_int4(shells[s2].l | (shells[s2].nprim << 8), shells[s2].prim_off, shells[s2].fn_off,
                            shells[s2].atom);
      std::vector<float4> prf(npr);
      std::vector<float2> pac(npr);
      for (size_t k = 0; k < (size_t)npr; ++k) {
        prf[k] = make_float4(alpha_f[k], alpha_f[npr + k], alpha_f[2 * npr + k], alpha_f[3 * npr + k]);
        pac[k] = make_float2(coef_f[k], coef_f[npr + k]);
      }
      if ((st = upload(P, &P->d_shell_f, shf.data(), shf.size())) != KLDI_OK) return fail(st);
      if ((st = upload(P, &P->d_prim_f, prf.data(), prf.size())) != KLDI_OK) return fail(st);
      if ((st = upload(P, &P->d_prim_ac, pac.data(), pac.size())) != KLDI_OK) return fail(st);
    }
    if ((st = upload(P, &P->d_bb_begin, bb_begin.data(), bb_begin.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_bb_end, bb_end.data(), bb_end.size())) != KLDI_OK) return fail(st);
    P->bb_nshell.resize(nbb);
    for (int64_t p = 0; p < nbb; ++p) P->bb_nshell[p] = std::max(0, bb_end[p] - bb_begin[p]);
    {
      // the kernels that give a block's shells to two groups of threads take
      // shells [0, split) and [split, nshell): about half of the block's
      // functions each (a shell's components inside the block counted)
      std::vector<int32_t> bb_split(nbb, 0);
      for (int64_t p = 0; p < nbb; ++p) {
        const int64_t lo = p * kBasisBlk, hi = std::min<int64_t>(lo + kBasisBlk, fn);
        int64_t tot = 0;
        for (int s = bb_begin[p]; s < bb_end[p]; ++s) {
          const int64_t f0 = shells[s].fn_off, f1 = f0 + (shells[s].l + 1) * (shells[s].l + 2) / 2;
          tot += std::min(f1, hi) - std::max(f0, lo);
        }
        int64_t acc = 0, best = INT64_MAX;
        int split = 0;
        for (int k = 0; k <= bb_end[p] - bb_begin[p]; ++k) {   // split before block-local shell k
          const int64_t d = std::llabs(2 * acc - tot);
          if (d < best) { best = d; split = k; }
          if (k < bb_end[p] - bb_begin[p]) {
            const int s = bb_begin[p] + k;
            const int64_t f0 = shells[s].fn_off, f1 = f0 + (shells[s].l + 1) * (shells[s].l + 2) / 2;
            acc += std::min(f1, hi) - std::max(f0, lo);
          }
        }
        bb_split[p] = split;
      }
      if ((st = upload(P, &P->d_bb_split, bb_split.data(), bb_split.size())) != KLDI_OK) return fail(st);
    }

    // ---- geometric candidates: shell extent R_s beyond which the value (and
    // gradient) bound r^l sum|c| e^{-a r^2} (+ l r^(l-1) .. + 2 a r^(l+1) ..) < t_b/2.
    const double tb = opt->t_b;
    std::vector<double> ext(ns, 0.0);
    for (int s = 0; s < ns; ++s) {
      const int l = shells[s].l, np = shells[s].nprim, o = shells[s].prim_off;
      double Rs = 0.0;
      for (double r = 60.0; r >= 0.0; r -= 0.01) {
        double v = 0.0, gd = 0.0;
        for (int k = 0; k < np; ++k) {
          const double e = std::fabs(coef[o + k]) * std::exp(-alpha[o + k] * r * r);
          v += e;
          gd += 2.0 * alpha[o + k] * e;
        }
        double b = std::pow(r, l) * v;
        if (P->gga) b = std::max(b, (l > 0 ? l * std::pow(r, l - 1) * v : 0.0) + std::pow(r, l + 1) * gd);
        if (b >= 0.5 * tb) { Rs = r + 0.05; break; }
      }
      ext[s] = tb > 0.0 ? Rs : 1e300;
    }
    std::vector<double> gc(nblk * 4);
    for (int64_t g = 0; g < nblk; ++g) {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int i = 0; i < kBlockPts; ++i)
        for (int c = 0; c < 3; ++c) {
          const double v = grid->xyz[(g * kBlockPts + i) * 3 + c];
          lo[c] = std::min(lo[c], v);
          hi[c] = std::max(hi[c], v);
        }
      double rad = 0.0;
      for (int c = 0; c < 3; ++c) {
        gc[g * 4 + c] = 0.5 * (lo[c] + hi[c]);
        rad += 0.25 * (hi[c] - lo[c]) * (hi[c] - lo[c]);
      }
      gc[g * 4 + 3] = std::sqrt(rad);
    }
    std::vector<std::vector<int32_t>> cand(nblk);
  #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t g = 0; g < nblk; ++g) {
      std::vector<char> mark(nbb, 0);
      for (int s = 0; s < ns; ++s) {
        const double dx = shells[s].cx - gc[g * 4], dy = shells[s].cy - gc[g * 4 + 1], dz = shells[s].cz - gc[g * 4 + 2];
        const double d = std::sqrt(dx * dx + dy * dy + dz * dz) - gc[g * 4 + 3];
        if (d <= ext[s]) {
          const int f0 = shells[s].fn_off, f1 = f0 + (shells[s].l + 1) * (shells[s].l + 2) / 2;
          for (int p = f0 / kBasisBlk; p <= (f1 - 1) / kBasisBlk; ++p) mark[p] = 1;
        }
      }
      for (int p = 0; p < nbb; ++p)
        if (mark[p]) cand[g].push_back(p);
    }
    std::vector<int64_t> cptr(nblk + 1, 0);
    for (int64_t g = 0; g < nblk; ++g) cptr[g + 1] = cptr[g] + (int64_t)cand[g].size();
    const int64_t ncand = cptr[nblk];
    std::vector<int32_t> cg(ncand), cp(ncand);
    for (int64_t g = 0; g < nblk; ++g)
      for (size_t k = 0; k < cand[g].size(); ++k) {
        cg[cptr[g] + k] = (int32_t)g;
        cp[cptr[g] + k] = cand[g][k];
      }
    int32_t *d_cg = nullptr, *d_cp = nullptr;
    double* d_cb = nullptr;
    std::vector<double> cb(ncand);
    if (ncand) {
      if (cudaMalloc(&d_cg, ncand * 4) != cudaSuccess || cudaMalloc(&d_cp, ncand * 4) != cudaSuccess ||
          cudaMalloc(&d_cb, ncand * 8) != cudaSuccess) {
        cudaFree(d_cg); cudaFree(d_cp); cudaFree(d_cb);
        set_error("kldi_screen: cudaMalloc of the candidate list failed");
        return fail(KLDI_ENOMEM);
      }
      cudaMemcpy(d_cg, cg.data(), ncand * 4, cudaMemcpyHostToDevice);
      cudaMemcpy(d_cp, cp.data(), ncand * 4, cudaMemcpyHostToDevice);
      st = launch_block_max(P, d_cg, d_cp, ncand, d_cb, 0);
      cudaError_t e = cudaMemcpy(cb.data(), d_cb, ncand * 8, cudaMemcpyDeviceToHost);
      cudaFree(d_cg); cudaFree(d_cp); cudaFree(d_cb);
      if (st != KLDI_OK) return fail(st);
      if (e != cudaSuccess) {
        set_error("kldi_screen: block summary kernel failed: %s", cudaGetErrorString(e));
        return fail(KLDI_ECUDA);
      }
    }
    // ---- retained lists S_g = {p : b_gp >= t_b}
    P->blk_ptr.assign(nblk + 1, 0);
    for (int64_t g = 0; g < nblk; ++g) {
      for (int64_t k = cptr[g]; k < cptr[g + 1]; ++k)
        if (cb[k] >= tb) {
          P->blk_idx.push_back(cp[k]);
          P->bmax.push_back(cb[k]);
        }
      if ((int64_t)P->blk_idx.size() > INT32_MAX) {
        set_error("kldi_screen: more than 2^31 retained tiles");
        return fail(KLDI_EUNSUPPORTED);
      }
      P->blk_ptr[g + 1] = (int32_t)P->blk_idx.size();
    }
    P->ntiles = (int64_t)P->blk_idx.size();
    P->rad_ptr.assign(P->ntiles + 1, 0);
    for (int64_t t = 0; t < P->ntiles; ++t) P->rad_ptr[t + 1] = P->rad_ptr[t] + P->bb_nshell[P->blk_idx[t]];
    if ((st = upload(P, &P->d_rad_ptr, P->rad_ptr.data(), P->rad_ptr.size())) != KLDI_OK) return fail(st);
    std::vector<int32_t> tile_of(nblk * nbb, -1);
    for (int64_t g = 0; g < nblk; ++g)
      for (int32_t t = P->blk_ptr[g]; t < P->blk_ptr[g + 1]; ++t) tile_of[g * nbb + P->blk_idx[t]] = t;
    if ((st = upload(P, &P->d_blk_ptr, P->blk_ptr.data(), P->blk_ptr.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_blk_idx, P->blk_idx.data(), P->blk_idx.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_bmax, P->bmax.data(), P->bmax.size())) != KLDI_OK) return fail(st);
    if ((st = upload(P, &P->d_tile_of, tile_of.data(), tile_of.size())) != KLDI_OK) return fail(st);
    {
      std::vector<int32_t> tile_g(std::max<int64_t>(P->ntiles, 1), 0);
      for (int64_t g = 0; g < nblk; ++g)
        for (int32_t t = P->blk_ptr[g]; t < P->blk_ptr[g + 1]; ++t) tile_g[t] = (int32_t)g;
      if ((st = upload(P, &P->d_tile_g, tile_g.data(), tile_g.size())) != KLDI_OK) return fail(st);
    }

    // ---- batches and V work lists (tile buffers are allocated at first use)
    {
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      int64_t cap = (int64_t)(0.35 * (double)free_b) / tile_bytes_max();
      if (const char* env = getenv("KLDI_TILE_CAP")) cap = std::max<int64_t>(1, atoll(env));
      if ((st = build_work(P, cap)) != KLDI_OK) return fail(st);
    }

    // ---- per-evaluation buffers
    const size_t nbf2 = (size_t)P->nbf * P->nbf;
    if ((st = dalloc(P, &P->d_D, nbf2)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_V, nbf2)) != KLDI_OK) return fail(st);
    if (!fnperm.empty()) {
      if ((st = upload(P, &P->d_fnperm, fnperm.data(), fnperm.size())) != KLDI_OK) return fail(st);
      if ((st = dalloc(P, &P->d_Dint, nbf2)) != KLDI_OK) return fail(st);
      if ((st = dalloc(P, &P->d_Vint, nbf2)) != KLDI_OK) return fail(st);
    }
    if ((st = dalloc(P, &P->d_dmax, (size_t)nbb * nbb)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_rho, (size_t)P->npoints)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_grad, (size_t)P->npoints * 3)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_xcoef, (size_t)P->npoints * 4)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_xdf, (size_t)P->npoints * 2)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_xmax, (size_t)std::max<int64_t>(P->ntiles, 1))) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_xmaxf, (size_t)std::max<int64_t>(P->ntiles, 1))) != KLDI_OK) return fail(st);
    {
      std::vector<float> bf(P->bmax.begin(), P->bmax.end());
      if ((st = upload(P, &P->d_bmaxf, bf.data(), bf.size())) != KLDI_OK) return fail(st);
    }
    if ((st = dalloc(P, &P->d_eblk, (size_t)nblk)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_exc, 1)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_err, 1)) != KLDI_OK) return fail(st);
    if ((st = dalloc(P, &P->d_vnext, 1)) != KLDI_OK) return fail(st);
    if (cudaMemset(P->d_err, 0, sizeof(int)) != cudaSuccess) { set_error("kldi_screen: memset failed"); return fail(KLDI_ECUDA); }
    *out = P;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_set_precision(kldi_plan* P, int prec) {
  return kldi::guarded("kldi_plan_set_precision", [&]() -> kldi_status {
    if (!P || prec < KLDI_FP64 || prec > KLDI_BF16X10) {
      set_error("kldi_plan_set_precision: bad argument");
      return KLDI_EINVAL;
    }
    KLDI_TRY(ensure_tile_buffers(P, prec));
    P->prec = prec;
    // the V work lists differ between the FP64 and the tensor-core products
    if ((prec == KLDI_FP64) != P->work_fp64) {
      KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
      KLDI_TRY(build_work(P, P->tile_cap));
    }
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_workspace_create(int64_t bytes, kldi_workspace** out) {
  return kldi::guarded("kldi_workspace_create", [&]() -> kldi_status {
    if (!out || bytes <= 0) {
      set_error("kldi_workspace_create: bad argument");
      return KLDI_EINVAL;
    }
    *out = nullptr;
    kldi_workspace* ws = new (std::nothrow) kldi_workspace;
    if (!ws) {
      set_error("kldi_workspace_create: out of host memory");
      return KLDI_ENOMEM;
    }
    cudaGetDevice(&ws->device);
    if (cudaMalloc(&ws->base, (size_t)bytes) != cudaSuccess) {
      cudaGetLastError();
      delete ws;
      set_error("kldi_workspace_create: cudaMalloc of %lld bytes failed", (long long)bytes);
      return KLDI_ENOMEM;
    }
    ws->bytes = bytes;
    *out = ws;
    return KLDI_OK;
  });
}

extern "C" void kldi_workspace_free(kldi_workspace* ws) {
  if (!ws) return;
  if (ws->base) cudaFree(ws->base);
  delete ws;
}

extern "C" kldi_status kldi_plan_set_workspace(kldi_plan* P, const kldi_workspace* ws) {
  return kldi::guarded("kldi_plan_set_workspace", [&]() -> kldi_status {
    if (!P) {
      set_error("kldi_plan_set_workspace: null plan");
      return KLDI_EINVAL;
    }
    int64_t cap;
    if (ws) {
      if (ws->device != P->device) {
        set_error("kldi_plan_set_workspace: workspace and plan live on different devices");
        return KLDI_EINVAL;
      }
      // tiles first, then the BF16X10 radial rows (2 KB each; 1.25 x the
      // plan's mean shells per tile reserved per tile)
      const double mean_rows = P->ntiles ? (double)P->rad_ptr[P->ntiles] / (double)P->ntiles : 1.0;
      const int64_t per_tile = tile_bytes_max() + (int64_t)std::ceil(1.25 * mean_rows) * kBlockPts * 16;
      cap = ws->bytes / per_tile;
      const int64_t rows_cap = (ws->bytes - cap * tile_bytes_max()) / (kBlockPts * 16);
      int64_t maxblk = 0, maxrows = 0;
      for (int64_t g = 0; g < P->nblocks; ++g) {
        maxblk = std::max<int64_t>(maxblk, P->blk_ptr[g + 1] - P->blk_ptr[g]);
        maxrows = std::max<int64_t>(maxrows, P->rad_ptr[P->blk_ptr[g + 1]] - P->rad_ptr[P->blk_ptr[g]]);
      }
      if (cap < maxblk || rows_cap < maxrows) {
        set_error("kldi_plan_set_workspace: %lld bytes hold %lld tiles, a grid block needs %lld", (long long)ws->bytes,
                  (long long)cap, (long long)maxblk);
        return KLDI_EINVAL;
      }
      P->rad_rows_cap = rows_cap;
    } else {
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      cap = (int64_t)(0.35 * (double)free_b) / tile_bytes_max();
      P->rad_rows_cap = INT64_MAX;
    }
    KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
    free_own_tile_buffers(P);
    if (P->d_rad && !P->ws) cudaFree(P->d_rad);   // a plan-owned radial buffer
    P->d_rad = nullptr;
    P->rad_cap = 0;
    P->ws = ws;
    KLDI_TRY(build_work(P, cap));
    if (ws) KLDI_TRY(ensure_tile_buffers(P, P->prec));
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_set_block_range(kldi_plan* P, int64_t g0, int64_t g1) {
  return kldi::guarded("kldi_plan_set_block_range", [&]() -> kldi_status {
    if (!P || g0 < 0 || g1 < g0 || g1 > P->nblocks) {
      set_error("kldi_plan_set_block_range: need 0 <= g0 <= g1 <= nblocks");
      return KLDI_EINVAL;
    }
    KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
    // blocks outside the range contribute nothing to E_xc
    KLDI_TRY_CUDA(cudaMemset(P->d_eblk, 0, sizeof(double) * P->nblocks));
    P->range_g0 = g0;
    P->range_g1 = g1;
    return build_work(P, P->tile_cap);
  });
}

extern "C" kldi_status kldi_plan_set_wait_limit(kldi_plan* P, uint64_t ns) {
  return kldi::guarded("kldi_plan_set_wait_limit", [&]() -> kldi_status {
    if (!P) {
      set_error("kldi_plan_set_wait_limit: null plan");
      return KLDI_EINVAL;
    }
    P->wait_ns = ns ? ns : 2000000000ull;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_set_withhold(kldi_plan* P, int64_t item) {
  return kldi::guarded("kldi_plan_set_withhold", [&]() -> kldi_status {
    if (!P || item < -1) {
      set_error("kldi_plan_set_withhold: bad argument");
      return KLDI_EINVAL;
    }
    P->withhold_item = item;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_set_tuning(kldi_plan* P, const kldi_tuning* t) {
  return kldi::guarded("kldi_plan_set_tuning", [&]() -> kldi_status {
    if (!P || !t || t->v_seg < 0 || (t->rho_ntile != 0 && t->rho_ntile != 64 && t->rho_ntile != 128) ||
        (t->v_align != 0 && t->v_align != 1 && t->v_align != 2 && t->v_align != 4)) {
      set_error("kldi_plan_set_tuning: bad argument (v_seg >= 0, rho_ntile 0, 64 or 128, v_align 0, 1, 2 or 4)");
      return KLDI_EINVAL;
    }
    if (P->prec == KLDI_BF16X10 && t->rho_ntile == 128) {
      set_error("kldi_plan_set_tuning: BF16X10 has only the 64-function density tile");
      return KLDI_EUNSUPPORTED;
    }
    KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
    const bool rebuild = t->v_seg != P->tune.v_seg || t->v_align != P->tune.v_align;
    P->tune = *t;
    return rebuild ? build_work(P, P->tile_cap) : KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_get_tuning(const kldi_plan* P, kldi_tuning* t) {
  return kldi::guarded("kldi_plan_get_tuning", [&]() -> kldi_status {
    if (!P || !t) {
      set_error("kldi_plan_get_tuning: null argument");
      return KLDI_EINVAL;
    }
    *t = P->tune;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_info(const kldi_plan* P, kldi_plan_stats* s) {
  return kldi::guarded("kldi_plan_info", [&]() -> kldi_status {
    if (!P || !s) { set_error("kldi_plan_info: null argument"); return KLDI_EINVAL; }
    s->nbf = P->nbf;
    s->nbasis_blocks = P->nbb;
    s->npoints = P->npoints;
    s->nblocks = P->nblocks;
    s->retained = P->ntiles;
    int64_t ps = 0;
    for (int64_t g = 0; g < P->nblocks; ++g) {
      const int64_t n = P->blk_ptr[g + 1] - P->blk_ptr[g];
      ps += n * n;
    }
    s->pair_slots = ps;
    s->vtile_work = P->vtile_work;
    s->workspace_bytes = P->workspace_bytes;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_export_lists(const kldi_plan* P, int32_t* blk_ptr, int32_t* blk_idx, double* bmax) {
  return kldi::guarded("kldi_plan_export_lists", [&]() -> kldi_status {
    if (!P) { set_error("kldi_plan_export_lists: null plan"); return KLDI_EINVAL; }
    if (blk_ptr) std::memcpy(blk_ptr, P->blk_ptr.data(), P->blk_ptr.size() * 4);
    if (blk_idx) std::memcpy(blk_idx, P->blk_idx.data(), P->blk_idx.size() * 4);
    if (bmax) std::memcpy(bmax, P->bmax.data(), P->bmax.size() * 8);
    return KLDI_OK;
  });
}

extern "C" void kldi_plan_free(kldi_plan* P) {
  if (!P) return;
  for (auto& e : P->prof_ev) cudaEventDestroy(e);
  free_plan_buffers(P);
  delete P;
}
