// Internal declarations of libkldi: handle structures, device views and the
// launchers shared between translation units.  Not part of the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <exception>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "kldi.h"

namespace kldi {

constexpr int kBlockPts = 128;   // grid block (points); one tcgen05 M = 128 tile
constexpr int kBasisBlk = 32;    // basis block d (Sec. IV numerical settings: d = 32)
constexpr int kVTile = 128;      // W output tile edge of the tensor-core V product (4 basis blocks)

void set_error(const char* fmt, ...);

#define KLDI_TRY_CUDA(expr)                                                                    \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      kldi::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return KLDI_ECUDA;                                                                       \
    }                                                                                          \
  } while (0)

#define KLDI_TRY(expr)            \
  do {                            \
    kldi_status s_ = (expr);      \
    if (s_ != KLDI_OK) return s_; \
  } while (0)

// Runs the body of a C-ABI call: host exceptions (allocation failures of the
// standard containers and the like) become a status and a message instead of
// unwinding through extern "C" into the caller.
template <typename F>
kldi_status guarded(const char* fn, F&& f) noexcept {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    set_error("%s: out of host memory", fn);
    return KLDI_ENOMEM;
  } catch (const std::exception& e) {
    set_error("%s: %s", fn, e.what());
    return KLDI_EINVAL;
  } catch (...) {
    set_error("%s: unexpected host exception", fn);
    return KLDI_EINVAL;
  }
}

// Runs f() once per device for the call site (each lambda type has its own
// state): kernel attributes such as the shared-memory opt-in belong to a
// device; the lock keeps plans built on several host threads from racing.
template <typename F>
kldi_status once_per_device(F&& f) {
  static std::mutex mu;
  static std::set<int> ready;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KLDI_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (ready.count(dev)) return KLDI_OK;
  const kldi_status st = f();
  if (st == KLDI_OK) ready.insert(dev);
  return st;
}

// One shell as the kernels see it.  coef[k] already carries the primitive norm
// (2a/pi)^(3/4) (4a)^(l/2) and the contraction rescale; the per-component factor
// 1/sqrt((2i-1)!!(2j-1)!!(2k-1)!!) is applied in the kernels.
struct DevShell {
  double cx, cy, cz;
  int32_t l;
  int32_t nprim;
  int32_t prim_off;
  int32_t fn_off;
  int32_t atom;
  int32_t pad;
};

// Read-only device view of basis, grid and retained lists.
struct BasisView {
  const DevShell* shells;
  const double* alpha;        // [nprim_total]
  const double* coef;         // [nprim_total]
  const float* alpha_f;       // FP32 hi/lo pairs (value = hi + lo to ~2^-48) of the
  const float* alpha_lo;      // exponents, coefficients and their products a*c,
  const float* coef_f;        // for the FP32 basis kernels
  const float* coef_lo;
  const float* ac_f;
  const float* ac_lo;
  const int32_t* bb_shell_begin;  // [nbb] first shell with a function in basis block p
  const int32_t* bb_shell_end;    // [nbb] one past the last such shell
  const int32_t* bb_split;        // [nbb] first shell (block-local) of the block's second half
  // FP32 evaluation in coordinates relative to an anchor atom: relatom[(a * natm + b) * 8 + 0..5]
  // = A_b - A_a as hi (0..2) and lo (3..5) FP32 parts
  const float* relatom;
  // packed copies for the FP32 kernels: per shell {l | nprim << 8, prim_off,
  // fn_off, atom}; per primitive {alpha hi, alpha lo, coef hi, coef lo} and
  // {alpha coef hi, lo}
  const int4* shell_f;
  const float4* prim_f;
  const float2* prim_ac;
  int32_t natm;
  int32_t nbf;
  int32_t nbb;
};

struct GridView {
  const double* xyz;   // [npoints*3]
  const double* w;     // [npoints]
  const float4* prel;  // [npoints] FP32 point coordinates relative to the block's anchor atom
  const float4* prel_lo;  // [npoints] their low parts (coordinate - hi, rounded to FP32)
  const int32_t* anchor;  // [nblocks] anchor atom of each grid block (atom of its first point)
  int64_t npoints;
  int64_t nblocks;
};

struct ListView {
  const int32_t* blk_ptr;  // [nblocks+1] CSR over grid blocks
  const int32_t* blk_idx;  // [ntiles] retained basis block p of tile t
  const double* bmax;      // [ntiles] b_gp
  const int32_t* tile_of;  // [nblocks*nbb] tile index of (g, p), -1 if not retained
  const int32_t* tile_g;   // [ntiles] grid block g of tile t
  int32_t nbb;
};

// Work item of the FP64 V product: one 32 x 32 block pair (p <= q) over the
// grid blocks list_g[beg, end).
struct VWork64 {
  int32_t p, q;
  int32_t beg, end;
};

// Work item of the tensor-core V product: one pair of 128-function windows
// (P, Q = the first of 4 consecutive basis blocks; P == Q, or P + 4 <= Q) over
// grid blocks list_g[beg, end).
struct VWorkTC {
  int32_t P, Q;
  int32_t beg, end;
};

struct Batch {
  int64_t g0 = 0, g1 = 0;     // grid blocks [g0, g1)
  int64_t t0 = 0, t1 = 0;     // tiles [t0, t1)
  // FP64 V product
  int32_t* d_v64_g = nullptr;  VWork64* d_v64_work = nullptr;  int64_t n_v64_work = 0;
  // tensor V product
  int32_t* d_vtc_g = nullptr;  VWorkTC* d_vtc_work = nullptr;  int64_t n_vtc_work = 0;
};

}  // namespace kldi

struct kldi_grid {
  std::vector<double> xyz;      // [npoints*3]
  std::vector<double> w;        // [npoints]
  std::vector<int32_t> atom;    // [npoints]
  int64_t npoints = 0, nreal = 0, nblocks = 0;
  int block = kldi::kBlockPts;
};

// Learned functional: FP32 master parameters, their FP16 copy used by the
// forward pass, Adam moments and the training box.
struct kldi_mlp {
  int device = 0;
  float* d_param = nullptr;          // [KLDI_MLP_NPARAMS] FP32 master
  __half* d_half = nullptr;          // [KLDI_MLP_NPARAMS] FP16 copy
  float* d_m = nullptr;              // Adam first moment
  float* d_v = nullptr;              // Adam second moment
  float* d_grad = nullptr;           // [KLDI_MLP_NPARAMS] scratch gradient
  float* d_part = nullptr;           // per-CTA partial gradients [cap][KLDI_MLP_NPARAMS + 2]
  int64_t part_cap = 0;              // CTAs the partial buffer holds
  float* d_loss = nullptr;           // [1 + loss history]
  int64_t step = 0;                  // Adam steps taken
  double box[4] = {0, 0, 0, 0};      // lo, hi of ln rho; lo, hi of ln sigma
};

// Shared device arena for the per-tile buffers of several plans.
struct kldi_workspace {
  int device = 0;
  void* base = nullptr;
  int64_t bytes = 0;
};

struct kldi_plan {
  kldi_options opt{};
  const kldi_workspace* ws = nullptr;   // shared per-tile buffers (not owned), or NULL
  kldi_tuning tune{0, 0, 0};
  bool work_fp64 = false;               // which V work lists the batches hold
  int64_t range_g0 = 0, range_g1 = -1;  // grid blocks evaluated: [range_g0, range_g1), -1 = all
  int gga = 0;
  const kldi_mlp* mlp = nullptr;   // learned functional for KLDI_XC_MLP (not owned)
  int prec = KLDI_FP64;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 148;
  int64_t nbf = 0, nbb = 0, nbf_pad = 0, npoints = 0, nblocks = 0, ntiles = 0, nshell = 0, nprim_total = 0;
  int* d_err = nullptr;         // device error word (bounded-wait timeouts)
  uint64_t wait_ns = 2000000000ull;   // limit of the tensor-core kernels' bounded waits
  int64_t withhold_item = -1;   // test hook: V work item not handed out (-1: none)
  int* d_vnext = nullptr;       // work-item counter of the tensor-core V product
  double* d_G = nullptr;        // [natm][3] nuclear gradient (allocated by the first kldi_exc_grad)

  // host copies of the retained lists
  std::vector<int32_t> blk_ptr, blk_idx;
  std::vector<double> bmax;

  // device: grid, basis, lists
  double* d_xyz = nullptr;
  double* d_w = nullptr;
  float4* d_prel = nullptr;
  float4* d_prel_lo = nullptr;
  int32_t* d_anchor = nullptr;
  float* d_relatom = nullptr;
  int32_t natm = 0;
  kldi::DevShell* d_shells = nullptr;
  double* d_alpha = nullptr;
  double* d_coef = nullptr;
  float* d_alpha_f = nullptr;   // [4][nprim]: alpha hi, alpha lo, coef hi, coef lo
  float* d_coef_f = nullptr;    // [2][nprim]: (alpha coef) hi, lo
  int4* d_shell_f = nullptr;    // packed per shell (BasisView::shell_f)
  float4* d_prim_f = nullptr;   // packed per primitive
  float2* d_prim_ac = nullptr;
  int32_t* d_bb_begin = nullptr;
  int32_t* d_bb_split = nullptr;
  int32_t* d_bb_end = nullptr;
  int32_t* d_blk_ptr = nullptr;
  int32_t* d_blk_idx = nullptr;
  double* d_bmax = nullptr;
  int32_t* d_tile_of = nullptr;
  int32_t* d_tile_g = nullptr;

  // device: per-evaluation buffers
  double* d_D = nullptr;        // staging copy of a host D
  double* d_V = nullptr;        // staging V when the caller passes host memory
  int32_t* d_fnperm = nullptr;  // [nbf] caller's index of each internal function (reordered plans)
  double* d_Dint = nullptr;     // D and V in the internal function order (reordered plans)
  double* d_Vint = nullptr;
  double* d_dmax = nullptr;     // [nbb*nbb]
  double* d_rho = nullptr;      // [npoints]
  double* d_grad = nullptr;     // [npoints*3]
  double* d_xcoef = nullptr;    // [npoints*4]: w v_rho / 2, 2 w v_sigma grad rho
  float4* d_xdf = nullptr;      // [npoints*2]: the same as FP32 hi, lo (the double-float X kernel)
  double* d_xmax = nullptr;     // [ntiles]
  float* d_xmaxf = nullptr;     // [ntiles] the same in FP32 (tensor-core V product's pair rule)
  float* d_bmaxf = nullptr;     // [ntiles] b_gp in FP32 (tensor-core V product's pair rule)
  double* d_eblk = nullptr;     // [nblocks]
  double* d_exc = nullptr;      // [1]
  // tiles of the current batch
  double* d_phi64 = nullptr;    // FP64: [tiles][32][128]
  double* d_x64 = nullptr;      // FP64: [tiles][32][128]
  uint16_t* d_phi_s = nullptr;  // Phi sliced per point: [tiles][NS planes][128][32] BF16 (room for 4 planes)
  uint16_t* d_phic_s = nullptr; // Phi sliced per function: [tiles][NS planes][128][32] BF16
  uint16_t* d_x_s = nullptr;    // X sliced per function: [tiles][NS planes][128][32] BF16
  float* d_phic_scale = nullptr;// [tiles][32] function scales of d_phic_s
  float* d_x_scale = nullptr;   // [tiles][32] function scales of d_x_s
  float* d_rowscale = nullptr;  // [npoints] point scales of d_phi_s
  float* d_pscale = nullptr;    // [npoints] per-point balance c_i: Phi c and X / c in the V product
  float* d_zscale = nullptr;    // [npoints] point scales of the gradient's Z tiles (first tensor-core gradient)
  bool rec_fit_all = true;      // every basis block fits a shared-memory shell record (40 shells, 80 primitives)
  // BF16X10: radial factors (g, gd) of every (tile, shell of its basis block, point) in hi / lo, written
  // by the Phi kernel and read by the density product's row-dot and the X kernel
  std::vector<int32_t> bb_nshell;   // [nbb] shells with a function in basis block p
  std::vector<int64_t> rad_ptr;     // [ntiles + 1] prefix of bb_nshell over the tiles
  int64_t* d_rad_ptr = nullptr;
  float4* d_rad = nullptr;          // [shells of the batch][128]: g hi, g lo, gd hi, gd lo
  int64_t rad_cap = 0;              // shell rows d_rad holds
  int64_t rad_rows_cap = INT64_MAX; // shell rows a batch may use (bounded when the rows live in a workspace)
  float* d_dscale = nullptr;    // [nbf_pad] column scales of d_dsplit
  uint16_t* d_dsplit = nullptr; // sliced D block pairs [nbb*nbb][NS planes][32][32]
  uint16_t* d_zero = nullptr;   // zero block (bulk-copy source for masked / absent blocks)
  int64_t tile_cap = 0;         // tiles per batch the buffers hold

  std::vector<kldi::Batch> batches;

  // stage timing (kldi_plan_profile)
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;       // pool, pairs (start, end)
  std::vector<int> prof_stage;            // stage of each recorded pair
  std::vector<int> prof_launches;         // kernel launches of each recorded pair
  int64_t launch_count = 0;               // kernels launched by this plan
  int64_t vtile_work = 0;
  int64_t workspace_bytes = 0;

  kldi::BasisView basis_view() const;
  kldi::GridView grid_view() const;
  kldi::ListView list_view() const;
};

namespace kldi {

// launchers (kernels.cu)
kldi_status launch_block_max(const kldi_plan* P, const int32_t* d_cand_g, const int32_t* d_cand_p,
                             int64_t ncand, double* d_out, cudaStream_t s);
kldi_status launch_dmax(const kldi_plan* P, const double* D, cudaStream_t s);
kldi_status launch_phi64(const kldi_plan* P, const Batch& b, cudaStream_t s);
kldi_status launch_rho64(const kldi_plan* P, const Batch& b, const double* D, double* rho, double* grad,
                         cudaStream_t s);
kldi_status launch_xc(const kldi_plan* P, const Batch& b, int xc, const double* rho, const double* grad,
                      cudaStream_t s);
kldi_status launch_x64(const kldi_plan* P, const Batch& b, cudaStream_t s);
kldi_status launch_v64(const kldi_plan* P, const Batch& b, double* V, cudaStream_t s);
kldi_status launch_finish(const kldi_plan* P, double* V, double* exc, cudaStream_t s);

// tensor-core path (tc.cu)
kldi_status launch_dsplit(const kldi_plan* P, const double* D, cudaStream_t s);
kldi_status launch_phi_split(const kldi_plan* P, const Batch& b, cudaStream_t s);
kldi_status launch_rho_tc(const kldi_plan* P, const Batch& b, double* rho, double* grad, cudaStream_t s);
kldi_status launch_x_split(const kldi_plan* P, const Batch& b, cudaStream_t s);
kldi_status launch_v_tc(const kldi_plan* P, const Batch& b, double* V, cudaStream_t s);
kldi_status prepare_tc_kernels();
kldi_status launch_grad64(const kldi_plan* P, const Batch& b, const double* D, double* G, cudaStream_t s);
// Reordered plans: dst[i][j] = src[fp[i]][fp[j]] (gather) or dst[fp[i]][fp[j]] = src[i][j].
kldi_status launch_permute(const kldi_plan* P, const double* src, double* dst, bool gather, cudaStream_t s);
kldi_status launch_grad_tc(const kldi_plan* P, const Batch& b, bool gga_xc, double* G, cudaStream_t s);
kldi_status becke_weights_device(int natm, const double* atom_xyz, const double* R, const int32_t* nbr,
                                 const double* xyz, const int32_t* owner, const double* raw_w, int64_t nreal,
                                 double* w);
kldi_status ensure_tile_buffers(kldi_plan* P, int prec);
kldi_status build_work(kldi_plan* P, int64_t cap);
int64_t tile_bytes_max();
void free_own_tile_buffers(kldi_plan* P);
kldi_status launch_xc_mlp(const kldi_plan* P, const Batch& b, const double* rho, const double* grad,
                          cudaStream_t s);
bool is_device_ptr(const void* p);

}  // namespace kldi
