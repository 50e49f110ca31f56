/*
 * kldi.h -- C ABI of the block-filtered exchange-correlation (EXC) quadrature
 * library for NVIDIA GB300 (sm_103a).
 *
 * What it computes (arxiv 2605.10363, Sec. II-A): for Gaussian basis functions
 * chi_mu, grid points r_i with weights w_i and a symmetric density matrix D,
 *   Phi_{mu i}  = chi_mu(r_i)                                  (Eq. phi_def)
 *   rho_i       = sum_{mu nu} D_{mu nu} chi_mu(r_i) chi_nu(r_i) (App. A), R = D Phi (Eq. r_equals_dphi)
 *   E_xc        = sum_i w_i f(rho_i, sigma_i),  sigma = |grad rho|^2
 *   V_{mu nu}   = sum_i w_i v_i chi_mu chi_nu  (Eq. exc_quadrature / fxc_matrix_form, b = 1),
 *                 generalised for the GGA to (Phi^T X + X^T Phi)_{mu nu} with
 *                 X_{i nu} = w_i (v_rho chi_nu / 2 + 2 v_sigma grad rho . grad chi_nu).
 * Both products run only over the retained, executable 32 x 32 block pairs
 * of the block-filtered representation (Sec. III-B-3 Eqs. block_summary_A..
 * retained_blocks_B, Sec. III-C-1 Eqs. block_pair_filter..executed_block_pairs).
 *
 * Conventions for every entry point
 *   - Units: bohr and Hartree.  Arrays are row-major.  Spin-restricted (b = 1).
 *   - Return value: a kldi_status; nothing aborts.  On failure the message is
 *     available from kldi_last_error() (thread-local, valid until the next call
 *     on the same thread).
 *   - Pointers passed to compute calls may be device or host memory; the
 *     library asks the CUDA runtime which one it is.  Host arrays are copied
 *     on the plan's stream; if any output is host memory the call synchronises
 *     the stream before returning, otherwise it returns after enqueueing.
 *   - Caller-owned: every array passed in.  Library-owned: the opaque handles,
 *     released with kldi_grid_free / kldi_plan_free.  Work buffers are
 *     allocated once when the plan is built; compute calls allocate nothing.
 *   - A plan is used by one host thread at a time.  All work goes on the
 *     stream given in kldi_options (0 = the legacy default stream).
 */
#ifndef KLDI_H
#define KLDI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kldi_grid kldi_grid;
typedef struct kldi_plan kldi_plan;

typedef enum {
  KLDI_OK = 0,
  KLDI_EINVAL = -1,       /* bad argument (null pointer, size, enum value)   */
  KLDI_ENOMEM = -2,       /* host or device allocation failed                */
  KLDI_ECUDA = -3,        /* a CUDA runtime/driver call failed               */
  KLDI_ETIMEOUT = -4,     /* a bounded device wait gave up                   */
  KLDI_EUNSUPPORTED = -5, /* valid request this build or device cannot serve */
  KLDI_EIO = -6           /* a file could not be opened, written or read     */
} kldi_status;

/* Functionals (Sec. III-F scope: local and semilocal).  KLDI_XC_LDA_X: Slater
 * exchange.  KLDI_XC_PBE: PBE exchange + PW92/PBE correlation.  KLDI_XC_MLP:
 * the learned 2-64-64-2 surrogate of the PBE form (see kldi_mlp_*). */
typedef enum { KLDI_XC_LDA_X = 1, KLDI_XC_PBE = 2, KLDI_XC_MLP = 3 } kldi_xc;

/* Arithmetic of the two block products.
 * KLDI_FP64: FP64 CUDA-core block products (the plain block form).
 * KLDI_BF16X3 / KLDI_BF16X6: tcgen05 tensor cores.  Every operand row (or
 * column) is scaled by a power of two to |a| <= 1 and cut into 2 (x3) or 3
 * (x6) BF16 slices on fixed-point grids of 2^-7, 2^-15, 2^-23; the products
 * of slices whose levels sum below the slice count (3 resp. 6 products) are
 * accumulated per level in FP32 tensor memory, where every partial sum of at
 * most 256 terms is exactly representable, so the accumulator never rounds.
 * Levels are combined and summed across K-segments in FP32/FP64 with
 * round-to-nearest.  Truncation error: 2^-16 (x3) or 2^-24 (x6) of the row /
 * column scale per element.
 * KLDI_BF16X10: four slices on the grids 2^-7, 2^-15, 2^-23, 2^-31 and the
 * ten products of levels 0..3; the basis values, X and the row-dot are
 * formed in double-float (FP32 hi + lo, ~2^-44 relative), so the truncation
 * error is 2^-32 of the row / column scale.  The density product keeps all
 * four levels exact (N tiles of 64 functions); the V product keeps levels 0
 * and 1 exact and accumulates levels 2 and 3 together (their rounding acts at
 * ~2^-40 of the scale).  This is the mode that meets |dE_xc| <= 1e-6 Ha and
 * max|dV| <= 1e-7 on whole grids of 10^7 points; it needs every basis block
 * to fit a shared-memory shell record (40 shells, 80 primitives), else
 * KLDI_EUNSUPPORTED.
 * KLDI_TF32X3: not provided (KLDI_EUNSUPPORTED): 11-bit slices cannot keep
 * 256-term partial sums exact, so the accumulator's rounding would bias the
 * result.
 * The functional, the E_xc reduction and the scatter into V are FP64 in
 * every mode. */
typedef enum { KLDI_FP64 = 0, KLDI_BF16X3 = 1, KLDI_TF32X3 = 2, KLDI_BF16X6 = 3, KLDI_BF16X10 = 4 } kldi_prec;

/* Atoms: natm nuclei, atomic numbers Z[natm], positions xyz[natm*3] in bohr. */
typedef struct {
  int natm;
  const int32_t* Z;
  const double* xyz;
} kldi_molecule;

/* Contracted Cartesian Gaussian shells (App. A, "Gaussian basis functions").
 * Shell s sits on atom atom[s], has angular momentum l[s] in {0,1,2} and
 * nprim[s] primitives; its exponents and raw contraction coefficients are
 * exps/coefs[off_s .. off_s + nprim[s]) with off_s = sum_{t<s} nprim[t].
 * Coefficients multiply unnormalised primitives x^i y^j z^k exp(-a r^2); the
 * library normalises each primitive and rescales the contraction to unit
 * self-overlap.  Function order: shell by shell; inside a shell
 * s | x y z | xx xy xz yy yz zz. */
typedef struct {
  int nshell;
  const int32_t* atom;
  const int32_t* l;
  const int32_t* nprim;
  const double* exps;
  const double* coefs;
} kldi_basis;

/* Atom-centred grid (App. A, "Numerical integration grids"): nrad radial
 * Treutler-Ahlrichs M4 points on Chebyshev nodes of the second kind; the
 * radial shells are split into nregions equal index ranges (inner to outer)
 * and range r uses the product angular rule ntheta[r] (Gauss-Legendre in
 * cos theta) x 2*ntheta[r] (uniform azimuth).  Becke partition (three
 * iterations).  Points are grouped by atom and stably sorted by the 60-bit
 * Morton key of App. B Eq. morton_code within each atom, then cut into
 * blocks of `block` points (only 128 is supported); the last block is padded
 * with copies of the last point at weight 0. */
typedef struct {
  int nrad;
  int nregions;
  const int32_t* ntheta;
  int block;
} kldi_grid_spec;

/* Thresholds and modes.  t_b: block-retention threshold (Eq. block_filter_A);
 * t_d: block-pair execution threshold (Eq. block_pair_filter); rho_min: points
 * with rho < rho_min contribute nothing; prec: kldi_prec; xc: the kldi_xc the
 * plan will serve (KLDI_XC_PBE/MLP need basis gradients, LDA does not);
 * stream: a cudaStream_t, or NULL for the legacy default stream;
 * shell_order: NULL, or a permutation of the nshell shells (e.g. from
 * kldi_order_shells; caller-owned, read during kldi_screen only) in which the
 * plan lays out its basis blocks (Sec. III-B).  The caller's D, V and any
 * other matrix stay in the caller's order: the compute calls permute D on the
 * way in and V on the way out (two gather kernels and two nbf x nbf buffers
 * held by the plan). */
typedef struct {
  double t_b;
  double t_d;
  double rho_min;
  int prec;
  int xc;
  void* stream;
  const int32_t* shell_order;
} kldi_options;

/* Plan statistics (kldi_plan_info). */
typedef struct {
  int64_t nbf;            /* basis functions                                  */
  int64_t nbasis_blocks;  /* ceil(nbf / 32)                                   */
  int64_t npoints;        /* grid points incl. padding (multiple of 128)     */
  int64_t nblocks;        /* grid blocks                                       */
  int64_t retained;       /* sum over grid blocks of |S_g| (retained tiles)    */
  int64_t pair_slots;     /* sum over grid blocks of |S_g|^2                   */
  int64_t vtile_work;     /* (V tile, grid block) work items of the V product */
  int64_t workspace_bytes;/* device bytes held by the plan                    */
} kldi_plan_stats;

/* Basis order by overlap signatures (Sec. III-B, appendix "Overlap-Signature
 * Construction and Basis-Function Clustering"), host preprocessing once per
 * geometry.  Units are shells (a Cartesian shell's functions stay together):
 * shell signature T_s = (||S[s,t]||_F)_t, cosine distance
 * d(s,t) = 1 - T_s.T_t / (|T_s||T_t|), agglomerative clustering with average
 * linkage, each merge orienting the two leaf sequences so that their closest end
 * leaves are adjacent.  nfn[nshell]: functions per shell in the current order;
 * S: the nbf x nbf overlap matrix in that order (row-major, host); perm[nshell]
 * (host, caller-owned) receives the new order: position k holds old shell
 * perm[k].  Ties are broken by the lower index, so the result is reproducible.
 * O(nshell^2) memory.  KLDI_EINVAL for a non-positive size or a shell with a
 * zero signature.  The caller reorders its basis and D with perm (the plan is
 * then built from the reordered basis). */
kldi_status kldi_order_shells(int nshell, const int* nfn, const double* S, int* perm);

/* Build the molecular grid on the host (preprocessing, run once per
 * geometry; Sec. III-D).  *out is library-owned. */
kldi_status kldi_make_grid(const kldi_molecule* mol, const kldi_grid_spec* spec, kldi_grid** out);

/* Grid sizes: total points (multiple of the block size), real points, blocks. */
kldi_status kldi_grid_info(const kldi_grid* grid, int64_t* npoints, int64_t* nreal, int64_t* nblocks);

/* Copy the grid into caller host buffers: xyz[npoints*3], w[npoints],
 * atom_of[npoints]; any of the three may be NULL. */
kldi_status kldi_grid_export(const kldi_grid* grid, double* xyz, double* w, int32_t* atom_of);

/* Save a grid to the file at path (created or replaced), and load one back,
 * so that a geometry's grid is built once (the Becke weights of Sec. III-D's
 * preprocessing are the costly part of building it).  File, host byte order:
 * the 8 bytes "KLDIGRD1"; int64 npoints, nreal, nblocks, block; then
 * xyz[npoints*3] and w[npoints] (double) and atom_of[npoints] (int32), as
 * kldi_grid_export gives them.  kldi_grid_load checks the header, the sizes
 * (block = 128, npoints = nblocks * block, npoints - block < nreal <= npoints),
 * the file length, the owning atoms (>= 0), finite coordinates and weights,
 * and zero weights on the padding; kldi_screen refuses a grid whose owning
 * atoms do not exist in its molecule.  KLDI_EINVAL: null argument or
 * malformed file; KLDI_EIO: the file cannot be opened, written or read in
 * full.  *out is library-owned (kldi_grid_free). */
kldi_status kldi_grid_save(const kldi_grid* grid, const char* path);
kldi_status kldi_grid_load(const char* path, kldi_grid** out);

/* Geometry-fixed preprocessing (Sec. III-B-3, III-D): upload grid and basis,
 * evaluate the block summaries b_gp = max |phi| (and |grad phi| for the GGA)
 * over every grid block x 32-function basis block in FP64 on the GPU, keep
 * S_g = {p : b_gp >= t_b} as a block-CSR list per grid block (the BCS(R)
 * analogue of App. C) and the per-V-tile lists of grid blocks (the BCS(C)
 * analogue), and allocate all work buffers.  The grid must stay alive while
 * the plan is used.  *out is library-owned.  Before any device work,
 * KLDI_EINVAL for: a null argument, a shell with l > 2 (KLDI_EUNSUPPORTED) or
 * nprim <= 0 or an atom outside the molecule, an exponent that is not positive
 * and finite, a non-finite coefficient or coordinate, negative thresholds, a
 * shell_order that is not a permutation, and a grid whose points belong to
 * atoms the molecule does not have. */
kldi_status kldi_screen(const kldi_grid* grid, const kldi_molecule* mol, const kldi_basis* basis,
                        const kldi_options* opt, kldi_plan** out);

kldi_status kldi_plan_info(const kldi_plan* plan, kldi_plan_stats* stats);

/* Export the retained lists for inspection: blk_ptr[nblocks+1] and
 * blk_idx[retained] (ascending basis-block indices per grid block) and the
 * summaries bmax[retained] (FP64).  Host buffers; any may be NULL. */
kldi_status kldi_plan_export_lists(const kldi_plan* plan, int32_t* blk_ptr, int32_t* blk_idx, double* bmax);

/* Density (Eq. r_equals_dphi then the row-dot of App. A): rho[npoints] and,
 * for a GGA plan, grad[npoints*3] (may be NULL for LDA).  D is nbf x nbf,
 * symmetric (only its values are used as given; no symmetrisation).  rho and
 * grad are both device or both host memory, else KLDI_EINVAL before any work. */
kldi_status kldi_density(kldi_plan* plan, const double* D, double* rho, double* grad);

/* Potential from a given density: E_xc (one double) and V[nbf*nbf]
 * (overwritten, symmetric) for functional xc; grad may be NULL for LDA. */
kldi_status kldi_vxc(kldi_plan* plan, int xc, const double* rho, const double* grad, double* V,
                     double* Exc);

/* The fused hot path: D -> rho (grad rho) -> functional -> E_xc and V. */
kldi_status kldi_exc(kldi_plan* plan, int xc, const double* D, double* V, double* Exc);

/* Many molecules / frames of uneven size in one call: plans[k], D[k], V[k]
 * and Exc[k] for k < nframes, captured into one CUDA graph (kldi_batch_*)
 * and run as one launch on the first plan's stream; synchronises.  Device
 * pointers only (KLDI_EINVAL otherwise). */
kldi_status kldi_exc_batched(kldi_plan* const* plans, int nframes, int xc, const double* const* D,
                             double* const* V, double* Exc);

/* Nuclear gradient of E_xc (the paper's energy + gradient workload, Sec. IV),
 * on the fixed grid (no grid-weight response), through the basis centres:
 *   dE/dR_A = -2 sum_{mu on A} sum_i [grad chi_mu Q_mu,i + (b_i . grad grad chi_mu) R_mu,i],
 *   R = Phi D, Q = Z D over the executed pairs E1_g,
 *   Z = w v_rho chi + 2 w v_sigma grad rho . grad chi, b = 2 w v_sigma grad rho.
 * G[natm*3] (row-major per atom, bohr, Hartree/bohr) and Exc[1]: each host or
 * device memory.  D as in kldi_exc.  FP64 plans use the FP64 block form;
 * BF16X3 / BF16X6 / BF16X10 plans run R and Q through the tensor-core density product
 * (Z sliced per point like Phi) and contract them with FP32 first and second
 * basis derivatives, one FP64 atomic per atom, component and warp (summation
 * order, hence the last bits, vary between calls).  KLDI_EUNSUPPORTED for a
 * tensor-core plan whose basis has a 32-function block with more than 40 shells
 * or 80 primitives.  The V product is not evaluated. */
kldi_status kldi_exc_grad(kldi_plan* plan, int xc, const double* D, double* G, double* Exc);

/* Stages of one evaluation, for kldi_plan_stage_times. */
typedef enum {
  KLDI_STAGE_DPREP = 0,   /* D block maxima (and slicing for tensor modes)        */
  KLDI_STAGE_PHI = 1,     /* basis values Phi of the retained tiles                */
  KLDI_STAGE_RHO = 2,     /* density product R = Phi D and the row-dot            */
  KLDI_STAGE_XC = 3,      /* functional, E_xc partial sums                         */
  KLDI_STAGE_X = 4,       /* X tiles (and the V-product operands)                  */
  KLDI_STAGE_V = 5,       /* potential product                                     */
  KLDI_STAGE_FINISH = 6,  /* E_xc reduction, V symmetrisation                      */
  KLDI_NSTAGES = 7
} kldi_stage;

/* Per-stage device timing with CUDA events on the plan's stream.  enable = 1
 * starts recording (and clears earlier records), 0 stops.  Recording adds two
 * event records per stage and batch; it allocates its events here, not in the
 * compute calls (at most 4096 stage records are kept per reset). */
kldi_status kldi_plan_profile(kldi_plan* plan, int enable);

/* Synchronise the plan's stream and return, per kldi_stage, the summed device
 * time in milliseconds (ms[KLDI_NSTAGES]) and the number of kernel launches
 * (launches[KLDI_NSTAGES]) recorded since kldi_plan_profile(plan, 1); either
 * pointer may be NULL.  Host buffers. */
kldi_status kldi_plan_stage_times(kldi_plan* plan, double* ms, int64_t* launches);

/* E_xc = sum_i w_i f(rho_i, sigma_i) of a density already on the device, for
 * callers that must not allocate device memory.  The paper has no
 * counterpart: this is an interface addition.  Callers that cannot allocate
 * include code running while a stream is captured into a CUDA graph (an
 * allocation cannot be captured), hosts that reserve all device memory up
 * front, and allocator callbacks that must not re-enter the allocator.
 *   xc: KLDI_XC_LDA_X or KLDI_XC_PBE; npoints points; rho[npoints],
 *   grad[npoints*3] (PBE only, may be NULL for LDA), w[npoints]: device
 *   arrays, FP64; points with rho < rho_min contribute nothing; Exc: one
 *   device double, written; stream: a cudaStream_t or NULL.
 * The per-block partial sums live in a fixed device array of 65536 slots, so
 * npoints may be at most 8,388,608 (KLDI_EINVAL beyond, and for host
 * pointers).  Allocates nothing and returns after enqueueing.  The first call
 * on a device resolves the array's address; make it outside stream capture.
 * Calls whose work overlaps on one GPU share the array and race. */
kldi_status kldi_exc_energy_noalloc(int xc, int64_t npoints, const double* rho, const double* grad,
                                    const double* w, double rho_min, double* Exc, void* stream);

/* ---- Many frames: shared workspace, tuning, one graph launch ------------
 * The paper runs many molecules and trajectory frames through the same
 * integration (Sec. IV; its multi-GPU pull scheduler, Sec. III-E, balances
 * their uneven sizes).  Here the frames share one device workspace for the
 * per-tile buffers, a tuner picks the V work decomposition, and all frames'
 * launches are captured into one CUDA graph that runs as one launch. */
typedef struct kldi_workspace kldi_workspace;

/* Device arena of `bytes` bytes for the per-tile buffers of any number of
 * plans on the current device.  Plans sharing it must not run concurrently
 * (use one stream, or one batch). */
kldi_status kldi_workspace_create(int64_t bytes, kldi_workspace** out);
void kldi_workspace_free(kldi_workspace* ws);

/* Use `ws` for the plan's per-tile buffers (NULL: the plan's own, sized from
 * free memory, allocated at the next compute call).  The grid blocks are
 * regrouped into batches that fit the workspace; KLDI_EINVAL if one grid
 * block's tiles do not fit.  Free the workspace after the plans. */
kldi_status kldi_plan_set_workspace(kldi_plan* plan, const kldi_workspace* ws);

/* Tunable shapes of the tensor-core products.
 * v_seg: the V product's decomposition: the grid blocks are cut into ranges
 * of v_seg consecutive blocks, a work item is one pair of 128-function
 * windows over the blocks of one range in its list, and items run range by
 * range (so concurrent items share the range's tiles in L2); 0 chooses 64.
 * rho_ntile: the density product's N tile, 128 functions (four basis
 * blocks, one TMEM buffer of the level accumulators for BF16X6) or 64 (two
 * basis blocks, two buffers, so the drains overlap the next tile's products,
 * and less padding where few blocks of a tile have executed pairs); 0 chooses
 * the mode's default (128; BF16X10 has only 64).
 * v_align: the V product's windows of 4 consecutive basis blocks start at
 * multiples of v_align blocks (4: fixed 128-function tiles; 2; 1: the
 * fewest windows that cover each grid block's retained blocks, hence the
 * fewest zero blocks in the products, but more distinct window pairs and so
 * shorter work items); 0 chooses 2. */
typedef struct {
  int v_seg;
  int rho_ntile;
  int v_align;
} kldi_tuning;

kldi_status kldi_plan_set_tuning(kldi_plan* plan, const kldi_tuning* tuning);
kldi_status kldi_plan_get_tuning(const kldi_plan* plan, kldi_tuning* tuning);

/* Time kldi_exc(plan, xc, D) (D on the device) with CUDA events over the
 * candidate tunings, `reps` timed calls each after one warm-up, and keep the
 * fastest on the plan: first the density product's N tile (128 and 64
 * functions for BF16X3 / BF16X6) at the default V decomposition, then the V
 * window alignment in {2, 4, 1}, then v_seg in {16, 32, 64, 128, 256} with
 * the chosen tile and alignment.  best (host, may be NULL) receives it, best_ms (host,
 * may be NULL) its mean time per call in milliseconds.  Overwrites the
 * plan's scratch outputs; synchronises. */
kldi_status kldi_plan_autotune(kldi_plan* plan, int xc, const double* D, int reps, kldi_tuning* best,
                               double* best_ms);

/* Restrict the plan to grid blocks [g0, g1) (0 <= g0 <= g1 <= nblocks): the
 * compute calls then produce this range's partial E_xc and V (and write rho
 * only on its points), so ranks holding complementary ranges sum to the full
 * result -- the one exchange step of the multi-GPU form (the paper's grid
 * blocks are independent work units, Sec. III-E).  (0, nblocks) restores
 * the whole grid. */
kldi_status kldi_plan_set_block_range(kldi_plan* plan, int64_t g0, int64_t g1);

typedef struct kldi_batch kldi_batch;

/* Capture kldi_exc for every frame k (plans[k], D[k] -> V[k], Exc[k]; all
 * device pointers, all plans on this device) into one CUDA graph, frames in
 * order, on `stream` (a cudaStream_t; NULL: a stream the batch creates).
 * Tile buffers are prepared before capture; the captured work allocates
 * nothing.  The pointers are baked into the graph: keep them valid. */
kldi_status kldi_batch_create(kldi_plan* const* plans, int nframes, int xc, const double* const* D,
                              double* const* V, double* Exc, void* stream, kldi_batch** out);

/* One graph launch of the whole batch on its stream (asynchronous). */
kldi_status kldi_batch_launch(kldi_batch* batch);

/* Synchronise the batch's stream and report a device-side error of its last
 * launch. */
kldi_status kldi_batch_sync(kldi_batch* batch);
void kldi_batch_free(kldi_batch* batch);

/* ---- Learned functional ------------------------------------------------
 * A 2 -> 64 -> 64 -> 2 MLP surrogate of the per-point GGA functional, the
 * evaluation that sits between the density product and the V product (Sec.
 * III-F; Eq. exc_quadrature gives the potential v_i it must supply).  The
 * paper has no learned part; the network is this project's addition:
 *   inputs  z = ((ln rho, ln max(sigma, 1e-30)) - centre) / half-width of the
 *           training box box[4] = {lo, hi of ln rho, lo, hi of ln sigma};
 *   layers  h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3;
 *   outputs f = e0(rho) o1, v_rho = v0(rho) o2 (e0, v0: Slater exchange and its
 *           derivative), v_sigma = e0 (d o1 / d z2) / (half-width_2 sigma);
 *   points outside the box use the analytic PBE-form functional; points with
 *   rho < rho_min contribute nothing.
 * Parameters (KLDI_MLP_NPARAMS floats, FP32 master copy): W1 [64][2], b1[64],
 * W2 [64][64] (row = output unit), b2[64], W3 [2][64], b3[2].  The forward
 * pass uses their FP16 values with FP32 arithmetic. */
#define KLDI_MLP_NPARAMS 4482
typedef struct kldi_mlp kldi_mlp;

typedef struct {
  int epochs;          /* passes over the training points                     */
  int batch;           /* points per Adam step (1 .. 65536)                   */
  double lr0, lr1;     /* learning rate: cosine schedule from lr0 to lr1      */
  double beta1, beta2, eps;   /* Adam                                         */
  double rho_min;      /* points with rho < rho_min or outside the box are not
                          trained on                                          */
  void* stream;        /* cudaStream_t or NULL                                */
} kldi_train_options;

/* New network with parameters params[KLDI_MLP_NPARAMS] (host or device, FP32)
 * and training box box[4] (host).  Owns its device memory. */
kldi_status kldi_mlp_create(const float* params, const double* box, kldi_mlp** out);

/* Copy the FP32 master parameters to params[KLDI_MLP_NPARAMS] (host). */
kldi_status kldi_mlp_get_params(const kldi_mlp* mlp, float* params);

/* Training checkpoint (the learned part's state; the paper has no
 * counterpart): state[3 * KLDI_MLP_NPARAMS] (host, FP32) holds the FP32
 * master parameters, then Adam's first and second moments; *step the Adam
 * steps taken.  kldi_mlp_set_state restores all of them (and the FP16 copy the
 * evaluation kernels read), so that training resumes bit for bit; the box is
 * the one the network was created with.  Both synchronise; KLDI_EINVAL for a
 * null argument or a negative step. */
kldi_status kldi_mlp_get_state(const kldi_mlp* mlp, float* state, int64_t* step);
kldi_status kldi_mlp_set_state(kldi_mlp* mlp, const float* state, int64_t step);

/* Mean loss over the valid points of (rho[n], sigma[n]) (host or device,
 * FP64) of (o1 - F*)^2 + (o2 - G*)^2 with F* = f / e0, G* = v_rho / v0 of the
 * analytic PBE-form functional, and its gradient grad[KLDI_MLP_NPARAMS]
 * (host, FP32); *loss (host).  Synchronises. */
kldi_status kldi_mlp_loss_grad(kldi_mlp* mlp, const double* rho, const double* sigma, int64_t n,
                               double rho_min, float* grad, float* loss);

/* One Adam step with gradient grad[KLDI_MLP_NPARAMS] (host or device, FP32),
 * learning rate lr; the step counter is kept by the network. */
kldi_status kldi_mlp_adam_step(kldi_mlp* mlp, const float* grad, double lr, double beta1, double beta2,
                               double eps);

/* Train on the GPU: per epoch one pass over all n points in a fixed
 * pseudo-random order (an affine permutation of the indices, new offset per
 * epoch), one Adam step per batch.  rho, sigma: host or device, FP64.
 * loss_per_epoch[epochs] (host, may be NULL): mean batch loss of each epoch.
 * Synchronises. */
kldi_status kldi_mlp_train(kldi_mlp* mlp, const double* rho, const double* sigma, int64_t n,
                           const kldi_train_options* opt, float* loss_per_epoch);

/* Evaluate the surrogate (with its fallback) at n points: f, vrho, vsigma
 * (FP64) and used[n] (1 where the network was used, int32), all host or all
 * device (used may be NULL; a mix is KLDI_EINVAL before any work).
 * Synchronises for host outputs. */
kldi_status kldi_mlp_eval(const kldi_mlp* mlp, const double* rho, const double* sigma, int64_t n,
                          double rho_min, double* f, double* vrho, double* vsigma, int32_t* used);

/* Attach a network to a GGA plan: kldi_vxc / kldi_exc with KLDI_XC_MLP then
 * evaluate it between the two products (fused into the functional kernel).
 * The plan keeps a reference: free the network after the plan or detach it
 * with mlp = NULL. */
kldi_status kldi_plan_set_mlp(kldi_plan* plan, const kldi_mlp* mlp);

void kldi_mlp_free(kldi_mlp* mlp);

/* Switch the product arithmetic of an existing plan (kldi_prec). */
kldi_status kldi_plan_set_precision(kldi_plan* plan, int prec);

/* ---- Bounded device waits (failure detection without a GPU fault) --------
 * Every wait of the tensor-core kernels on an mbarrier (a copy that has not
 * landed, a product not finished, a consumer not done) gives up after `ns`
 * nanoseconds of the GPU's global timer (default 2e9), records a code in the
 * plan's device error word and stops the kernel's other roles; the kernel
 * still waits for its own copies and products in flight and frees its tensor
 * memory before it exits.  The compute call then returns KLDI_ETIMEOUT (when
 * it synchronises; otherwise the next synchronising call on the plan does)
 * and the plan stays usable.  ns = 0 restores the default. */
kldi_status kldi_plan_set_wait_limit(kldi_plan* plan, uint64_t ns);

/* Test hook of the timeout path: the tensor-core V product does not hand out
 * work item `item` (0-based, in the order its CTAs take items) to its
 * consumers, whose bounded wait then runs out; nothing is in flight for that
 * item.  -1 (the default) turns it off. */
kldi_status kldi_plan_set_withhold(kldi_plan* plan, int64_t item);

/* Self-test of the bounded wait: one CTA waits `limit_ns` nanoseconds on an
 * mbarrier at which, with arrive = 0, nothing arrives (nothing else in
 * flight); returns KLDI_ETIMEOUT, or KLDI_OK when arrive = 1.  Synchronises
 * `stream` (a cudaStream_t, NULL = legacy default stream). */
kldi_status kldi_selftest_wait(uint64_t limit_ns, int arrive, void* stream);

void kldi_plan_free(kldi_plan* plan);
void kldi_grid_free(kldi_grid* grid);
const char* kldi_last_error(void);

/* Version string of the library build. */
const char* kldi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KLDI_H */
