/*
 * mg.h -- C ABI of the GB300 (sm_103a) masked-domain multigrid Poisson solver.
 *
 * Method: Guillet & Teyssier, "A Simple Multigrid Scheme for Solving the
 * Poisson Equation with Arbitrary Domain Boundaries", arXiv:1104.1703.
 * The library solves Laplacian(Phi) = rho on the active cells of one AMR
 * level inside a Cartesian box, with Dirichlet values on the outer faces of
 * the active domain (Section 2, problem statement; Fig. 1), by multigrid
 * iterations (Section 2 recipe) with red-black Gauss-Seidel smoothing, R1
 * restriction and P2 prolongation (Fig. 3), the mask-based second-order
 * boundary reconstruction (Section 3, Fig. 5), the first-order coarse fix
 * for sub-cell boundary features (Section 4) and its run-time switch
 * (Section 4, threshold eta).
 *
 * Conventions for every entry point:
 *  - Grids are cell centred, x fastest: element (i, j, k) of an nx*ny*nz array
 *    is at index (k*ny + j)*nx + i.  Cell (i,j,k) has its centre at
 *    ((i+1/2)h, (j+1/2)h, (k+1/2)h).
 *  - `where` says whether a pointer is host memory (MG_MEM_HOST, any pageable
 *    or pinned host pointer) or device memory of the hierarchy's GPU
 *    (MG_MEM_DEVICE).  An MG_MEM_DEVICE pointer that is not device (or
 *    managed) memory of that GPU is refused with MG_ERR_INVALID_ARG before
 *    any copy or launch.  The caller owns every buffer it passes; the library
 *    copies what it needs before returning and never keeps a caller pointer.
 *    All library memory is device memory owned by the hierarchy.
 *  - Work is issued on the hierarchy's CUDA stream.  Calls that return host
 *    data (solve, norms, copies to MG_MEM_HOST) synchronise that stream; calls
 *    that write device data into caller buffers (MG_MEM_DEVICE) are ordered
 *    on the stream and complete asynchronously.
 *  - Values at inactive cells are ignored on input and written as 0 on output.
 *  - Every call returns an mg_status; nothing is thrown across the ABI.  On
 *    error mg_last_error() describes the failure.  A hierarchy stays usable
 *    after MG_ERR_NOT_CONVERGED and MG_ERR_DIVERGED; after MG_ERR_CUDA the
 *    CUDA context may be unusable.
 *  - One hierarchy must not be used from two host threads at once.
 */
#ifndef GBMG_MG_H
#define GBMG_MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_hierarchy mg_hierarchy; /* opaque, library-owned */

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,   /* bad pointer, size, option or level index */
  MG_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  MG_ERR_OOM = 3,           /* device allocation failed; nothing leaked */
  MG_ERR_EMPTY_DOMAIN = 4,  /* the mask has no active cell */
  MG_ERR_NOT_CONVERGED = 5, /* max_cycles reached above the tolerance */
  MG_ERR_DIVERGED = 6,      /* a residual norm became non-finite */
  MG_ERR_INTERNAL = 7
} mg_status;

typedef enum { MG_MEM_HOST = 0, MG_MEM_DEVICE = 1 } mg_mem;

/* Parameters of the multigrid iteration.
 *  n_pre, n_post   Gauss-Seidel sweeps before and after the coarse correction
 *                  (Section 2, recipe steps 1 and 8; the paper uses 2 and 2).
 *  n_cycles        coarse iterations per level, 1..4: 1 = V-cycle, 2 =
 *                  W-cycle, 3 and 4 the deeper recursions of Section 5.3
 *                  (N_cycles).
 *  coarse_sweeps   red-black sweeps on the deepest level that has an active
 *                  cell (the paper does not specify the coarsest solve).
 *  order           0 = automatic switch (start in second order, Section 4),
 *                  1 = always first order on coarse levels, 2 = always second.
 *  eta             switch threshold on ||r_{n+1}|| / ||r_n|| (Section 4; 0.5).
 *  hold_solves     solves that stay in first order after a switch
 *                  (Section 4: "for the next 10 solves").
 *  use_graphs      1 = replay each V-cycle from a captured CUDA graph.
 *  precision       0 = the method in FP64 throughout; 1 = mixed: each
 *                  multigrid iteration is the paper's V-cycle run in FP32 on
 *                  the error equation A e = b - A Phi, inside FP64 iterative
 *                  refinement (the residual, its norm, the update Phi += e
 *                  and the folded boundary data stay FP64).  The paper has
 *                  no counterpart; the stopping test and the order switch
 *                  act on the FP64 residual norms as in FP64 mode.
 *  inner_cycles    FP32 V-cycles per refinement step (precision 1), 1..16.
 *                  The stopping test and the switch act once per step; the
 *                  switch compares the step's residual ratio with
 *                  eta^inner_cycles (eta per multigrid iteration).
 *  coarse_cluster  1 = run the middle coarse levels (4096 to 131072 cells per
 *                  colour) and the bottom levels of a V-cycle as one launch of
 *                  one thread-block cluster; 0 = one launch per step (faster
 *                  on GB300: the replayed graph pipelines the launches, while
 *                  each cluster-wide step costs a barrier).  The results are
 *                  the same.
 *  smoother_pass   mixed form: 1 = run each pair of FP32 Gauss-Seidel sweeps
 *                  of the fine level (N_pre = N_post = 2 is one pair) as one
 *                  temporal-blocked pass over the level (a z-wavefront over
 *                  tiles staged in shared memory); 0 = four list half-sweeps
 *                  (faster on GB300: the pass moves fewer bytes but waits on
 *                  its chain of barrier-separated stages).  The results are
 *                  bit-identical.
 *  fp64_sum        level-0 FP64 kernels (the FP64 form's Gauss-Seidel
 *                  sweeps, residual norms and residual + restriction, and
 *                  the mixed form's FP64 residual): 1 = form each cell's sum
 *                  of its six neighbour values in 64-bit integer arithmetic
 *                  (exponent-aligned fixed point, rounded once to the
 *                  nearest double; subnormal values count as zero), so that
 *                  a sweep's update issues one FP64 instruction instead of
 *                  six; 0 = five FP64 additions.  Both are accurate to about
 *                  one rounding of the sum; the results differ in the last
 *                  bits.
 *  fine_segments   mixed form, level-0 FP32 Gauss-Seidel sweeps: 1, 2 = one
 *                  thread per slot of the row segments (8, 16 slots of one
 *                  colour's half-row) that hold an active cell, so that a
 *                  warp reads whole runs of every array; 3 = 16-slot
 *                  segments with two consecutive slots per thread (8-byte
 *                  loads); 0 = one thread per active cell of the colour's
 *                  compact list.  The results are bit-identical.  (The FP64
 *                  sweeps always use the cell lists.)
 *  coarse_matrix   1 = solve the coarsest level, when it has at most 64
 *                  unknowns and runs inside the one-CTA bottom cycle, through
 *                  the precomputed affine map of its coarse_sweeps red-black
 *                  sweeps (built once per mask, one launch): a small
 *                  matrix-vector product instead of 2 * coarse_sweeps
 *                  dependent half-sweeps per visit, the same result up to
 *                  rounding; 0 = the sweeps.  (Batched patches use the
 *                  sweeps.) */
typedef struct {
  int n_pre, n_post, n_cycles, coarse_sweeps, hold_solves;
  double eta;
  int order;
  int use_graphs;
  int precision;
  int inner_cycles;
  int coarse_cluster;
  int smoother_pass;
  int fp64_sum;
  int fine_segments;
  int coarse_matrix;
} mg_options;

#define MG_HIST_MAX 256

/* Result of mg_solve.  hist[n] = ||r_n|| for n = 0..min(cycles, MG_HIST_MAX)
 * with r_0 the residual of the initial guess; r_zero = ||r(Phi = 0)|| is the
 * reference of the relative residual rel = ||r_final|| / r_zero.  Norms are
 * unscaled L2 norms of r = Laplacian(Phi) - rho over the active fine cells. */
typedef struct {
  int cycles;     /* multigrid iterations performed (mixed form: refinement steps) */
  int order_used; /* coarse reconstruction order at exit (1 or 2) */
  int switched;   /* 1 if this solve switched from second to first order */
  int status;     /* the mg_status returned by mg_solve */
  long long cell_updates; /* Gauss-Seidel updates of active cells, all levels */
  double r_zero, r_init, r_final, rel;
  double hist[MG_HIST_MAX + 1];
} mg_solve_info;

/* Fills *opt with the paper's parameters: n_pre = n_post = 2, n_cycles = 1,
 * coarse_sweeps = 50, hold_solves = 10, eta = 0.5, order = 0, use_graphs = 1,
 * precision = 0 (FP64), inner_cycles = 1, coarse_cluster = 0, smoother_pass = 0,
 * fp64_sum = 1, fine_segments = 3, coarse_matrix = 1. */
void mg_default_options(mg_options* opt);

/* Builds the multigrid hierarchy of one AMR level (Section 2, Fig. 2):
 * levels of size ceil(n/2) down to at most 2 cells per axis, the mask
 * averaged recursively (Section 3; kept as exact integer sums of the +1/-1
 * colours), the per-level active sets of both reconstruction orders and the
 * modified-Laplacian diagonals (Sections 3 and 4).
 *  mask         nx*ny*nz int8: > 0 active, <= 0 inactive (Omega = {m > 0}).
 *  nx, ny, nz   1..2048 each, and (nz+2)*(ny+2)*pitch < 2^31 with pitch =
 *               (nx+1)/2 + 1 rounded up to 8: each colour array of the padded
 *               red/black layout must hold fewer than 2^31 elements (about
 *               1600^3 cells for a cube); larger grids return INVALID_ARG.
 *  h            fine cell size, > 0.
 *  opt          NULL for mg_default_options.
 *  cuda_stream  a cudaStream_t of the current device, or NULL for a stream
 *               the library creates (and destroys with the hierarchy); that
 *               stream synchronises with the legacy default stream.
 *  out          receives the new hierarchy (NULL on failure).
 * The solution starts at 0, rho at 0 and the Dirichlet values at 0.
 * Errors: INVALID_ARG, EMPTY_DOMAIN (no active cell), OOM, CUDA. */
mg_status mg_create_hierarchy(const int8_t* mask, mg_mem where, int nx, int ny, int nz, double h,
                              const mg_options* opt, void* cuda_stream, mg_hierarchy** out);

/* Rebuilds the mask hierarchy for a new mask of the same dimensions without
 * reallocating (the AMR level changed shape).  The solution is reset to 0
 * and the right-hand side and Dirichlet values must be set again.
 * Errors: INVALID_ARG, EMPTY_DOMAIN (the previous mask stays in force), CUDA. */
mg_status mg_update_mask(mg_hierarchy* hier, const int8_t* mask, mg_mem where);

/* Releases every device buffer, graph and (if library-created) the stream.
 * NULL is accepted. */
mg_status mg_destroy_hierarchy(mg_hierarchy* hier);

/* rho: nx*ny*nz doubles, the right-hand side of Laplacian(Phi) = rho
 * (Section 1, Poisson equation).  Errors: INVALID_ARG, CUDA. */
mg_status mg_set_rhs(mg_hierarchy* hier, const double* rho, mg_mem where);

/* Dirichlet values on the faces of the fine level (Fig. 1: the boundary
 * conditions live at the border cell faces).
 *  bx  (nx+1)*ny*nz: value on the x-face between cells (i-1,j,k) and (i,j,k),
 *      at index (k*ny + j)*(nx+1) + i, centred at (i h, (j+1/2) h, (k+1/2) h);
 *  by  nx*(ny+1)*nz, index (k*(ny+1) + j)*nx + i;  bz nx*ny*(nz+1), index
 *      (k*ny + j)*nx + i with k in 0..nz.
 * Only faces between an active cell and an inactive or out-of-box cell are
 * read.  A NULL array means 0 on that face family.
 * Errors: INVALID_ARG, CUDA. */
mg_status mg_set_dirichlet(mg_hierarchy* hier, const double* bx, const double* by, const double* bz,
                           mg_mem where);

/* One-way interface (Section 1; Fig. 1 caption): the Dirichlet values are
 * linearly (trilinearly) interpolated, at each boundary face centre, from
 * the solution of the coarser AMR level.
 *  phi_c        cnx*cny*cnz doubles, the coarse-level potential, cell size 2h.
 *  ox, oy, oz   lower corner of coarse cell (0,0,0) in fine-cell units: the
 *               coarse cell (I,J,K) spans [ox+2I, ox+2I+2] x ... so its
 *               centre is at ox+2I+1.  Typical: -2 (one coarse ghost cell).
 * Errors: INVALID_ARG (including a boundary face outside the coarse centres),
 * CUDA. */
mg_status mg_set_dirichlet_from_coarse(mg_hierarchy* hier, const double* phi_c, mg_mem where, int cnx,
                                       int cny, int cnz, int ox, int oy, int oz);

/* The values mg_set_dirichlet_from_coarse would fold, as face arrays in
 * mg_set_dirichlet's layout: each boundary face of the hierarchy's active
 * domain gets the coarse potential trilinearly interpolated at its centre
 * (Section 1 one-way interface); every other face is 0.  bx, by, bz are
 * device buffers of the hierarchy's GPU ((nx+1) ny nz, nx (ny+1) nz,
 * nx ny (nz+1) doubles).  Errors: INVALID_ARG (including a boundary face
 * outside the coarse cell centres), CUDA. */
mg_status mg_faces_from_coarse(mg_hierarchy* hier, const double* phi_c, mg_mem where, int cnx, int cny, int cnz, int ox,
                               int oy, int oz, double* bx, double* by, double* bz);

/* Initial guess (NULL = 0) and read-back of the fine solution, nx*ny*nz.
 * Errors: INVALID_ARG, CUDA. */
mg_status mg_set_solution(mg_hierarchy* hier, const double* phi, mg_mem where);
mg_status mg_get_solution(mg_hierarchy* hier, double* phi, mg_mem where);

/* One multigrid iteration (Section 2 recipe, applied recursively N_cycles
 * times per level) in the current order (option order 1 or 2; for order 0,
 * first order while the hold counter is positive, else second order).  No
 * order switching happens here.  rel_residual_out (nullable) receives
 * ||r|| / ||r(Phi = 0)|| after the iteration; passing NULL keeps the call
 * asynchronous.  Errors: CUDA, DIVERGED (non-finite norm). */
mg_status mg_vcycle(mg_hierarchy* hier, double* rel_residual_out);

/* Iterates until ||r_n|| / ||r(Phi = 0)|| < tol (relative residual, Section
 * 5.2 measures the reduction from a zero first guess), with the run-time
 * order switch of Section 4 when option order = 0: a solve starts in second
 * order unless the hold counter is positive (then first order, counter - 1);
 * when ||r_n|| / ||r_{n-1}|| > eta it switches to first order for the rest of
 * the solve and for the next hold_solves solves.  On a switch the iterate is
 * kept unless its residual exceeds the initial one, in which case the
 * initial guess is restored.  The ratio test is skipped once ||r_n|| <
 * 100 * DBL_EPSILON * ||r(0)||.  If rho and the Dirichlet values are all 0 the
 * solution is set to 0 and the call returns at once.
 *  tol > 0, max_cycles >= 0; info nullable.
 * Errors: INVALID_ARG, NOT_CONVERGED (the best iterate is kept), DIVERGED,
 * CUDA. */
mg_status mg_solve(mg_hierarchy* hier, double tol, int max_cycles, mg_solve_info* info);

/* ||r|| and ||r(Phi = 0)|| (unscaled L2 over the active fine cells) for the
 * current solution.  Either output may be NULL.  Errors: CUDA. */
mg_status mg_residual_norm(mg_hierarchy* hier, double* norm_out, double* norm_zero_out);

/* 1 if the fine level's FP32 sweeps run as temporal-blocked passes (mixed
 * form with option smoother_pass on a fine level larger than the one-CTA
 * smoother's, and the GPU accepted the pass's tensor maps), else 0. */
mg_status mg_get_smoother_pass(const mg_hierarchy* hier, int* active);

/* Order-switch state: solves left in forced first order. */
mg_status mg_get_hold(const mg_hierarchy* hier, int* hold);
mg_status mg_set_hold(mg_hierarchy* hier, int hold);

/* Message of the last failed call on this hierarchy, or of the last failed
 * create on this thread when hier is NULL.  Never NULL. */
const char* mg_last_error(const mg_hierarchy* hier);
const char* mg_status_string(mg_status status);

/* ---------------------------------------------------------------------------
 * Level access.  These expose the individual steps of the Section 2 recipe
 * on one level of the hierarchy, for verification and for callers that
 * drive their own schedule.  Level 0 is the fine level.
 * ------------------------------------------------------------------------- */

/* Number of levels built, and the deepest level with an active cell in
 * second (deepest2) and first (deepest1) order.  Any output may be NULL. */
mg_status mg_num_levels(const mg_hierarchy* hier, int* nlev, int* deepest2, int* deepest1);

/* dims3 receives {nx, ny, nz} of the level; active2/active1 the number of
 * unknowns in second and first order (Omega^l = {m > 0}, Section 3; cells
 * with m = 1, Section 4).  Outputs nullable. */
mg_status mg_level_info(const mg_hierarchy* hier, int level, int* dims3, long long* active2,
                        long long* active1);

/* Fields of a level, in natural x-fastest layout of the level's dimensions:
 *  MG_FIELD_PHI     double  level 0: Phi; level >= 1: the correction dPhi
 *  MG_FIELD_RHS     double  the right-hand side scaled by the level's cell
 *                           size squared: level 0 h^2 rho minus the folded
 *                           Dirichlet terms, level l >= 1 h_l^2 times the
 *                           coarse right-hand side -R(r)
 *  MG_FIELD_MASKSUM int32   sum of the +1/-1 fine colours under each cell
 *                           (m_l = S / 8^l; Section 3)
 *  MG_FIELD_INVDIAG double  1 / D of the second-order operator, D the sum
 *                           over the six faces of 1 (active neighbour) or
 *                           1/theta (ghost) (Section 3), 0 on inactive cells
 * mg_level_set accepts MG_FIELD_PHI and MG_FIELD_RHS only. */
enum { MG_FIELD_PHI = 0, MG_FIELD_RHS = 1, MG_FIELD_MASKSUM = 2, MG_FIELD_INVDIAG = 3 };
mg_status mg_level_get(mg_hierarchy* hier, int level, int field, void* out, mg_mem where);
mg_status mg_level_set(mg_hierarchy* hier, int level, int field, const void* in, mg_mem where);

/* Recipe step 1/8 on one level: `sweeps` red-black Gauss-Seidel sweeps
 * (red = (i+j+k) even first) in the given order (1 or 2).  Inactive cells
 * are not touched.  Errors: INVALID_ARG, CUDA. */
mg_status mg_level_smooth(mg_hierarchy* hier, int level, int order, int sweeps);

/* Recipe steps 2-5 on one level: the residual of level `level` is restricted
 * by R1 into the right-hand side of level+1 (as -R(r)) and the correction of
 * level+1 is zeroed.  The residual is taken at every active cell.
 * Errors: INVALID_ARG (no coarser level), CUDA. */
mg_status mg_level_restrict(mg_hierarchy* hier, int level, int order);

/* Recipe steps 6-7 on one level: Phi_level += P2(dPhi_{level+1}) on the
 * active cells of `level` in the given order.  Errors: INVALID_ARG, CUDA. */
mg_status mg_level_prolong(mg_hierarchy* hier, int level, int order);

/* ---------------------------------------------------------------------------
 * Allocation-free residual norm
 * ------------------------------------------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory.  Examples are AMR codes and frameworks
 * that reserve the GPU's memory up front in their own pool, where a
 * cudaMalloc outside the pool can fail, and host code that must not block
 * on the allocator.  It computes ||r|| = ||Laplacian(Phi) - rho||_2 over the
 * active cells of a fine level, with the same operator, boundary treatment
 * and norm as mg_residual_norm, directly from the caller's device buffers,
 * with no hierarchy and no allocation of any kind (no cudaMalloc, cudaFree
 * or allocating library call).
 *  mask, phi, rho   device, nx*ny*nz, natural layout (as mg_create_hierarchy,
 *                   mg_set_solution and mg_set_rhs); values of phi and rho on
 *                   inactive cells are ignored.
 *  bx, by, bz       device face arrays as in mg_set_dirichlet; NULL = 0.
 *  nx, ny, nz       1..2048 each; larger sizes return MG_ERR_INVALID_ARG.
 *  h                fine cell size, > 0.
 *  norm_out         device pointer to one double that receives ||r||.
 *  cuda_stream      stream of the current device (NULL: legacy default).
 * The work is enqueued on the stream and the call returns without waiting;
 * norm_out is valid once the stream reaches that point.  Scratch: 4096
 * doubles (32 KB) of static device memory in the library, which every GPU
 * that loads the library holds until the process exits.  Each call looks up
 * that array's device address (cudaGetSymbolAddress); the first call on a
 * device also loads the library's kernels for it, so make the first call on
 * each device before any stream capture.  All calls on a device share the
 * array: calls that can overlap on the GPU (different streams, no ordering
 * between them) race on it and must be serialised by the caller.
 * Errors (mg_last_error(NULL)): INVALID_ARG, CUDA. */
mg_status mg_residual_norm_noalloc(const int8_t* mask, const double* phi, const double* rho, const double* bx,
                                   const double* by, const double* bz, int nx, int ny, int nz, double h,
                                   double* norm_out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched solve of many independent patches
 *
 * An AMR level is made of many patches of uneven size, each with its own
 * mask and its own Dirichlet values from the coarser level (Section 2
 * problem statement, one per patch; Fig. 1).  A batch owns one hierarchy per
 * patch and runs the multigrid iteration of all of them together: one
 * launch per step of the Section 2 recipe covers that level of every patch,
 * the small coarse levels of each patch run as a one-CTA V-cycle (one CTA
 * per patch, all patches in one launch), and one cycle of the whole batch is
 * replayed from a CUDA graph.  Each patch keeps its own convergence test,
 * order switch and hold counter (Section 4), with the same decisions as
 * mg_solve on that patch alone.  FP64 only, V-cycles only (options
 * precision = 0, n_cycles = 1).
 * ------------------------------------------------------------------------- */

typedef struct mg_batch mg_batch; /* opaque, library-owned */

/* Launch parameters of a batch (results do not depend on them, except the
 * smoother schedule n_pre / n_post, which is part of the method):
 *  threads          threads per block of the chunked kernels: 128, 256 or
 *                   512
 *  persistent_ctas  0: one block per chunk; 1 .. 2^20: at most this many
 *                   blocks, each looping over chunks
 *  bottom_slots     a patch's coarse levels with at most this many cells per
 *                   colour (64 .. 16384) run inside the one-CTA bottom cycle
 *  n_pre, n_post    Gauss-Seidel sweeps around the coarse correction (0..8)
 *  ms_per_cycle     output of mg_batch_autotune: the measured time of one
 *                   batched cycle with these parameters (0 if not measured)
 *  chunk            the tile shape of the chunked kernels: list entries per
 *                   chunk (a block works on one chunk at a time, 2 entries
 *                   per thread in flight): 64 .. 65536, or 0 for
 *                   2 * threads */
typedef struct {
  int threads;
  int persistent_ctas;
  int bottom_slots;
  int n_pre, n_post;
  double ms_per_cycle;
  int chunk;
} mg_batch_tuning;

/* Creates a batch of n_patches (1 .. 4096) patches.  masks[p] points to
 * the nx*ny*nz int8 mask of patch p (layout as mg_create_hierarchy), all in
 * memory of kind `where`; dims[3p .. 3p+2] = nx, ny, nz of patch p; h[p] its
 * cell size.  opt as in mg_create_hierarchy (nullable) with precision 0 and
 * n_cycles 1.  All patches work on the batch's stream (cuda_stream, or a
 * new stream when NULL).  Errors: INVALID_ARG (a patch's dims, h or mask is
 * invalid; the message names the patch), EMPTY_DOMAIN (a patch has no
 * active cell), OOM, CUDA. */
mg_status mg_batch_create(int n_patches, const int8_t* const* masks, mg_mem where, const int* dims, const double* h,
                          const mg_options* opt, void* cuda_stream, mg_batch** out);
mg_status mg_batch_destroy(mg_batch* batch);

/* The hierarchy of patch p, owned by the batch (do not destroy it).  Its
 * right-hand side, Dirichlet values and initial guess are set, and its
 * solution read, with the mg_hierarchy calls above.  Errors: INVALID_ARG. */
mg_status mg_batch_patch(mg_batch* batch, int p, mg_hierarchy** out);

/* One multigrid iteration of every patch in its current order (as
 * mg_vcycle; no order switching).  rel_out (nullable) receives n_patches
 * relative residuals.  Errors: CUDA, DIVERGED (a non-finite norm). */
mg_status mg_batch_vcycle(mg_batch* batch, double* rel_out);

/* Solves every patch to relative residual tol (as mg_solve on each patch,
 * with its own order switch, hold counter and stopping test); patches that
 * converge stop iterating while the others go on.  infos (nullable) receives
 * n_patches results.  Returns OK when every patch converged, else
 * NOT_CONVERGED or DIVERGED (the worst over the patches; each patch's own
 * status is in infos[p].status).  Errors: INVALID_ARG, CUDA. */
mg_status mg_batch_solve(mg_batch* batch, double tol, int max_cycles, mg_solve_info* infos);

/* Current launch parameters; setting them validates the values and rebuilds
 * the chunk tables and the cycle graph.  Errors: INVALID_ARG, CUDA. */
mg_status mg_batch_get_tuning(const mg_batch* batch, mg_batch_tuning* out);
mg_status mg_batch_set_tuning(mg_batch* batch, const mg_batch_tuning* tuning);

/* Autotuner: times candidate launch parameters (threads 128/256/512, one
 * block per chunk or 4 / 8 resident blocks per multiprocessor, bottom_slots
 * 1024/2048/4096) on `reps` batched cycles each (CUDA events on the batch's
 * stream) and keeps the fastest; then, with those, the chunk lengths 1, 2,
 * 4 and 8 times threads.  With flags & MG_TUNE_SCHEDULE it then
 * times whole solves to tol from a zero initial guess for the smoother
 * schedules (n_pre, n_post) = (1,1), (2,1), (2,2), (3,3) and keeps the one
 * with the shortest time to tolerance.  Each patch's solution and hold
 * counter are restored afterwards.  best (nullable) receives the result.
 * Errors: INVALID_ARG, CUDA, OOM. */
#define MG_TUNE_SCHEDULE 1
mg_status mg_batch_autotune(mg_batch* batch, int reps, double tol, int max_cycles, int flags,
                            mg_batch_tuning* best);

/* Kernels the last batched cycle graph holds (launches per cycle). */
mg_status mg_batch_launches_per_cycle(const mg_batch* batch, long long* launches);

const char* mg_batch_last_error(const mg_batch* batch);

/* ---------------------------------------------------------------------------
 * Learned initial guess (no counterpart in the paper)
 *
 * A 3D U-Net that predicts the fine solution Phi of one AMR patch from three
 * input channels (the right-hand side, the mask and the Dirichlet values),
 * used as the initial guess of mg_solve, whose stopping test and order switch
 * (Sections 4 and 5.2) stay the judge: a poor guess costs cycles, never
 * accuracy.  Architecture, for L levels and c base channels (level l: c 2^l
 * channels, grid n / 2^l): down path of two 3x3x3 convolutions with bias and
 * ReLU per level, 2x2x2 mean pooling between levels; up path of nearest
 * upsampling by 2, concatenation after the level's down output and two
 * 3x3x3 convolutions with ReLU; a 1x1x1 head to one channel times the active
 * mask.  Weights and activations are BF16 and every convolution accumulates
 * in FP32 on the tensor cores (tcgen05 with TMEM accumulators).
 * Parameters are ordered, per convolution down0.0, down0.1, ..., down(L-1).1,
 * up0.0, up0.1, ..., up(L-2).1 and then the head: the weights
 * [cout][cin][3][3][3] followed by the bias [cout] (head: [c], then [1]).
 * Tensors at the C ABI are FP32 in natural layout [channel][z][y][x].
 * ------------------------------------------------------------------------- */

typedef struct mg_unet mg_unet; /* opaque, library-owned */

/* levels 1..6, base a multiple of 16 with base * 2^(levels-1) <= 128, grid
 * nx*ny*nz with each size 1..1024 and divisible by 2^(levels-1).  All
 * parameters start at 0 (set them with mg_unet_set_params).  cuda_stream as
 * in mg_create_hierarchy.  Errors: INVALID_ARG, OOM, CUDA. */
mg_status mg_unet_create(int levels, int base, int nx, int ny, int nz, void* cuda_stream, mg_unet** out);
mg_status mg_unet_destroy(mg_unet* net);
mg_status mg_unet_num_params(const mg_unet* net, long long* n);
/* All parameters in the order above, FP64 (rounded to FP32 masters and BF16
 * working copies on the device).  Errors: INVALID_ARG, CUDA. */
mg_status mg_unet_set_params(mg_unet* net, const double* params, mg_mem where);
mg_status mg_unet_get_params(mg_unet* net, double* params, mg_mem where);
/* Forward pass: x [3][nz][ny][nx] input channels (FP32); pred (nullable)
 * receives [nz][ny][nx] (FP32).  Errors: INVALID_ARG, CUDA, INTERNAL (a
 * kernel's bounded wait ran out). */
mg_status mg_unet_forward(mg_unet* net, const float* x, mg_mem where, float* pred, mg_mem pred_where);
/* Backward pass after mg_unet_forward: g_pred [nz][ny][nx] (FP32) is
 * dL/dpred; the gradient of every parameter (order above) is computed on the
 * GPU (weight gradients as tcgen05 GEMMs over the voxels) and kept in the
 * network; mg_unet_get_grads copies it out (FP64).  Errors: INVALID_ARG,
 * CUDA, INTERNAL. */
mg_status mg_unet_backward(mg_unet* net, const float* g_pred, mg_mem where);
mg_status mg_unet_get_grads(mg_unet* net, double* grads, mg_mem where);
/* One Adam update (Kingma & Ba, Algorithm 1, with bias correction) of every
 * parameter from the current gradients; FP32 master parameters, then the
 * BF16 working weights are rounded again.  Errors: INVALID_ARG, CUDA. */
mg_status mg_unet_adam_step(mg_unet* net, double lr, double beta1, double beta2, double eps);
/* One training step on one sample: forward pass on x [3][nz][ny][nx], loss
 * sum over active cells of (pred - y)^2 / sum of y^2 there (y [nz][ny][nx],
 * active = x channel 1 > 0), backward pass and one Adam update (beta1 0.9,
 * beta2 0.999, eps 1e-8).  loss (nullable) receives the loss before the
 * update.  Errors: INVALID_ARG, CUDA, INTERNAL. */
mg_status mg_unet_train_step(mg_unet* net, const float* x, const float* y, mg_mem where, double lr, double* loss);
/* The network's input channels for one patch of the network's grid size,
 * from device buffers: mask (int8), rho (double) and the Dirichlet face
 * arrays bx, by, bz of mg_set_dirichlet's layout (nullable = 0); h the cell
 * size.  Channel 0 is h^2 n^2 rho / s on active cells (n the largest grid
 * size), channel 1 is +1 on active and -1 on inactive cells, channel 2 the
 * mean Dirichlet value over the cell's boundary faces / s (0 without
 * boundary faces), with s the root of the mean square of channel 0's
 * numerator over active cells plus that of the boundary-face values (so
 * scaling rho and the boundary values together leaves the channels alone).
 * x (nullable) receives [3][nz][ny][nx] FP32, scale (nullable, host) s. */
mg_status mg_unet_features(mg_unet* net, const int8_t* mask, const double* rho, const double* bx, const double* by,
                           const double* bz, double h, float* x, mg_mem where, double* scale);
/* The learned initial guess: phi (device, [nz][ny][nx] doubles) = s times
 * the network's prediction from the patch's input channels.  Enqueued on the
 * network's stream.  Errors: INVALID_ARG, CUDA. */
mg_status mg_unet_predict(mg_unet* net, const int8_t* mask, const double* rho, const double* bx, const double* by,
                          const double* bz, double h, double* phi);
/* One training step on a solved patch: target phi / s (phi device, the
 * patch's solution), then as mg_unet_train_step.  Errors: INVALID_ARG, CUDA,
 * INTERNAL. */
mg_status mg_unet_train_patch(mg_unet* net, const int8_t* mask, const double* rho, const double* bx, const double* by,
                              const double* bz, double h, const double* phi, double lr, double* loss);
/* The ReLU output of convolution `layer` (parameter order) after the last
 * forward pass, [c][d][h][w] FP32; dims4 = {c, d, h, w}.  For verification. */
mg_status mg_unet_layer_info(const mg_unet* net, int layer, int* dims4);
mg_status mg_unet_layer_output(mg_unet* net, int layer, float* out, mg_mem where);
/* The gradient of the loss w.r.t. convolution `layer`'s pre-activation after
 * the last backward pass, same shape as its output.  For verification. */
mg_status mg_unet_layer_grad(mg_unet* net, int layer, float* out, mg_mem where);
const char* mg_unet_last_error(const mg_unet* net);

/* Synthetic AMR patch on the GPU (input synthesis for training and
 * evaluating the learned guess; no part of the method): the blob-patch
 * recipe, a mask from white noise (SplitMix64 stream of `seed`, Box-Muller)
 * smoothed by a periodic Gaussian of corr_cells cells and thresholded at 0,
 * rho ~ U[-1, 1], and a coarse potential of 6 random low Fourier modes on
 * ((nz+1)/2+2) x ((ny+1)/2+2) x ((nx+1)/2+2) cells (origin -2 in fine-cell
 * units).  Device buffers: scratch 2 nx ny nz + 8 corr_cells + 2 floats,
 * mask nx ny nz int8, rho nx ny nz doubles, phi_c the coarse grid.  Sizes
 * 1..2048, corr_cells in (0, 64].  Enqueued on cuda_stream.
 * Errors (mg_last_error(NULL)): INVALID_ARG, CUDA. */
mg_status mg_generate_blob_patch(unsigned long long seed, int nx, int ny, int nz, double corr_cells, float* scratch,
                                 int8_t* mask, double* rho, double* phi_c, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Instrumentation
 * ------------------------------------------------------------------------- */

/* Number of kernels this library has launched in the process (a graph
 * replay counts each of its kernel nodes). */
unsigned long long mg_launch_count(void);

/* Kernel timing: when enabled, every launch of the fine-level (level 0)
 * Gauss-Seidel half-sweep kernel is bracketed by CUDA events on the stream
 * it runs on (inside the replayed graph when use_graphs is set; those are
 * accumulated each time mg_solve or mg_vcycle with a non-null output waits
 * for a cycle).  mg_timing_read synchronises the stream and returns the
 * number of timed launches and their total time in ms, then resets the
 * accumulators.  Errors: CUDA. */
mg_status mg_timing_enable(mg_hierarchy* hier, int enable);
mg_status mg_timing_read(mg_hierarchy* hier, long long* launches, double* total_ms);

/* Measured FP64 fused multiply-add throughput of the current GPU, in FP64
 * lane operations (one FMA per lane) per second: 8 independent FMA chains of
 * `iters` steps (1 .. 2^20; 4096 is plenty) per thread, 8 blocks of 256
 * threads per multiprocessor, the best of three timed launches (CUDA events
 * on the legacy default stream, after one warm-up launch).  This is the
 * ceiling of the FP64 form's Gauss-Seidel sweeps, which issue more FP64
 * instructions per byte than the GPU's FP64 pipe retires at the HBM rate.
 * Allocates nothing.  Errors: INVALID_ARG, CUDA. */
mg_status mg_probe_fp64_rate(int iters, double* lane_ops_per_s);

/* ---------------------------------------------------------------------------
 * Debugging aids
 * ------------------------------------------------------------------------- */

/* 1 if this library was built with MG_CHECKED: every kernel that reads a
 * compact list of unknowns checks each entry against its level's slots,
 * skips an entry outside them and records the kernel site; the entry point
 * that ran the kernel then returns MG_ERR_INTERNAL and mg_last_error names
 * the site.  0 for the normal build, which has no such checks. */
int mg_checked_build(void);

/* Test hook: the nth device or pinned-host allocation the library makes from
 * now on (nth >= 1) fails as if the device were out of memory; nth = 0
 * disarms the hook.  It fires once.  The failing call returns MG_ERR_OOM and
 * releases everything it had allocated. */
void mg_debug_fail_alloc(int nth);

/* Test hook of the temporal-blocked smoothing pass (option smoother_pass):
 * while on, passes captured or launched from now on make their first CTA
 * wait on a barrier that nothing completes, so that its bounded wait runs out
 * (after about a second); the CTA then leaves the pass and the solve or
 * V-cycle returns MG_ERR_INTERNAL.  0 turns it off. */
void mg_debug_stall_pass(int on);

#ifdef __cplusplus
}
#endif
#endif /* GBMG_MG_H */
