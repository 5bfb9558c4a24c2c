/*
 * mr.h -- C-ABI of the GB300 (sm_103a) library for the adaptive-multiresolution
 * Strang step of Descombes, Duarte, Dumont, Guillet, Louvet, Massot,
 * "Task-based adaptive multiresolution for time-space multi-scale
 * reaction-diffusion systems on multi-core architectures" (arXiv:1506.04651).
 *
 * The library advances du_i/dt - div(D_i grad u_i) = f_i(u) on [0,1]^d with
 * homogeneous Neumann conditions (Sec. 1, Eq. thesystem) by the Strang scheme
 * U_{n+1} = R_{dt/2} D_dt R_{dt/2} U_n (Sec. 2.1) on the leaves of a graded
 * dyadic tree adapted every step by multiresolution (Sec. 2.2, Sec. 3.1).
 *
 * Conventions shared by every entry point:
 *   - Every call returns mr_status; nothing throws across the ABI.
 *   - Pointers are plain host or device pointers; an `on_device` flag (0 host,
 *     1 device) says which.  The caller owns every buffer it passes; the
 *     context owns all device memory it allocates (freed by mr_destroy).
 *   - Work is ordered on the CUDA stream given to mr_create (0 = legacy
 *     default stream).  Calls synchronise that stream before returning.
 *   - Leaf order: by level, then by Morton abscissa within a level (the key
 *     order below).  Leaf values are structure-of-arrays: values[i*n + r] is
 *     species i of leaf r (Sec. 3.2: one contiguous array per unknown).
 *   - Keys follow Sec. 3.1.1 / Fig. 2: bits 0-47 the Morton abscissa of the
 *     cell at its level (x digit first in each digit group), bits 48-51 the
 *     level, bits 52-63 zero.
 *   - Errors: MR_EINVAL for bad arguments (checked before any GPU work),
 *     MR_ENOMEM when a capacity is exceeded, MR_ECUDA for a CUDA runtime
 *     error, per-cell Radau5 failures as MR_ERADAU_* (first one wins; the
 *     leaf values are then those reached when the failing cell stopped).
 *     mr_last_error() gives a one-line message.
 */
#ifndef MR_GB300_H
#define MR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mr_ctx mr_ctx;

typedef enum {
  MR_OK = 0,
  MR_EINVAL = -1,
  MR_ENOMEM = -2,
  MR_ECUDA = -3,
  MR_ESTATE = -4,
  MR_ERADAU_HMIN = -10,
  MR_ERADAU_MAXSTEPS = -11,
  MR_ERADAU_SINGULAR = -12,
  MR_EROCK_STEP = -20,
  MR_ENONFINITE = -30,
  MR_ETIMEOUT = -40,
  MR_EIO = -50
} mr_status;

enum { MR_MODEL_BZ = 1, MR_MODEL_NAGUMO = 2, MR_MODEL_NETWORK = 3, MR_MODEL_IONIC = 4 };
enum { MR_FP64 = 0, MR_MIXED = 1, MR_MIXED_F32_DETAILS = 2 };
enum { MR_RADAU_THREAD = 0, MR_RADAU_POOL = 1 };

#define MR_MAX_SPECIES 32
#define MR_IONIC_SPECIES 21
#define MR_MAX_LEVEL 16
#define MR_MAX_REACTIONS 32

/*
 * Problem description (Sec. 1, Eq. thesystem).
 *   dim       d in {2, 3}
 *   J         finest level (Sec. 2.2); d*J <= 30
 *   jmin      no leaf is coarser than jmin (1 <= jmin <= J)
 *   m         number of species (BZ: 3, NAGUMO: 1, NETWORK: 2..16, IONIC: 21)
 *   model     MR_MODEL_BZ: params = (eps, mu, f, q) of
 *               f_a = (-q a - a b + f c)/mu, f_b = (b - b^2 + a (q - b))/eps, f_c = b - c
 *               (Sec. 1 item II; the paper prints q = 0.02)
 *             MR_MODEL_NAGUMO: params = (k) of f = k u^2 (1 - u) (Sec. 1 item I)
 *             MR_MODEL_NETWORK: a stiff mass-action reaction network (a
 *               synthetic stand-in for the paper's large-mechanism case, Sec.
 *               1 item III); no params, the reactions are given by
 *               mr_set_network before the first reaction sub-step
 *             MR_MODEL_IONIC: a synthetic 21-species membrane model, the
 *               stand-in for the paper's STROKE case (Sec. 1 item III: 21
 *               equations, voltage-gated channels with steep sigmoid gates,
 *               log Nernst potentials, Jacobian eigenvalues down to about
 *               -1e8, Jacobian computed numerically); no params.  Species:
 *               e_0..e_3 (extracellular ions), g (transmitter), c_0..c_3
 *               (intracellular ions), V (membrane potential), a_0..a_3,
 *               b_0..b_3 (gates), E (energy), B (buffer), S (energy supply,
 *               f = 0).  The Jacobian is formed by forward differences, one
 *               column per species, with the increment
 *               sqrt(1e-16 max(1e-5, |y_j|)).
 *   D         m diffusion coefficients (when m > 16 the species are
 *             diffused in windows of 16; windows whose coefficients are
 *             all zero cost nothing)
 *   precision MR_FP64, or MR_MIXED: Radau5 factorises and solves its Newton
 *             systems in FP32 and forms the starting values and tolerance
 *             scales of each step attempt in FP32, and the ROCK4 stages and
 *             finishing procedure
 *             run on FP32 increments from the FP64 state (y_{n+1} - y_n and
 *             the stage differences; L y_n is applied in FP64 once per
 *             sub-step), so rounding is relative to the change a step makes
 *             (Radau5 residuals, both error norms, step control, the state,
 *             details and mass stay FP64), or
 *             MR_MIXED_F32_DETAILS: MR_MIXED with the MR details (Eq.
 *             detail) also predicted and differenced in FP32 from the FP64
 *             node values (thresholds and the normalisation stay FP64); the
 *             adapted grid may then differ from the FP64 one where a detail
 *             lies within FP32 rounding of its threshold
 *   max_leaves leaf capacity; 0 means 2^(d J)
 */
typedef struct {
  int dim, J, jmin, m, model, nparams, precision, reserved;
  double params[8];
  double D[MR_MAX_SPECIES];
  int64_t max_leaves;
} mr_problem;

/* Counters of the last completed calls (see each field). */
typedef struct {
  int64_t leaves, nodes;
  int64_t leaves_per_level[MR_MAX_LEVEL + 1];
  double compression_ratio;       /* CR = (1 - N/2^(dJ)) 100, Sec. 4.1 */
  /* last react_radau5 call (App. A complexity: fev + m * jac) */
  int64_t radau_fev, radau_jac, radau_steps, radau_accept, radau_reject, radau_newton, radau_dec;
  /* last diffuse_rock4 call, summed over species */
  int64_t rock_steps, rock_reject, rock_stages, rock_matvec;
  int32_t rock_smax, reserved0;
  double rock_rho;                /* Gershgorin bound of the species-free operator */
  int64_t irregular_rows, irregular_nnz;
  double ms_adapt, ms_react, ms_diffuse; /* device time of the last strang_step phases */
  int64_t kernel_launches;        /* cumulative kernels launched by this context */
  /* cumulative since mr_create, from CUDA events around each launch on the
   * context stream: the Radau5 kernel and the ROCK4 sweep kernel, with their
   * algorithmic work (Radau5: FP64 operations counted from the kernel's
   * source per counted event, applied to radau_counters as a lower bound --
   * for BZ (m = 3): right-hand side 13, Jacobian 10, factorisations 110,
   * Newton iteration 249 plus 6 for its contraction monitor from the second
   * iteration on, step attempt 73, extrapolated starting values 142,
   * accepted step 77; ROCK4: bytes each sweep must move at least) */
  double radau_kernel_ms, radau_alg_flops;
  int64_t radau_kernel_launches;
  double rock_kernel_ms, rock_alg_bytes;
  int64_t rock_kernel_launches;
  /* cumulative Radau5 counters since mr_create: f evaluations, Jacobians, step
   * attempts, accepted, rejected, Newton iterations, factorisations, cells */
  int64_t radau_counters[8];
  /* cumulative arithmetic of the ROCK4 sweeps since mr_create: per operator
   * application 2d + 1 per regular leaf and 2 per merged-row entry, plus the
   * stage and finishing combinations (5 per stage, 3 + 3 + 8 + 4 for the
   * finishing sweeps, 8 for the estimate, 3 for the first stage); FP64
   * operations in the FP64 form, FP32 in the mixed form.  rock_alg_bytes
   * counts the merged rows too (12 bytes per entry in FP64, 8 in the mixed
   * form, 8 per row). */
  double rock_alg_flops;
} mr_stats;

/* Create a context for `prob` on `cuda_stream` (a cudaStream_t or NULL).
 * Allocates the device capacity for the full tree once.  MR_EINVAL on bad
 * sizes, MR_ENOMEM if the device cannot hold the capacity. */
mr_status mr_create(const mr_problem *prob, void *cuda_stream, mr_ctx **out);
void mr_destroy(mr_ctx *ctx);

/* Initial grid: u0 holds m x 2^(dJ) values at level J, lexicographic with x
 * fastest; the full tree is projected (Sec. 2.2) and then adapted with
 * threshold eta until no family can be deleted (Sec. 3.1.2). */
mr_status mr_build(mr_ctx *ctx, const double *u0, int on_device, double eta);

/* Reactions of an MR_MODEL_NETWORK context: nr (1..MR_MAX_REACTIONS)
 * reversible mass-action reactions u_a + u_b <-> u_c + u_d, species[4 r + t]
 * = (a, b, c, d) of reaction r (four distinct indices in [0, m)), rates
 * kf[r], kb[r] >= 0:  w_r = kf_r u_a u_b - kb_r u_c u_d, f_a -= w_r,
 * f_b -= w_r, f_c += w_r, f_d += w_r.  Host arrays, copied.  MR_EINVAL for
 * another model or bad data. */
mr_status mr_set_network(mr_ctx *ctx, int nr, const int32_t *species, const double *kf,
                         const double *kb);

/* Replace the tree by the n given leaves (keys as above, values m x n).
 * MR_EINVAL unless they tile the domain as a graded tree whose levels below
 * jmin are all refined. */
mr_status mr_set_leaves(mr_ctx *ctx, int64_t n, const uint64_t *keys, const double *values,
                        int on_device);

mr_status mr_num_leaves(const mr_ctx *ctx, int64_t *n);

/* Copy the current leaves out (keys may be NULL).  cap is the capacity of
 * `keys` (entries) and of each species row of `values`; MR_ENOMEM if short. */
mr_status mr_get_leaves(mr_ctx *ctx, uint64_t *keys, double *values, int64_t cap, int64_t *n,
                        int on_device);

/* One grid adaptation (Sec. 3.1.2): projection, details d = u - P P u
 * (Eq. detail) against eps_j = 2^((d/2)(j-J)) eta, refinement of tagged
 * leaves, grading to the least graded tree, coarsening to a fixed point.
 * eta = 0 on the uniform level-J grid is the identity (every node is tagged,
 * nothing can be refined or coarsened) and returns at once.  MR_EINVAL for a
 * negative or non-finite eta; MR_ESTATE if a detail is not finite (the state
 * holds NaN or infinity); MR_ENOMEM if the adapted tree outgrows the leaf
 * capacity given to mr_create (max_leaves). */
mr_status mr_adapt(mr_ctx *ctx, double eta);

/* Reaction sub-step R_dt (Sec. 2.1): every leaf integrates u' = f(u) over dt
 * with Radau5 (3-stage Radau IIA, simplified Newton, step-size control;
 * rtol, atol > 0).  MR_EINVAL for dt <= 0 or tolerances <= 0; per-cell
 * failures MR_ERADAU_HMIN (step size underflow), MR_ERADAU_MAXSTEPS (over
 * 100000 attempts), MR_ERADAU_SINGULAR (five singular Newton matrices in a
 * row), MR_ENONFINITE (a non-finite state); MR_ESTATE for a network model
 * whose reactions are not set.  With the MR_RADAU_POOL schedule also
 * MR_ENOMEM if its slot buffer (about 64 MB, allocated on the first pooled
 * launch of the context) cannot be allocated, and MR_ETIMEOUT if one of its
 * bounded waits runs out. */
mr_status react_radau5(mr_ctx *ctx, double dt, double rtol, double atol);

/* Schedule of the Radau5 launches of BZ and NAGUMO contexts (the network
 * and membrane models have their team kernels only):
 *   MR_RADAU_THREAD  one thread integrates one cell at a time, taking cells
 *                    from a device work queue; a pass is one step attempt;
 *   MR_RADAU_POOL    the cells in flight are held in a shared-memory pool per
 *                    SM, and each warp runs one phase of a step attempt
 *                    (prepare: Jacobian, factorisations, starting values; one
 *                    Newton iteration; error estimate and step control) for
 *                    up to 32 cells that are in that phase.
 * Both run the same operations per cell in the same order, so results and
 * complexity counts are bit-identical.  New contexts use MR_RADAU_THREAD,
 * the faster of the two on the measured workloads.
 * MR_EINVAL for another value. */
mr_status mr_set_radau_schedule(mr_ctx *ctx, int schedule);

/* Diffusion sub-step D_dt (Sec. 2.1, Sec. 3.2.1): every species integrates
 * u' = D_i L u with the ROCK4-type stabilized method (tol > 0).  Species
 * with D_i = 0 are left unchanged.  MR_EINVAL for dt <= 0 or tol <= 0;
 * MR_EROCK_STEP if the step size collapses (below 1e-14 dt) or the step
 * limit is reached; MR_ENONFINITE if the error norm is not finite. */
mr_status diffuse_rock4(mr_ctx *ctx, double dt, double tol);

/* One Strang step: mr_adapt(eta); R_{dt/2}; D_dt; R_{dt/2}.  Errors as for
 * the three calls; the first failing phase ends the step. */
mr_status strang_step(mr_ctx *ctx, double dt, double eta, double rtol, double atol,
                      double rock_tol);

/*
 * Batched serving: n independent instances (own grid depth, parameters and
 * threshold each) stepped together on the current device.
 *   mr_batch_create  n contexts (probs[i], each with its own CUDA stream) and
 *                    a pool of `threads` host threads (<= 0: one per core, at
 *                    most 32).  MR_EINVAL for n outside [1, 4096] or a bad
 *                    problem (as mr_create).
 *   mr_batch_context the i-th instance's context, for mr_build / mr_set_leaves
 *                    / mr_get_leaves / mr_mass ... (owned by the batch; NULL
 *                    for a bad index).  Do not destroy it.
 *   mr_batch_run     nsteps Strang steps of every instance, eta[i] its
 *                    threshold: the adaptation of all instances runs
 *                    concurrently on their streams; each reaction half step
 *                    of all instances is one persistent Radau5 launch over
 *                    the union of their leaves (when all instances use the
 *                    BZ or all the NAGUMO model with one precision; otherwise
 *                    one launch per instance), and the diffusion sub-step of
 *                    all instances is one persistent ROCK4 launch (when all
 *                    are 2D with one or three species, the same species
 *                    count and precision; otherwise one launch per instance,
 *                    run concurrently).  Every cell is integrated with the
 *                    same arithmetic as by strang_step, so reaction results
 *                    equal stepping each context alone; in the joint
 *                    diffusion each instance keeps its own step control, but
 *                    its error norm is summed in another order, so its
 *                    results agree with stepping it alone to rounding (and
 *                    an accept / reject decision at the tolerance's edge may
 *                    differ).  Synchronises before returning; the first
 *                    error wins (per-instance detail in each context's last
 *                    error).
 *   mr_batch_diffuse the diffusion sub-step alone (diffuse_rock4 of every
 *                    instance over dt with tolerance tol), joint or per
 *                    instance as in mr_batch_run.  MR_EINVAL for dt <= 0 or
 *                    not finite, or tol <= 0; synchronises before returning.
 *   mr_batch_get_stats counters of the last mr_batch_run or mr_batch_diffuse.  In the joint form
 *                    the Radau5 counters are batch totals (the contexts' own
 *                    Radau5 counters are not updated); the ROCK4 counters of
 *                    each context are its own in either form.
 */
typedef struct mr_batch mr_batch;
typedef struct {
  int64_t instances, threads, steps;
  int64_t leaf_updates;        /* sum over steps and instances of the leaves after adaptation */
  double ms_device;            /* device time of the run: start event to end event */
  double ms_react_kernel;      /* summed device time of the joint Radau5 launches */
  int64_t react_launches;      /* joint Radau5 launches */
  int64_t radau_fev, radau_jac, radau_steps, radau_accept, radau_reject, radau_newton, radau_dec;
  double radau_alg_flops;      /* algorithmic FP64 operations of the joint launches */
  int32_t joint_reaction;      /* 1: the reaction sub-steps ran as joint launches */
  int32_t joint_diffusion;     /* 1: the diffusion sub-steps ran as joint launches */
  double ms_adapt_phase, ms_diffuse_phase; /* host wall time of the adaptation and diffusion
                                              phases over the run */
  double ms_diffuse_kernel;    /* summed device time of the joint ROCK4 launches */
  int64_t diffuse_launches;    /* joint ROCK4 launches */
} mr_batch_stats;

/*
 * The batch's autotuner (no counterpart in the paper; the launch shapes of
 * the batched form are chosen by timed trials).  The joint Radau5 launch has
 * four candidate shapes -- 128 or 64 threads per block, cells taken from the
 * finest level down or in leaf order -- and the joint ROCK4 launch two -- 2
 * or 1 blocks of 256 threads per SM.  None changes a result (cells are
 * integrated independently; the joint ROCK4 error norms are summed in fixed
 * chunks), so tuning is online: the first launches of mr_batch_run /
 * mr_batch_diffuse try each candidate twice, rank them by algorithmic work
 * per millisecond (Radau5: FP64 operations as in mr_stats; ROCK4: sweep
 * bytes), and the fastest is kept.  On by default.
 *   mr_batch_set_autotune  on = 1 restarts the trials, on = 0 fixes the
 *                          default shapes (128 threads, finest first; 2
 *                          blocks per SM); MR_EINVAL otherwise
 *   mr_batch_tuning        the trial table: one entry per candidate (the
 *                          six Radau5 shapes: the thread schedule with
 *                          128 or 64 threads per block, then the pooled
 *                          schedule, each in both queue orders; then the
 *                          two ROCK4 shapes);
 *                          *n gets the number of entries, MR_ENOMEM if cap
 *                          is smaller
 */
typedef struct {
  int32_t phase;       /* 0: joint Radau5 launch, 1: joint ROCK4 launch */
  int32_t block;       /* threads per block */
  int32_t per_sm;      /* ROCK4: blocks per SM; Radau5: 0 (as many as fit) */
  int32_t order;       /* Radau5: 1 finest levels first, 0 leaf order */
  int64_t launches;    /* launches run with this shape */
  double ms, work, rate; /* their summed device time and algorithmic work, work per ms */
  int32_t chosen;
  int32_t schedule;    /* Radau5: MR_RADAU_THREAD or MR_RADAU_POOL (block 128 = 4 warps per SM) */
} mr_tune_entry;

mr_status mr_batch_create(int n, const mr_problem *probs, int threads, mr_batch **out);
mr_ctx *mr_batch_context(mr_batch *b, int i);
mr_status mr_batch_run(mr_batch *b, int nsteps, double dt, const double *eta, double rtol, double atol,
                       double rock_tol);
mr_status mr_batch_diffuse(mr_batch *b, double dt, double tol);
mr_status mr_batch_get_stats(const mr_batch *b, mr_batch_stats *out);
mr_status mr_batch_set_autotune(mr_batch *b, int on);
mr_status mr_batch_tuning(const mr_batch *b, mr_tune_entry *out, int cap, int *n);
void mr_batch_destroy(mr_batch *b);

/* Checkpoint and resume.  mr_save writes the current leaves to `path`:
 * a 64-byte header (8-byte magic "MRGB300\0"; int32 format version 2, dim,
 * J, jmin, m, model, precision, 0; int64 leaf count; 16 zero bytes), the model parameters
 * and diffusion coefficients of the problem (8 + MR_MAX_SPECIES doubles;
 * version-1 files, written with 16 coefficients, still load), the leaf keys
 * (n uint64, the key layout above) and the values (m x n doubles, species
 * major), all little-endian.  mr_load replaces the context's tree by the
 * file's leaves; the file must have been written for the same dim, J, jmin,
 * m and model (MR_EINVAL otherwise, the context unchanged).  MR_EIO if the
 * file cannot be opened, written or read in full.  Resuming from a file gives
 * the same results as continuing the saved context: the tree, its values and
 * everything the next step computes from them are restored exactly. */
mr_status mr_save(mr_ctx *ctx, const char *path);
mr_status mr_load(mr_ctx *ctx, const char *path);

mr_status mr_get_stats(const mr_ctx *ctx, mr_stats *out);

/* Per-leaf complexity of the last react_radau5 call: f evaluations plus m
 * per Jacobian (App. A counts the analytic BZ Jacobian as three). */
mr_status mr_get_complexity(mr_ctx *ctx, int32_t *out, int64_t cap, int on_device);

/* Integral of each species over the domain, sum over leaves h^d u_i (FP64). */
mr_status mr_mass(mr_ctx *ctx, double *mass);

/* Apply the species-free finite-volume leaf operator L (Eq. discretise,
 * App. C; D_i L is the diffusion operator of species i) to one leaf vector
 * u_in (length N) into out.  Also returns its Gershgorin bound in *rho
 * (may be NULL).  For checking the operator the library builds. */
mr_status mr_apply_operator(mr_ctx *ctx, const double *u_in, double *out, int on_device,
                            double *rho);

/* The two storage forms of the leaf operator L and their cost per
 * application: the comparison of App. C (Table 5: the paper's compact
 * operator against a CSR matrix of the same operator).  "Compact" is the form
 * the ROCK4 sweeps use: a regular-leaf table (the leaf, its 2d same-level
 * neighbours and its level; weights 1/h^2 implicit) and one merged
 * (leaf, weight) row per leaf at a level jump.  "CSR" assembles every row
 * into one compressed sparse row matrix.  Each form is applied `reps` times
 * (1..10000) to one FP64 vector of the current tree after a warm-up; *ms_* get
 * the mean device time of one application (CUDA events on the context
 * stream), *csr_nnz the CSR matrix's entries and *max_rel_diff max |L_csr u -
 * L_compact u| / max |L_compact u|.  The CSR matrix and the vectors are
 * allocated for the call and freed before it returns.  MR_EINVAL for bad
 * arguments; MR_ECUDA if an allocation or launch fails. */
mr_status mr_operator_forms(mr_ctx *ctx, int reps, double *ms_compact, double *ms_csr, int64_t *csr_nnz,
                            double *max_rel_diff);

/* The library's ROCK4-type coefficients for s stages (5 <= s <= 152): the
 * recurrence P_{j+1} = mu[j+1] P_j + nu[j+1] P_{j-1} + kap[j+1] z P_j
 * (arrays of length s-3), the finishing quartic w[0..4] (w[0] = 1) and the
 * embedded-estimate weights errc[0..3]; *ell = 0.336 s^2 - 2.7. */
mr_status mr_rock4_coefficients(int s, double *mu, double *nu, double *kap, double *w,
                                double *errc, double *ell);

/* The per-event FP64 operation counts of the one-thread-per-cell Radau5
 * kernel (App. A counts right-hand sides and Jacobians; the other events
 * follow the method's steps, Hairer and Wanner Sec. IV.8) from which
 * mr_stats.radau_alg_flops is formed, for model MR_MODEL_BZ or
 * MR_MODEL_NAGUMO with m species: out[0..7] = right-hand side, Jacobian,
 * factorisations, Newton iteration without its right-hand sides,
 * contraction monitor, step attempt, extrapolated starting values,
 * accepted step.  A launch's work is rhs fev + jac njac + dec ndec + newton
 * nnewton + monitor (nnewton - steps) + attempt steps + extrap max(0, steps -
 * cells - reject) + accept naccept.  Host only; MR_EINVAL for another model
 * or a null out. */
mr_status mr_radau_work(int model, int m, double *out);

/*
 * Reaction of a plain array of cells that allocates nothing.  The paper has
 * no counterpart; this entry point is for callers that cannot allocate device
 * memory themselves or through a context: code that runs while another
 * component (a caching allocator, a host application handing out device
 * pointers) owns the device's memory, or code that must not call into the CUDA
 * allocator at all.  It integrates u' = f(u) over dt in every cell with the same
 * Radau5 kernel and control as react_radau5.
 *   model, params, nparams  as in mr_problem (BZ: m = 3; NAGUMO: m = 1)
 *   u           device pointer; species i of cell r is u[i*ld + r]; updated in place
 *   n, ld       number of cells and row stride (0 <= n <= MR_NOALLOC_MAX_CELLS, ld >= n)
 *   dt, rtol, atol  as in react_radau5 (all > 0)
 *   complexity  device pointer to n int32 (f evaluations + m per Jacobian), or NULL
 *   cuda_stream stream the work is ordered on (NULL: legacy default stream); the
 *               call synchronises it before returning
 * Scratch: the work-queue head, the status word and the step counters live in a
 * 512-byte static device array that every GPU which loads this library holds
 * until the process exits; no cudaMalloc/cudaFree or allocating library call is
 * made.  The first call on a device looks up that array's device address and
 * caches it, so make that first call before any stream capture; the cached
 * address belongs to the device's primary context and is not valid after
 * cudaDeviceReset (do not call this entry point after a reset in the same
 * process).  The work-queue head is 64-bit, so the tickets the grid draws past
 * the last cell cannot wrap at any n up to the maximum.  All calls share
 * the array (it keeps the last call's contents; each call clears it first), so
 * calls whose work overlaps on the GPU -- other streams, other host threads --
 * race on it and must be serialised by the caller.
 * Errors: MR_EINVAL for a bad model or parameters, n outside [0,
 * MR_NOALLOC_MAX_CELLS], ld < n or a NULL u (checked before any GPU work);
 * MR_ECUDA if the device address of the scratch cannot be obtained or a launch
 * fails; per-cell Radau5 failures as in react_radau5.
 */
#define MR_NOALLOC_MAX_CELLS 2147483647LL
mr_status mr_react_radau5_noalloc(int model, const double *params, int nparams, double *u,
                                  int64_t n, int64_t ld, double dt, double rtol, double atol,
                                  int32_t *complexity, void *cuda_stream);

/* Measurement aid (no counterpart in the paper): FP64 fused multiply-add
 * throughput of the current device in TFLOP/s (2 flops per FMA), from a
 * kernel of independent FMA chains on every SM timed with CUDA events; used
 * as the denominator of the Radau5 arithmetic roofline.  *mhz gets the SM
 * clock the driver reports during the run (may be NULL). */
mr_status mr_fp64_fma_rate(double *tflops, double *mhz);

const char *mr_status_str(mr_status s);
mr_status mr_last_error(const mr_ctx *ctx, char *buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif
