/*
 * Oracle for the adaptive-multiresolution Strang step of Descombes, Duarte,
 * Dumont, Guillet, Louvet, Massot, "Task-based adaptive multiresolution for
 * time-space multi-scale reaction-diffusion systems on multi-core
 * architectures" (arXiv:1506.04651).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU
 * restatement of what the GPU path computes.  Only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load it.  It
 * shares no code, header, table or constant generator with the CUDA library:
 * every constant below (Radau IIA tableau, its T-transformation, the ROCK4-type
 * polynomials) is recomputed here from its definition.
 *
 * Files:
 *   radau5.c  models f, J (Sec. 1 items I-II; BZ printed in Sec. 1; a
 *             synthetic stiff mass-action network standing in for the
 *             paper's large-mechanism case, Sec. 1 item III; a synthetic
 *             21-species membrane model with a numerical Jacobian standing
 *             in for the paper's STROKE model, Sec. 1 item III) and the
 *             Radau5 reaction integrator (Sec. 2.1, App. A; algorithm of
 *             Hairer-Wanner, Solving ODEs II, Sec. IV.8, cited as MR1439506)
 *   rock4.c   ROCK4-type stabilized polynomials and the linear diffusion
 *             integrator (Sec. 3.2.1, Eq. (RKscheme), Horner form; Abdulle's
 *             construction cited as MR1923724)
 *   parallel.c a parallel-for (one chunk per thread) for the threaded form of
 *             the timed CPU baseline; one thread by default
 *   mrtree.c  dyadic tree, projection, prediction (Eq. inter_1d), details
 *             (Eq. detail), thresholds, graded refinement and coarsening
 *             (Sec. 2.2, Sec. 3.1.2), finite-volume leaf operator (Eq.
 *             discretise, App. C), Strang step (Sec. 2.1), mass.
 *
 * Parity pins: see tests/test_oracle_*.py.  Every function is pinned by a
 * closed form, an invariant or brute force.  The whole multi-step trajectory
 * (adaptation, Radau5, ROCK4, splitting) is pinned by the exact travelling
 * front of the NAGUMO model; the multi-step BZ trajectory itself has no
 * closed form and no published worked example ("parity unpinned" for that
 * model's trajectory beyond its per-step pins).  Trees are 2D or 3D.
 */
#ifndef MR_ORACLE_H
#define MR_ORACLE_H
#include <stdint.h>

#define ORC_MAXM 32
#define ORC_MAXL 16
#define ORC_MAXR 32

enum { ORC_MODEL_BZ = 1, ORC_MODEL_NAGUMO = 2, ORC_MODEL_LINEAR = 3, ORC_MODEL_NETWORK = 4, ORC_MODEL_IONIC = 5 };

/* IONIC: the synthetic 21-species membrane model (radau5.c) */
#define ORC_IONIC_M 21

enum {
  ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ESTATE = -4,
  ORC_ERADAU_HMIN = -10, ORC_ERADAU_MAXSTEPS = -11, ORC_ERADAU_SINGULAR = -12,
  ORC_ERADAU_NEWTON = -13, ORC_EROCK_STEP = -20, ORC_ENONFINITE = -30
};

typedef struct {
  int kind, m;
  double p[8];                 /* BZ: eps, mu, f, q.  NAGUMO: k */
  double K[ORC_MAXM * ORC_MAXM]; /* LINEAR: f(u) = K u (row-major) */
  /* NETWORK: nr reversible mass-action reactions u_a + u_b <-> u_c + u_d,
   * species (a, b, c, d) = sp[r][0..3], rates kf[r] (forward), kb[r] */
  int nr;
  int sp[ORC_MAXR][4];
  double kf[ORC_MAXR], kb[ORC_MAXR];
} orc_model;

typedef struct {
  int64_t nfev, njac, nstep, naccept, nreject, nnewton, ndec;
  int status;
} orc_radau_stats;

typedef struct {
  int64_t nsteps, naccept, nreject, nstages, nmatvec;
  int smax, status;
} orc_rock_stats;

/* ---- parallel.c (threaded form of the timed CPU baseline only) ---- */
typedef void (*orc_body)(void *ctx, int64_t lo, int64_t hi, int chunk);
void orc_set_threads(int t);
int orc_get_threads(void);
/* body(ctx, lo, hi, chunk index) over chunks of `chunk` iterations */
void orc_parallel_for(int64_t n, int64_t chunk, orc_body body, void *ctx);

/* ---- radau5.c ---- */
void orc_model_f(const orc_model *md, const double *y, double *f);
void orc_model_jac(const orc_model *md, const double *y, double *J);
void orc_radau_constants(double c[3], double A[9], double T[9], double Tinv[9],
                         double lam[3], double bhat[3], double e[3]);
int orc_radau5(const orc_model *md, double *y, double tend, double rtol,
               double atol, double hfix, orc_radau_stats *st);

/* ---- rock4.c ---- */
double orc_rock4_ell(int s);
int orc_rock4_coeffs(int s, double *mu, double *nu, double *kap, double w[5],
                     double errc[4], double xc[5]);
int orc_rock4_choose(double rho_dt, int *s, double *ell);
int orc_rock4_linear(int64_t n, const int64_t *rowptr, const int32_t *col,
                     const double *val, double D, double rho, double *y,
                     double dt, double tol, double hfix, orc_rock_stats *st);

/* ---- mrtree.c ---- */
typedef struct orc_tree orc_tree;
orc_tree *orc_tree_new(int d, int J, int jmin, int m);
void orc_tree_free(orc_tree *T);
int orc_tree_set_full(orc_tree *T, const double *u0);
int orc_tree_set_leaves(orc_tree *T, int64_t n, const uint64_t *keys,
                        const double *vals);
int64_t orc_tree_num_leaves(orc_tree *T);
int orc_tree_get_leaves(orc_tree *T, uint64_t *keys, double *vals);
int orc_tree_num_nodes(orc_tree *T, int64_t *per_level);
int orc_tree_is_graded(orc_tree *T);
void orc_project(orc_tree *T);
int orc_details(orc_tree *T, int64_t cap, uint64_t *keys, double *delta);
double orc_value(orc_tree *T, int j, const int32_t *k, int i);
int orc_adapt(orc_tree *T, double eta);
int orc_operator(orc_tree *T, int64_t cap, int64_t *rowptr, int32_t *col,
                 double *val, double *rho);
int orc_apply_literal(orc_tree *T, const double *u, double *out);
int orc_react(orc_tree *T, const orc_model *md, double dt, double rtol,
              double atol, orc_radau_stats *agg, int32_t *complexity);
int orc_diffuse(orc_tree *T, const double *D, double dt, double tol,
                orc_rock_stats *agg);
int orc_strang(orc_tree *T, const orc_model *md, const double *D, double dt,
               double eta, double rtol, double atol, double rock_tol);
void orc_mass(orc_tree *T, double *mass);
uint64_t orc_key(int d, int j, const int32_t *k);
void orc_key_decode(int d, uint64_t key, int *j, int32_t *k);

#endif
