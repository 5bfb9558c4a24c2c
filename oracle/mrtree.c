/*
 * Oracle (test infrastructure only): dyadic multiresolution tree, adaptation,
 * finite-volume leaf operator, reaction/diffusion sweeps and the Strang step.
 *
 * Storage is the plainest one that can be checked by eye: for every level j a
 * dense array over all 2^(d j) cells (lexicographic, x fastest) holding a
 * status (absent / leaf / internal) and the m values.  Nothing here follows
 * the GPU layout; keys are produced only for input/output.
 *
 * Paper passages restated here:
 *   Sec. 2.2   levels 0..J, 2^(dj) cells at level j, leaves = adapted grid,
 *              values stored at all nodes; projection = exact average of the
 *              2^d children; prediction = centred interpolation of order 3
 *              (l = 1), Eq. inter_1d, extended by tensor product (3^d stencil);
 *              details, Eq. detail; thresholds eps_j = 2^((d/2)(j-J)) eps in an
 *              L2 normalisation; graded tree = every prediction stencil present.
 *   Sec. 3.1.1 node key: Morton abscissa (x digit first) in bits 0-47, level
 *              in bits 48-51 (Fig. 2).
 *   Sec. 3.1.2 refinement (tag by details, refine, tag extra nodes for grading,
 *              repeat until graded) and coarsening (delete leaves whose parent
 *              was not tagged when grading survives; repeat until no deletion).
 *   Eq. discretise, App. C: centred second-order finite volumes, 5/7-point on a
 *              Cartesian mesh; coefficients depend on the neighbour's level.
 *   Sec. 2.1   Strang step U_{n+1} = R_{dt/2} D_dt R_{dt/2} U_n.
 *
 * Readings where the paper is silent:
 *   - boundary: out-of-range stencil cells are mirrored (k -> -1-k,
 *     k -> 2^(j+1)-1-k), the even reflection of homogeneous Neumann data;
 *   - detail norm: delta = max_i |d_i| / s_i with s_i = max over leaves |u_i|
 *     (floor 1e-30); a node is tagged iff delta >= eps_j (so eta = 0 refines all);
 *   - the root and all levels below jmin are always refined;
 *   - coarsening deletes the children of P when P was internal before the
 *     adaptation, P is untagged, P's level >= jmin, all children are leaves
 *     and no node two levels below P needs a child of P in its stencil;
 *   - new nodes are valued by prediction from the tree as it was before the
 *     adaptation (recursively where the stencil itself was absent);
 *   - ghost values across a level jump come from the same recursive value
 *     function; a coarse cell facing finer leaves receives minus the mean of
 *     their fluxes, so the operator conserves mass exactly.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ABSENT = 0, LEAF = 1, INTERNAL = 2 };

struct orc_tree {
  int d, J, jmin, m;
  int64_t n[ORC_MAXL + 1];
  uint8_t *st[ORC_MAXL + 1];
  double *v[ORC_MAXL + 1];
  int32_t *lidx[ORC_MAXL + 1];
};

/* ---------------- keys ---------------- */

uint64_t orc_key(int d, int j, const int32_t *k) {
  uint64_t s = 0;
  for (int b = 0; b < j; b++)
    for (int a = 0; a < d; a++)
      s |= (uint64_t)((k[a] >> b) & 1) << (d * b + (d - 1 - a));
  return s | ((uint64_t)j << 48);
}

void orc_key_decode(int d, uint64_t key, int *j, int32_t *k) {
  *j = (int)((key >> 48) & 15);
  for (int a = 0; a < 3; a++) k[a] = 0;
  for (int b = 0; b < *j; b++)
    for (int a = 0; a < d; a++)
      k[a] |= (int32_t)((key >> (d * b + (d - 1 - a))) & 1) << b;
}

/* ---------------- basic helpers ---------------- */

static int64_t pos(const orc_tree *T, int j, const int32_t *k) {
  int64_t p = 0;
  for (int a = T->d - 1; a >= 0; a--) p = (p << j) | k[a];
  return p;
}

static void unpos(const orc_tree *T, int j, int64_t p, int32_t *k) {
  k[0] = k[1] = k[2] = 0;
  for (int a = 0; a < T->d; a++) { k[a] = (int32_t)(p & ((1 << j) - 1)); p >>= j; }
}

static int in_range(const orc_tree *T, int j, const int32_t *k) {
  for (int a = 0; a < T->d; a++)
    if (k[a] < 0 || k[a] >= (1 << j)) return 0;
  return 1;
}

static int32_t mirror(int32_t k, int j) {
  if (k < 0) return -1 - k;
  if (k >= (1 << j)) return (2 << j) - 1 - k;
  return k;
}

/* 1D prediction weight for child offset a in {0,1} and coarse offset o in {-1,0,1} */
static double wpred(int a, int o) {
  if (o == 0) return 1.0;
  return ((o == -1) == (a == 0)) ? 0.125 : -0.125;
}

/* d in {2, 3}: the dimensions of the method's problems and of the GPU path
 * (the one-dimensional case is not supported) */
orc_tree *orc_tree_new(int d, int J, int jmin, int m) {
  if (d < 2 || d > 3 || J < 1 || J > ORC_MAXL || m < 1 || m > ORC_MAXM) return NULL;
  if ((int64_t)d * J > 48 || jmin < 1 || jmin > J) return NULL;
  orc_tree *T = calloc(1, sizeof *T);
  T->d = d; T->J = J; T->jmin = jmin; T->m = m;
  for (int j = 0; j <= J; j++) {
    T->n[j] = (int64_t)1 << (d * j);
    T->st[j] = calloc(T->n[j], 1);
    T->v[j] = calloc(T->n[j] * m, sizeof(double));
    T->lidx[j] = malloc(sizeof(int32_t) * T->n[j]);
    if (!T->st[j] || !T->v[j] || !T->lidx[j]) { orc_tree_free(T); return NULL; }
  }
  return T;
}

void orc_tree_free(orc_tree *T) {
  if (!T) return;
  for (int j = 0; j <= T->J; j++) { free(T->st[j]); free(T->v[j]); free(T->lidx[j]); }
  free(T);
}

/* leaves in key order (level, then Morton) get indices 0..N-1 */
static int64_t index_leaves(orc_tree *T) {
  int64_t cnt = 0;
  int32_t k[3];
  for (int j = 0; j <= T->J; j++) {
    for (int64_t p = 0; p < T->n[j]; p++) T->lidx[j][p] = -1;
    for (int64_t s = 0; s < T->n[j]; s++) {
      orc_key_decode(T->d, (uint64_t)s | ((uint64_t)j << 48), &(int){0}, k);
      int64_t p = pos(T, j, k);
      if (T->st[j][p] == LEAF) T->lidx[j][p] = (int32_t)cnt++;
    }
  }
  return cnt;
}

/* projection P^j_{j-1}: parent = mean of its 2^d children (Sec. 2.2) */
void orc_project(orc_tree *T) {
  const int d = T->d, m = T->m, nc = 1 << d;
  int32_t k[3], c[3] = {0, 0, 0};
  for (int j = T->J - 1; j >= 0; j--) {
    for (int64_t p = 0; p < T->n[j]; p++) {
      if (T->st[j][p] != INTERNAL) continue;
      unpos(T, j, p, k);
      for (int i = 0; i < m; i++) {
        double s = 0.0;
        for (int t = 0; t < nc; t++) {
          for (int a = 0; a < d; a++) c[a] = 2 * k[a] + ((t >> (d - 1 - a)) & 1);
          s += T->v[j + 1][(int64_t)i * T->n[j + 1] + pos(T, j + 1, c)];
        }
        T->v[j][(int64_t)i * T->n[j] + p] = s / nc;
      }
    }
  }
}

/* recursive value v(j,k): stored value if the node exists, else the
 * prediction from level j-1 (tensor product of Eq. inter_1d), mirror BC */
static double vrec(const orc_tree *T, int j, const int32_t *kin, int i) {
  int32_t k[3] = {0, 0, 0};
  for (int a = 0; a < T->d; a++) k[a] = mirror(kin[a], j);
  int64_t p = pos(T, j, k);
  if (T->st[j][p] != ABSENT) return T->v[j][(int64_t)i * T->n[j] + p];
  int32_t par[3] = {0, 0, 0}, q[3] = {0, 0, 0};
  for (int a = 0; a < T->d; a++) par[a] = k[a] >> 1;
  double s = 0.0;
  int nst = 1;
  for (int a = 0; a < T->d; a++) nst *= 3;
  for (int o = 0; o < nst; o++) {
    double w = 1.0;
    int oo = o;
    for (int a = 0; a < T->d; a++) {
      int off = oo % 3 - 1;
      oo /= 3;
      q[a] = par[a] + off;
      w *= wpred(k[a] & 1, off);
    }
    s += w * vrec(T, j - 1, q, i);
  }
  return s;
}

double orc_value(orc_tree *T, int j, const int32_t *k, int i) { return vrec(T, j, k, i); }

/* prediction of node (j,k) from its parent's 3^d stencil (j >= 1) */
static double predict(const orc_tree *T, int j, const int32_t *k, int i) {
  int32_t par[3] = {0, 0, 0}, q[3] = {0, 0, 0};
  for (int a = 0; a < T->d; a++) par[a] = k[a] >> 1;
  int nst = 1;
  for (int a = 0; a < T->d; a++) nst *= 3;
  double s = 0.0;
  for (int o = 0; o < nst; o++) {
    double w = 1.0;
    int oo = o;
    for (int a = 0; a < T->d; a++) {
      int off = oo % 3 - 1;
      oo /= 3;
      q[a] = par[a] + off;
      w *= wpred(k[a] & 1, off);
    }
    s += w * vrec(T, j - 1, q, i);
  }
  return s;
}

static int graded_at(const orc_tree *T, int j, const int32_t *k) {
  if (j < 1) return 1;
  int32_t par[3] = {0, 0, 0}, q[3] = {0, 0, 0};
  for (int a = 0; a < T->d; a++) par[a] = k[a] >> 1;
  int nst = 1;
  for (int a = 0; a < T->d; a++) nst *= 3;
  for (int o = 0; o < nst; o++) {
    int oo = o;
    for (int a = 0; a < T->d; a++) { q[a] = par[a] + (oo % 3 - 1); oo /= 3; }
    if (!in_range(T, j - 1, q)) continue;
    if (T->st[j - 1][pos(T, j - 1, q)] == ABSENT) return 0;
  }
  return 1;
}

int orc_tree_is_graded(orc_tree *T) {
  int32_t k[3];
  for (int j = 1; j <= T->J; j++)
    for (int64_t p = 0; p < T->n[j]; p++) {
      if (T->st[j][p] == ABSENT) continue;
      unpos(T, j, p, k);
      if (!graded_at(T, j, k)) return 0;
    }
  return 1;
}

static void clear_tree(orc_tree *T) {
  for (int j = 0; j <= T->J; j++) {
    memset(T->st[j], 0, T->n[j]);
    memset(T->v[j], 0, sizeof(double) * T->n[j] * T->m);
  }
}

/* full tree with leaves at level J; u0 is m x 2^(dJ), x fastest */
int orc_tree_set_full(orc_tree *T, const double *u0) {
  clear_tree(T);
  for (int j = 0; j < T->J; j++) memset(T->st[j], INTERNAL, T->n[j]);
  memset(T->st[T->J], LEAF, T->n[T->J]);
  memcpy(T->v[T->J], u0, sizeof(double) * T->n[T->J] * T->m);
  orc_project(T);
  return ORC_OK;
}

int orc_tree_set_leaves(orc_tree *T, int64_t n, const uint64_t *keys, const double *vals) {
  clear_tree(T);
  int32_t k[3];
  int j;
  for (int64_t r = 0; r < n; r++) {
    orc_key_decode(T->d, keys[r], &j, k);
    if (j > T->J) return ORC_EINVAL;
    int64_t p = pos(T, j, k);
    if (T->st[j][p] != ABSENT) return ORC_EINVAL;
    T->st[j][p] = LEAF;
    for (int i = 0; i < T->m; i++) T->v[j][(int64_t)i * T->n[j] + p] = vals[(int64_t)i * n + r];
  }
  /* mark ancestors internal */
  for (int jj = T->J; jj >= 1; jj--)
    for (int64_t p = 0; p < T->n[jj]; p++) {
      if (T->st[jj][p] == ABSENT) continue;
      unpos(T, jj, p, k);
      for (int a = 0; a < T->d; a++) k[a] >>= 1;
      int64_t pp = pos(T, jj - 1, k);
      if (T->st[jj - 1][pp] == LEAF) return ORC_EINVAL;
      T->st[jj - 1][pp] = INTERNAL;
    }
  if (T->st[0][0] == ABSENT) return ORC_EINVAL;
  /* every internal node has its complete family of children */
  const int nc = 1 << T->d;
  int32_t c[3] = {0, 0, 0};
  for (int jj = 0; jj < T->J; jj++)
    for (int64_t p = 0; p < T->n[jj]; p++) {
      if (T->st[jj][p] != INTERNAL) continue;
      unpos(T, jj, p, k);
      for (int t = 0; t < nc; t++) {
        for (int a = 0; a < T->d; a++) c[a] = 2 * k[a] + ((t >> a) & 1);
        if (T->st[jj + 1][pos(T, jj + 1, c)] == ABSENT) return ORC_EINVAL;
      }
    }
  for (int jj = 0; jj < T->jmin; jj++)
    for (int64_t p = 0; p < T->n[jj]; p++)
      if (T->st[jj][p] != INTERNAL) return ORC_EINVAL;
  if (!orc_tree_is_graded(T)) return ORC_EINVAL;
  orc_project(T);
  return ORC_OK;
}

int64_t orc_tree_num_leaves(orc_tree *T) { return index_leaves(T); }

int orc_tree_num_nodes(orc_tree *T, int64_t *per_level) {
  for (int j = 0; j <= T->J; j++) {
    int64_t c = 0;
    for (int64_t p = 0; p < T->n[j]; p++) c += T->st[j][p] != ABSENT;
    per_level[j] = c;
  }
  return ORC_OK;
}

int orc_tree_get_leaves(orc_tree *T, uint64_t *keys, double *vals) {
  int64_t N = index_leaves(T);
  int32_t k[3];
  for (int j = 0; j <= T->J; j++)
    for (int64_t p = 0; p < T->n[j]; p++) {
      int32_t r = T->lidx[j][p];
      if (r < 0) continue;
      unpos(T, j, p, k);
      if (keys) keys[r] = orc_key(T->d, j, k);
      if (vals)
        for (int i = 0; i < T->m; i++) vals[(int64_t)i * N + r] = T->v[j][(int64_t)i * T->n[j] + p];
    }
  return ORC_OK;
}

static void set_leaf_values(orc_tree *T, const double *vals, int64_t N) {
  int32_t k[3];
  for (int j = 0; j <= T->J; j++)
    for (int64_t p = 0; p < T->n[j]; p++) {
      int32_t r = T->lidx[j][p];
      if (r < 0) continue;
      (void)k;
      for (int i = 0; i < T->m; i++) T->v[j][(int64_t)i * T->n[j] + p] = vals[(int64_t)i * N + r];
    }
}

/* ---------------- details and thresholds ---------------- */

static void scales(orc_tree *T, double *s) {
  for (int i = 0; i < T->m; i++) s[i] = 0.0;
  for (int j = 0; j <= T->J; j++)
    for (int64_t p = 0; p < T->n[j]; p++)
      if (T->st[j][p] == LEAF)
        for (int i = 0; i < T->m; i++)
          s[i] = fmax(s[i], fabs(T->v[j][(int64_t)i * T->n[j] + p]));
  for (int i = 0; i < T->m; i++) s[i] = fmax(s[i], 1e-30);
}

/* delta = max_i |v_i - P^{j-1}_j P^j_{j-1} v_i| / s_i (Eq. detail) */
static double detail(const orc_tree *T, int j, const int32_t *k, const double *s) {
  double dmax = 0.0;
  int64_t p = pos(T, j, k);
  for (int i = 0; i < T->m; i++) {
    double dd = fabs(T->v[j][(int64_t)i * T->n[j] + p] - predict(T, j, k, i)) / s[i];
    if (dd > dmax) dmax = dd;
  }
  return dmax;
}

static double eps_level(const orc_tree *T, int j, double eta) {
  return eta * pow(2.0, 0.5 * T->d * (j - T->J));
}

int orc_details(orc_tree *T, int64_t cap, uint64_t *keys, double *delta) {
  orc_project(T);
  double s[ORC_MAXM];
  scales(T, s);
  int64_t c = 0;
  int32_t k[3];
  for (int j = 1; j <= T->J; j++)
    for (int64_t q = 0; q < T->n[j]; q++) {
      orc_key_decode(T->d, (uint64_t)q | ((uint64_t)j << 48), &(int){0}, k);
      int64_t p = pos(T, j, k);
      if (T->st[j][p] == ABSENT) continue;
      if (c < cap) { keys[c] = orc_key(T->d, j, k); delta[c] = detail(T, j, k, s); }
      c++;
    }
  return (int)(c > cap ? -1 : 0);
}

/* ---------------- adaptation (Sec. 3.1.2) ---------------- */

typedef struct { uint8_t *st[ORC_MAXL + 1]; double *v[ORC_MAXL + 1]; int64_t n[ORC_MAXL + 1]; int d, J, m; } snap_t;

static void refine_leaf(orc_tree *T, const orc_tree *S, int j, const int32_t *k, uint8_t **added) {
  const int nc = 1 << T->d;
  int32_t c[3] = {0, 0, 0};
  T->st[j][pos(T, j, k)] = INTERNAL;
  for (int t = 0; t < nc; t++) {
    for (int a = 0; a < T->d; a++) c[a] = 2 * k[a] + ((t >> a) & 1);
    int64_t p = pos(T, j + 1, c);
    T->st[j + 1][p] = LEAF;
    added[j + 1][p] = 1;
    for (int i = 0; i < T->m; i++) T->v[j + 1][(int64_t)i * T->n[j + 1] + p] = vrec(S, j + 1, c, i);
  }
}

int orc_adapt(orc_tree *T, double eta) {
  const int d = T->d, J = T->J, m = T->m;
  orc_project(T);
  /* snapshot of the tree before adaptation: the source of every new value */
  orc_tree S = *T;
  for (int j = 0; j <= J; j++) {
    S.st[j] = malloc(T->n[j]);
    S.v[j] = malloc(sizeof(double) * T->n[j] * m);
    memcpy(S.st[j], T->st[j], T->n[j]);
    memcpy(S.v[j], T->v[j], sizeof(double) * T->n[j] * m);
    S.lidx[j] = NULL;
  }
  uint8_t *tag[ORC_MAXL + 1], *added[ORC_MAXL + 1];
  double s[ORC_MAXM];
  scales(T, s);
  int32_t k[3], q[3] = {0, 0, 0}, c[3] = {0, 0, 0};
  for (int j = 0; j <= J; j++) {
    tag[j] = calloc(T->n[j], 1);
    added[j] = calloc(T->n[j], 1);
    if (j == 0) continue;
    double ej = eps_level(T, j, eta);
    for (int64_t p = 0; p < T->n[j]; p++) {
      if (S.st[j][p] == ABSENT) continue;
      unpos(T, j, p, k);
      tag[j][p] = detail(&S, j, k, s) >= ej;
    }
  }
  /* refinement of tagged leaves (all at once, from the snapshot) */
  for (int j = 1; j < J; j++)
    for (int64_t p = 0; p < T->n[j]; p++)
      if (S.st[j][p] == LEAF && tag[j][p]) {
        unpos(T, j, p, k);
        refine_leaf(T, &S, j, k, added);
      }
  /* tag-and-refine until every prediction stencil is present */
  const int nst = d == 2 ? 9 : 27;
  for (int changed = 1; changed;) {
    changed = 0;
    for (int j = J; j >= 2; j--)
      for (int64_t p = 0; p < T->n[j]; p++) {
        if (T->st[j][p] == ABSENT) continue;
        unpos(T, j, p, k);
        for (int o = 0; o < nst; o++) {
          int oo = o;
          for (int a = 0; a < d; a++) { q[a] = (k[a] >> 1) + (oo % 3 - 1); oo /= 3; }
          if (!in_range(T, j - 1, q)) continue;
          if (T->st[j - 1][pos(T, j - 1, q)] != ABSENT) continue;
          /* refine the deepest existing ancestor of (j-1, q): it is a leaf */
          int jj = j - 1;
          int32_t aq[3] = {q[0], q[1], q[2]};
          while (T->st[jj][pos(T, jj, aq)] == ABSENT) {
            for (int a = 0; a < d; a++) aq[a] >>= 1;
            jj--;
          }
          refine_leaf(T, &S, jj, aq, added);
          changed = 1;
        }
      }
  }
  /* coarsening passes until no deletion */
  const int nc = 1 << d;
  int64_t *cand = NULL;
  int64_t ccap = 0;
  for (int deleted = 1; deleted;) {
    deleted = 0;
    for (int j = J - 1; j >= T->jmin; j--) {
      int64_t nc_list = 0;
      for (int64_t p = 0; p < T->n[j]; p++) {
        if (T->st[j][p] != INTERNAL || S.st[j][p] != INTERNAL || tag[j][p]) continue;
        unpos(T, j, p, k);
        int ok = 1;
        for (int t = 0; t < nc && ok; t++) {
          for (int a = 0; a < d; a++) c[a] = 2 * k[a] + ((t >> a) & 1);
          if (T->st[j + 1][pos(T, j + 1, c)] != LEAF) ok = 0;
        }
        /* no node at level j+2 has a child of P in its prediction stencil */
        if (ok && j + 2 <= J) {
          int32_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
          for (int a = 0; a < d; a++) {
            lo[a] = 4 * k[a] - 2; hi[a] = 4 * k[a] + 5;
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > (1 << (j + 2)) - 1) hi[a] = (1 << (j + 2)) - 1;
          }
          int32_t g[3] = {0, 0, 0};
          for (g[2] = lo[2]; g[2] <= hi[2] && ok; g[2]++)
            for (g[1] = lo[1]; g[1] <= hi[1] && ok; g[1]++)
              for (g[0] = lo[0]; g[0] <= hi[0] && ok; g[0]++)
                if (T->st[j + 2][pos(T, j + 2, g)] != ABSENT) ok = 0;
        }
        if (!ok) continue;
        if (nc_list == ccap) { ccap = ccap ? 2 * ccap : 1024; cand = realloc(cand, sizeof(int64_t) * ccap); }
        cand[nc_list++] = p;
      }
      for (int64_t r = 0; r < nc_list; r++) {
        unpos(T, j, cand[r], k);
        for (int t = 0; t < nc; t++) {
          for (int a = 0; a < d; a++) c[a] = 2 * k[a] + ((t >> a) & 1);
          T->st[j + 1][pos(T, j + 1, c)] = ABSENT;
        }
        T->st[j][cand[r]] = LEAF; /* keeps its projected value */
        deleted = 1;
      }
    }
  }
  free(cand);
  for (int j = 0; j <= J; j++) { free(S.st[j]); free(S.v[j]); free(tag[j]); free(added[j]); }
  orc_project(T);
  return orc_tree_is_graded(T) ? ORC_OK : ORC_ESTATE;
}

/* ---------------- finite-volume leaf operator (Eq. discretise, App. C) ---- */

typedef struct { int32_t *col; double *w; int64_t n, cap; } row_t;

static void row_add(row_t *r, int32_t col, double w) {
  if (r->n == r->cap) {
    r->cap = r->cap ? 2 * r->cap : 64;
    r->col = realloc(r->col, sizeof(int32_t) * r->cap);
    r->w = realloc(r->w, sizeof(double) * r->cap);
  }
  r->col[r->n] = col;
  r->w[r->n] = w;
  r->n++;
}

/* symbolic value: v(j,k) as a linear combination of leaf values */
static void vsym(const orc_tree *T, int j, const int32_t *kin, double w, row_t *r) {
  int32_t k[3] = {0, 0, 0};
  for (int a = 0; a < T->d; a++) k[a] = mirror(kin[a], j);
  int64_t p = pos(T, j, k);
  if (T->st[j][p] == LEAF) { row_add(r, T->lidx[j][p], w); return; }
  if (T->st[j][p] == INTERNAL) {
    const int nc = 1 << T->d;
    int32_t c[3] = {0, 0, 0};
    for (int t = 0; t < nc; t++) {
      for (int a = 0; a < T->d; a++) c[a] = 2 * k[a] + ((t >> a) & 1);
      vsym(T, j + 1, c, w / nc, r);
    }
    return;
  }
  int32_t par[3] = {0, 0, 0}, q[3] = {0, 0, 0};
  for (int a = 0; a < T->d; a++) par[a] = k[a] >> 1;
  int nst = T->d == 2 ? 9 : 27;
  for (int o = 0; o < nst; o++) {
    double ww = 1.0;
    int oo = o;
    for (int a = 0; a < T->d; a++) {
      int off = oo % 3 - 1;
      oo /= 3;
      q[a] = par[a] + off;
      ww *= wpred(k[a] & 1, off);
    }
    vsym(T, j - 1, q, w * ww, r);
  }
}

static int cmp_col(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* row of leaf (j,k): (L u)_L = (1/h_j) sum over faces of the face flux */
static void leaf_row(const orc_tree *T, int j, const int32_t *k, row_t *r) {
  const int d = T->d;
  const double ih = ldexp(1.0, j), ih1 = ldexp(1.0, j + 1);
  const int32_t self = T->lidx[j][pos(T, j, k)];
  int32_t nk[3], c[3], g[3];
  for (int a = 0; a < d; a++)
    for (int sg = -1; sg <= 1; sg += 2) {
      memcpy(nk, k, sizeof nk);
      nk[a] += sg;
      if (!in_range(T, j, nk)) continue; /* homogeneous Neumann: zero flux */
      uint8_t stn = T->st[j][pos(T, j, nk)];
      if (stn == LEAF || stn == ABSENT) {
        vsym(T, j, nk, ih * ih, r); /* same-level leaf or predicted ghost */
        row_add(r, self, -ih * ih);
      } else {
        /* finer side: minus the mean of the fluxes into the 2^(d-1) children of
         * the neighbour that touch the face, each computed at level j+1 against
         * the predicted value of the adjacent child cell of this leaf */
        const int nc = 1 << d;
        const double coef = ih * ih1 / (double)(nc / 2);
        for (int t = 0; t < nc; t++) {
          for (int b = 0; b < d; b++) c[b] = 2 * nk[b] + ((t >> b) & 1);
          if (c[a] != 2 * nk[a] + (sg > 0 ? 0 : 1)) continue;
          memcpy(g, c, sizeof g);
          g[a] -= sg;
          vsym(T, j + 1, g, -coef, r);
          vsym(T, j + 1, c, coef, r);
        }
      }
    }
  /* merge duplicate columns (weights are dyadic: the sums are exact) */
  int64_t n = r->n;
  /* sort (col, w) pairs by col */
  struct cw { int32_t col; int32_t pad; double w; } *tmp = malloc(sizeof(struct cw) * (n ? n : 1));
  for (int64_t e = 0; e < n; e++) { tmp[e].col = r->col[e]; tmp[e].pad = 0; tmp[e].w = r->w[e]; }
  qsort(tmp, n, sizeof(struct cw), cmp_col);
  int64_t o = 0;
  for (int64_t e = 0; e < n;) {
    int32_t cc = tmp[e].col;
    double s = 0.0;
    while (e < n && tmp[e].col == cc) s += tmp[e++].w;
    if (s != 0.0) { r->col[o] = cc; r->w[o] = s; o++; }
  }
  r->n = o;
  free(tmp);
}

/* Rows of the operator, one per leaf in leaf (key) order.  Rows are
 * independent: with several oracle threads they are built by the
 * parallel-for in fixed chunks of consecutive leaves, each chunk into its own
 * buffer, and the chunks are concatenated in order, so the result is that of
 * the serial loop. */
typedef struct {
  const orc_tree *T;
  const int8_t *lj;     /* level of leaf r */
  const int32_t *lk;    /* coordinates of leaf r (3 per leaf) */
  row_t *chunk_rows;    /* per chunk: the concatenated rows */
  int64_t *cnt;         /* per leaf: entries of its row */
  double *chunk_rmax;   /* per chunk: largest absolute row sum */
} op_args;

static void op_rows(void *ctx, int64_t lo, int64_t hi, int c) {
  op_args *a = (op_args *)ctx;
  row_t row = {0};
  row_t *out = &a->chunk_rows[c];
  double rmax = 0.0;
  for (int64_t r = lo; r < hi; r++) {
    row.n = 0;
    leaf_row(a->T, a->lj[r], a->lk + 3 * r, &row);
    double sa = 0.0;
    for (int64_t e = 0; e < row.n; e++) {
      sa += fabs(row.w[e]);
      row_add(out, row.col[e], row.w[e]);
    }
    rmax = fmax(rmax, sa);
    a->cnt[r] = row.n;
  }
  a->chunk_rmax[c] = rmax;
  free(row.col);
  free(row.w);
}

int orc_operator(orc_tree *T, int64_t cap, int64_t *rowptr, int32_t *col, double *val, double *rho) {
  int64_t N = index_leaves(T);
  int8_t *lj = malloc(N ? N : 1);
  int32_t *lk = calloc(3 * (N ? N : 1), sizeof(int32_t));
  int32_t k[3];
  for (int j = 0; j <= T->J; j++)
    for (int64_t sm = 0; sm < T->n[j]; sm++) { /* leaves in key order */
      orc_key_decode(T->d, (uint64_t)sm | ((uint64_t)j << 48), &(int){0}, k);
      int32_t r = T->lidx[j][pos(T, j, k)];
      if (r < 0) continue;
      lj[r] = (int8_t)j;
      memcpy(lk + 3 * (int64_t)r, k, sizeof k);
    }
  const int64_t chunk = 512, nchunks = (N + chunk - 1) / chunk;
  op_args a = {T, lj, lk, calloc(nchunks ? nchunks : 1, sizeof(row_t)), malloc(sizeof(int64_t) * (N ? N : 1)),
               calloc(nchunks ? nchunks : 1, sizeof(double))};
  orc_parallel_for(N, chunk, op_rows, &a);
  int64_t nnz = 0;
  double rmax = 0.0;
  int over = 0;
  for (int64_t c = 0; c < nchunks; c++) {
    const row_t *cr = &a.chunk_rows[c];
    for (int64_t e = 0; e < cr->n; e++)
      if (nnz + e < cap) { col[nnz + e] = cr->col[e]; val[nnz + e] = cr->w[e]; }
    for (int64_t r = c * chunk; r < N && r < (c + 1) * chunk; r++) {
      rowptr[r] = nnz;
      nnz += a.cnt[r];
    }
    if (nnz > cap) over = 1;
    rmax = fmax(rmax, a.chunk_rmax[c]);
    free(cr->col);
    free(cr->w);
  }
  rowptr[N] = nnz;
  free(a.chunk_rows);
  free(a.cnt);
  free(a.chunk_rmax);
  free(lj);
  free(lk);
  if (rho) *rho = rmax;
  return over ? -1 : 0;
}

/* literal evaluation of L u with the numeric value function (cross-check of
 * the explicit rows): u and out are m x N in leaf order */
int orc_apply_literal(orc_tree *T, const double *u, double *out) {
  int64_t N = index_leaves(T);
  set_leaf_values(T, u, N);
  orc_project(T);
  const int d = T->d, m = T->m;
  int32_t k[3], nk[3], c[3], g[3];
  for (int j = 0; j <= T->J; j++)
    for (int64_t p = 0; p < T->n[j]; p++) {
      int32_t r = T->lidx[j][p];
      if (r < 0) continue;
      unpos(T, j, p, k);
      const double hj = ldexp(1.0, -j), hj1 = ldexp(1.0, -(j + 1));
      for (int i = 0; i < m; i++) {
        double uL = T->v[j][(int64_t)i * T->n[j] + p], acc = 0.0;
        for (int a = 0; a < d; a++)
          for (int sg = -1; sg <= 1; sg += 2) {
            memcpy(nk, k, sizeof nk);
            nk[a] += sg;
            if (!in_range(T, j, nk)) continue;
            uint8_t stn = T->st[j][pos(T, j, nk)];
            double F;
            if (stn != INTERNAL) {
              F = (vrec(T, j, nk, i) - uL) / hj;
            } else {
              const int nc = 1 << d;
              double sum = 0.0;
              for (int t = 0; t < nc; t++) {
                for (int b = 0; b < d; b++) c[b] = 2 * nk[b] + ((t >> b) & 1);
                if (c[a] != 2 * nk[a] + (sg > 0 ? 0 : 1)) continue;
                memcpy(g, c, sizeof g);
                g[a] -= sg;
                sum += (vrec(T, j + 1, g, i) - vrec(T, j + 1, c, i)) / hj1;
              }
              F = -sum / (double)(nc / 2);
            }
            acc += F / hj;
          }
        out[(int64_t)i * N + r] = acc;
      }
    }
  return ORC_OK;
}

/* ---------------- reaction, diffusion, Strang, mass ---------------- */

/* every leaf integrates its own ODE: a parallel-for over the leaves (in leaf
 * order); per-chunk counters and first errors are combined in chunk order, so
 * the outcome is that of the serial loop */
typedef struct {
  orc_tree *T;
  const orc_model *md;
  double dt, rtol, atol;
  int32_t *complexity;
  int32_t (*leaf)[2]; /* (level, position) of every leaf, in leaf order */
  orc_radau_stats *part;
} react_args;

static void react_leaves(void *p, int64_t lo, int64_t hi, int chunk) {
  react_args *a = (react_args *)p;
  orc_tree *T = a->T;
  const int m = T->m;
  orc_radau_stats *agg = &a->part[chunk];
  double y[ORC_MAXM];
  for (int64_t q = lo; q < hi; q++) {
    const int j = a->leaf[q][0];
    const int64_t pos = a->leaf[q][1];
    for (int i = 0; i < m; i++) y[i] = T->v[j][(int64_t)i * T->n[j] + pos];
    orc_radau_stats st;
    int rc = orc_radau5(a->md, y, a->dt, a->rtol, a->atol, 0.0, &st);
    if (rc && agg->status == ORC_OK) agg->status = rc;
    for (int i = 0; i < m; i++) T->v[j][(int64_t)i * T->n[j] + pos] = y[i];
    if (a->complexity) a->complexity[q] = (int32_t)(st.nfev + (int64_t)m * st.njac);
    agg->nfev += st.nfev; agg->njac += st.njac; agg->nstep += st.nstep;
    agg->naccept += st.naccept; agg->nreject += st.nreject;
    agg->nnewton += st.nnewton; agg->ndec += st.ndec;
  }
}

int orc_react(orc_tree *T, const orc_model *md, double dt, double rtol, double atol,
              orc_radau_stats *agg, int32_t *complexity) {
  int64_t N = index_leaves(T);
  int32_t (*leaf)[2] = malloc(sizeof(int32_t[2]) * (N > 0 ? N : 1));
  for (int j = 0; j <= T->J; j++)
    for (int64_t p = 0; p < T->n[j]; p++) {
      int32_t r = T->lidx[j][p];
      if (r < 0) continue;
      leaf[r][0] = j;
      leaf[r][1] = (int32_t)p;
    }
  const int64_t chunk = 64, nchunks = (N + chunk - 1) / chunk;
  orc_radau_stats *part = calloc(nchunks > 0 ? nchunks : 1, sizeof(orc_radau_stats));
  react_args a = {T, md, dt, rtol, atol, complexity, leaf, part};
  orc_parallel_for(N, chunk, react_leaves, &a);
  orc_radau_stats tot;
  memset(&tot, 0, sizeof tot);
  for (int64_t q = 0; q < nchunks; q++) {
    if (part[q].status && tot.status == ORC_OK) tot.status = part[q].status;
    tot.nfev += part[q].nfev; tot.njac += part[q].njac; tot.nstep += part[q].nstep;
    tot.naccept += part[q].naccept; tot.nreject += part[q].nreject;
    tot.nnewton += part[q].nnewton; tot.ndec += part[q].ndec;
  }
  free(part);
  free(leaf);
  if (agg) *agg = tot;
  return tot.status;
}

int orc_diffuse(orc_tree *T, const double *D, double dt, double tol, orc_rock_stats *agg) {
  int64_t N = index_leaves(T);
  int64_t cap = N * 32 + 1024;
  int64_t *rp = malloc(sizeof(int64_t) * (N + 1));
  int32_t *col = NULL;
  double *val = NULL, rho = 0.0;
  for (;;) {
    col = realloc(col, sizeof(int32_t) * cap);
    val = realloc(val, sizeof(double) * cap);
    if (orc_operator(T, cap, rp, col, val, &rho) == 0) break;
    cap = rp[N] + 16;
  }
  double *u = malloc(sizeof(double) * N * T->m);
  orc_tree_get_leaves(T, NULL, u);
  int status = ORC_OK;
  if (agg) memset(agg, 0, sizeof *agg);
  for (int i = 0; i < T->m; i++) {
    orc_rock_stats st = {0};
    int rc = orc_rock4_linear(N, rp, col, val, D[i], rho, u + (int64_t)i * N, dt, tol, 0.0, &st);
    if (rc && status == ORC_OK) status = rc;
    if (agg) {
      agg->nsteps += st.nsteps; agg->naccept += st.naccept; agg->nreject += st.nreject;
      agg->nstages += st.nstages; agg->nmatvec += st.nmatvec;
      if (st.smax > agg->smax) agg->smax = st.smax;
    }
  }
  set_leaf_values(T, u, N);
  free(rp); free(col); free(val); free(u);
  if (agg) agg->status = status;
  return status;
}

int orc_strang(orc_tree *T, const orc_model *md, const double *D, double dt,
               double eta, double rtol, double atol, double rock_tol) {
  int rc = orc_adapt(T, eta);
  if (rc) return rc;
  if ((rc = orc_react(T, md, 0.5 * dt, rtol, atol, NULL, NULL))) return rc;
  if ((rc = orc_diffuse(T, D, dt, rock_tol, NULL))) return rc;
  if ((rc = orc_react(T, md, 0.5 * dt, rtol, atol, NULL, NULL))) return rc;
  return ORC_OK;
}

void orc_mass(orc_tree *T, double *mass) {
  for (int i = 0; i < T->m; i++) mass[i] = 0.0;
  for (int j = 0; j <= T->J; j++) {
    double vol = ldexp(1.0, -T->d * j);
    for (int64_t p = 0; p < T->n[j]; p++)
      if (T->st[j][p] == LEAF)
        for (int i = 0; i < T->m; i++) mass[i] += vol * T->v[j][(int64_t)i * T->n[j] + p];
  }
}
