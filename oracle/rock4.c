/*
 * Oracle (test infrastructure only): ROCK4-type stabilized explicit
 * integrator for the linear diffusion sub-step D_dt.
 *
 * Paper, Sec. 3.2.1: ROCK4 is the composition of (i) s-4 stages of a
 * three-term recurrence of orthogonal polynomials whose number depends on the
 * spectral radius of the Jacobian and (ii) an explicit 4-stage Runge-Kutta
 * finishing procedure (Eq. RKscheme).  For the linear problem y' = A y the
 * finishing procedure is y_{n+1} = pi(dt A) y with pi a polynomial evaluated
 * by Horner's rule (it has complex roots, so it is not factorised); the
 * spectral radius comes from Gershgorin's theorem.
 *
 * The coefficient tables of the published ROCK4 code are not available, so
 * the polynomials are recomputed here from Abdulle's construction (MR1923724):
 *   R_s(z) = w(x) P_{s-4}(x),  x = 1 + 2 z / l_s,  z in [-l_s, 0] <-> x in [-1, 1],
 *   P_j orthogonal on [-1,1] for the weight w(x)^2 / sqrt(1 - x^2), P_j(1) = 1,
 *   w a quartic with w(1) = 1 fixed by the order conditions R_s(z) = e^z + O(z^5).
 * The pair (w, P) is the fixed point of: P <- orthogonal family of w^2/sqrt(1-x^2)
 * (Stieltjes procedure on Gauss-Chebyshev nodes, exact for these degrees);
 * w <- Taylor series of exp(l t/2) / P(1 + t) truncated after t^4.
 * The interval length is fixed by formula, l_s = 0.336 s^2 - 2.7 (about 95% of
 * the largest stable length of this family, which grows like 0.354 s^2).
 *
 * Embedded estimate: the difference between y_{n+1} and an order-3 solution
 * built from the same vectors, E = a y_P + b1 h1 + b2 h2 + y_{n+1} + d dt A y_{n+1},
 * where h_k are the Horner partial sums and (a, b1, b2, d) make E = O(z^4).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SMIN 5
#define SMAX 152

double orc_rock4_ell(int s) { return 0.336 * (double)s * s - 2.7; }

static int gauss_solve(int n, double *a, double *b) {
  for (int k = 0; k < n; k++) {
    int p = k;
    for (int i = k + 1; i < n; i++)
      if (fabs(a[i * n + k]) > fabs(a[p * n + k])) p = i;
    if (a[p * n + k] == 0.0) return -1;
    if (p != k) {
      for (int j = 0; j < n; j++) { double t = a[k*n+j]; a[k*n+j] = a[p*n+j]; a[p*n+j] = t; }
      double t = b[k]; b[k] = b[p]; b[p] = t;
    }
    for (int i = k + 1; i < n; i++) {
      double l = a[i * n + k] / a[k * n + k];
      for (int j = k; j < n; j++) a[i * n + j] -= l * a[k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int k = n - 1; k >= 0; k--) {
    double s = b[k];
    for (int j = k + 1; j < n; j++) s -= a[k * n + j] * b[j];
    b[k] = s / a[k * n + k];
  }
  return 0;
}

/*
 * Coefficients for s stages (n = s - 4 recurrence stages):
 *   P_{j+1} = mu[j+1] P_j + nu[j+1] P_{j-1} + kap[j+1] z P_j,  j = 0..n-1
 *   w(z) = sum_k w[k] z^k (w[0] = 1), errc = (a, b1, b2, d), xc = w in (x-1).
 */
int orc_rock4_coeffs(int s, double *mu, double *nu, double *kap, double w[5],
                     double errc[4], double xc[5]) {
  if (s < SMIN || s > SMAX) return ORC_EINVAL;
  const int n = s - 4;
  const double l = orc_rock4_ell(s);
  const int M = 2 * n + 64;
  double *x = malloc(sizeof(double) * M), *wt = malloc(sizeof(double) * M);
  double *pc = malloc(sizeof(double) * M), *pp = malloc(sizeof(double) * M);
  double *a = malloc(sizeof(double) * (n + 1)), *b = malloc(sizeof(double) * (n + 1));
  for (int k = 0; k < M; k++) x[k] = cos((2.0 * k + 1.0) * M_PI / (2.0 * M));
  double c[5], cn[5], E[5];
  double fact = 1.0;
  for (int k = 0; k < 5; k++) {
    if (k) fact *= k;
    E[k] = pow(l / 2.0, k) / fact;
    c[k] = E[k];
  }
  int it, conv = 0;
  for (it = 0; it < 300; it++) {
    /* weight w(x)^2 at the Chebyshev nodes; Stieltjes procedure */
    for (int k = 0; k < M; k++) {
      double t = x[k] - 1.0, wx = c[4];
      for (int q = 3; q >= 0; q--) wx = wx * t + c[q];
      wt[k] = wx * wx;
      pc[k] = 1.0;
      pp[k] = 0.0;
    }
    double nprev = 1.0;
    for (int j = 0; j < n; j++) {
      double nr = 0.0, xr = 0.0;
      for (int k = 0; k < M; k++) { nr += wt[k] * pc[k] * pc[k]; xr += wt[k] * x[k] * pc[k] * pc[k]; }
      a[j] = xr / nr;
      b[j] = j ? nr / nprev : 0.0;
      nprev = nr;
      for (int k = 0; k < M; k++) {
        double nx = (x[k] - a[j]) * pc[k] - b[j] * pp[k];
        pp[k] = pc[k];
        pc[k] = nx;
      }
    }
    /* Taylor coefficients (in t = x - 1) of the normalised P_n, P_n(1) = 1 */
    double P[5] = {1, 0, 0, 0, 0}, Pm[5] = {0, 0, 0, 0, 0}, rho = 0.0;
    for (int j = 0; j < n; j++) {
      double den = (1.0 - a[j]) - b[j] * rho;
      double Pn[5];
      for (int q = 0; q < 5; q++)
        Pn[q] = ((1.0 - a[j]) * P[q] + (q ? P[q - 1] : 0.0) - b[j] * rho * Pm[q]) / den;
      memcpy(Pm, P, sizeof P);
      memcpy(P, Pn, sizeof P);
      rho = 1.0 / den;
    }
    /* w = E / P truncated after t^4 */
    for (int q = 0; q < 5; q++) {
      double acc = E[q];
      for (int r = 0; r < q; r++) acc -= cn[r] * P[q - r];
      cn[q] = acc / P[0];
    }
    double dmax = 0.0, cmax = 0.0;
    for (int q = 0; q < 5; q++) { dmax = fmax(dmax, fabs(cn[q] - c[q])); cmax = fmax(cmax, fabs(cn[q])); }
    memcpy(c, cn, sizeof c);
    if (dmax <= 1e-14 * cmax) { conv = 1; break; }
  }
  if (!conv) { free(x); free(wt); free(pc); free(pp); free(a); free(b); return ORC_ESTATE; }
  /* recurrence coefficients for the converged weight */
  for (int k = 0; k < M; k++) {
    double t = x[k] - 1.0, wx = c[4];
    for (int q = 3; q >= 0; q--) wx = wx * t + c[q];
    wt[k] = wx * wx;
    pc[k] = 1.0;
    pp[k] = 0.0;
  }
  double nprev = 1.0;
  for (int j = 0; j < n; j++) {
    double nr = 0.0, xr = 0.0;
    for (int k = 0; k < M; k++) { nr += wt[k] * pc[k] * pc[k]; xr += wt[k] * x[k] * pc[k] * pc[k]; }
    a[j] = xr / nr;
    b[j] = j ? nr / nprev : 0.0;
    nprev = nr;
    for (int k = 0; k < M; k++) {
      double nx = (x[k] - a[j]) * pc[k] - b[j] * pp[k];
      pp[k] = pc[k];
      pc[k] = nx;
    }
  }
  double rho = 0.0;
  mu[0] = nu[0] = kap[0] = 0.0;
  for (int j = 0; j < n; j++) {
    double den = (1.0 - a[j]) - b[j] * rho;
    mu[j + 1] = (1.0 - a[j]) / den;
    nu[j + 1] = -b[j] * rho / den;
    kap[j + 1] = (2.0 / l) / den;
    rho = 1.0 / den;
  }
  for (int q = 0; q < 5; q++) {
    xc[q] = c[q];
    w[q] = c[q] * pow(2.0 / l, q);
  }
  /* embedded combination: (a, b1, b2, d) with
   *   a*1 + b1*h1(z) + b2*h2(z) + w(z) + d*z*w(z) = O(z^4)
   * h1 = w1 + w2 z + w3 z^2 + w4 z^3,  h2 = w2 + w3 z + w4 z^2 */
  double Mx[16] = {
      1.0, w[1], w[2], 0.0,
      0.0, w[2], w[3], 1.0,
      0.0, w[3], w[4], w[1],
      0.0, w[4], 0.0,  w[2]};
  double rhs[4] = {-w[0], -w[1], -w[2], -w[3]};
  int bad = gauss_solve(4, Mx, rhs);
  for (int q = 0; q < 4; q++) errc[q] = rhs[q];
  free(x); free(wt); free(pc); free(pp); free(a); free(b);
  return bad ? ORC_ESTATE : ORC_OK;
}

/* smallest s in [5,152] with l_s >= rho*dt; 1 if even s = 152 is too short */
int orc_rock4_choose(double rho_dt, int *s, double *ell) {
  for (int q = SMIN; q <= SMAX; q++)
    if (orc_rock4_ell(q) >= rho_dt) { *s = q; *ell = orc_rock4_ell(q); return 0; }
  *s = SMAX;
  *ell = orc_rock4_ell(SMAX);
  return 1;
}

typedef struct {
  const int64_t *rp;
  const int32_t *col;
  const double *val, *x;
  double scale, *y;
} mv_args;

static void matvec_rows(void *p, int64_t lo, int64_t hi, int chunk) {
  const mv_args *a = (const mv_args *)p;
  (void)chunk;
  for (int64_t r = lo; r < hi; r++) {
    double acc = 0.0;
    for (int64_t e = a->rp[r]; e < a->rp[r + 1]; e++) acc += a->val[e] * a->x[a->col[e]];
    a->y[r] = a->scale * acc;
  }
}

/* y = scale * (A x), rows independent (parallel-for over rows) */
static void matvec(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                   double scale, const double *x, double *y) {
  mv_args a = {rp, col, val, x, scale, y};
  orc_parallel_for(n, 4096, matvec_rows, &a);
}

/*
 * Integrate y' = D L y over [0, dt] in place, L given as CSR, rho = Gershgorin
 * bound of L (so D rho bounds the spectral radius of D L).
 * hfix > 0: fixed steps, no error control (order pins); else adaptive with
 *   err = WRMS(E / (tol + tol max(|y_n|, |y_{n+1}|))), accept err <= 1,
 *   dt_new = dt clamp(0.8 err^(-1/4), 0.2, 2), first step = whole interval.
 */
int orc_rock4_linear(int64_t n, const int64_t *rowptr, const int32_t *col,
                     const double *val, double D, double rho, double *y,
                     double dt, double tol, double hfix, orc_rock_stats *st) {
  double *P0 = malloc(sizeof(double) * n), *P1 = malloc(sizeof(double) * n);
  double *P2 = malloc(sizeof(double) * n), *Av = malloc(sizeof(double) * n);
  double *h1 = malloc(sizeof(double) * n), *h2 = malloc(sizeof(double) * n);
  double *yP = malloc(sizeof(double) * n);
  double mu[SMAX], nu[SMAX], kap[SMAX], w[5], ec[4], xc[5];
  int status = ORC_OK;
  double t = 0.0, h = hfix > 0 ? hfix : dt;
  while (t < dt) {
    int last = 0, s;
    double ell;
    if (t + 1.0001 * h >= dt) { h = dt - t; last = 1; }
    if (orc_rock4_choose(D * rho * h, &s, &ell)) { h = ell / (D * rho); last = 0; }
    if (h <= 1e-14 * dt) { status = ORC_EROCK_STEP; break; }
    if (orc_rock4_coeffs(s, mu, nu, kap, w, ec, xc)) { status = ORC_ESTATE; break; }
    const int ns = s - 4;
    if (s > st->smax) st->smax = s;
    st->nsteps++;
    st->nstages += s;
    /* recurrence stages P_1..P_ns from P_0 = y */
    memcpy(P0, y, sizeof(double) * n);
    double *pm = NULL, *pc = P0;
    double *bufs[3] = {P1, P2, yP};
    int bi = 0;
    for (int j = 1; j <= ns; j++) {
      double *pn = bufs[bi];
      bi = (bi + 1) % 3;
      if (pn == pm || pn == pc) { pn = bufs[bi]; bi = (bi + 1) % 3; }
      matvec(n, rowptr, col, val, D * h, pc, Av);
      st->nmatvec++;
      for (int64_t r = 0; r < n; r++)
        pn[r] = mu[j] * pc[r] + kap[j] * Av[r] + (pm ? nu[j] * pm[r] : 0.0);
      pm = pc;
      pc = pn;
    }
    if (pc != yP) memcpy(yP, pc, sizeof(double) * n);
    /* Horner: h3 = w3 yP + w4 zyP; h2 = w2 yP + z h3; h1 = w1 yP + z h2; y1 = yP + z h1 */
    matvec(n, rowptr, col, val, D * h, yP, Av);
    for (int64_t r = 0; r < n; r++) P1[r] = w[3] * yP[r] + w[4] * Av[r]; /* h3 */
    matvec(n, rowptr, col, val, D * h, P1, Av);
    for (int64_t r = 0; r < n; r++) h2[r] = w[2] * yP[r] + Av[r];
    matvec(n, rowptr, col, val, D * h, h2, Av);
    for (int64_t r = 0; r < n; r++) h1[r] = w[1] * yP[r] + Av[r];
    matvec(n, rowptr, col, val, D * h, h1, Av);
    for (int64_t r = 0; r < n; r++) P2[r] = yP[r] + Av[r]; /* y_{n+1} */
    st->nmatvec += 4;
    if (hfix > 0) {
      memcpy(y, P2, sizeof(double) * n);
      st->naccept++;
      t = last ? dt : t + h;
      continue;
    }
    matvec(n, rowptr, col, val, D * h, P2, Av);
    st->nmatvec++;
    double err = 0.0;
    for (int64_t r = 0; r < n; r++) {
      double e = ec[0] * yP[r] + ec[1] * h1[r] + ec[2] * h2[r] + P2[r] + ec[3] * Av[r];
      double sc = tol + tol * fmax(fabs(y[r]), fabs(P2[r]));
      err += (e / sc) * (e / sc);
    }
    err = sqrt(err / (double)n);
    double fac = err == 0.0 ? 2.0 : fmin(2.0, fmax(0.2, 0.8 * pow(err, -0.25)));
    if (err <= 1.0) {
      memcpy(y, P2, sizeof(double) * n);
      st->naccept++;
      t = last ? dt : t + h;
    } else {
      st->nreject++;
    }
    h *= fac;
  }
  free(P0); free(P1); free(P2); free(Av); free(h1); free(h2); free(yP);
  st->status = status;
  return status;
}
