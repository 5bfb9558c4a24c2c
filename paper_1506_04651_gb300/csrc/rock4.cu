// Diffusion sub-step D_dt (Sec. 2.1, Sec. 3.2.1): each species integrates the
// linear system u' = D_i L u with a ROCK4-type stabilized explicit method:
// s-4 stages of an orthogonal-polynomial three-term recurrence (count chosen
// from the Gershgorin bound of the spectral radius) followed by the 4-stage
// finishing procedure, which for a linear problem is the quartic w(dt A)
// evaluated by Horner's rule (Eq. RKscheme and the Horner remark of Sec.
// 3.2.1).  The polynomials follow Abdulle's construction (MR1923724):
// R_s(z) = w(x) P_{s-4}(x), x = 1 + 2z/l_s, P_j orthogonal on [-1, 1] for
// w^2/sqrt(1-x^2), w fixed by R_s(z) = e^z + O(z^5), l_s = 0.336 s^2 - 2.7.
// They are recomputed here on the host (orthonormal Lanczos recurrence on
// Gauss-Chebyshev nodes, fixed point in w).
//
// GPU design.  Every recurrence stage, Horner step and the embedded error
// estimate is one bandwidth-bound sweep over the leaves: a thread per leaf
// reads its 2d neighbour indices once and applies the operator to all active
// species (structure-of-arrays, coalesced).  Leaves whose faces all meet
// same-level leaves (or the boundary, stored as a self index) use the implicit
// 5/7-point weights 1/h_j^2; the few leaves at level jumps use a
// precomputed merged row of (leaf, weight) pairs.  The error norm is a
// deterministic two-pass reduction.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mr_internal.cuh"

namespace mrg {
namespace {

constexpr int kSmin = 5, kSmax = 152;

enum Mode { M_STAGE = 0, M_H3 = 1, M_H2 = 2, M_H1 = 3, M_H0 = 4, M_FSAL = 5 };

struct SpecOp {
  const double* x;  // vector the operator is applied to
  const double* a;  // first additive vector
  const double* b;  // second additive vector (may be null)
  double* out;
  double* acc;      // error accumulator
  const double* yn; // state at the step start (FSAL scaling)
  double ca, cb, cl;
  double e0, e1, e2, tol;  // error combination weights, tolerance
};

struct StageArgs {
  int nspec, mode, D;
  SpecOp op[kMaxM];
};

__constant__ double c_ih2[kMaxL + 1];

template <int D>
__device__ inline double apply_L(const double* __restrict__ x, int64_t r, const int32_t* __restrict__ nbr,
                                 int64_t capL, int32_t n0, double ih2, const int64_t* __restrict__ irr_ptr,
                                 const int32_t* __restrict__ irr_col, const double* __restrict__ irr_w) {
  if (n0 >= 0) {
    double s = x[n0];
#pragma unroll
    for (int f = 1; f < 2 * D; f++) s += x[nbr[f * capL + r]];
    return (s - 2.0 * D * x[r]) * ih2;
  }
  const int64_t row = -(int64_t)n0 - 1;
  double s = 0.0;
  for (int64_t e = irr_ptr[row]; e < irr_ptr[row + 1]; e++) s += irr_w[e] * x[irr_col[e]];
  return s;
}

template <int D>
__global__ void __launch_bounds__(kBlock) k_rock(StageArgs A, int64_t N, int64_t capL,
                                                 const int32_t* __restrict__ nbr, const uint8_t* __restrict__ lvl,
                                                 const int64_t* __restrict__ irr_ptr,
                                                 const int32_t* __restrict__ irr_col,
                                                 const double* __restrict__ irr_w, double* __restrict__ red) {
  __shared__ double sh[kBlock];
  double errs[kMaxM];
  for (int i = 0; i < A.nspec; i++) errs[i] = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t n0 = nbr[r];
    const double ih2 = c_ih2[lvl[r]];
    for (int i = 0; i < A.nspec; i++) {
      const SpecOp& o = A.op[i];
      double Lx = apply_L<D>(o.x, r, nbr, capL, n0, ih2, irr_ptr, irr_col, irr_w);
      switch (A.mode) {
        case M_STAGE:
          o.out[r] = o.ca * o.a[r] + (o.b ? o.cb * o.b[r] : 0.0) + o.cl * Lx;
          break;
        case M_H3:
        case M_H2:
          o.out[r] = o.ca * o.a[r] + o.cl * Lx;
          break;
        case M_H1: {
          double v = o.ca * o.a[r] + o.cl * Lx;  // h1 = w1 yP + z h2
          o.out[r] = v;
          o.acc[r] = o.e0 * o.a[r] + o.e1 * v + o.e2 * o.x[r];
          break;
        }
        case M_H0: {
          double v = o.a[r] + o.cl * Lx;  // y_{n+1} = yP + z h1
          o.out[r] = v;
          o.acc[r] += v;
          break;
        }
        default: {  // M_FSAL: e = acc + d z y_{n+1}
          double e = o.acc[r] + o.cl * Lx;
          double sc = o.tol + o.tol * fmax(fabs(o.yn[r]), fabs(o.x[r]));
          errs[i] += (e / sc) * (e / sc);
        }
      }
    }
  }
  if (A.mode != M_FSAL) return;
  for (int i = 0; i < A.nspec; i++) {
    sh[threadIdx.x] = errs[i];
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) red[i * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void k_reduce_rows(const double* __restrict__ red, int nb, int nspec, double* __restrict__ out) {
  __shared__ double sh[kBlock];
  for (int i = 0; i < nspec; i++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += red[i * nb + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------ host coefficients
struct Coeffs {
  int s = 0;
  double ell = 0;
  std::vector<double> mu, nu, kap;
  double w[5], errc[4];
};

int build_coeffs(int s, Coeffs& C) {
  if (s < kSmin || s > kSmax) return -1;
  const int n = s - 4;
  const double l = rock4_ell(s);
  const int M = n + 48;
  std::vector<double> x(M), om(M), q0(M), q1(M), al(n + 1), be(n + 2);
  for (int k = 0; k < M; k++) x[k] = cos(M_PI * (k + 0.5) / M);
  double q[5];
  double f = 1.0;
  for (int k = 0; k < 5; k++) {
    if (k) f *= k;
    q[k] = pow(0.5 * l, k) / f;
  }
  // orthonormal recurrence for the discrete weight om_k = w(x_k)^2:
  // be_{j+1} phi_{j+1} = (x - al_j) phi_j - be_j phi_{j-1}
  auto lanczos = [&](const double* qq) {
    double tot = 0.0;
    for (int k = 0; k < M; k++) {
      double t = x[k] - 1.0;
      double wv = (((qq[4] * t + qq[3]) * t + qq[2]) * t + qq[1]) * t + qq[0];
      om[k] = wv * wv;
      tot += om[k];
    }
    double inv = 1.0 / sqrt(tot);
    for (int k = 0; k < M; k++) {
      q0[k] = 0.0;
      q1[k] = inv;
    }
    be[0] = 0.0;
    for (int j = 0; j < n; j++) {
      double a = 0.0;
      for (int k = 0; k < M; k++) a += om[k] * x[k] * q1[k] * q1[k];
      al[j] = a;
      double nrm = 0.0;
      for (int k = 0; k < M; k++) {
        double v = (x[k] - a) * q1[k] - be[j] * q0[k];
        q0[k] = v;
        nrm += om[k] * v * v;
      }
      nrm = sqrt(nrm);
      be[j + 1] = nrm;
      for (int k = 0; k < M; k++) {
        double v = q0[k] / nrm;
        q0[k] = q1[k];
        q1[k] = v;
      }
    }
  };
  bool conv = false;
  for (int it = 0; it < 300 && !conv; it++) {
    lanczos(q);
    // monic recurrence p_{j+1} = (x - al_j) p_j - be_j^2 p_{j-1}; Taylor series
    // of P_n(1 + t) = p_n(1 + t)/p_n(1) through the ratio r_j = p_{j-1}(1)/p_j(1)
    double P[5] = {1, 0, 0, 0, 0}, Pm[5] = {0, 0, 0, 0, 0}, r = 0.0;
    for (int j = 0; j < n; j++) {
      double bj = j ? be[j] * be[j] : 0.0;
      double den = (1.0 - al[j]) - bj * r;
      double Pn[5];
      for (int k = 0; k < 5; k++) Pn[k] = ((1.0 - al[j]) * P[k] + (k ? P[k - 1] : 0.0) - bj * r * Pm[k]) / den;
      memcpy(Pm, P, sizeof P);
      memcpy(P, Pn, sizeof P);
      r = 1.0 / den;
    }
    double qn[5], E[5];
    f = 1.0;
    for (int k = 0; k < 5; k++) {
      if (k) f *= k;
      E[k] = pow(0.5 * l, k) / f;
    }
    for (int k = 0; k < 5; k++) {
      double acc = E[k];
      for (int i = 0; i < k; i++) acc -= qn[i] * P[k - i];
      qn[k] = acc / P[0];
    }
    double dm = 0.0, cm = 0.0;
    for (int k = 0; k < 5; k++) {
      dm = std::max(dm, fabs(qn[k] - q[k]));
      cm = std::max(cm, fabs(qn[k]));
    }
    memcpy(q, qn, sizeof q);
    conv = dm <= 1e-14 * cm;
  }
  if (!conv) return -2;
  lanczos(q);
  C.s = s;
  C.ell = l;
  C.mu.assign(n + 1, 0.0);
  C.nu.assign(n + 1, 0.0);
  C.kap.assign(n + 1, 0.0);
  double r = 0.0;
  for (int j = 0; j < n; j++) {
    double bj = j ? be[j] * be[j] : 0.0;
    double den = (1.0 - al[j]) - bj * r;
    C.mu[j + 1] = (1.0 - al[j]) / den;
    C.nu[j + 1] = -bj * r / den;
    C.kap[j + 1] = (2.0 / l) / den;
    r = 1.0 / den;
  }
  for (int k = 0; k < 5; k++) C.w[k] = q[k] * pow(2.0 / l, k);
  // embedded weights (a, b1, b2, d): a + b1 h1 + b2 h2 + w + d z w = O(z^4)
  const double* w = C.w;
  double Mx[4][5] = {{1.0, w[1], w[2], 0.0, -w[0]},
                     {0.0, w[2], w[3], 1.0, -w[1]},
                     {0.0, w[3], w[4], w[1], -w[2]},
                     {0.0, w[4], 0.0, w[2], -w[3]}};
  for (int k = 0; k < 4; k++) {
    int p = k;
    for (int i = k + 1; i < 4; i++)
      if (fabs(Mx[i][k]) > fabs(Mx[p][k])) p = i;
    for (int j = 0; j < 5; j++) std::swap(Mx[k][j], Mx[p][j]);
    for (int i = 0; i < 4; i++) {
      if (i == k) continue;
      double fct = Mx[i][k] / Mx[k][k];
      for (int j = k; j < 5; j++) Mx[i][j] -= fct * Mx[k][j];
    }
  }
  for (int k = 0; k < 4; k++) C.errc[k] = Mx[k][4] / Mx[k][k];
  return 0;
}

std::vector<Coeffs>& coeff_cache() {
  static std::vector<Coeffs> cache(kSmax + 1);
  return cache;
}

const Coeffs* get_coeffs(int s) {
  Coeffs& C = coeff_cache()[s];
  if (C.s != s && build_coeffs(s, C)) return nullptr;
  return &C;
}

}  // namespace

double rock4_ell(int s) { return 0.336 * (double)s * s - 2.7; }

int rock4_coeffs(int s, double* mu, double* nu, double* kap, double* w, double* errc) {
  const Coeffs* C = get_coeffs(s);
  if (!C) return -1;
  for (int j = 0; j <= s - 4; j++) {
    mu[j] = C->mu[j];
    nu[j] = C->nu[j];
    kap[j] = C->kap[j];
  }
  for (int k = 0; k < 5; k++) w[k] = C->w[k];
  for (int k = 0; k < 4; k++) errc[k] = C->errc[k];
  return 0;
}

// minimum bytes one sweep moves: per leaf the 2d neighbour indices and the
// level, per species the vectors the mode reads once and writes once, plus
// the merged rows of the leaves at level jumps
static double sweep_bytes(const mr_ctx* c, const StageArgs& A, int64_t N) {
  double per_leaf = 0.0;
  for (int i = 0; i < A.nspec; i++) {
    const SpecOp& o = A.op[i];
    switch (A.mode) {
      case M_STAGE: per_leaf += o.b ? 24 : 16; break;
      case M_H3: per_leaf += 16; break;
      case M_H2: per_leaf += 24; break;
      case M_H1: per_leaf += 32; break;
      case M_H0: per_leaf += 40; break;
      default: per_leaf += 24;
    }
  }
  return N * (per_leaf + 8.0 * c->d + 1.0) + 12.0 * c->stats.irregular_nnz + 8.0 * c->stats.irregular_rows;
}

static void launch_rock(mr_ctx* c, const StageArgs& A, int64_t N, int nb, int* nev = nullptr) {
  if (nev && *nev < 256) cudaEventRecord(c->tev[2 * *nev], c->stream);
  if (c->d == 2)
    k_rock<2><<<nb, kBlock, 0, c->stream>>>(A, N, c->cap_leaves, c->nbr, c->leaf_lvl, c->irr_ptr, c->irr_col,
                                            c->irr_w, c->red);
  else
    k_rock<3><<<nb, kBlock, 0, c->stream>>>(A, N, c->cap_leaves, c->nbr, c->leaf_lvl, c->irr_ptr, c->irr_col,
                                            c->irr_w, c->red);
  c->launches++;
  if (nev && *nev < 256) {
    cudaEventRecord(c->tev[2 * *nev + 1], c->stream);
    c->stats.rock_alg_bytes += sweep_bytes(c, A, N);
    c->stats.rock_kernel_launches++;
    (*nev)++;
  }
}

mr_status apply_operator(mr_ctx* c, const double* in, double* out) {
  mr_status st = build_tables(c);
  if (st) return st;
  double ih2[kMaxL + 1];
  for (int j = 0; j <= kMaxL; j++) ih2[j] = ldexp(1.0, 2 * j);
  MR_CUDA(c, cudaMemcpyToSymbolAsync(c_ih2, ih2, sizeof ih2, 0, cudaMemcpyHostToDevice, c->stream));
  StageArgs A;
  memset(&A, 0, sizeof A);
  A.nspec = 1;
  A.mode = M_H2;
  A.D = c->d;
  A.op[0].x = in;
  A.op[0].a = in;
  A.op[0].out = out;
  A.op[0].ca = 0.0;
  A.op[0].cl = 1.0;
  const int64_t N = c->tb[c->cur].nleaves;
  launch_rock(c, A, N, grid_for(N));
  MR_CUDA(c, cudaGetLastError());
  MR_CUDA(c, cudaStreamSynchronize(c->stream));
  return MR_OK;
}

mr_status diffuse(mr_ctx* c, double dt, double tol) {
  mr_status st = build_tables(c);
  if (st) return st;
  const int m = c->m;
  const int64_t N = c->tb[c->cur].nleaves, cap = c->cap_leaves;
  double ih2[kMaxL + 1];
  for (int j = 0; j <= kMaxL; j++) ih2[j] = ldexp(1.0, 2 * j);
  MR_CUDA(c, cudaMemcpyToSymbolAsync(c_ih2, ih2, sizeof ih2, 0, cudaMemcpyHostToDevice, c->stream));
  double* U = c->tb[c->cur].U;
  const int nb = std::max(1, std::min(grid_for(N), 152 * 8));
  struct Sp {
    double t = 0, h = 0, rho = 0;
    bool done = false, last = false;
    const Coeffs* C = nullptr;
    int n = 0, a = 0;
  } sp[kMaxM];
  for (int i = 0; i < m; i++) {
    sp[i].h = dt;
    sp[i].rho = c->prob.D[i] * c->rho;
    sp[i].done = !(dt > 0.0) || c->prob.D[i] == 0.0 || N == 0;
  }
  mr_stats& S = c->stats;
  S.rock_steps = S.rock_reject = S.rock_stages = S.rock_matvec = 0;
  S.rock_smax = 0;
  auto W = [&](int q, int i) { return c->work[q] + (int64_t)i * cap; };
  for (int round = 0;; round++) {
    int act[kMaxM], na = 0, nmax = 0, nev = 0;
    for (int i = 0; i < m; i++) {
      if (sp[i].done) continue;
      Sp& p = sp[i];
      if (p.h <= 1e-14 * dt) {
        c->last_error = "ROCK4 step size underflow";
        return MR_EROCK_STEP;
      }
      p.last = false;
      if (p.t + 1.0001 * p.h >= dt) {
        p.h = dt - p.t;
        p.last = true;
      }
      int s = kSmax;
      for (int q = kSmin; q <= kSmax; q++)
        if (rock4_ell(q) >= p.rho * p.h) {
          s = q;
          break;
        }
      if (rock4_ell(s) < p.rho * p.h) {
        p.h = rock4_ell(kSmax) / p.rho;
        p.last = false;
      }
      p.C = get_coeffs(s);
      if (!p.C) return MR_ESTATE;
      p.n = s - 4;
      p.a = (p.n - 1) % 3;
      nmax = std::max(nmax, p.n);
      S.rock_steps++;
      S.rock_stages += s;
      S.rock_smax = std::max(S.rock_smax, s);
      act[na++] = i;
    }
    if (na == 0) break;
    if (round > 100000) return MR_EROCK_STEP;
    // recurrence stages: P_j -> W[(j-1) % 3]
    for (int j = 1; j <= nmax; j++) {
      StageArgs A;
      memset(&A, 0, sizeof A);
      A.mode = M_STAGE;
      A.D = c->d;
      for (int q = 0; q < na; q++) {
        Sp& p = sp[act[q]];
        if (j > p.n) continue;
        const int i = act[q];
        SpecOp& o = A.op[A.nspec++];
        const double hd = p.h * c->prob.D[i];
        o.x = j == 1 ? U + (int64_t)i * cap : W((j - 2) % 3, i);
        o.a = o.x;
        o.b = j == 1 ? nullptr : (j == 2 ? U + (int64_t)i * cap : W((j - 3) % 3, i));
        o.out = W((j - 1) % 3, i);
        o.ca = p.C->mu[j];
        o.cb = p.C->nu[j];
        o.cl = p.C->kap[j] * hd;
        S.rock_matvec++;
      }
      launch_rock(c, A, N, nb, &nev);
    }
    // Horner steps and the error estimate
    for (int mode = M_H3; mode <= M_FSAL; mode++) {
      StageArgs A;
      memset(&A, 0, sizeof A);
      A.mode = mode;
      A.D = c->d;
      for (int q = 0; q < na; q++) {
        Sp& p = sp[act[q]];
        const int i = act[q];
        const int a = p.a, b = (p.a + 1) % 3, cc = (p.a + 2) % 3;
        const double hd = p.h * c->prob.D[i];
        const double* w = p.C->w;
        SpecOp& o = A.op[A.nspec++];
        o.tol = tol;
        switch (mode) {
          case M_H3:  // h3 = w3 yP + w4 z yP
            o.x = W(a, i); o.a = W(a, i); o.out = W(b, i); o.ca = w[3]; o.cl = w[4] * hd;
            break;
          case M_H2:  // h2 = w2 yP + z h3
            o.x = W(b, i); o.a = W(a, i); o.out = W(cc, i); o.ca = w[2]; o.cl = hd;
            break;
          case M_H1:  // h1 = w1 yP + z h2 ; acc = e0 yP + e1 h1 + e2 h2
            o.x = W(cc, i); o.a = W(a, i); o.out = W(b, i); o.acc = W(3, i); o.ca = w[1]; o.cl = hd;
            o.e0 = p.C->errc[0]; o.e1 = p.C->errc[1]; o.e2 = p.C->errc[2];
            break;
          case M_H0:  // y1 = yP + z h1 ; acc += y1
            o.x = W(b, i); o.a = W(a, i); o.out = W(cc, i); o.acc = W(3, i); o.cl = hd;
            break;
          default:  // e = acc + d z y1
            o.x = W(cc, i); o.acc = W(3, i); o.yn = U + (int64_t)i * cap; o.cl = p.C->errc[3] * hd;
        }
        S.rock_matvec++;
      }
      launch_rock(c, A, N, nb, &nev);
    }
    k_reduce_rows<<<1, kBlock, 0, c->stream>>>(c->red, nb, na, c->red_out);
    c->launches++;
    double err2[kMaxM];
    MR_CUDA(c, cudaMemcpyAsync(err2, c->red_out, sizeof(double) * na, cudaMemcpyDeviceToHost, c->stream));
    MR_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < nev; q++) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->tev[2 * q], c->tev[2 * q + 1]);
      S.rock_kernel_ms += ms;
    }
    for (int q = 0; q < na; q++) {
      const int i = act[q];
      Sp& p = sp[i];
      double err = sqrt(err2[q] / (double)N);
      if (!isfinite(err)) {
        c->last_error = "non-finite ROCK4 error estimate";
        return MR_ENONFINITE;
      }
      double fac = err == 0.0 ? 2.0 : std::min(2.0, std::max(0.2, 0.8 * pow(err, -0.25)));
      if (err <= 1.0) {
        MR_CUDA(c, cudaMemcpyAsync(U + (int64_t)i * cap, W((p.a + 2) % 3, i), sizeof(double) * N,
                                   cudaMemcpyDeviceToDevice, c->stream));
        p.t = p.last ? dt : p.t + p.h;
        if (p.last) p.done = true;
      } else {
        S.rock_reject++;
      }
      p.h *= fac;
    }
  }
  MR_CUDA(c, cudaGetLastError());
  MR_CUDA(c, cudaStreamSynchronize(c->stream));
  return MR_OK;
}

}  // namespace mrg
