// Pieces shared by the Radau5 kernels (one thread per cell, csrc/radau5.cu;
// one team of 16 or 32 lanes per cell for larger systems, csrc/radau5_net.cu):
// the method's constants as the kernels take them, per-cell counters, and
// two small helpers.
#pragma once
#include "mr_internal.cuh"

namespace mrg {

struct RadauC {
  double c1, c2;
  double T[9], Ti[9];
  double gam, alp, bet;
  double ge[3];        // gam * e_j (embedded estimate weights times gam)
  double idn[4][4];    // 1 / (nd[a] - nd[b]) for the nodes (0, c1, c2, 1)
  double rt, at, fnewt;  // transformed tolerances and Newton tolerance (per call)
  double ifnewt;         // 1 / fnewt
  double fac[8];       // min(0.9, 0.9 (1 + 2 kmax)/(k + 2 kmax)), k Newton iterations
  // starting values: the Lagrange weight of node a (1..3) at stage time
  // 1 + c_s r as a cubic in the step ratio r, Lc[s][a-1][0..3] (ascending)
  double Lc[3][3][4];
  // FP32 copies for the mixed form's starting values and tolerance scales
  float c1f, c2f, Tif[9], idnf[4][4], Lcf[3][3][4];
  float rtf, atf;  // set with rt, at
};

struct CellCount {
  int nfev, njac, nstep, naccept, nreject, nnewton, ndec;
};

__device__ inline double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// x^(1/4) through two square roots (hardware-assisted) instead of pow
__device__ inline double root4(double x) { return sqrt(sqrt(x)); }

// x^0.8 (x in [1e-16, 100]) for the Newton-stopping factor of each step
// attempt, without FP64 division: x^0.8 = x z with z = x^(-1/5), from an FP32
// estimate refined by two Newton steps on z^-5 = x written as
// z <- z (1 + (1 - x z^5) / 5) (quadratic convergence); within a few ulps of
// pow (the factor only enters the comparison with the Newton tolerance)
__device__ inline double pow08(double x) {
  double z = (double)exp2f(__fmul_rn(-0.2f, log2f((float)x)));
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const double z2 = z * z, z5 = z2 * z2 * z;
    const double e = fma(-x, z5, 1.0);
    z = fma(z * e, 0.2, z);
  }
  return x * z;
}

// the mixed form's x^0.8: the FP32 estimate alone (the factor only enters
// the comparison with the Newton tolerance)
__device__ inline double pow08_f32(double x) { return (double)exp2f(__fmul_rn(0.8f, log2f((float)x))); }

// kernel-side constants from radau_constants' array (tolerances unset)
RadauC constants_from(const double* rc);

// Algorithmic FP64 work of k_radau (one thread per cell, m = M species),
// counted operation by operation from its source: every addition,
// subtraction, multiplication, division and square root is one operation,
// a*b + c is two whether or not it is fused, and fabs, fmin, fmax,
// comparisons and negations are none.  Per event:
//   rhs, jac   one right-hand side, one Jacobian (model-specific)
//   dec        forming gam/h I - J and (alp + i bet)/h I - J and factorising
//              them: 6 + 2M + LU_real(M) + LU_cplx(M), where
//              LU_real = M + M(M-1)/2 + M(M-1)(2M-1)/3 and
//              LU_cplx = M(M+1)/2 + 6M + 3M(M-1) + 4M(M-1)(2M-1)/3
//   newton     one simplified Newton iteration without its three right-hand
//              sides: stage arguments 3M, T^-1 F 15M, residuals 10M, real
//              solve M + 2M(M-1), complex solve 6M + 8M(M-1), increment norm
//              9M + 2, W update 3M, Z = T W 15M, stopping test 1
//              = 62M + 10M(M-1) + 3
//   monitor    contraction rate and its test (iterations k >= 2): 6
//   attempt    every step attempt: step-size floor 2, W = T^-1 Z 15M, scales
//              3M, faccon^0.8 14, shifted eigenvalues 3 = 19 + 18M
//   extrap     starting values extrapolated from the last accepted step:
//              the step ratio 1, nine Lagrange weights as cubics in it
//              (Horner, 3 fused multiply-adds = 6 each) and the stage values
//              6M per stage: 1 + 3 (18 + 6M) = 55 + 18M
//   accept     error estimate 5 + 13M + solve_real(M), step-size factor 4,
//              accepted-step control, update and time 11 + M
// Where the source trades divisions for multiplications (the tolerance
// scales as one reciprocal of their product, the contraction monitor with
// one division, faccon^0.8 without division) the table keeps the smaller
// division forms' counts.  A launch's work is taken as the lower bound
//   rhs nfev + jac njac + dec ndec + newton nnewton + monitor (nnewton - nstep)
//   + attempt nstep + extrap max(0, nstep - ncells - nreject) + accept naccept
// (an attempt extrapolates unless it precedes its cell's first accepted
// step, so at least nstep - ncells - nreject attempts do; error estimates of
// rejected steps and the refiltered estimate are left out).
struct RadauWork {
  double rhs, jac, dec, newton, monitor, attempt, extrap, accept;
};
RadauWork radau_work(int model, int M);
// counters in the order of DevCounters::radau (fev, jac, steps, accept,
// reject, newton, dec)
double radau_alg_flops(const RadauWork& w, const unsigned long long* cnt, int64_t ncells);

// Reaction sub-steps of the network and membrane models (team kernels); C
// carries the transformed tolerances of the call.
mr_status react_network(mr_ctx* c, const RadauC& C, double dt);
mr_status react_ionic(mr_ctx* c, const RadauC& C, double dt);

}  // namespace mrg
