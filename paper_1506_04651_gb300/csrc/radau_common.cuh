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
};

struct CellCount {
  int nfev, njac, nstep, naccept, nreject, nnewton, ndec;
};

__device__ inline double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// x^(1/4) through two square roots (hardware-assisted) instead of pow
__device__ inline double root4(double x) { return sqrt(sqrt(x)); }

// x^0.8 (x in [1e-16, 100]) for the Newton-stopping factor of each step
// attempt: an FP32 estimate refined by two FP64 Newton steps on y^5 = x^4,
// within a few ulps of pow at a fraction of its FP64 instructions (the factor
// only enters the comparison with the Newton tolerance)
__device__ inline double pow08(double x) {
  double y = (double)exp2f(0.8f * log2f((float)x));
  const double x2 = x * x, x4 = x2 * x2;
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const double y2 = y * y;
    y = y + (x4 / (y2 * y2) - y) * 0.2;
  }
  return y;
}

// kernel-side constants from radau_constants' array (tolerances unset)
RadauC constants_from(const double* rc);

// Reaction sub-steps of the network and membrane models (team kernels); C
// carries the transformed tolerances of the call.
mr_status react_network(mr_ctx* c, const RadauC& C, double dt);
mr_status react_ionic(mr_ctx* c, const RadauC& C, double dt);

}  // namespace mrg
