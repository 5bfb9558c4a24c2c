// Pieces shared by the Radau5 kernels (one thread per cell, csrc/radau5.cu;
// one team of 16 lanes per cell for larger systems, csrc/radau5_net.cu):
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
  double fac[8];       // min(0.9, 0.9 (1 + 2 kmax)/(k + 2 kmax)), k Newton iterations
};

struct CellCount {
  int nfev, njac, nstep, naccept, nreject, nnewton, ndec;
};

__device__ inline double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// x^(1/4) through two square roots (hardware-assisted) instead of pow
__device__ inline double root4(double x) { return sqrt(sqrt(x)); }

// kernel-side constants from radau_constants' array (tolerances unset)
RadauC constants_from(const double* rc);

// Reaction sub-step of the network model (team kernel); C carries the
// transformed tolerances of the call.
mr_status react_network(mr_ctx* c, const RadauC& C, double dt);

}  // namespace mrg
