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
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
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
__constant__ float c_ih2f[kMaxL + 1];

struct IrrRows {
  const int32_t* cnt;
  const int32_t* col;
  const double* w;
  const float* wf;  // the same weights in FP32 (exact: dyadic), for the mixed form
  int slot;
};

template <int D>
__device__ inline double apply_L(const double* __restrict__ x, int64_t r, const int32_t* __restrict__ nbr,
                                 int64_t capL, int32_t n0, double ih2, const IrrRows& R) {
  if (n0 >= 0) {
    double s = x[n0];
#pragma unroll
    for (int f = 1; f < 2 * D; f++) s += x[nbr[f * capL + r]];
    return (s - 2.0 * D * x[r]) * ih2;
  }
  const int64_t row = -(int64_t)n0 - 1;
  const int32_t* col = R.col + row * R.slot;
  const double* w = R.w + row * R.slot;
  const int n = R.cnt[row];
  double s = 0.0;
  for (int e = 0; e < n; e++) s += w[e] * x[col[e]];
  return s;
}

template <int D>
__global__ void __launch_bounds__(kBlock) k_rock(StageArgs A, int64_t N, int64_t capL,
                                                 const int32_t* __restrict__ nbr, const uint8_t* __restrict__ lvl,
                                                 IrrRows R, double* __restrict__ red) {
  __shared__ double sh[kBlock];
  double errs[kMaxM];
  for (int i = 0; i < A.nspec; i++) errs[i] = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t n0 = nbr[r];
    const double ih2 = c_ih2[lvl[r]];
    for (int i = 0; i < A.nspec; i++) {
      const SpecOp& o = A.op[i];
      double Lx = apply_L<D>(o.x, r, nbr, capL, n0, ih2, R);
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

// ------------------------------------------------------------ persistent driver
// One cooperative launch integrates a whole diffusion sub-step D_dt for every
// species: ROCK4 steps are taken, accepted or rejected and resized on the
// device, with grid-wide barriers between sweeps (the vectors of the
// benchmark's grids are L2-resident, so a barrier is far cheaper than a kernel
// launch and a host round trip per step).
//
// Every block keeps its own copy of the step control in shared memory and
// runs the same control arithmetic on the same per-block error partials in
// the same order, so all copies agree and no barrier is spent on a control
// section.  An accepted step swaps the state with the buffer holding the
// candidate (no copy sweep), and the operator applied to the candidate by the
// embedded-estimate sweep is kept: it is L y_n of the next step, so the first
// recurrence stage of every step but the first is a plain axpy.

// coefficient table for s = 5..152: [l_s, w0..w4, e0..e3, mu_1..n, nu_1..n, kap_1..n]
struct RockTab {
  const double* data;
  int off[kSmax + 1];
};

struct RockCtl {
  double t[kMaxM], h[kMaxM], err[kMaxM];
  int done[kMaxM], last[kMaxM], s[kMaxM], n[kMaxM], a[kMaxM], acc_prev[kMaxM], c_prev[kMaxM];
  int nmax, finished, status, rounds;
  long long steps, rejects, stages, matvecs;
  int smax;
  double bytes, flops;
};

// Work of one sweep shared by the species (the regular-leaf table, none on the
// uniform grid, and the merged rows) and the arithmetic of one operator
// application of one species: (2d + 1) per regular leaf (the neighbour sum
// and the centre term) and 2 per merged-row entry
struct SweepWork {
  double tab_bytes, op_flops;
  int inc;  // the mixed form (FP32 increments)
};

struct PersArgs {
  int m, D, nb;
  int J;         // finest level (the uniform-grid form's leaves are all at J)
  SweepWork work;
  int64_t N, capL;
  double dt, tol, rho;
  double Dc[kMaxM];
  double* U;     // the state; buffer 0 of each species' pool of four
  double* W[6];  // W0..W2: pool buffers 1..3; W3: error accumulator; W4, W5: L y
  double* part;  // [kMaxM][nb] per-block partial sums of the error norm
  RockCtl* ctl;  // initial control in, final control out
  RockTab tab;
};

__device__ inline double ell_dev(int s) { return 0.336 * (double)s * s - 2.7; }

// choose the next step of every species (one thread per block, on the
// block's copy of the control)
__device__ void rock_prepare(int m, double dt, const double* Dc, double rho_L, RockCtl& C, int64_t N,
                             const SweepWork& W) {
  const bool inc = W.inc;
  int nmax = 0, any = 0;
  double bytes = 0.0, flops = 0.0;
  for (int i = 0; i < m; i++) {
    if (C.done[i]) continue;
    if (C.h[i] <= 1e-14 * dt) {
      C.status = MR_EROCK_STEP;
      C.finished = 1;
      return;
    }
    const double rho = Dc[i] * rho_L;
    C.last[i] = 0;
    if (C.t[i] + 1.0001 * C.h[i] >= dt) {
      C.h[i] = dt - C.t[i];
      C.last[i] = 1;
    }
    int s = kSmax;
    for (int q = kSmin; q <= kSmax; q++)
      if (ell_dev(q) >= rho * C.h[i]) {
        s = q;
        break;
      }
    if (ell_dev(s) < rho * C.h[i]) {
      C.h[i] = ell_dev(kSmax) / rho;
      C.last[i] = 0;
    }
    C.s[i] = s;
    C.n[i] = s - 4;
    C.a[i] = (s - 5) % 3;
    nmax = max(nmax, s - 4);
    C.steps++;
    C.stages += s;
    C.smax = max(C.smax, s);
    C.matvecs += s + 1;
    // vector bytes per leaf, each vector read or written once.  FP64: stage
    // 1 24, stages 2..n 24, Horner 16+24+32+40, embedded estimate 24 + 8
    // (keeps L y_{n+1}).  Mixed form (FP32 increments, FP64 state): stage 1
    // 8 plus the FP64 state update 20, stage 2 12, stages 3..n 16, Horner
    // 12+16+20+24, embedded estimate 24 (with the FP64 state for its scale)
    if (inc)
      bytes += N * (28.0 + (s >= 6 ? 12.0 + 16.0 * (s - 6) : 0.0) + 72.0 + 24.0);
    else
      bytes += N * (24.0 * (s - 4) + 112.0 + 32.0);
    // n + 4 operator applications (stages 2..n, Horner, estimate) and the
    // combinations per leaf: stages 5 each, Horner 3 + 3 + 8 + 4, estimate 8,
    // first stage 3
    flops += (s - 4 + 4) * W.op_flops + N * (5.0 * (s - 5) + 29.0);
    any = 1;
  }
  C.nmax = nmax;
  // tables and merged rows: one gather sweep per stage 2..n and per finishing sweep
  C.bytes += bytes + (double)(nmax - 1 + 5) * W.tab_bytes;
  C.flops += flops;
  if (!any) C.finished = 1;
}

// operands of one species in one sweep
enum { K_STAGE = 0, K_H3, K_H2, K_H1, K_H0, K_FSAL, K_STAGE1 };
constexpr int kPhaseFinish = 1000;  // phases 2..n: stages; kPhaseFinish + K_*: the other sweeps

// VT: arithmetic of the stage vectors (double, or float in the mixed form);
// the error norm is accumulated in double either way.
//
// The mixed form integrates increments: with y_n the FP64 state at the start
// of a ROCK4 step and g = L y_n, every FP32 vector holds a difference from
// y_n (or from its image under the Horner partial sums), so rounding is
// relative to the change a step makes, not to the state.  Since every
// stability polynomial is 1 at z = 0 (mu_j + nu_j = 1, w(0) = 1, and the
// embedded estimate vanishes at z = 0), the recurrence and the finishing
// procedure keep their form, with the term z y_n = h D g added:
//   delta_1 = kap_1 h D g,
//   delta_j = mu_j delta_{j-1} + nu_j delta_{j-2} + kap_j h D (g + L delta_{j-1}),
//   eta_3 = w_3 delta + w_4 h D (g + L delta),
//   eta_k = w_k delta + w_{k+1} h D g + h D L eta_{k+1}   (k = 2, 1),
//   Delta = delta + w_1 h D g + h D L eta_1,   y_{n+1} = y_n + Delta (in FP64),
//   E = e_0 delta + e_1 eta_1 + e_2 eta_2 + Delta + e_3 h D (g + L Delta),
// and L y_{n+1} = g + L Delta is kept for the next step.  g itself is L y_n
// applied in FP64 once per sub-step.
template <typename VT>
struct Ops {
  const VT *x, *a, *b, *yn;
  VT *out, *acc, *lx;
  VT ca, cb, cl, e0, e1, e2;
  int kind;
  const VT* g;      // mixed form: L y_n (null in FP64)
  VT cg;            // mixed form: weight of g
  const double* u;  // mixed form: the FP64 state y_n (the error scale)
};

// d: the unscaled stencil sum (sum of the neighbours minus 2D times the
// leaf) at a regular leaf, with ih2 = 1 / h^2 of its level and beta = cl ih2;
// L y itself at a merged row (ih2 = 1, beta = cl).  ih2 is a power of two, so
// beta d equals cl (d ih2) exactly and the sweeps that do not keep L y save
// the scaling multiply.
template <typename VT>
__device__ inline void combine(const Ops<VT>& o, int64_t r, VT d, VT ih2, VT beta, double tol, double& err) {
  if constexpr (!std::is_same<VT, double>::value) {  // the mixed form's increments
    switch (o.kind) {
      case K_STAGE:
        o.out[r] = o.ca * o.a[r] + (o.b ? o.cb * o.b[r] : (VT)0) + o.cl * o.g[r] + beta * d;
        break;
      case K_H3:
      case K_H2:
        o.out[r] = o.ca * o.a[r] + o.cg * o.g[r] + beta * d;
        break;
      case K_H1: {
        const VT v = o.ca * o.a[r] + o.cg * o.g[r] + beta * d;
        o.out[r] = v;
        o.acc[r] = o.e0 * o.a[r] + o.e1 * v + o.e2 * o.x[r];
        break;
      }
      case K_H0: {
        const VT v = o.a[r] + o.cg * o.g[r] + beta * d;  // Delta
        o.out[r] = v;
        o.acc[r] += v;
        break;
      }
      case K_FSAL: {  // L y_{n+1} = g + L Delta is kept; scale from y_n and y_n + Delta
        const VT ly1 = o.g[r] + d * ih2;
        o.lx[r] = ly1;
        const double ee = (double)(o.acc[r] + o.cl * ly1);
        const double yv = o.u[r];
        const double sc = tol + tol * fmax(fabs(yv), fabs(yv + (double)o.x[r]));
        err += (ee / sc) * (ee / sc);
        break;
      }
      default:
        break;  // K_STAGE1: the first stage reads the FP64 state (the g sweep)
    }
    return;
  }
  switch (o.kind) {
    case K_STAGE:
      o.out[r] = o.ca * o.a[r] + o.cb * o.b[r] + beta * d;
      break;
    case K_STAGE1: {  // first step only: P_1 = y + kap_1 h L y, keeping L y
      const VT Lx = d * ih2;
      o.lx[r] = Lx;
      o.out[r] = o.ca * o.a[r] + o.cl * Lx;
      break;
    }
    case K_H3:
    case K_H2:
      o.out[r] = o.ca * o.a[r] + beta * d;
      break;
    case K_H1: {
      const VT v = o.ca * o.a[r] + beta * d;  // h1 = w1 yP + z h2
      o.out[r] = v;
      o.acc[r] = o.e0 * o.a[r] + o.e1 * v + o.e2 * o.x[r];
      break;
    }
    case K_H0: {
      const VT v = o.a[r] + beta * d;  // y_{n+1} = yP + z h1
      o.out[r] = v;
      o.acc[r] += v;
      break;
    }
    default: {  // embedded estimate e = acc + d z y_{n+1}; L y_{n+1} is kept
      const VT Lx = d * ih2;
      o.lx[r] = Lx;
      const double ee = (double)(o.acc[r] + o.cl * Lx);
      const double sc = tol + tol * fmax(fabs((double)o.yn[r]), fabs((double)o.x[r]));
      err += (ee / sc) * (ee / sc);
    }
  }
}

// The faces of the level-J cell with Morton code c on the uniform grid, in
// the regular-leaf table's order (x-, x+, y-, y+, z-, z+): the neighbour's
// code, or c itself at the domain boundary (no flux, as in the table).
template <int D>
__device__ inline void uniform_faces(uint32_t c, int J, int* v) {
  int k[3];
  unmorton<D>(c, k);
  const int lim = 1 << J;
#pragma unroll
  for (int f = 0; f < 2 * D; f++) {
    const int a = f >> 1, sg = (f & 1) ? 1 : -1;
    int q[3] = {k[0], k[1], k[2]};
    q[a] += sg;
    v[f] = (q[a] >= 0 && q[a] < lim) ? (int)morton<D>(q) : (int)c;
  }
}

// CM: the uniform level-J grid (a Cartesian mesh: every leaf at level J, no
// merged rows).  The leaf index is then the Morton code, and the sweeps take
// the 2d neighbours from the code instead of the regular-leaf table, saving
// its 32 bytes per leaf and sweep.
template <int D, int M, typename VT, bool CM = false>
__global__ void __launch_bounds__(kBlock, M > 4 ? 1 : 2)
    k_rock_persistent(PersArgs P, const int4* __restrict__ reg, int64_t nreg, IrrRows R,
                      const int32_t* __restrict__ irr_leaf, int64_t nirr) {
  constexpr bool kF64 = std::is_same<VT, double>::value;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[kBlock];
  __shared__ RockCtl C;         // this block's copy of the step control
  __shared__ int s_py[kMaxM];   // pool index of the state
  __shared__ int s_pr[kMaxM][3];  // pool indices of the three recurrence buffers
  __shared__ int s_ly[kMaxM];   // which of W4 / W5 holds L y of the state
  __shared__ int s_pend[kMaxM];  // mixed form: an accepted increment not yet added to the state
  __shared__ double s_err2[kMaxM];
  __shared__ Ops<VT> s_ops[M];
  __shared__ int s_act[M];
  __shared__ VT s_beta[M][kMaxL + 1];  // cl / h^2 of every level
  const int64_t N = P.N, capL = P.capL;
  if (threadIdx.x == 0) {
    C = *P.ctl;
    for (int i = 0; i < M; i++) {
      s_pend[i] = 0;
      s_py[i] = 0;
      s_pr[i][0] = 1;
      s_pr[i][1] = 2;
      s_pr[i][2] = 3;
      s_ly[i] = 0;
    }
  }
  // thread index dealt warp by warp round the blocks (warp w of block b is
  // warp b + nb w of the grid), so that when the leaves fill the grid only
  // partly, or a little more than once, every SM gets the same share of them
  // (the sweeps are bound by the narrow FP64 pipe of each SM)
  const int64_t tid = (threadIdx.x & 31) + 32 * (blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5)),
                nth = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  // vector q of species i: FP64: the state U (pool 0), W0..W2 (pool 1..3),
  // W3 (error accumulator), W4, W5 (L y); FP32: twelve float vectors carved
  // from the six work buffers, pool 0..3 = vectors 0..3 (vector 0 holds a
  // float copy of the state), accumulator 4, L y 5 and 6
  auto fvec = [&](int q, int i) -> VT* {
    return reinterpret_cast<VT*>(reinterpret_cast<float*>(P.W[q >> 1]) + (q & 1) * (int64_t)P.m * capL) +
           (int64_t)i * capL;
  };
  auto pool = [&](int i, int k) -> VT* {
    if constexpr (kF64)
      return reinterpret_cast<VT*>(k == 0 ? P.U : P.W[k - 1]) + (int64_t)i * capL;
    else
      return fvec(k, i);
  };
  auto Wp = [&](int q, int i) -> VT* {  // q = 3 accumulator, 4 / 5 L y
    if constexpr (kF64)
      return reinterpret_cast<VT*>(P.W[q]) + (int64_t)i * capL;
    else
      return fvec(q + 1, i);
  };
  auto Y = [&](int i) { return pool(i, s_py[i]); };
  auto Rb = [&](int i, int q) { return pool(i, s_pr[i][q]); };
  auto LY = [&](int i) { return Wp(4 + s_ly[i], i); };
  auto LC = [&](int i) { return Wp(5 - s_ly[i], i); };
  // operands of species i in `phase`; false if the species sits it out
  auto ops_for = [&](int phase, int i, Ops<VT>& o) -> bool {
    if (C.done[i]) return false;
    const double* tb = P.tab.data + P.tab.off[C.s[i]];
    const double hd = C.h[i] * P.Dc[i];
    const int n = C.n[i];
    o.b = nullptr;
    o.acc = nullptr;
    o.lx = nullptr;
    o.yn = Y(i);
    o.g = nullptr;
    o.cg = (VT)0;
    o.u = nullptr;
    if constexpr (!kF64) {  // increments: g = L y_n, the FP64 state for the error scale
      o.g = LY(i);
      o.u = P.U + (int64_t)i * capL;
    }
    if (phase < kPhaseFinish) {  // stage j >= 2
      const int j = phase;
      if (j > n) return false;
      o.kind = K_STAGE;
      o.x = Rb(i, (j - 2) % 3);
      o.a = o.x;
      // P_0 = y_n: its increment delta_0 is zero
      o.b = j == 2 ? (kF64 ? Y(i) : nullptr) : Rb(i, (j - 3) % 3);
      o.out = Rb(i, (j - 1) % 3);
      o.ca = (VT)tb[10 + (j - 1)];
      o.cb = (VT)tb[10 + n + (j - 1)];
      o.cl = (VT)(tb[10 + 2 * n + (j - 1)] * hd);
      return true;
    }
    const double* w = tb + 1;
    const double* e = tb + 6;
    const int a = C.a[i], b = (a + 1) % 3, cc = (a + 2) % 3;
    o.kind = phase - kPhaseFinish;
    switch (o.kind) {
      case K_STAGE1:
        o.x = Y(i); o.a = Y(i); o.out = Rb(i, 0); o.lx = LY(i);
        o.ca = (VT)tb[10]; o.cl = (VT)(tb[10 + 2 * n] * hd);
        break;
      case K_H3:
        o.x = Rb(i, a); o.a = Rb(i, a); o.out = Rb(i, b); o.ca = (VT)w[3]; o.cl = (VT)(w[4] * hd);
        o.cg = (VT)(w[4] * hd);
        break;
      case K_H2:
        o.x = Rb(i, b); o.a = Rb(i, a); o.out = Rb(i, cc); o.ca = (VT)w[2]; o.cl = (VT)hd; o.cg = (VT)(w[3] * hd);
        break;
      case K_H1:
        o.x = Rb(i, cc); o.a = Rb(i, a); o.out = Rb(i, b); o.acc = Wp(3, i); o.ca = (VT)w[1]; o.cl = (VT)hd;
        o.e0 = (VT)e[0]; o.e1 = (VT)e[1]; o.e2 = (VT)e[2]; o.cg = (VT)(w[2] * hd);
        break;
      case K_H0:
        o.x = Rb(i, b); o.a = Rb(i, a); o.out = Rb(i, cc); o.acc = Wp(3, i); o.ca = (VT)1; o.cl = (VT)hd;
        o.cg = (VT)(w[1] * hd);
        break;
      default:
        o.x = Rb(i, cc); o.a = nullptr; o.out = nullptr; o.acc = Wp(3, i); o.lx = LC(i); o.cl = (VT)(e[3] * hd);
    }
    return true;
  };
  auto build_ops = [&](int phase) {
    __syncthreads();
    if (threadIdx.x < M) s_act[threadIdx.x] = ops_for(phase, threadIdx.x, s_ops[threadIdx.x]);
    __syncthreads();
    for (int q = threadIdx.x; q < M * (kMaxL + 1); q += blockDim.x) {
      const int i = q / (kMaxL + 1), j = q % (kMaxL + 1);
      if (s_act[i]) {
        if constexpr (kF64)
          s_beta[i][j] = s_ops[i].cl * c_ih2[j];
        else
          s_beta[i][j] = s_ops[i].cl * c_ih2f[j];
      }
    }
    __syncthreads();
  };
  // one operator sweep: regular leaves one thread each from the compact
  // table (neighbour indices loaded once for all species), merged rows G
  // lanes each
  // lanes per merged row: 2D rows are short (~30 entries), 3D rows long
  // (~100); measured best 2 and 4
  constexpr int G = D == 2 ? 2 : 4;
  constexpr int MG = (M + G - 1) / G;  // species a merged-row lane finishes
  const int sub = lane & (G - 1);
  auto sweep = [&](double* err, double* err_row) {
    const Ops<VT>* o = s_ops;
    const int* act = s_act;
    for (int64_t q = tid; q < nreg; q += nth) {
      int v[8];
      if constexpr (CM) {
        v[0] = (int)q;
        uniform_faces<D>((uint32_t)q, P.J, v + 1);
        v[1 + 2 * D] = P.J;
      } else {
        const int4 e0 = reg[2 * q], e1 = reg[2 * q + 1];
        v[0] = e0.x; v[1] = e0.y; v[2] = e0.z; v[3] = e0.w;
        v[4] = e1.x; v[5] = e1.y; v[6] = e1.z; v[7] = e1.w;
      }
      const int64_t r = v[0];
      const int lev = v[1 + 2 * D];
      VT ih2;
      if constexpr (kF64)
        ih2 = c_ih2[lev];
      else
        ih2 = c_ih2f[lev];
#pragma unroll
      for (int i = 0; i < M; i++) {
        if (!act[i]) continue;
        const VT* x = o[i].x;
        VT sx = x[v[1]];
#pragma unroll
        for (int f = 1; f < 2 * D; f++) sx += x[v[1 + f]];
        combine<VT>(o[i], r, sx - (VT)(2 * D) * x[r], ih2, s_beta[i][lev], P.tol, err[i]);
      }
    }
    // 2D: merged rows are taken from the last threads, which have no regular
    // leaf when the leaves number fewer than the threads (fewer threads do
    // both kinds of work)
    const int64_t grp = (D == 2 ? nth - 1 - tid : tid) / G, ngrp = nth / G;
    const int64_t rounds = (nirr + ngrp - 1) / ngrp;
    for (int64_t k = 0; k < rounds; k++) {
      const int64_t row = grp + k * ngrp;
      const bool have = row < nirr;
      VT v[M];
#pragma unroll
      for (int i = 0; i < M; i++) v[i] = (VT)0;
      int32_t r = 0;
      if (have) {
        r = irr_leaf[row];
        const int cnt = R.cnt[row];
        const int32_t* col = R.col + row * (int64_t)R.slot;
        const VT* wr;
        if constexpr (kF64)
          wr = R.w + row * (int64_t)R.slot;
        else
          wr = R.wf + row * (int64_t)R.slot;
#pragma unroll 4
        for (int e = sub; e < cnt; e += G) {
          const int32_t cidx = col[e];
          const VT we = wr[e];
#pragma unroll
          for (int i = 0; i < M; i++)
            if (act[i]) v[i] += we * o[i].x[cidx];
        }
      }
#pragma unroll
      for (int i = 0; i < M; i++)
        for (int sft = G / 2; sft > 0; sft >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], sft);
      // every lane of the group holds the row's sums; lane `sub` finishes
      // species sub, sub + G, ... (one instruction stream for the species)
      if (have) {
#pragma unroll
        for (int i0 = 0; i0 < M; i0 += G) {
          const int i = i0 + sub;
          VT vi = v[i0];
#pragma unroll
          for (int u = 1; u < G; u++)
            if (i0 + u < M && sub == u) vi = v[i0 + u];
          if (i < M && act[i]) combine<VT>(o[i], r, vi, (VT)1, o[i].cl, P.tol, err_row[i0 / G]);
        }
      }
    }
  };
  // mixed form, first stage of a sub-step: g = L y_n applied to the FP64
  // state in FP64 (kept as the float L y) and delta_1 = kap_1 h D g
  auto gsweep = [&]() {
    const Ops<VT>* o = s_ops;
    const int* act = s_act;
    for (int64_t q = tid; q < nreg; q += nth) {
      int v[8];
      if constexpr (CM) {
        v[0] = (int)q;
        uniform_faces<D>((uint32_t)q, P.J, v + 1);
        v[1 + 2 * D] = P.J;
      } else {
        const int4 e0 = reg[2 * q], e1 = reg[2 * q + 1];
        v[0] = e0.x; v[1] = e0.y; v[2] = e0.z; v[3] = e0.w;
        v[4] = e1.x; v[5] = e1.y; v[6] = e1.z; v[7] = e1.w;
      }
      const int64_t r = v[0];
      const double ih2 = c_ih2[v[1 + 2 * D]];
#pragma unroll
      for (int i = 0; i < M; i++) {
        if (!act[i]) continue;
        const double* u = P.U + (int64_t)i * capL;
        double sx = u[v[1]];
#pragma unroll
        for (int f = 1; f < 2 * D; f++) sx += u[v[1 + f]];
        const double gv = (sx - 2.0 * D * u[r]) * ih2;
        o[i].lx[r] = (VT)gv;
        o[i].out[r] = (VT)((double)o[i].cl * gv);
      }
    }
    const int64_t grp = (D == 2 ? nth - 1 - tid : tid) / G, ngrp = nth / G;
    const int64_t rounds = (nirr + ngrp - 1) / ngrp;
    for (int64_t k = 0; k < rounds; k++) {
      const int64_t row = grp + k * ngrp;
      const bool have = row < nirr;
      double v[M];
#pragma unroll
      for (int i = 0; i < M; i++) v[i] = 0.0;
      int32_t r = 0;
      if (have) {
        r = irr_leaf[row];
        const int cnt = R.cnt[row];
        const int32_t* col = R.col + row * (int64_t)R.slot;
        const double* wr = R.w + row * (int64_t)R.slot;
        for (int e = sub; e < cnt; e += G) {
          const int32_t cidx = col[e];
          const double we = wr[e];
#pragma unroll
          for (int i = 0; i < M; i++)
            if (act[i]) v[i] += we * P.U[(int64_t)i * capL + cidx];
        }
      }
#pragma unroll
      for (int i = 0; i < M; i++)
        for (int sft = G / 2; sft > 0; sft >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], sft);
      if (have && sub == 0) {
#pragma unroll
        for (int i = 0; i < M; i++)
          if (act[i]) {
            o[i].lx[r] = (VT)v[i];
            o[i].out[r] = (VT)((double)o[i].cl * v[i]);
          }
      }
    }
  };
  __syncthreads();
  if (threadIdx.x == 0) rock_prepare(P.m, P.dt, P.Dc, P.rho, C, N, P.work);
  __syncthreads();
  bool first = true;
  for (int round = 0; round < 20000; round++) {
    if (C.finished) break;
    double err[M], err_row[MG];  // err_row[q]: the merged rows' share of species q G + sub
#pragma unroll
    for (int i = 0; i < M; i++) err[i] = 0.0;
#pragma unroll
    for (int q = 0; q < MG; q++) err_row[q] = 0.0;
    // stage 1: P_1 = y + kap_1 h L y (an operator sweep in the first step,
    // then an axpy on the kept L y)
    if (first) {
      build_ops(kPhaseFinish + K_STAGE1);
      if constexpr (kF64)
        sweep(err, err_row);
      else
        gsweep();
    } else {
      for (int i = 0; i < M; i++) {
        if (C.done[i]) continue;
        const double* tb = P.tab.data + P.tab.off[C.s[i]];
        const VT ca = (VT)tb[10], cl = (VT)(tb[10 + 2 * C.n[i]] * C.h[i] * P.Dc[i]);
        const VT *y = Y(i), *ly = LY(i);
        VT* out = Rb(i, 0);
        if constexpr (kF64) {
          for (int64_t r = tid; r < N; r += nth) out[r] = ca * y[r] + cl * ly[r];
        } else if (s_pend[i]) {
          // the last accepted increment joins the FP64 state (it may share
          // the buffer delta_1 goes to: read before the write)
          double* u = P.U + (int64_t)i * capL;
          const VT* dl = Rb(i, C.c_prev[i]);
          for (int64_t r = tid; r < N; r += nth) {
            const VT dv = dl[r];
            u[r] += (double)dv;
            out[r] = cl * ly[r];
          }
        } else {
          for (int64_t r = tid; r < N; r += nth) out[r] = cl * ly[r];
        }
      }
    }
    first = false;
    grid.sync();
    // recurrence stages P_j -> R[(j-1) % 3]
    for (int j = 2; j <= C.nmax; j++) {
      build_ops(j);
      sweep(err, err_row);
      grid.sync();
    }
    // Horner finishing procedure and the embedded estimate
    for (int mode = K_H3; mode <= K_FSAL; mode++) {
      build_ops(kPhaseFinish + mode);
      sweep(err, err_row);
      if (mode == K_FSAL) {
#pragma unroll
        for (int i = 0; i < M; i++) {
          if (C.done[i]) continue;  // uniform across the grid
          sh[threadIdx.x] = err[i] + (i % G == sub ? err_row[i / G] : 0.0);
          __syncthreads();
          for (int w = kBlock / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
          }
          if (threadIdx.x == 0) P.part[i * P.nb + blockIdx.x] = sh[0];
          __syncthreads();
        }
      }
      grid.sync();
    }
    // control, in every block: the per-block partial sums reduced in a fixed
    // order (strided by thread, then a tree), then accept / reject and size
    // the next steps
    for (int i = 0; i < M; i++) {
      if (C.done[i]) continue;
      double v = 0.0;
      for (int b = threadIdx.x; b < P.nb; b += blockDim.x) v += __ldcg(&P.part[i * P.nb + b]);
      sh[threadIdx.x] = v;
      __syncthreads();
      for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
      }
      if (threadIdx.x == 0) s_err2[i] = sh[0];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i < M; i++) {
        C.acc_prev[i] = 0;
        if (C.done[i]) continue;
        s_pend[i] = 0;  // consumed by this round's first stage
        const double err2 = sqrt(s_err2[i] / (double)N);
        C.err[i] = err2;
        if (!isfinite(err2)) {
          C.status = MR_ENONFINITE;
          C.finished = 1;
          break;
        }
        const double fac = err2 == 0.0 ? 2.0 : fmin(2.0, fmax(0.2, 0.8 * pow(err2, -0.25)));
        if (err2 <= 1.0) {
          // the candidate (recurrence buffer (a+2) % 3) becomes the state:
          // FP64 by a buffer swap; the mixed form's increment Delta is added
          // to the FP64 state by the next first stage (or at the end)
          const int cp = (C.a[i] + 2) % 3;
          if constexpr (kF64) {
            const int t = s_py[i];
            s_py[i] = s_pr[i][cp];
            s_pr[i][cp] = t;
          } else {
            s_pend[i] = 1;
          }
          s_ly[i] ^= 1;
          C.acc_prev[i] = 1;
          C.c_prev[i] = cp;
          C.t[i] = C.last[i] ? P.dt : C.t[i] + C.h[i];
          if (C.last[i]) C.done[i] = 1;
        } else {
          C.rejects++;
        }
        C.h[i] *= fac;
      }
      C.rounds++;
      if (!C.finished) rock_prepare(P.m, P.dt, P.Dc, P.rho, C, N, P.work);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && !C.finished) C.status = MR_EROCK_STEP;
  // the final state into the state array where a swap moved it (FP64), or
  // the last accepted increment added to it (mixed form)
  for (int i = 0; i < P.m; i++) {
    double* u = P.U + (int64_t)i * capL;
    if constexpr (kF64) {
      if (s_py[i] == 0) continue;
      const VT* y = Y(i);
      for (int64_t r = tid; r < N; r += nth) u[r] = (double)y[r];
    } else {
      if (!s_pend[i]) continue;
      const VT* dl = Rb(i, C.c_prev[i]);
      for (int64_t r = tid; r < N; r += nth) u[r] += (double)dl[r];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *P.ctl = C;
}

// ------------------------------------------------------------ joint driver (batches)
// One cooperative launch integrates the diffusion sub-step of every instance
// of a batch (2D, same species count and precision).  Every (instance,
// species) pair keeps its own step control, stage count and buffers, as in
// the one-instance driver; block 0 takes the control of all pairs and
// publishes it through global memory (one more grid barrier per step).  Each
// sweep runs over the concatenated tables of the instances that still have a
// pair in that sweep (compacted per sweep, so instances that finished early,
// or whose stage count is lower, cost nothing), and each error norm is summed
// from per-leaf terms in fixed chunks, so results do not depend on the
// schedule.
constexpr int kChunk = 8192;  // leaves per partial sum of an error norm

struct JInst {
  double* U;
  double* W[6];
  double* E2;  // [m][capL]: per leaf and species, the squared scaled error of the step
  const int4* reg;
  const int32_t* irr_leaf;
  const int32_t* cnt;
  const int32_t* col;
  const double* w;
  const float* wf;
  int64_t N, capL, nreg, nirr;
  int slot;
  double rho;
  double Dc[kMaxM];
  SweepWork work;
};

struct JArgs {
  const JInst* inst;
  int n, m;
  const int64_t* off;  // [4][n + 1] prefix offsets: regular leaves, merged rows, leaves, error chunks
  double dt, tol;
  RockCtl* ctl;  // [n]
  int* ptr;      // [n * kMaxM][5]: pool index of the state, of the three recurrence buffers, L y slot
  double* part;  // [chunks][kMaxM]: chunk sums of the squared scaled errors
  int* flags;    // [0] every instance finished, [1] largest recurrence stage count
  RockTab tab;
};

// a pair's control as read at the start of a round
struct PairCtl {
  double h;
  int s, n, a, on;  // on: the pair steps in this round
  int py, pr[3], ly;  // pool indices; in the mixed form py is instead 1 while an
                      // accepted increment waits to join the FP64 state
  int cp;             // recurrence buffer of the last accepted candidate
};

// last k in [0, cnt) with off[k] <= q
__device__ inline int bisect(const int64_t* off, int cnt, int64_t q) {
  int lo = 0, hi = cnt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= q)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int M, typename VT>
__global__ void __launch_bounds__(kBlock, 2) k_rock_joint(JArgs A) {
  constexpr bool kF64 = std::is_same<VT, double>::value;
  constexpr int D = 2, G = 2;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char jsm[];
  const int n = A.n, L = n * M;
  Ops<VT>* s_ops = reinterpret_cast<Ops<VT>*>(jsm);
  PairCtl* s_pc = reinterpret_cast<PairCtl*>(s_ops + L);
  int64_t* s_off = reinterpret_cast<int64_t*>(s_pc + L);  // [4][n + 1] as A.off
  int64_t* s_coff = s_off + 4 * (n + 1);                    // [3][n + 1] the same over the active instances
  int* s_cmap = reinterpret_cast<int*>(s_coff + 3 * (n + 1));  // the active instances
  int* s_act = s_cmap + n;                                     // [L]
  VT* s_beta = reinterpret_cast<VT*>((reinterpret_cast<uintptr_t>(s_act + L) + 7) & ~uintptr_t(7));
  // s_beta: [L][kMaxL + 1], cl / h^2 of every level
  __shared__ double sh[kBlock];
  __shared__ int s_nact;
  for (int q = threadIdx.x; q < 4 * (n + 1); q += blockDim.x) s_off[q] = A.off[q];
  __syncthreads();
  const int64_t* reg_off = s_off;
  const int64_t* irr_off = s_off + (n + 1);
  const int64_t* leaf_off = s_off + 2 * (n + 1);
  const int64_t* chk_off = s_off + 3 * (n + 1);
  const int64_t* creg = s_coff;
  const int64_t* cirr = s_coff + (n + 1);
  const int64_t* cleaf = s_coff + 2 * (n + 1);
  const int64_t tid = (threadIdx.x & 31) + 32 * (blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5)),
                nth = (int64_t)gridDim.x * blockDim.x;  // dealt as in the one-instance driver
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  // a thread's indices increase: its cursor is found once by bisection,
  // then walks forward
  auto seek = [&](const int64_t* off, int cnt, int64_t q, int& k) {
    if (k < 0)
      k = bisect(off, cnt, q);
    else
      while (off[k + 1] <= q) k++;
  };

  auto fvec = [&](const JInst& I, int q, int sp) -> VT* {
    return reinterpret_cast<VT*>(reinterpret_cast<float*>(I.W[q >> 1]) + (q & 1) * (int64_t)A.m * I.capL) +
           (int64_t)sp * I.capL;
  };
  auto pool = [&](const JInst& I, int sp, int k) -> VT* {
    if constexpr (kF64)
      return reinterpret_cast<VT*>(k == 0 ? I.U : I.W[k - 1]) + (int64_t)sp * I.capL;
    else
      return fvec(I, k, sp);
  };
  auto Wp = [&](const JInst& I, int sp, int q) -> VT* {  // q = 3 accumulator, 4 / 5 L y
    if constexpr (kF64)
      return reinterpret_cast<VT*>(I.W[q]) + (int64_t)sp * I.capL;
    else
      return fvec(I, q + 1, sp);
  };
  // the published control of every pair, once per round
  auto load_ctl = [&]() {
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
      const int i = l / M, sp = l % M;
      PairCtl p;
      p.on = 0;
      if (sp < A.m) {
        const RockCtl& C = A.ctl[i];
        p.on = !__ldcg(&C.done[sp]) && !__ldcg(&C.finished);
        if (p.on) {
          const int* pt = A.ptr + 5 * (i * kMaxM + sp);
          p.h = __ldcg(&C.h[sp]);
          p.s = __ldcg(&C.s[sp]);
          p.n = __ldcg(&C.n[sp]);
          p.a = __ldcg(&C.a[sp]);
          p.py = __ldcg(pt);
          p.pr[0] = __ldcg(pt + 1);
          p.pr[1] = __ldcg(pt + 2);
          p.pr[2] = __ldcg(pt + 3);
          p.ly = __ldcg(pt + 4);
          p.cp = __ldcg(&C.c_prev[sp]);
        }
      }
      s_pc[l] = p;
    }
    __syncthreads();
  };
  // operands of pair l = (instance, species) in `phase`; false if it sits out
  auto ops_for = [&](int phase, int l, Ops<VT>& o) -> bool {
    const PairCtl& p = s_pc[l];
    if (!p.on) return false;
    const int i = l / M, sp = l % M;
    const JInst& I = A.inst[i];
    const double* tb = A.tab.data + A.tab.off[p.s];
    const double hd = p.h * I.Dc[sp];
    const int nn = p.n;
    VT* Y = pool(I, sp, kF64 ? p.py : 0);
    auto Rb = [&](int q) { return pool(I, sp, p.pr[q]); };
    o.b = nullptr;
    o.acc = nullptr;
    o.lx = nullptr;
    o.yn = Y;
    o.g = nullptr;
    o.cg = (VT)0;
    o.u = nullptr;
    if constexpr (!kF64) {  // increments: g = L y_n, the FP64 state for the error scale
      o.g = Wp(I, sp, 4 + p.ly);
      o.u = I.U + (int64_t)sp * I.capL;
    }
    if (phase < kPhaseFinish) {  // stage j >= 2
      const int j = phase;
      if (j > nn) return false;
      o.kind = K_STAGE;
      o.x = Rb((j - 2) % 3);
      o.a = o.x;
      o.b = j == 2 ? (kF64 ? Y : nullptr) : Rb((j - 3) % 3);
      o.out = Rb((j - 1) % 3);
      o.ca = (VT)tb[10 + (j - 1)];
      o.cb = (VT)tb[10 + nn + (j - 1)];
      o.cl = (VT)(tb[10 + 2 * nn + (j - 1)] * hd);
      return true;
    }
    const double* w = tb + 1;
    const double* e = tb + 6;
    const int a = p.a, b = (a + 1) % 3, cc = (a + 2) % 3;
    o.kind = phase - kPhaseFinish;
    switch (o.kind) {
      case K_STAGE1:
        o.x = Y; o.a = Y; o.out = Rb(0); o.lx = Wp(I, sp, 4 + p.ly);
        o.ca = (VT)tb[10]; o.cl = (VT)(tb[10 + 2 * nn] * hd);
        // mixed form: the accepted increment still to be added to the state
        if (!kF64 && p.py) o.b = Rb(p.cp);
        break;
      case K_H3:
        o.x = Rb(a); o.a = Rb(a); o.out = Rb(b); o.ca = (VT)w[3]; o.cl = (VT)(w[4] * hd); o.cg = (VT)(w[4] * hd);
        break;
      case K_H2: o.x = Rb(b); o.a = Rb(a); o.out = Rb(cc); o.ca = (VT)w[2]; o.cl = (VT)hd; o.cg = (VT)(w[3] * hd); break;
      case K_H1:
        o.x = Rb(cc); o.a = Rb(a); o.out = Rb(b); o.acc = Wp(I, sp, 3); o.ca = (VT)w[1]; o.cl = (VT)hd;
        o.e0 = (VT)e[0]; o.e1 = (VT)e[1]; o.e2 = (VT)e[2]; o.cg = (VT)(w[2] * hd);
        break;
      case K_H0:
        o.x = Rb(b); o.a = Rb(a); o.out = Rb(cc); o.acc = Wp(I, sp, 3); o.ca = (VT)1; o.cl = (VT)hd;
        o.cg = (VT)(w[1] * hd);
        break;
      default:
        o.x = Rb(cc); o.a = nullptr; o.out = nullptr; o.acc = Wp(I, sp, 3); o.lx = Wp(I, sp, 5 - p.ly);
        o.cl = (VT)(e[3] * hd);
    }
    return true;
  };
  // operands of every pair in `phase`, then the instances with an active
  // pair compacted (warp 0: ballot for the positions, shuffle scans for the
  // offsets)
  auto build_ops = [&](int phase) {
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) s_act[l] = ops_for(phase, l, s_ops[l]);
    __syncthreads();
    for (int q = threadIdx.x; q < L * (kMaxL + 1); q += blockDim.x) {
      const int l = q / (kMaxL + 1), j = q % (kMaxL + 1);
      if (s_act[l]) {
        if constexpr (kF64)
          s_beta[q] = s_ops[l].cl * c_ih2[j];
        else
          s_beta[q] = s_ops[l].cl * c_ih2f[j];
      }
    }
    if (threadIdx.x < 32) {
      int cnt = 0;
      int64_t c0 = 0, c1 = 0, c2 = 0;
      if (lane == 0) s_coff[0] = s_coff[n + 1] = s_coff[2 * (n + 1)] = 0;
      for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        bool on = false;
        if (i < n)
#pragma unroll
          for (int sp = 0; sp < M; sp++) on = on || s_act[i * M + sp];
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        int64_t v0 = on ? reg_off[i + 1] - reg_off[i] : 0;
        int64_t v1 = on ? irr_off[i + 1] - irr_off[i] : 0;
        int64_t v2 = on ? leaf_off[i + 1] - leaf_off[i] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int64_t t0 = __shfl_up_sync(0xffffffffu, v0, d), t1 = __shfl_up_sync(0xffffffffu, v1, d),
                        t2 = __shfl_up_sync(0xffffffffu, v2, d);
          if (lane >= d) {
            v0 += t0;
            v1 += t1;
            v2 += t2;
          }
        }
        if (on) {
          const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
          s_cmap[pos] = i;
          s_coff[pos + 1] = c0 + v0;
          s_coff[(n + 1) + pos + 1] = c1 + v1;
          s_coff[2 * (n + 1) + pos + 1] = c2 + v2;
        }
        cnt += __popc(bal);
        c0 += __shfl_sync(0xffffffffu, v0, 31);
        c1 += __shfl_sync(0xffffffffu, v1, 31);
        c2 += __shfl_sync(0xffffffffu, v2, 31);
      }
      if (lane == 0) s_nact = cnt;
    }
    __syncthreads();
  };
  // the embedded estimate of one leaf: its squared scaled error goes to E2
  auto finish = [&](const Ops<VT>& o, const JInst& I, int sp, int64_t r, VT d, VT ih2, VT beta) {
    if (o.kind == K_FSAL) {
      double ee, sc;
      if constexpr (kF64) {
        const VT Lx = d * ih2;
        o.lx[r] = Lx;
        ee = (double)(o.acc[r] + o.cl * Lx);
        sc = A.tol + A.tol * fmax(fabs((double)o.yn[r]), fabs((double)o.x[r]));
      } else {  // increments: L y_{n+1} = g + L Delta, scale from y_n and y_n + Delta
        const VT ly1 = o.g[r] + d * ih2;
        o.lx[r] = ly1;
        ee = (double)(o.acc[r] + o.cl * ly1);
        const double yv = o.u[r];
        sc = A.tol + A.tol * fmax(fabs(yv), fabs(yv + (double)o.x[r]));
      }
      I.E2[(int64_t)sp * I.capL + r] = (ee / sc) * (ee / sc);
    } else {
      double unused = 0.0;
      combine<VT>(o, r, d, ih2, beta, A.tol, unused);
    }
  };
  // one operator sweep over the active instances: regular leaves one thread
  // each, merged rows G lanes each (taken from the last threads)
  auto sweep = [&]() {
    const int na = s_nact;
    const int64_t nreg = creg[na], nirr = cirr[na];
    int k = -1;
    for (int64_t q = tid; q < nreg; q += nth) {
      seek(creg, na, q, k);
      const int i = s_cmap[k];
      const JInst& I = A.inst[i];
      const int64_t ql = q - creg[k];
      const int4 e0 = I.reg[2 * ql], e1 = I.reg[2 * ql + 1];
      const int v[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
      const int64_t r = v[0];
      const int lev = v[1 + 2 * D];
      VT ih2;
      if constexpr (kF64)
        ih2 = c_ih2[lev];
      else
        ih2 = c_ih2f[lev];
#pragma unroll
      for (int sp = 0; sp < M; sp++) {
        const int l = i * M + sp;
        if (!s_act[l]) continue;
        const Ops<VT>& o = s_ops[l];
        const VT* x = o.x;
        VT sx = x[v[1]];
#pragma unroll
        for (int f = 1; f < 2 * D; f++) sx += x[v[1 + f]];
        finish(o, I, sp, r, sx - (VT)(2 * D) * x[r], ih2, s_beta[l * (kMaxL + 1) + lev]);
      }
    }
    const int64_t grp = (nth - 1 - tid) / G, ngrp = nth / G;
    const int64_t rounds = (nirr + ngrp - 1) / ngrp;
    k = -1;
    for (int64_t kk = 0; kk < rounds; kk++) {
      const int64_t row = grp + kk * ngrp;
      const bool have = row < nirr;
      int i = 0;
      VT vs[M];
#pragma unroll
      for (int sp = 0; sp < M; sp++) vs[sp] = (VT)0;
      int32_t r = 0;
      if (have) {
        seek(cirr, na, row, k);
        i = s_cmap[k];
        const JInst& I = A.inst[i];
        const int64_t rl = row - cirr[k];
        r = I.irr_leaf[rl];
        const int cnt = I.cnt[rl];
        const int32_t* col = I.col + rl * (int64_t)I.slot;
        const VT* wr;
        if constexpr (kF64)
          wr = I.w + rl * (int64_t)I.slot;
        else
          wr = I.wf + rl * (int64_t)I.slot;
#pragma unroll 4
        for (int e = sub; e < cnt; e += G) {
          const int32_t cidx = col[e];
          const VT we = wr[e];
#pragma unroll
          for (int sp = 0; sp < M; sp++)
            if (s_act[i * M + sp]) vs[sp] += we * s_ops[i * M + sp].x[cidx];
        }
      }
#pragma unroll
      for (int sp = 0; sp < M; sp++)
        for (int sft = G / 2; sft > 0; sft >>= 1) vs[sp] += __shfl_xor_sync(0xffffffffu, vs[sp], sft);
      if (have && sub == 0) {
        const JInst& I = A.inst[i];
#pragma unroll
        for (int sp = 0; sp < M; sp++)
          if (s_act[i * M + sp]) finish(s_ops[i * M + sp], I, sp, r, vs[sp], (VT)1, s_ops[i * M + sp].cl);
      }
    }
  };
  // mixed form, first stage of the sub-step: g = L y_n of every active pair
  // applied to the FP64 state in FP64 (kept as the float L y) and
  // delta_1 = kap_1 h D g, over the active instances as in sweep()
  auto gsweep = [&]() {
    const int na = s_nact;
    const int64_t nreg = creg[na], nirr = cirr[na];
    int k = -1;
    for (int64_t q = tid; q < nreg; q += nth) {
      seek(creg, na, q, k);
      const int i = s_cmap[k];
      const JInst& I = A.inst[i];
      const int64_t ql = q - creg[k];
      const int4 e0 = I.reg[2 * ql], e1 = I.reg[2 * ql + 1];
      const int v[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
      const int64_t r = v[0];
      const double ih2 = c_ih2[v[1 + 2 * D]];
#pragma unroll
      for (int sp = 0; sp < M; sp++) {
        const int l = i * M + sp;
        if (!s_act[l]) continue;
        const Ops<VT>& o = s_ops[l];
        const double* u = I.U + (int64_t)sp * I.capL;
        double sx = u[v[1]];
#pragma unroll
        for (int f = 1; f < 2 * D; f++) sx += u[v[1 + f]];
        const double gv = (sx - 2.0 * D * u[r]) * ih2;
        o.lx[r] = (VT)gv;
        o.out[r] = (VT)((double)o.cl * gv);
      }
    }
    const int64_t grp = (nth - 1 - tid) / G, ngrp = nth / G;
    const int64_t rounds = (nirr + ngrp - 1) / ngrp;
    k = -1;
    for (int64_t kk = 0; kk < rounds; kk++) {
      const int64_t row = grp + kk * ngrp;
      const bool have = row < nirr;
      int i = 0;
      double vs[M];
#pragma unroll
      for (int sp = 0; sp < M; sp++) vs[sp] = 0.0;
      int32_t r = 0;
      if (have) {
        seek(cirr, na, row, k);
        i = s_cmap[k];
        const JInst& I = A.inst[i];
        const int64_t rl = row - cirr[k];
        r = I.irr_leaf[rl];
        const int cnt = I.cnt[rl];
        const int32_t* col = I.col + rl * (int64_t)I.slot;
        const double* wr = I.w + rl * (int64_t)I.slot;
        for (int e = sub; e < cnt; e += G) {
          const int32_t cidx = col[e];
          const double we = wr[e];
#pragma unroll
          for (int sp = 0; sp < M; sp++)
            if (s_act[i * M + sp]) vs[sp] += we * I.U[(int64_t)sp * I.capL + cidx];
        }
      }
#pragma unroll
      for (int sp = 0; sp < M; sp++)
        for (int sft = G / 2; sft > 0; sft >>= 1) vs[sp] += __shfl_xor_sync(0xffffffffu, vs[sp], sft);
      if (have && sub == 0) {
#pragma unroll
        for (int sp = 0; sp < M; sp++)
          if (s_act[i * M + sp]) {
            const Ops<VT>& o = s_ops[i * M + sp];
            o.lx[r] = (VT)vs[sp];
            o.out[r] = (VT)((double)o.cl * vs[sp]);
          }
      }
    }
  };
  // accept / reject and the next step of instance i (one thread of block 0)
  auto control = [&](int i) {
    RockCtl& C = A.ctl[i];
    const JInst& I = A.inst[i];
    for (int sp = 0; sp < A.m; sp++) {
      C.acc_prev[sp] = 0;
      if (C.done[sp]) continue;
      double e2 = 0.0;
      for (int64_t c = chk_off[i]; c < chk_off[i + 1]; c++) e2 += __ldcg(&A.part[c * kMaxM + sp]);
      const double err = sqrt(e2 / (double)I.N);
      C.err[sp] = err;
      if (!isfinite(err)) {
        C.status = MR_ENONFINITE;
        C.finished = 1;
        break;
      }
      const double fac = err == 0.0 ? 2.0 : fmin(2.0, fmax(0.2, 0.8 * pow(err, -0.25)));
      int* pt = A.ptr + 5 * (i * kMaxM + sp);
      if (!kF64) pt[0] = 0;  // the pending increment was added by this round's first stage
      if (err <= 1.0) {
        // the candidate (recurrence buffer (a+2) % 3) becomes the state: by a
        // buffer swap (FP64), or its increment joins the FP64 state at the
        // next first stage or at the end (mixed form)
        const int cp = (C.a[sp] + 2) % 3;
        if constexpr (kF64) {
          const int t = pt[0];
          pt[0] = pt[1 + cp];
          pt[1 + cp] = t;
        } else {
          pt[0] = 1;
        }
        pt[4] ^= 1;
        C.acc_prev[sp] = 1;
        C.c_prev[sp] = cp;
        C.t[sp] = C.last[sp] ? A.dt : C.t[sp] + C.h[sp];
        if (C.last[sp]) C.done[sp] = 1;
      } else {
        C.rejects++;
      }
      C.h[sp] *= fac;
    }
    C.rounds++;
    if (!C.finished) rock_prepare(A.m, A.dt, I.Dc, I.rho, C, I.N, I.work);
  };
  auto publish = [&]() {  // block 0: the flags every block reads after the next barrier
    if (blockIdx.x == 0) {
      __syncthreads();
      if (threadIdx.x == 0) {
        int fin = 1, nmax = 0;
        for (int i = 0; i < n; i++) {
          const bool f = A.ctl[i].finished || A.ctl[i].status;
          fin = fin && f;
          if (!f) nmax = max(nmax, A.ctl[i].nmax);
        }
        A.flags[0] = fin;
        A.flags[1] = nmax;
      }
      __threadfence();
    }
  };

  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const JInst& I = A.inst[i];
      rock_prepare(A.m, A.dt, I.Dc, I.rho, A.ctl[i], I.N, I.work);
      for (int sp = 0; sp < kMaxM; sp++) {
        int* pt = A.ptr + 5 * (i * kMaxM + sp);
        pt[0] = 0;
        pt[1] = 1;
        pt[2] = 2;
        pt[3] = 3;
        pt[4] = 0;
      }
    }
  }
  publish();
  const int64_t nleaf_all = leaf_off[n];
  grid.sync();
  bool first = true;
  for (int round = 0; round < 20000; round++) {
    if (__ldcg(&A.flags[0])) break;
    const int nmax = __ldcg(&A.flags[1]);
    load_ctl();
    // stage 1: P_1 = y + kap_1 h L y (an operator sweep in the first step,
    // then an axpy on the kept L y)
    build_ops(kPhaseFinish + K_STAGE1);
    if (first) {
      if constexpr (kF64)
        sweep();
      else
        gsweep();
    } else {
      const int na = s_nact;
      const int64_t nl = cleaf[na];
      int k = -1;
      for (int64_t q = tid; q < nl; q += nth) {
        seek(cleaf, na, q, k);
        const int i = s_cmap[k];
        const int64_t r = q - cleaf[k];
#pragma unroll
        for (int sp = 0; sp < M; sp++) {
          const int l = i * M + sp;
          if (!s_act[l]) continue;
          const Ops<VT>& o = s_ops[l];
          if constexpr (kF64) {
            o.out[r] = o.ca * o.a[r] + o.cl * o.lx[r];
          } else {
            if (o.b) {  // the accepted increment joins the FP64 state (read before delta_1 is written)
              const VT dv = o.b[r];
              A.inst[i].U[(int64_t)sp * A.inst[i].capL + r] += (double)dv;
            }
            o.out[r] = o.cl * o.lx[r];
          }
        }
      }
    }
    first = false;
    grid.sync();
    for (int j = 2; j <= nmax; j++) {  // recurrence stages P_j -> R[(j-1) % 3]
      build_ops(j);
      sweep();
      grid.sync();
    }
    for (int mode = K_H3; mode <= K_FSAL; mode++) {  // finishing procedure, embedded estimate
      build_ops(kPhaseFinish + mode);
      sweep();
      grid.sync();
    }
    // chunk sums of the error terms (the pairs of the last sweep), one block
    // per chunk in a fixed order
    for (int64_t c = blockIdx.x; c < chk_off[n]; c += gridDim.x) {
      const int i = bisect(chk_off, n, c);
      const JInst& I = A.inst[i];
      const int64_t r0 = (c - chk_off[i]) * kChunk, r1 = min(I.N, r0 + kChunk);
      for (int sp = 0; sp < M; sp++) {
        if (!s_act[i * M + sp]) continue;
        double v = 0.0;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) v += __ldcg(&I.E2[(int64_t)sp * I.capL + r]);
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = kBlock / 2; w > 0; w >>= 1) {
          if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
          __syncthreads();
        }
        if (threadIdx.x == 0) A.part[c * kMaxM + sp] = sh[0];
        __syncthreads();
      }
    }
    grid.sync();
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (!A.ctl[i].finished) control(i);
    publish();
    grid.sync();
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (!A.ctl[i].finished) A.ctl[i].status = MR_EROCK_STEP;
  // the final states into the state arrays where a swap moved them (FP64),
  // or the last accepted increments added to them (mixed form)
  int k = -1;
  for (int64_t q = tid; q < nleaf_all; q += nth) {
    seek(leaf_off, n, q, k);
    const JInst& I = A.inst[k];
    const int64_t r = q - leaf_off[k];
    for (int sp = 0; sp < A.m; sp++) {
      const int* pt = A.ptr + 5 * (k * kMaxM + sp);
      const int py = __ldcg(pt);
      if (py == 0) continue;
      if constexpr (kF64) {
        I.U[(int64_t)sp * I.capL + r] = (double)pool(I, sp, py)[r];
      } else {
        const int cp = __ldcg(&A.ctl[k].c_prev[sp]);
        I.U[(int64_t)sp * I.capL + r] += (double)pool(I, sp, __ldcg(pt + 1 + cp))[r];
      }
    }
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

// every stage count's coefficients, built once per process (thread-safe:
// contexts on several host threads share them)
std::vector<Coeffs>& coeff_cache() {
  static std::vector<Coeffs> cache = [] {
    std::vector<Coeffs> v(kSmax + 1);
    for (int s = kSmin; s <= kSmax; s++)
      if (build_coeffs(s, v[s])) v[s].s = 0;
    return v;
  }();
  return cache;
}

const Coeffs* get_coeffs(int s) {
  if (s < kSmin || s > kSmax) return nullptr;
  const Coeffs& C = coeff_cache()[s];
  return C.s == s ? &C : nullptr;
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

// the sweep work of context c's current tree (see SweepWork); cm: the
// uniform-grid form (no table)
static SweepWork sweep_work(const mr_ctx* c, bool cm, bool inc) {
  const double N = (double)c->tb[c->cur].nleaves, nirr = (double)c->stats.irregular_rows,
               nnz = (double)c->stats.irregular_nnz;
  SweepWork W;
  W.tab_bytes = (cm ? 0.0 : (N - nirr) * (8.0 * c->d + 1.0)) + (inc ? 8.0 : 12.0) * nnz + 8.0 * nirr;
  W.op_flops = (2.0 * c->d + 1.0) * (N - nirr) + 2.0 * nnz;
  W.inc = inc;
  return W;
}

// 1/h_j^2 of every level in constant memory, written once per device
static std::mutex g_ih2_mu;
static bool g_ih2_done[256] = {false};

static mr_status init_ih2(mr_ctx* c) {
  int dev = 0;
  MR_CUDA(c, cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_ih2_mu);
  if (dev >= 0 && dev < 256 && g_ih2_done[dev]) return MR_OK;
  double ih2[kMaxL + 1];
  float ih2f[kMaxL + 1];
  for (int j = 0; j <= kMaxL; j++) {
    ih2[j] = ldexp(1.0, 2 * j);
    ih2f[j] = ldexpf(1.0f, 2 * j);
  }
  MR_CUDA(c, cudaMemcpyToSymbol(c_ih2, ih2, sizeof ih2));
  MR_CUDA(c, cudaMemcpyToSymbol(c_ih2f, ih2f, sizeof ih2f));
  if (dev >= 0 && dev < 256) g_ih2_done[dev] = true;
  return MR_OK;
}

static void launch_rock(mr_ctx* c, const StageArgs& A, int64_t N, int nb, int* nev = nullptr) {
  if (nev && *nev < 256) cudaEventRecord(c->tev[2 * *nev], c->stream);
  IrrRows R{c->irr_cnt, c->irr_col, c->irr_w, c->irr_wf, c->irr_slot};
  if (c->d == 2)
    k_rock<2><<<nb, kBlock, 0, c->stream>>>(A, N, c->cap_leaves, c->nbr, c->leaf_lvl, R, c->red);
  else
    k_rock<3><<<nb, kBlock, 0, c->stream>>>(A, N, c->cap_leaves, c->nbr, c->leaf_lvl, R, c->red);
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
  MR_TRY(init_ih2(c));
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

// device coefficient table for every s (built once per process on the host)
struct HostTable {
  std::vector<double> data;
  int off[kSmax + 1] = {0};
  bool ok = true;
};

static const HostTable& host_table() {
  static const HostTable T = [] {
    HostTable t;
    for (int s = kSmin; s <= kSmax; s++) {
      const Coeffs* C = get_coeffs(s);
      if (!C) {
        t.ok = false;
        break;
      }
      t.off[s] = (int)t.data.size();
      const int n = s - 4;
      t.data.push_back(C->ell);
      for (int k = 0; k < 5; k++) t.data.push_back(C->w[k]);
      for (int k = 0; k < 4; k++) t.data.push_back(C->errc[k]);
      for (int j = 1; j <= n; j++) t.data.push_back(C->mu[j]);
      for (int j = 1; j <= n; j++) t.data.push_back(C->nu[j]);
      for (int j = 1; j <= n; j++) t.data.push_back(C->kap[j]);
    }
    return t;
  }();
  return T;
}

static const double* device_table(mr_ctx* c, RockTab* tab) {
  const HostTable& T = host_table();
  if (!T.ok) return nullptr;
  const std::vector<double>& host = T.data;
  const int* off = T.off;
  if (!c->rock_tab) {
    if (cudaMalloc(&c->rock_tab, sizeof(double) * host.size()) != cudaSuccess) return nullptr;
    if (cudaMemcpy(c->rock_tab, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return nullptr;
  }
  for (int s = 0; s <= kSmax; s++) tab->off[s] = s >= kSmin ? off[s] : 0;
  tab->data = c->rock_tab;
  return c->rock_tab;
}

mr_status diffuse(mr_ctx* c, double dt, double tol) {
  mr_status st = build_tables(c);
  if (st) return st;
  const int m = c->m;
  const int64_t N = c->tb[c->cur].nleaves;
  MR_TRY(init_ih2(c));
  PersArgs P;
  memset(&P, 0, sizeof P);
  if (!device_table(c, &P.tab)) {
    c->last_error = "ROCK4 coefficient table";
    return MR_ESTATE;
  }
  int dev = 0, nsm = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // kernels for 1, 3 and up to 16 species (unused species of the 16-wide
  // kernel are marked done); more species run in windows of 16
  const int M = m == 1 ? 1 : (m == 3 ? 3 : 16);
  // FP64 stage vectors, or FP32 in the mixed form
  const bool f32 = c->prob.precision != MR_FP64;
  // the uniform finest grid (Cartesian mesh) sweeps without the table
  const bool cm = N == c->n_level[c->J] && c->stats.irregular_rows == 0 && (M == 1 || M == 3);
  const void* kern;
  if (cm) {
    if (!f32)
      kern = c->d == 2 ? (M == 1 ? (const void*)k_rock_persistent<2, 1, double, true>
                                 : (const void*)k_rock_persistent<2, 3, double, true>)
                       : (M == 1 ? (const void*)k_rock_persistent<3, 1, double, true>
                                 : (const void*)k_rock_persistent<3, 3, double, true>);
    else
      kern = c->d == 2 ? (M == 1 ? (const void*)k_rock_persistent<2, 1, float, true>
                                 : (const void*)k_rock_persistent<2, 3, float, true>)
                       : (M == 1 ? (const void*)k_rock_persistent<3, 1, float, true>
                                 : (const void*)k_rock_persistent<3, 3, float, true>);
  } else if (!f32)
    kern = c->d == 2 ? (M == 1 ? (const void*)k_rock_persistent<2, 1, double>
                               : (M == 3 ? (const void*)k_rock_persistent<2, 3, double>
                                         : (const void*)k_rock_persistent<2, 16, double>))
                     : (M == 1 ? (const void*)k_rock_persistent<3, 1, double>
                               : (M == 3 ? (const void*)k_rock_persistent<3, 3, double>
                                         : (const void*)k_rock_persistent<3, 16, double>));
  else
    kern = c->d == 2 ? (M == 1 ? (const void*)k_rock_persistent<2, 1, float>
                               : (M == 3 ? (const void*)k_rock_persistent<2, 3, float>
                                         : (const void*)k_rock_persistent<2, 16, float>))
                     : (M == 1 ? (const void*)k_rock_persistent<3, 1, float>
                               : (M == 3 ? (const void*)k_rock_persistent<3, 3, float>
                                         : (const void*)k_rock_persistent<3, 16, float>));
  MR_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0));
  if (per_sm < 1) return MR_ECUDA;
  // enough blocks to cover the leaves, at most two co-resident per SM
  const int64_t want = std::max<int64_t>(1, (N + kBlock - 1) / kBlock);
  const int nb = (int)std::min<int64_t>(want, (int64_t)nsm * std::min(per_sm, 2));
  mr_stats& S = c->stats;
  S.rock_steps = S.rock_reject = S.rock_stages = S.rock_matvec = 0;
  S.rock_smax = 0;
  for (int w0 = 0; w0 < m; w0 += M) {
    const int mw = std::min(M, m - w0);  // species of this window
    bool any = false;
    for (int i = 0; i < mw; i++) any = any || c->prob.D[w0 + i] != 0.0;
    if (!any && w0 > 0) continue;  // nothing diffuses in this window
    RockCtl hctl;
    memset(&hctl, 0, sizeof hctl);
    for (int i = 0; i < kMaxM; i++) {
      hctl.h[i] = dt;
      hctl.done[i] = i >= mw || !(dt > 0.0) || c->prob.D[w0 + i] == 0.0 || N == 0;
    }
    RockCtl* dctl = reinterpret_cast<RockCtl*>(c->rock_ctl);
    MR_CUDA(c, cudaMemcpyAsync(dctl, &hctl, sizeof hctl, cudaMemcpyHostToDevice, c->stream));
    P.m = mw;
    P.D = c->d;
    P.J = c->J;
    P.nb = nb;
    P.N = N;
    P.capL = c->cap_leaves;
    P.dt = dt;
    P.tol = tol;
    P.rho = c->rho;
    P.work = sweep_work(c, cm, f32);
    for (int i = 0; i < mw; i++) P.Dc[i] = c->prob.D[w0 + i];
    // the window's species: rows w0.. of the state and of every work buffer
    P.U = c->tb[c->cur].U + (int64_t)w0 * c->cap_leaves;
    for (int q = 0; q < 6; q++) P.W[q] = c->work[q] + (int64_t)w0 * c->cap_leaves;
    P.part = c->red;
    P.ctl = dctl;
    IrrRows R{c->irr_cnt, c->irr_col, c->irr_w, c->irr_wf, c->irr_slot};
    const int4* reg = c->reg_tab;
    const int32_t* irr_leaf = c->irr_leaf;
    int64_t nirr = c->stats.irregular_rows;
    int64_t nreg = N - nirr;
    void* args[] = {&P, (void*)&reg, &nreg, &R, (void*)&irr_leaf, &nirr};
    MR_CUDA(c, cudaEventRecord(c->tev[0], c->stream));
    MR_CUDA(c, cudaLaunchCooperativeKernel(kern, nb, kBlock, args, 0, c->stream));
    MR_CUDA(c, cudaEventRecord(c->tev[1], c->stream));
    c->launches++;
    MR_CUDA(c, cudaMemcpyAsync(&hctl, dctl, sizeof hctl, cudaMemcpyDeviceToHost, c->stream));
    MR_CUDA(c, cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->tev[0], c->tev[1]);
    S.rock_steps += hctl.steps;
    S.rock_reject += hctl.rejects;
    S.rock_stages += hctl.stages;
    S.rock_matvec += hctl.matvecs;
    S.rock_smax = std::max(S.rock_smax, (int32_t)hctl.smax);
    S.rock_kernel_ms += ms;
    S.rock_kernel_launches++;
    S.rock_alg_bytes += hctl.bytes;
    S.rock_alg_flops += hctl.flops;
    if (hctl.status) {
      c->last_error = "ROCK4 step control failed";
      return (mr_status)hctl.status;
    }
  }
  return MR_OK;
}


// ------------------------------------------------------------ joint driver (host)
namespace {
template <int M, typename VT>
const void* joint_kernel() {
  return (const void*)k_rock_joint<M, VT>;
}
}  // namespace

void free_batch_rock(BatchRockScratch& S) {
  cudaFree(S.inst);
  cudaFree(S.off);
  cudaFree(S.ctl);
  cudaFree(S.ptr);
  cudaFree(S.part);
  cudaFree(S.flags);
  for (int q = 0; q < 2; q++)
    if (S.ev[q]) cudaEventDestroy(S.ev[q]);
  S = BatchRockScratch{};
}

mr_status diffuse_batch(mr_ctx* const* cs, int n, double dt, double tol, cudaStream_t stream, BatchRockScratch& S,
                        double* kernel_ms, int blocks_per_sm) {
  if (blocks_per_sm != 1 && blocks_per_sm != 2) return MR_EINVAL;
  if (n < 1) return MR_EINVAL;
  const int m = cs[0]->m, prec = cs[0]->prob.precision;
  if (cs[0]->d != 2 || (m != 1 && m != 3)) return MR_EINVAL;
  for (int b = 1; b < n; b++)
    if (cs[b]->d != 2 || cs[b]->m != m || cs[b]->prob.precision != prec) return MR_EINVAL;
  for (int b = 0; b < n; b++) {
    MR_TRY(build_tables(cs[b]));
    MR_TRY(init_ih2(cs[b]));
    if (!cs[b]->e2buf) MR_CUDA(cs[b], cudaMalloc(&cs[b]->e2buf, sizeof(double) * (size_t)m * cs[b]->cap_leaves));
  }
  JArgs A;
  memset(&A, 0, sizeof A);
  if (!device_table(cs[0], &A.tab)) return MR_ESTATE;
  std::vector<JInst> hin(n);
  std::vector<int64_t> off(4 * (n + 1), 0);
  std::vector<RockCtl> hctl(n);
  for (int b = 0; b < n; b++) {
    mr_ctx* c = cs[b];
    JInst& I = hin[b];
    memset(&I, 0, sizeof I);
    I.U = c->tb[c->cur].U;
    for (int q = 0; q < 6; q++) I.W[q] = c->work[q];
    I.E2 = c->e2buf;
    I.reg = c->reg_tab;
    I.irr_leaf = c->irr_leaf;
    I.cnt = c->irr_cnt;
    I.col = c->irr_col;
    I.w = c->irr_w;
    I.wf = c->irr_wf;
    I.N = c->tb[c->cur].nleaves;
    I.capL = c->cap_leaves;
    I.nirr = c->stats.irregular_rows;
    I.nreg = I.N - I.nirr;
    I.slot = c->irr_slot;
    I.rho = c->rho;
    I.work = sweep_work(c, false, prec != MR_FP64);
    for (int i = 0; i < m; i++) I.Dc[i] = c->prob.D[i];
    off[b + 1] = off[b] + I.nreg;
    off[(n + 1) + b + 1] = off[(n + 1) + b] + I.nirr;
    off[2 * (n + 1) + b + 1] = off[2 * (n + 1) + b] + I.N;
    off[3 * (n + 1) + b + 1] = off[3 * (n + 1) + b] + (I.N + kChunk - 1) / kChunk;
    RockCtl& C = hctl[b];
    memset(&C, 0, sizeof C);
    for (int i = 0; i < kMaxM; i++) {
      C.h[i] = dt;
      C.done[i] = i >= m || !(dt > 0.0) || c->prob.D[i] == 0.0 || I.N == 0;
    }
  }
  const int64_t chunks = std::max<int64_t>(1, off[4 * (n + 1) - 1]);
  if (S.cap < n || S.part_cap < chunks) {
    free_batch_rock(S);
    if (cudaMalloc(&S.inst, sizeof(JInst) * n) != cudaSuccess ||
        cudaMalloc(&S.off, sizeof(int64_t) * 4 * (n + 1)) != cudaSuccess ||
        cudaMalloc(&S.ctl, sizeof(RockCtl) * n) != cudaSuccess ||
        cudaMalloc(&S.ptr, sizeof(int) * 5 * kMaxM * n) != cudaSuccess ||
        cudaMalloc(&S.part, sizeof(double) * kMaxM * 2 * chunks) != cudaSuccess ||
        cudaMalloc(&S.flags, sizeof(int) * 2) != cudaSuccess || cudaEventCreate(&S.ev[0]) != cudaSuccess ||
        cudaEventCreate(&S.ev[1]) != cudaSuccess) {
      free_batch_rock(S);
      return MR_ENOMEM;
    }
    S.cap = n;
    S.part_cap = 2 * chunks;
  }
  if (cudaMemcpyAsync(S.inst, hin.data(), sizeof(JInst) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(S.off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(S.ctl, hctl.data(), sizeof(RockCtl) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return MR_ECUDA;
  const bool f32 = prec != MR_FP64;
  const void* kern = m == 3 ? (f32 ? joint_kernel<3, float>() : joint_kernel<3, double>())
                            : (f32 ? joint_kernel<1, float>() : joint_kernel<1, double>());
  const int L = n * (m == 3 ? 3 : 1);
  const size_t smem = (size_t)L * ((f32 ? sizeof(Ops<float>) : sizeof(Ops<double>)) + sizeof(PairCtl) + sizeof(int)) +
                      sizeof(int64_t) * 7 * (n + 1) + sizeof(int) * (n + 1) +
                      (size_t)L * (kMaxL + 1) * (f32 ? sizeof(float) : sizeof(double)) + 8;
  if (smem > 200 * 1024) return MR_EINVAL;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MR_ECUDA;
  int dev = 0, nsm = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem) != cudaSuccess || per_sm < 1)
    return MR_ECUDA;
  A.inst = reinterpret_cast<const JInst*>(S.inst);
  A.n = n;
  A.m = m;
  A.off = S.off;
  A.dt = dt;
  A.tol = tol;
  A.ctl = reinterpret_cast<RockCtl*>(S.ctl);
  A.ptr = S.ptr;
  A.part = S.part;
  A.flags = S.flags;
  void* args[] = {&A};
  const int nb = nsm * std::min(per_sm, blocks_per_sm);
  cudaEventRecord(S.ev[0], stream);
  if (cudaLaunchCooperativeKernel(kern, nb, kBlock, args, smem, stream) != cudaSuccess) return MR_ECUDA;
  cudaEventRecord(S.ev[1], stream);
  if (cudaMemcpyAsync(hctl.data(), S.ctl, sizeof(RockCtl) * n, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return MR_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, S.ev[0], S.ev[1]);
  if (kernel_ms) *kernel_ms = ms;
  mr_status st = MR_OK;
  for (int b = 0; b < n; b++) {
    mr_stats& s = cs[b]->stats;
    s.rock_steps = hctl[b].steps;
    s.rock_reject = hctl[b].rejects;
    s.rock_stages = hctl[b].stages;
    s.rock_matvec = hctl[b].matvecs;
    s.rock_smax = hctl[b].smax;
    s.rock_alg_bytes += hctl[b].bytes;
    s.rock_alg_flops += hctl[b].flops;
    if (hctl[b].status && !st) {
      cs[b]->last_error = "ROCK4 step control failed";
      st = (mr_status)hctl[b].status;
    }
  }
  return st;
}

}  // namespace mrg
