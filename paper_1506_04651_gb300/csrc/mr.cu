// Multiresolution kernels: projection, details and thresholds, graded
// refinement and coarsening, tree reconstruction, new-node prediction, leaf
// lists, and the finite-volume leaf operator tables.
//
// Paper: Sec. 2.2 (dyadic tree, projection = exact average of the 2^d
// children, prediction Eq. inter_1d by tensor product, details Eq. detail,
// thresholds eps_j = 2^((d/2)(j-J)) eps, graded tree), Sec. 3.1.2 (refine
// tagged leaves, tag extra nodes until graded, coarsen untagged families while
// grading survives, repeat until no deletion), Eq. discretise and App. C
// (finite-volume leaf operator with level-dependent coefficients).
//
// GPU formulation.  A tree is the set R of refined (internal) cells: the nodes
// are the root and the children of R.  Grading holds iff every refined cell
// (i, p), i >= 1, forces the cells (i-1, floor((p+o)/2)), o in {-1,0,1}^d, to
// be refined.  One adaptation is then a single sweep from level J-1 down to
// 0 over dense per-level byte flags:
//   candidate(P) = refined before, or a tagged leaf, or forced from level i+1;
//   keep(P)      = forced, or new, or tagged, or level < jmin;
// kept cells force their level i-1 neighbours.  This reaches the same tree
// as repeating "refine, grade, coarsen until no deletion": grading only adds
// cells below a refined one, and a deletion only relaxes forcing one level
// down.  Nodes are then renumbered without sorting: an exclusive scan over
// the refined flags of all levels gives each refined cell its rank g, and its
// children are nodes 1 + 2^d g ... 2^d (g + 1) (level-major Morton order).
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include <type_traits>

#include "mr_internal.cuh"

namespace mrg {
namespace {

constexpr uint8_t F_OLD_INT = 1, F_TAG = 2, F_LEAF_TAG = 4;

__device__ inline int mirror(int k, int j) {
  if (k < 0) return -1 - k;
  if (k >= (1 << j)) return (2 << j) - 1 - k;
  return k;
}

// 1D prediction weight (Eq. inter_1d): child parity a, coarse offset o
__device__ inline double wpred(int a, int o) {
  if (o == 0) return 1.0;
  return ((o == -1) == (a == 0)) ? 0.125 : -0.125;
}

struct Level {
  int64_t doff[kMaxL + 2];
  int64_t noff[kMaxL + 2];
};

// thresholds eps_j = 2^((d/2)(j - J)) eta of every level, computed on the host
struct Thresholds {
  double eps[kMaxL + 1];
};

// ------------------------------------------------------------ projection
// parent = mean of its 2^d children, summed in child order (Sec. 2.2)
template <int D>
__device__ inline void project_node(double* __restrict__ V, const int32_t* __restrict__ first_child, int64_t n,
                                    int m, int64_t capN) {
  int32_t fc = first_child[n];
  if (fc < 0) return;
  for (int i = 0; i < m; i++) {
    const double* v = V + i * capN + fc;
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < (1 << D); t++) s = __dadd_rn(s, v[t]);
    V[i * capN + n] = s / (double)(1 << D);
  }
}

// The whole projection in one cooperative launch: the leaf values into the
// node array, then levels J-1 .. 0 bottom-up with a grid barrier between
// levels (one launch instead of J + 1).
template <int D>
__global__ void k_project_all(const double* __restrict__ U, const int32_t* __restrict__ leaf_node,
                              double* __restrict__ V, const int32_t* __restrict__ first_child, Level L, int J,
                              int64_t N, int m, int64_t capL, int64_t capN) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = tid; r < N; r += nth) {
    const int32_t n = leaf_node[r];
    for (int i = 0; i < m; i++) V[i * capN + n] = U[i * capL + r];
  }
  for (int j = J - 1; j >= 0; j--) {
    grid.sync();
    for (int64_t n = L.noff[j] + tid; n < L.noff[j + 1]; n += nth) project_node<D>(V, first_child, n, m, capN);
  }
}

// ------------------------------------------------------------ scales
__global__ void k_scale(const double* __restrict__ U, int64_t N, int m, int64_t capL,
                        unsigned long long* bits) {
  for (int i = 0; i < m; i++) {
    double mx = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x)
      mx = fmax(mx, fabs(U[i * capL + r]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&bits[i], (unsigned long long)__double_as_longlong(mx));
  }
}

// prediction of node value from the 3^d stencil of its parent, literal tensor
// sum in a fixed order with round-to-nearest products and sums (no fused
// multiply-add), values looked up through the level-(j-1) map
template <int D>
__device__ inline double predict(const double* __restrict__ V, const int32_t* __restrict__ dmap_pl,
                                 const int* k, int jm1, int64_t capN, int i) {
  int par[3] = {k[0] >> 1, k[1] >> 1, D == 3 ? k[2] >> 1 : 0};
  double s = 0.0;
  constexpr int NST = D == 2 ? 9 : 27;
#pragma unroll 1
  for (int o = 0; o < NST; o++) {
    int oo = o;
    double w = 1.0;
    int q[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; a++) {
      int off = oo % 3 - 1;
      oo /= 3;
      q[a] = mirror(par[a] + off, jm1);
      w = __dmul_rn(w, wpred(k[a] & 1, off));
    }
    int32_t idx = dmap_pl[morton<D>(q)];
    if (idx < 0) return __longlong_as_double(0x7ff8000000000000ll);  // not graded: NaN
    s = __dadd_rn(s, __dmul_rn(w, V[i * capN + idx]));
  }
  return s;
}

// round-to-nearest sums and products without contraction, in the detail
// arithmetic's precision
__device__ inline double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ inline float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ inline double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ inline float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// DT: arithmetic of the prediction and the difference (double, or float in
// the mixed form with FP32 details: node values rounded to float, weights
// exact in either); the normalised detail is compared with eps_j in double
template <int D, typename DT = double>
__global__ void k_details(const double* __restrict__ V, const uint32_t* __restrict__ code,
                          const uint8_t* __restrict__ lvl, const int32_t* __restrict__ dmap,
                          Level L, int64_t nnodes, int m, int64_t capN,
                          const unsigned long long* __restrict__ scale_bits, Thresholds T, uint8_t* __restrict__ tag,
                          double* __restrict__ delta_out, DevCounters* dc) {
  // the 3^d prediction weights of each child parity, built in the order
  // predict() multiplies them (they are products of 1 and +-1/8, exact)
  constexpr int NST = D == 2 ? 9 : 27;
  __shared__ DT sw[1 << D][NST];
  for (int q = threadIdx.x; q < (1 << D) * NST; q += blockDim.x) {
    const int par = q / NST;
    int oo = q % NST;
    double w = 1.0;
    for (int a = 0; a < D; a++) {
      const int off = oo % 3 - 1;
      oo /= 3;
      w = __dmul_rn(w, wpred((par >> a) & 1, off));
    }
    sw[par][q % NST] = (DT)w;  // a product of 1 and +-1/8: exact in float too
  }
  // s_i = max(max over leaves |u_i|, 1e-30), from the ordered bits k_scale left
  __shared__ double s_scale[kMaxM];
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_scale[i] = fmax(__longlong_as_double(scale_bits[i]), 1e-30);
  __syncthreads();
  for (int64_t n = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nnodes;
       n += (int64_t)gridDim.x * blockDim.x) {
    int j = lvl[n];
    int k[3];
    unmorton<D>(code[n], k);
    const int32_t* dm = dmap + L.doff[j - 1];
    // the parent-level stencil, looked up once for all species
    const int par[3] = {k[0] >> 1, k[1] >> 1, D == 3 ? k[2] >> 1 : 0};
    const int parity = (k[0] & 1) | ((k[1] & 1) << 1) | (D == 3 ? (k[2] & 1) << 2 : 0);
    int32_t idx[NST];
    bool graded = true;
#pragma unroll
    for (int o = 0; o < NST; o++) {
      int oo = o, q[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < D; a++) {
        q[a] = mirror(par[a] + oo % 3 - 1, j - 1);
        oo /= 3;
      }
      idx[o] = dm[morton<D>(q)];
      graded = graded && idx[o] >= 0;
    }
    double dmax = 0.0;
    bool finite = true;  // fmax drops a NaN operand, so non-finite details are caught here
    if (!graded) {
      dmax = __longlong_as_double(0x7ff8000000000000ll);  // a stencil cell is missing: NaN
    } else {
      for (int i = 0; i < m; i++) {
        const double* Vi = V + i * capN;
        DT p = DT(0);  // same products and sums, in the same order, as predict()
#pragma unroll
        for (int o = 0; o < NST; o++) p = add_rn(p, mul_rn(sw[parity][o], (DT)Vi[idx[o]]));
        const DT dd = fabs(add_rn((DT)Vi[n], -p)) / (DT)s_scale[i];
        finite = finite && isfinite(dd);
        dmax = fmax(dmax, (double)dd);
      }
    }
    if (isnan(dmax) || !finite) atomicCAS(&dc->status, 0, (int)MR_ESTATE);
    tag[n] = dmax >= T.eps[j];
    if (delta_out) delta_out[n] = dmax;
  }
}

// ------------------------------------------------------------ adaptation sweep
// the flags of node n (of a level < J) in the dense level maps
__device__ inline void flags_node(const uint32_t* __restrict__ code, const uint8_t* __restrict__ lvl,
                                  const int32_t* __restrict__ first_child, const uint8_t* __restrict__ tag,
                                  const Level& L, int64_t n, uint8_t* __restrict__ state) {
  int j = lvl[n];
  uint8_t f = 0;
  if (first_child[n] >= 0) f |= F_OLD_INT;
  if (n > 0 && tag[n]) {
    f |= F_TAG;
    if (first_child[n] < 0) f |= F_LEAF_TAG;
  }
  state[L.doff[j] + code[n]] = f;
}

template <int D>
__device__ inline void sweep_cell(const uint8_t* __restrict__ state, uint8_t* __restrict__ forced,
                                  uint8_t* __restrict__ final_, const Level& L, int i, int jmin, int64_t p) {
  const int64_t base = L.doff[i];
  {
    uint8_t st = state[base + p];
    uint8_t fo = forced[base + p];
    bool cand = (st & (F_OLD_INT | F_LEAF_TAG)) || fo;
    bool keep = fo || !(st & F_OLD_INT) || (st & F_TAG) || i < jmin;
    bool r = cand && keep;
    final_[base + p] = r;
    if (r && i >= 1) {
      int k[3];
      unmorton<D>((uint32_t)p, k);
      const int64_t pb = L.doff[i - 1];
      const int lim = 1 << i;
      constexpr int NST = D == 2 ? 9 : 27;
      for (int o = 0; o < NST; o++) {
        int oo = o, q[3] = {0, 0, 0};
        bool in = true;
        for (int a = 0; a < D; a++) {
          q[a] = k[a] + oo % 3 - 1;
          oo /= 3;
          in = in && q[a] >= 0 && q[a] < lim;
          q[a] >>= 1;
        }
        if (in) forced[pb + morton<D>(q)] = 1;
      }
    }
  }
}

// The flags and the whole downward sweep in one cooperative launch: the
// flags of the old tree's nodes of levels < J, then levels J-1 .. 0 with a
// grid barrier between levels (a level's cells force cells one level down).
template <int D>
__global__ void k_sweep_all(const uint32_t* __restrict__ code, const uint8_t* __restrict__ lvl,
                            const int32_t* __restrict__ first_child, const uint8_t* __restrict__ tag, Level L,
                            int64_t nint, int J, int jmin, uint8_t* __restrict__ state,
                            uint8_t* __restrict__ forced, uint8_t* __restrict__ final_) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = tid; n < nint; n += nth) flags_node(code, lvl, first_child, tag, L, n, state);
  for (int i = J - 1; i >= 0; i--) {
    grid.sync();
    const int64_t ncell = (int64_t)1 << (D * i);
    for (int64_t p = tid; p < ncell; p += nth) sweep_cell<D>(state, forced, final_, L, i, jmin, p);
  }
}

// ------------------------------------------------------------ tree reconstruction
__global__ void k_level_offsets(const int32_t* __restrict__ grank, const int32_t* total, Level L,
                                int J, int D, DevCounters* dc) {
  // level_internal[j] = refined cells in levels < j (exclusive scan at doff[j])
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int j = 0; j < J; j++) dc->level_internal[j] = grank[L.doff[j]];
    dc->level_internal[J] = *total;
  }
  (void)D;
}

__global__ void k_fill_int(int32_t* p, int64_t n, int32_t v) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    p[r] = v;
}

template <int D>
__global__ void k_children(const uint8_t* __restrict__ final_, const int32_t* __restrict__ grank,
                           Level L, int J, uint32_t* __restrict__ code, uint8_t* __restrict__ lvl,
                           int32_t* __restrict__ first_child, int32_t* __restrict__ dmap) {
  const int64_t nint = L.doff[J];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nint;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (!final_[p]) continue;
    int i = 0;
    while (L.doff[i + 1] <= p) i++;
    uint32_t c = (uint32_t)(p - L.doff[i]);
    int64_t self;
    if (i == 0) {
      self = 0;
    } else {
      int64_t pp = L.doff[i - 1] + (c >> D);
      self = 1 + ((int64_t)grank[pp] << D) + (c & ((1u << D) - 1));
    }
    int64_t fc = 1 + ((int64_t)grank[p] << D);
    first_child[self] = (int32_t)fc;
    for (int t = 0; t < (1 << D); t++) {
      uint32_t cc = (c << D) | t;
      code[fc + t] = cc;
      lvl[fc + t] = (uint8_t)(i + 1);
      dmap[L.doff[i + 1] + cc] = (int32_t)(fc + t);
    }
  }
}

__global__ void k_root(uint32_t* code, uint8_t* lvl, int32_t* dmap) {
  code[0] = 0;
  lvl[0] = 0;
  dmap[0] = 0;
}

__global__ void k_leaf_flags(const int32_t* __restrict__ first_child, int64_t nn, int32_t* flag) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn;
       n += (int64_t)gridDim.x * blockDim.x)
    flag[n] = first_child[n] < 0;
}

__global__ void k_leaf_lists(const int32_t* __restrict__ first_child, const int32_t* __restrict__ lrank,
                             int64_t nn, int32_t* __restrict__ leaf_node, int32_t* __restrict__ node_leaf) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn;
       n += (int64_t)gridDim.x * blockDim.x) {
    if (first_child[n] < 0) {
      int32_t r = lrank[n];
      leaf_node[r] = (int32_t)n;
      node_leaf[n] = r;
    } else {
      node_leaf[n] = -1;
    }
  }
}

// values of the new tree, level j: old nodes keep their value, new nodes are
// predicted from the new tree's level j-1 (whose stencils exist: graded)
template <int D>
__device__ inline void new_value_node(const uint32_t* __restrict__ code, int64_t n, int j,
                                      const int32_t* __restrict__ dmap_old, const int32_t* __restrict__ dmap_new,
                                      const Level& L, const double* __restrict__ Vold, double* __restrict__ Vnew,
                                      int m, int64_t capN, DevCounters* dc) {
  uint32_t c = code[n];
  int32_t o = dmap_old[L.doff[j] + c];
  if (o >= 0) {
    for (int i = 0; i < m; i++) Vnew[i * capN + n] = Vold[i * capN + o];
  } else {
    int k[3];
    unmorton<D>(c, k);
    const int32_t* dm = dmap_new + L.doff[j - 1];
    for (int i = 0; i < m; i++) {
      double v = predict<D>(Vnew, dm, k, j - 1, capN, i);
      if (isnan(v)) atomicCAS(&dc->status, 0, (int)MR_ESTATE);
      Vnew[i * capN + n] = v;
    }
  }
}

// The new tree's values in one cooperative launch.  Every node that the old
// tree had copies its value at once (no order needed); the nodes the
// adaptation created are listed per level and predicted level by level from
// the new tree's level j - 1 (1 .. J, a grid barrier after every level that
// has any), then the
// leaves are gathered into the state array.  L holds the new tree's node
// offsets; list has room for every node; level_new starts at zero.
template <int D>
__global__ void k_new_values_all(const uint32_t* __restrict__ code, const uint8_t* __restrict__ lvl, int J,
                                 const int32_t* __restrict__ dmap_old, const int32_t* __restrict__ dmap_new, Level L,
                                 const double* __restrict__ Vold, double* __restrict__ Vnew, int m, int64_t capN,
                                 const int32_t* __restrict__ leaf_node, double* __restrict__ U, int64_t N,
                                 int64_t capL, int32_t* __restrict__ list, int32_t* __restrict__ level_new,
                                 DevCounters* dc) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = tid; n < L.noff[J + 1]; n += nth) {
    const int j = lvl[n];
    const int32_t o = dmap_old[L.doff[j] + code[n]];
    if (o >= 0) {
      for (int i = 0; i < m; i++) Vnew[i * capN + n] = Vold[i * capN + o];
    } else {
      list[L.noff[j] + atomicAdd(&level_new[j], 1)] = (int32_t)n;
    }
  }
  grid.sync();
  // the per-level counts are final now and read alike by every thread, so
  // levels without created nodes cost no barrier (usually all but the finest
  // one or two)
  for (int j = 1; j <= J; j++) {
    const int cnt = __ldcg(&level_new[j]);
    if (cnt == 0) continue;
    for (int64_t q = tid; q < cnt; q += nth)
      new_value_node<D>(code, list[L.noff[j] + q], j, dmap_old, dmap_new, L, Vold, Vnew, m, capN, dc);
    grid.sync();
  }
  for (int64_t r = tid; r < N; r += nth) {
    const int32_t n = leaf_node[r];
    for (int i = 0; i < m; i++) U[i * capL + r] = Vnew[i * capN + n];
  }
}

// ------------------------------------------------------------ full tree / explicit leaves
template <int D>
__global__ void k_full_values(const double* __restrict__ u0, const uint32_t* __restrict__ code,
                              int64_t lo, int64_t N, int J, int m, int64_t capL,
                              double* __restrict__ U) {
  const int64_t nJ = (int64_t)1 << (D * J);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    int k[3];
    unmorton<D>(code[lo + r], k);
    int64_t lex = (int64_t)k[0] + ((int64_t)k[1] << J) + (D == 3 ? ((int64_t)k[2] << (2 * J)) : 0);
    for (int i = 0; i < m; i++) U[i * capL + r] = u0[i * nJ + lex];
  }
}

template <int D>
__global__ void k_mark_ancestors(const uint64_t* __restrict__ keys, int64_t n, Level L, int J,
                                 uint8_t* __restrict__ final_, DevCounters* dc) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = keys[r];
    int j = (int)((key >> 48) & 15);
    uint64_t s = key & ((1ull << 48) - 1);
    if (j > J || (key >> 52) != 0 || (s >> (D * j)) != 0) {
      atomicCAS(&dc->status, 0, (int)MR_EINVAL);
      continue;
    }
    for (int i = j - 1; i >= 0; i--) final_[L.doff[i] + (uint32_t)(s >> (D * (j - i)))] = 1;
  }
}

template <int D>
__global__ void k_place_leaves(const uint64_t* __restrict__ keys, const double* __restrict__ vals,
                               int64_t n, Level L, const int32_t* __restrict__ dmap,
                               const int32_t* __restrict__ node_leaf, int m, int64_t capL,
                               double* __restrict__ U, int32_t* __restrict__ seen, DevCounters* dc) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = keys[r];
    int j = (int)((key >> 48) & 15);
    uint32_t c = (uint32_t)(key & ((1ull << 48) - 1));
    int32_t idx = dmap[L.doff[j] + c];
    int32_t li = idx >= 0 ? node_leaf[idx] : -1;
    if (li < 0) {
      atomicCAS(&dc->status, 0, (int)MR_EINVAL);
      continue;
    }
    if (atomicAdd(&seen[li], 1) != 0) atomicCAS(&dc->status, 0, (int)MR_EINVAL);  // duplicate key
    for (int i = 0; i < m; i++) U[i * capL + li] = vals[i * n + r];
  }
}

template <int D>
__global__ void k_check_graded(const uint32_t* __restrict__ code, const uint8_t* __restrict__ lvl,
                               const int32_t* __restrict__ dmap, Level L, int64_t nn,
                               DevCounters* dc) {
  for (int64_t n = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn;
       n += (int64_t)gridDim.x * blockDim.x) {
    int j = lvl[n];
    if (j < 2) continue;
    int k[3];
    unmorton<D>(code[n], k);
    const int lim = 1 << (j - 1);
    constexpr int NST = D == 2 ? 9 : 27;
    for (int o = 0; o < NST; o++) {
      int oo = o, q[3] = {0, 0, 0};
      bool in = true;
      for (int a = 0; a < D; a++) {
        q[a] = (k[a] >> 1) + oo % 3 - 1;
        oo /= 3;
        in = in && q[a] >= 0 && q[a] < lim;
      }
      if (in && dmap[L.doff[j - 1] + morton<D>(q)] < 0) atomicCAS(&dc->status, 0, (int)MR_EINVAL);
    }
  }
}

// ------------------------------------------------------------ leaf operator tables
template <int D>
__global__ void k_classify(const int32_t* __restrict__ leaf_node, const uint32_t* __restrict__ code,
                           const uint8_t* __restrict__ lvl, const int32_t* __restrict__ dmap,
                           const int32_t* __restrict__ node_leaf, Level L, int64_t N, int64_t capL,
                           int32_t* __restrict__ nbr, uint8_t* __restrict__ leaf_lvl,
                           int32_t* __restrict__ irr_flag, unsigned long long* rho_bits) {
  double rmax = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t n = leaf_node[r];
    int j = lvl[n];
    int k[3];
    unmorton<D>(code[n], k);
    leaf_lvl[r] = (uint8_t)j;
    bool irr = false;
    int inner = 0;
    const int lim = 1 << j;
    for (int f = 0; f < 2 * D; f++) {
      int a = f >> 1, sg = (f & 1) ? 1 : -1;
      int q[3] = {k[0], k[1], k[2]};
      q[a] += sg;
      int32_t nb = (int32_t)r;
      if (q[a] >= 0 && q[a] < lim) {
        int32_t idx = dmap[L.doff[j] + morton<D>(q)];
        int32_t li = idx >= 0 ? node_leaf[idx] : -1;
        if (li >= 0) {
          nb = li;
          inner++;
        } else {
          irr = true;
        }
      }
      nbr[f * capL + r] = nb;
    }
    irr_flag[r] = irr;
    if (!irr) rmax = fmax(rmax, 2.0 * inner * ldexp(1.0, 2 * j));
  }
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(rho_bits, (unsigned long long)__double_as_longlong(rmax));
}

__global__ void k_irr_index(const int32_t* __restrict__ irr_flag, const int32_t* __restrict__ irank,
                            int64_t N, int64_t capL, int32_t* __restrict__ nbr,
                            int32_t* __restrict__ irr_leaf) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (!irr_flag[r]) continue;
    int32_t row = irank[r];
    irr_leaf[row] = (int32_t)r;
    nbr[r] = -(row + 1);
  }
}

// Compact table of the regular leaves (every face meets a same-level leaf or
// the boundary), in leaf order: leaf index, the 2d neighbour indices and the
// level in two 16-byte words, so that a sweep thread loads everything it
// needs with two vector loads and no thread of a sweep idles on a leaf at a
// level jump.
__global__ void k_reg_table(const int32_t* __restrict__ irr_flag, const int32_t* __restrict__ irank,
                            const int32_t* __restrict__ nbr, const uint8_t* __restrict__ leaf_lvl, int64_t N,
                            int64_t capL, int D, int4* __restrict__ reg) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (irr_flag[r]) continue;
    const int64_t k = r - irank[r];
    int v[8] = {(int)r, 0, 0, 0, 0, 0, 0, 0};
    for (int f = 0; f < 2 * D; f++) v[1 + f] = nbr[f * capL + r];
    v[1 + 2 * D] = leaf_lvl[r];
    reg[2 * k] = make_int4(v[0], v[1], v[2], v[3]);
    reg[2 * k + 1] = make_int4(v[4], v[5], v[6], v[7]);
  }
}

// Merged rows of the leaves at level jumps.  One warp builds one row.  The
// row's faces name cells (level, position, weight): the same-level neighbour
// and the row's own leaf, or, across a finer face, the touching children and
// the row's own (absent) children.  Cells are merged in a shared-memory table
// keyed by (level, Morton code) as they are named, and resolved level by
// level so that every cell is expanded once with its summed weight:
//   up:   absent cells from the finest level to the coarsest, each replaced by
//         its parent's 3^d prediction stencil (Eq. inter_1d, mirror cells at
//         the boundary);
//   down: internal cells from the coarsest level to the finest, each replaced
//         by its 2^d children with weight / 2^d (projection).
// An absent cell only names cells one level coarser and an internal cell only
// existing cells one level finer, so each cell's weight is complete when its
// level is resolved.  What remains are leaves; the row is sorted by leaf index
// (so the sweeps' sums are reproducible run to run) and written to a fixed
// slot.  Weights are dyadic, so merging is exact in any order.
// Table sizes per warp.  3D rows are built first with a half-size table (more
// resident warps); the few rows that do not fit (more than 512 cells or 320
// leaves) are rebuilt by a second launch with the full-size table.
struct IrrCfg2 {
  static constexpr int kCells = 256, kSort = kIrrSlot2, kWarps = 4;
};
struct IrrCfg3 {
  static constexpr int kCells = 1024, kSort = kIrrSlot3, kWarps = 3;
};
struct IrrCfg3Small {
  static constexpr int kCells = 512, kSort = 320, kWarps = 4;
};

template <class Cfg>
constexpr bool fits_in_keys() {
  return sizeof(int32_t) * Cfg::kSort + sizeof(double) * Cfg::kSort <= sizeof(unsigned long long) * Cfg::kCells;
}
static_assert(fits_in_keys<IrrCfg2>() && fits_in_keys<IrrCfg3>() && fits_in_keys<IrrCfg3Small>(),
              "a row's leaves fit in the key bytes");

constexpr unsigned long long kEmptyCell = ~0ull;
constexpr int32_t kAbsent = -1, kInternal = -2, kUnresolved = -3;

template <int D, class Cfg>
struct IrrShared {
  // the keys are dead once every cell is resolved, and the row's leaves are
  // collected into the same bytes for placement
  union {
    unsigned long long key[Cfg::kCells];  // (level << 48) | Morton code
    struct {
      int32_t skey[Cfg::kSort];
      double sval[Cfg::kSort];
    } row;
  };
  double w[Cfg::kCells];
  int32_t st[Cfg::kCells];  // leaf index, kAbsent or kInternal
  int16_t order[Cfg::kCells];  // table slots in the order the cells were named
  int16_t list[Cfg::kCells];   // slots of the cells one pass expands
  int n, cnt, lo, hi, bad;
};

// per cell of every level (dense, level offsets L.doff): the leaf index, -2
// for an internal node, -1 for a cell that is not in the tree
struct IrrMaps {
  const int32_t* smap;
};

__global__ void k_status_map(const uint32_t* __restrict__ code, const uint8_t* __restrict__ lvl,
                             const int32_t* __restrict__ node_leaf, Level L, int64_t nnodes,
                             int32_t* __restrict__ smap) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nnodes;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int32_t li = node_leaf[n];
    smap[L.doff[lvl[n]] + code[n]] = li >= 0 ? li : -2;
  }
}

// name a cell: shared memory only; its status (leaf, internal, absent) is
// looked up afterwards for all the cells a pass named at once (resolve)
template <int D, class Cfg>
__device__ inline void cell_add(IrrShared<D, Cfg>& S, int j, const int* k, double w) {
  constexpr int kC = Cfg::kCells;
  const uint32_t code = morton<D>(k);
  const unsigned long long key = ((unsigned long long)j << 48) | code;
  uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & (kC - 1);
  for (int probe = 0; probe < kC; probe++) {
    const unsigned long long old = atomicCAS(&S.key[h], kEmptyCell, key);
    if (old == kEmptyCell) {
      S.st[h] = kUnresolved;
      const int pos = atomicAdd(&S.n, 1);
      S.order[pos] = (int16_t)h;
      atomicMin(&S.lo, j);
      atomicMax(&S.hi, j);
      atomicAdd(&S.w[h], w);
      return;
    }
    if (old == key) {
      atomicAdd(&S.w[h], w);
      return;
    }
    h = (h + 1) & (kC - 1);
  }
  atomicExch(&S.bad, 1);
}

// status of the cells named in order[from, to): one lane per cell, the
// direct-map and leaf-index loads of all of them in flight together
template <int D, class Cfg>
__device__ inline void resolve(IrrShared<D, Cfg>& S, const IrrMaps& M, const Level& L, int from, int to, int lane) {
#pragma unroll 4
  for (int e = from + lane; e < to; e += 32) {
    const int h = S.order[e];
    const unsigned long long key = S.key[h];
    const int j = (int)(key >> 48);
    S.st[h] = M.smap[L.doff[j] + (int64_t)(key & 0xffffffffffffull)];  // leaf, kInternal or kAbsent
  }
}

// rowlist: the rows to build (null: all nrows); retry: where rows that do
// not fit this table go (null: a row that does not fit its slot is an error)
template <int D, class Cfg>
__global__ void __launch_bounds__(32 * Cfg::kWarps, 2)
    k_irr_rows(const int32_t* __restrict__ irr_leaf, int64_t nrows, const int32_t* __restrict__ rowlist,
               const int32_t* __restrict__ leaf_node, const uint32_t* __restrict__ code,
               const uint8_t* __restrict__ lvl, const int32_t* __restrict__ smap, Level L, int slot,
               int32_t* __restrict__ cnt, int32_t* __restrict__ col, double* __restrict__ wout,
               float* __restrict__ wout_f, unsigned long long* rho_bits, int32_t* __restrict__ retry,
               DevCounters* dc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kC = Cfg::kCells, kS = Cfg::kSort;
  IrrShared<D, Cfg>& S = reinterpret_cast<IrrShared<D, Cfg>*>(smem_raw)[threadIdx.x >> 5];
  const IrrMaps M{smap};
  const int lane = threadIdx.x & 31;
  for (int q = lane; q < kC; q += 32) {
    S.key[q] = kEmptyCell;
    S.w[q] = 0.0;
  }
  if (lane == 0) S.n = 0;
  __syncwarp();
  for (int64_t item = (int64_t)blockIdx.x * Cfg::kWarps + (threadIdx.x >> 5); item < nrows;
       item += (int64_t)gridDim.x * Cfg::kWarps) {
    const int64_t row = rowlist ? rowlist[item] : item;
    if (lane == 0) {
      S.cnt = S.bad = 0;
      S.lo = 1 << 20;
      S.hi = -1;
    }
    __syncwarp();
    const int32_t r = irr_leaf[row];
    const int32_t n = leaf_node[r];
    const int j = lvl[n];
    int k[3] = {0, 0, 0};
    unmorton<D>(code[n], k);
    const int lim = 1 << j;
    const double ih2 = ldexp(1.0, 2 * j);
    const double coef = ldexp(1.0, 2 * j + 1 - (D - 1));
    if (lane < 2 * D) {
      const int a = lane >> 1, sg = (lane & 1) ? 1 : -1;
      int q[3] = {k[0], k[1], k[2]};
      q[a] += sg;
      if (q[a] >= 0 && q[a] < lim) {  // homogeneous Neumann: no flux through the boundary
        if (smap[L.doff[j] + morton<D>(q)] != kInternal) {
          cell_add<D, Cfg>(S, j, q, ih2);  // same-level leaf, or ghost by prediction
          cell_add<D, Cfg>(S, j, k, -ih2);
        } else {
          // finer side: minus the mean of the fluxes into the touching children
          for (int t = 0; t < (1 << D); t++) {
            int c[3] = {0, 0, 0};
            for (int b = 0; b < D; b++) c[b] = 2 * q[b] + ((t >> b) & 1);
            if (c[a] != 2 * q[a] + (sg > 0 ? 0 : 1)) continue;
            int g[3] = {c[0], c[1], c[2]};
            g[a] -= sg;
            cell_add<D, Cfg>(S, j + 1, g, -coef);
            cell_add<D, Cfg>(S, j + 1, c, coef);
          }
        }
      }
    }
    __syncwarp();
    resolve<D, Cfg>(S, M, L, 0, S.n, lane);
    __syncwarp();
    // gather the table slots of the cells at level jj with status st into
    // S.list (ballot compaction, every lane in step); returns their count
    auto gather = [&](int jj, int32_t want, int ne) {
      int nl = 0;
      for (int e0 = 0; e0 < ne; e0 += 32) {
        const int e = e0 + lane;
        int h = 0;
        bool take = false;
        if (e < ne) {
          h = S.order[e];
          take = (int)(S.key[h] >> 48) == jj && S.st[h] == want;
        }
        const unsigned b = __ballot_sync(0xffffffffu, take);
        if (take) S.list[nl + __popc(b & ((1u << lane) - 1))] = (int16_t)h;
        nl += __popc(b);
      }
      __syncwarp();
      return nl;
    };
    // up: absent cells, finest level first; the (cell, stencil offset) pairs
    // of a level are spread over the lanes
    // (the pass's bounds are read by every lane before any lane adds a cell)
    constexpr int NST = D == 2 ? 9 : 27;
    for (int jj = S.hi;; jj--) {
      const bool go = jj >= 1 && jj >= S.lo && !S.bad;
      const int ne = S.n;
      __syncwarp();
      if (!go) break;
      const int nl = gather(jj, kAbsent, ne);
      for (int it = lane; it < nl * NST; it += 32) {
        const int h = S.list[it / NST];
        int c[3] = {0, 0, 0};
        unmorton<D>((uint32_t)(S.key[h] & 0xffffffffffffull), c);
        int oo = it % NST, st[3] = {0, 0, 0};
        double w = S.w[h];
        for (int a = 0; a < D; a++) {
          const int off = oo % 3 - 1;
          oo /= 3;
          st[a] = mirror((c[a] >> 1) + off, jj - 1);
          w *= wpred(c[a] & 1, off);
        }
        cell_add<D, Cfg>(S, jj - 1, st, w);
      }
      __syncwarp();
      resolve<D, Cfg>(S, M, L, ne, S.n, lane);
      __syncwarp();
    }
    // down: internal cells, coarsest level first, (cell, child) pairs over
    // the lanes
    for (int jj = S.lo;; jj++) {
      const bool go = jj <= S.hi && !S.bad;
      const int ne = S.n;
      __syncwarp();
      if (!go) break;
      const int nl = gather(jj, kInternal, ne);
      for (int it = lane; it < (nl << D); it += 32) {
        const int h = S.list[it >> D];
        const int t = it & ((1 << D) - 1);
        int c[3] = {0, 0, 0};
        unmorton<D>((uint32_t)(S.key[h] & 0xffffffffffffull), c);
        const double w = S.w[h] * (1.0 / (1 << D));
        int ch[3] = {0, 0, 0};
        for (int a = 0; a < D; a++) ch[a] = 2 * c[a] + ((t >> a) & 1);
        cell_add<D, Cfg>(S, jj + 1, ch, w);
      }
      __syncwarp();
      resolve<D, Cfg>(S, M, L, ne, S.n, lane);
      __syncwarp();
    }
    // collect the leaves with non-zero weight, then sort them by leaf index
    const int ne = S.n;
    for (int e = lane; e < ne; e += 32) {
      const int h = S.order[e];
      if (S.st[h] >= 0 && S.w[h] != 0.0) {
        const int pos = atomicAdd(&S.cnt, 1);
        if (pos < kS) {
          S.row.skey[pos] = S.st[h];
          S.row.sval[pos] = S.w[h];
        } else {
          atomicExch(&S.bad, 1);
        }
      }
    }
    __syncwarp();
    // each entry's place in the row is its rank by leaf index (the leaves are
    // distinct), so the row comes out sorted without a sort network; the
    // absolute row sum is exact in any order (dyadic weights)
    const int cntr = min(S.cnt, kS);
    double sa = 0.0;
    const bool ok = !S.bad && cntr <= slot;
    for (int q = lane; q < cntr; q += 32) {
      const int32_t kq = S.row.skey[q];
      int rank = 0;
#pragma unroll 8
      for (int p = 0; p < cntr; p++) rank += S.row.skey[p] < kq;
      sa += fabs(S.row.sval[q]);
      if (ok) {
        col[row * (int64_t)slot + rank] = kq;
        wout[row * (int64_t)slot + rank] = S.row.sval[q];
        wout_f[row * (int64_t)slot + rank] = (float)S.row.sval[q];
      }
    }
    for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(0xffffffffu, sa, o);
    // empty the table for the next row: every key (the placement overwrote
    // them), the weights of the slots this row used
    __syncwarp();
    for (int q = lane; q < kC; q += 32) S.key[q] = kEmptyCell;
    for (int e = lane; e < ne; e += 32) S.w[S.order[e]] = 0.0;
    if (lane == 0) {
      cnt[row] = ok ? cntr : 0;
      if (ok) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&dc->irr_nnz), (unsigned long long)cntr);
        atomicMax(rho_bits, (unsigned long long)__double_as_longlong(sa));
      } else if (retry) {
        retry[atomicAdd(&dc->nretry, 1)] = (int32_t)row;
      } else {
        atomicExch(&dc->overflow, 1);
      }
      S.n = 0;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ mass
__global__ void k_mass_partial(const double* __restrict__ U, const uint8_t* __restrict__ leaf_lvl,
                               int64_t N, int m, int64_t capL, int D, double* __restrict__ part) {
  __shared__ double sh[kBlock];
  for (int i = 0; i < m; i++) {
    double s = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x)
      s += ldexp(1.0, -D * leaf_lvl[r]) * U[i * capL + r];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[i * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void k_mass_final(const double* __restrict__ part, int nb, int m, double* __restrict__ out) {
  int i = threadIdx.x;
  if (i < m) {
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[i * nb + b];
    out[i] = s;
  }
}

Level make_level(const mr_ctx* c, const TreeBuf& t) {
  Level L;
  for (int j = 0; j <= kMaxL + 1; j++) {
    L.doff[j] = c->doff[j];
    L.noff[j] = t.noff[j];
  }
  return L;
}

}  // namespace

mr_status sync_counts(mr_ctx* c) {
  MR_CUDA(c, cudaMemcpyAsync(&c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream));
  MR_CUDA(c, cudaStreamSynchronize(c->stream));
  return MR_OK;
}

// Build node arrays of buffer `dst` from c->fl_final (refined cells of levels < J).
mr_status tree_from_final(mr_ctx* c, int dst, bool /*keep_values*/) {
  TreeBuf& t = c->tb[dst];
  const int D = c->d, J = c->J;
  Level L = make_level(c, t);
  int32_t* total = &c->dc->level_internal[kMaxL];
  scan_u8(c, c->fl_final, c->grank, c->cap_dense_int, total);
  k_level_offsets<<<1, 32, 0, c->stream>>>(c->grank, total, L, J, D, c->dc);
  c->launches++;
  MR_TRY(sync_counts(c));
  // node offsets: level j+1 starts at 1 + 2^d (refined cells of levels < j)
  t.noff[0] = 0;
  t.noff[1] = 1;
  for (int j = 1; j <= J; j++) t.noff[j + 1] = 1 + ((int64_t)c->hc.level_internal[j] << D);
  for (int j = J + 2; j <= kMaxL + 1; j++) t.noff[j] = t.noff[J + 1];
  t.nnodes = t.noff[J + 1];
  if (t.nnodes > c->cap_nodes) return MR_ENOMEM;
  L = make_level(c, t);
  MR_CUDA(c, cudaMemsetAsync(t.dmap, 0xff, sizeof(int32_t) * c->cap_dense, c->stream));
  k_fill_int<<<grid_for(t.nnodes), kBlock, 0, c->stream>>>(t.first_child, t.nnodes, -1);
  k_root<<<1, 1, 0, c->stream>>>(t.code, t.lvl, t.dmap);
  if (D == 2)
    k_children<2><<<grid_for(c->cap_dense_int), kBlock, 0, c->stream>>>(
        c->fl_final, c->grank, L, J, t.code, t.lvl, t.first_child, t.dmap);
  else
    k_children<3><<<grid_for(c->cap_dense_int), kBlock, 0, c->stream>>>(
        c->fl_final, c->grank, L, J, t.code, t.lvl, t.first_child, t.dmap);
  k_leaf_flags<<<grid_for(t.nnodes), kBlock, 0, c->stream>>>(t.first_child, t.nnodes, c->itmp);
  scan_i32(c, c->itmp, t.node_leaf, t.nnodes, &c->dc->nleaves);
  c->launches += 4;
  MR_TRY(sync_counts(c));
  t.nleaves = c->hc.nleaves;
  if (t.nleaves > c->cap_leaves) return MR_ENOMEM;  // checked before any leaf is written
  k_leaf_lists<<<grid_for(t.nnodes), kBlock, 0, c->stream>>>(t.first_child, t.node_leaf, t.nnodes,
                                                             t.leaf_node, t.node_leaf);
  c->launches++;
  // leaves per level: nodes of level j minus refined cells of level j
  t.loff[0] = 0;
  for (int j = 0; j <= J; j++) {
    int64_t nodes_j = t.noff[j + 1] - t.noff[j];
    int64_t ref_j = j < J ? (int64_t)c->hc.level_internal[j + 1] - c->hc.level_internal[j] : 0;
    t.loff[j + 1] = t.loff[j] + nodes_j - ref_j;
  }
  for (int j = J + 2; j <= kMaxL + 1; j++) t.loff[j] = t.loff[J + 1];
  c->tables_valid = false;
  return MR_OK;
}

mr_status build_full(mr_ctx* c, const double* u0_dev) {
  MR_CUDA(c, cudaMemsetAsync(c->fl_final, 1, c->cap_dense_int, c->stream));
  mr_status s = tree_from_final(c, c->cur, false);
  if (s) return s;
  TreeBuf& t = c->tb[c->cur];
  if (c->d == 2)
    k_full_values<2><<<grid_for(t.nleaves), kBlock, 0, c->stream>>>(
        u0_dev, t.code, t.noff[c->J], t.nleaves, c->J, c->m, c->cap_leaves, t.U);
  else
    k_full_values<3><<<grid_for(t.nleaves), kBlock, 0, c->stream>>>(
        u0_dev, t.code, t.noff[c->J], t.nleaves, c->J, c->m, c->cap_leaves, t.U);
  c->launches++;
  MR_CUDA(c, cudaGetLastError());
  return MR_OK;
}

mr_status set_leaves(mr_ctx* c, int64_t n, const uint64_t* keys_dev, const double* vals_dev) {
  const int D = c->d;
  MR_CUDA(c, cudaMemsetAsync(c->fl_final, 0, c->cap_dense_int, c->stream));
  MR_CUDA(c, cudaMemsetAsync(&c->dc->status, 0, sizeof(int), c->stream));
  TreeBuf& t = c->tb[c->cur];
  Level L = make_level(c, t);
  if (D == 2)
    k_mark_ancestors<2><<<grid_for(n), kBlock, 0, c->stream>>>(keys_dev, n, L, c->J, c->fl_final, c->dc);
  else
    k_mark_ancestors<3><<<grid_for(n), kBlock, 0, c->stream>>>(keys_dev, n, L, c->J, c->fl_final, c->dc);
  c->launches++;
  MR_TRY(sync_counts(c));
  if (c->hc.status) return MR_EINVAL;
  mr_status s = tree_from_final(c, c->cur, false);
  if (s) return s;
  if (t.nleaves != n) return MR_EINVAL;
  for (int j = 0; j < c->jmin; j++)
    if (c->hc.level_internal[j + 1] - c->hc.level_internal[j] != c->n_level[j]) return MR_EINVAL;
  L = make_level(c, t);
  MR_CUDA(c, cudaMemsetAsync(c->itmp, 0, sizeof(int32_t) * n, c->stream));
  if (D == 2) {
    k_place_leaves<2><<<grid_for(n), kBlock, 0, c->stream>>>(keys_dev, vals_dev, n, L, t.dmap,
                                                             t.node_leaf, c->m, c->cap_leaves, t.U, c->itmp, c->dc);
    k_check_graded<2><<<grid_for(t.nnodes), kBlock, 0, c->stream>>>(t.code, t.lvl, t.dmap, L, t.nnodes, c->dc);
  } else {
    k_place_leaves<3><<<grid_for(n), kBlock, 0, c->stream>>>(keys_dev, vals_dev, n, L, t.dmap,
                                                             t.node_leaf, c->m, c->cap_leaves, t.U, c->itmp, c->dc);
    k_check_graded<3><<<grid_for(t.nnodes), kBlock, 0, c->stream>>>(t.code, t.lvl, t.dmap, L, t.nnodes, c->dc);
  }
  c->launches += 2;
  MR_TRY(sync_counts(c));
  return c->hc.status ? MR_EINVAL : MR_OK;
}

// One cooperative launch of kern (every block co-resident, for its grid
// barriers): at most 2 kBlock-thread blocks per SM, no more than the work
// needs.  A grid barrier costs more with more blocks, and these loops pass
// one per level over levels that are mostly small.
template <typename... Args>
static mr_status coop_launch(mr_ctx* c, void (*kern)(Args...), int64_t work, Args... args) {
  int dev = 0, nsm = 152, per_sm = 0;
  MR_CUDA(c, cudaGetDevice(&dev));
  MR_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  MR_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0));
  if (per_sm < 1) return MR_ECUDA;
  const int64_t want = std::max<int64_t>(1, (work + kBlock - 1) / kBlock);
  const int grid = (int)std::min<int64_t>(want, (int64_t)nsm * std::min(per_sm, 2));
  void* a[] = {(void*)&args...};
  MR_CUDA(c, cudaLaunchCooperativeKernel((const void*)kern, grid, kBlock, a, 0, c->stream));
  c->launches++;
  return MR_OK;
}

// project the current leaves to all nodes: V = leaf values, then bottom-up means
static mr_status project(mr_ctx* c, const TreeBuf& t) {
  const Level L = make_level(c, t);
  const auto kern = c->d == 2 ? k_project_all<2> : k_project_all<3>;
  return coop_launch(c, kern, std::max<int64_t>(t.nleaves, t.noff[c->J] - t.noff[c->J - 1]),
                     (const double*)t.U, (const int32_t*)t.leaf_node, c->V, (const int32_t*)t.first_child, L, c->J,
                     (int64_t)t.nleaves, c->m, c->cap_leaves, c->cap_nodes);
}

mr_status adapt(mr_ctx* c, double eta) {
  const int D = c->d, J = c->J, m = c->m;
  // eta = 0 on the uniform finest grid (as many leaves as level-J cells):
  // every node is tagged (delta >= 0 = eps_j) and no leaf can be refined or
  // coarsened, so the adaptation is the identity and the tables stay valid
  if (eta == 0.0 && c->tb[c->cur].nleaves == c->n_level[J]) return MR_OK;
  const int src = c->cur, dst = 1 - c->cur;
  TreeBuf& t = c->tb[src];
  Level L = make_level(c, t);
  MR_CUDA(c, cudaMemsetAsync(&c->dc->status, 0, sizeof(int), c->stream));
  MR_TRY(project(c, t));
  // scales s_i = max over leaves |u_i|
  MR_CUDA(c, cudaMemsetAsync(c->dc->scale_bits, 0, sizeof(c->dc->scale_bits), c->stream));
  k_scale<<<grid_for(t.nleaves), kBlock, 0, c->stream>>>(t.U, t.nleaves, m, c->cap_leaves,
                                                          c->dc->scale_bits);
  c->launches++;
  // the details kernel reads the scales from the device; the thresholds
  // depend on eta, d and J only (no host round trip)
  Thresholds th;
  for (int j = 0; j <= kMaxL; j++) th.eps[j] = j <= J ? eta * pow(2.0, 0.5 * D * (j - J)) : 0.0;
  const bool f32d = c->prob.precision == MR_MIXED_F32_DETAILS;
  const auto details = D == 2 ? (f32d ? k_details<2, float> : k_details<2, double>)
                              : (f32d ? k_details<3, float> : k_details<3, double>);
  details<<<grid_for(t.nnodes), kBlock, 0, c->stream>>>(c->V, t.code, t.lvl, t.dmap, L, t.nnodes, m, c->cap_nodes,
                                                        c->dc->scale_bits, th, c->tag, nullptr, c->dc);
  c->launches++;
  // flags and the level sweep
  MR_CUDA(c, cudaMemsetAsync(c->fl_state, 0, c->cap_dense_int, c->stream));
  MR_CUDA(c, cudaMemsetAsync(c->fl_forced, 0, c->cap_dense_int, c->stream));
  {
    const auto kern = D == 2 ? k_sweep_all<2> : k_sweep_all<3>;
    MR_TRY(coop_launch(c, kern, std::max<int64_t>(t.noff[J], c->n_level[J - 1]), (const uint32_t*)t.code,
                       (const uint8_t*)t.lvl, (const int32_t*)t.first_child, (const uint8_t*)c->tag, L,
                       (int64_t)t.noff[J], J, c->jmin, c->fl_state, c->fl_forced, c->fl_final));
  }
  mr_status s = tree_from_final(c, dst, true);
  if (s) return s;
  TreeBuf& nt = c->tb[dst];
  Level Ln = make_level(c, nt);
  {
    MR_CUDA(c, cudaMemsetAsync(c->level_new, 0, sizeof(int32_t) * (kMaxL + 2), c->stream));
    const auto kern = D == 2 ? k_new_values_all<2> : k_new_values_all<3>;
    MR_TRY(coop_launch(c, kern, std::max<int64_t>(nt.nleaves, nt.noff[J + 1]), (const uint32_t*)nt.code,
                       (const uint8_t*)nt.lvl, J, (const int32_t*)t.dmap, (const int32_t*)nt.dmap, Ln,
                       (const double*)c->V, c->Vnew, m, c->cap_nodes, (const int32_t*)nt.leaf_node, nt.U,
                       (int64_t)nt.nleaves, c->cap_leaves, c->itmp, c->level_new, c->dc));
  }
  MR_CUDA(c, cudaGetLastError());
  MR_TRY(sync_counts(c));
  if (c->hc.status) {
    c->last_error = "adaptation: a detail is not finite (NaN or infinity in the state) or a prediction stencil is missing";
    return (mr_status)c->hc.status;
  }
  c->cur = dst;
  c->tables_valid = false;
  return MR_OK;
}

mr_status build_tables(mr_ctx* c) {
  if (c->tables_valid) return MR_OK;
  TreeBuf& t = c->tb[c->cur];
  const int D = c->d;
  const int64_t N = t.nleaves;
  Level L = make_level(c, t);
  MR_CUDA(c, cudaMemsetAsync(c->rho_bits, 0, sizeof(unsigned long long), c->stream));
  MR_CUDA(c, cudaMemsetAsync(&c->dc->overflow, 0, sizeof(int), c->stream));
  MR_CUDA(c, cudaMemsetAsync(&c->dc->irr_nnz, 0, sizeof(long long), c->stream));
  int32_t* irr_flag = c->itmp;
  if (D == 2)
    k_classify<2><<<grid_for(N), kBlock, 0, c->stream>>>(t.leaf_node, t.code, t.lvl, t.dmap, t.node_leaf, L, N,
                                                         c->cap_leaves, c->nbr, c->leaf_lvl, irr_flag, c->rho_bits);
  else
    k_classify<3><<<grid_for(N), kBlock, 0, c->stream>>>(t.leaf_node, t.code, t.lvl, t.dmap, t.node_leaf, L, N,
                                                         c->cap_leaves, c->nbr, c->leaf_lvl, irr_flag, c->rho_bits);
  int32_t* irank = c->itmp + c->cap_leaves;
  scan_i32(c, irr_flag, irank, N, &c->dc->irr_rows);
  k_reg_table<<<grid_for(N), kBlock, 0, c->stream>>>(irr_flag, irank, c->nbr, c->leaf_lvl, N, c->cap_leaves, D,
                                                     c->reg_tab);
  k_irr_index<<<grid_for(N), kBlock, 0, c->stream>>>(irr_flag, irank, N, c->cap_leaves, c->nbr, c->irr_leaf);
  c->launches += 3;
  MR_TRY(sync_counts(c));
  const int64_t nrows = c->hc.irr_rows;
  const int slot = D == 2 ? kIrrSlot2 : kIrrSlot3;
  if (nrows > 0) {
    const int64_t need = nrows * (int64_t)slot;
    if (need > c->irr_cap) {
      cudaFree(c->irr_col);
      cudaFree(c->irr_w);
      cudaFree(c->irr_wf);
      c->irr_col = nullptr;
      c->irr_w = nullptr;
      c->irr_wf = nullptr;
      c->irr_cap = need + need / 2 + 1024;
      MR_CUDA(c, cudaMalloc(&c->irr_col, sizeof(int32_t) * c->irr_cap));
      MR_CUDA(c, cudaMalloc(&c->irr_w, sizeof(double) * c->irr_cap));
      MR_CUDA(c, cudaMalloc(&c->irr_wf, sizeof(float) * c->irr_cap));
    }
    int nsm = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // status of every cell of every level, for one-load lookups while the
    // rows are built
    MR_CUDA(c, cudaMemsetAsync(c->smap, 0xff, sizeof(int32_t) * c->cap_dense, c->stream));
    k_status_map<<<grid_for(t.nnodes), kBlock, 0, c->stream>>>(t.code, t.lvl, t.node_leaf, L, t.nnodes, c->smap);
    c->launches++;
    auto launch = [&](auto cfg, auto dim, const int32_t* rowlist, int64_t count, int32_t* retry) -> mr_status {
      using Cfg = decltype(cfg);
      constexpr int DD = decltype(dim)::value;
      const size_t sm = sizeof(IrrShared<DD, Cfg>) * Cfg::kWarps;
      MR_CUDA(c, cudaFuncSetAttribute(k_irr_rows<DD, Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      const int grid = (int)std::min<int64_t>((count + Cfg::kWarps - 1) / Cfg::kWarps, (int64_t)nsm * 16);
      k_irr_rows<DD, Cfg><<<grid, 32 * Cfg::kWarps, sm, c->stream>>>(
          c->irr_leaf, count, rowlist, t.leaf_node, t.code, t.lvl, c->smap, L, slot, c->irr_cnt, c->irr_col,
          c->irr_w, c->irr_wf, c->rho_bits, retry, c->dc);
      c->launches++;
      MR_CUDA(c, cudaGetLastError());
      return MR_OK;
    };
    if (D == 2) {
      MR_TRY(launch(IrrCfg2{}, std::integral_constant<int, 2>{}, nullptr, nrows, nullptr));
    } else {
      // half-size tables first, the rows that do not fit again with full-size ones
      int32_t* retry = c->itmp;
      MR_CUDA(c, cudaMemsetAsync(&c->dc->nretry, 0, sizeof(int), c->stream));
      MR_TRY(launch(IrrCfg3Small{}, std::integral_constant<int, 3>{}, nullptr, nrows, retry));
      MR_TRY(sync_counts(c));
      if (c->hc.nretry > 0)
        MR_TRY(launch(IrrCfg3{}, std::integral_constant<int, 3>{}, retry, c->hc.nretry, nullptr));
    }
  }
  c->irr_slot = slot;
  MR_TRY(sync_counts(c));
  if (c->hc.overflow) {
    c->last_error = "an operator row at a level jump exceeds its slot";
    return MR_ESTATE;
  }
  unsigned long long rb = 0;
  MR_CUDA(c, cudaMemcpyAsync(&rb, c->rho_bits, sizeof rb, cudaMemcpyDeviceToHost, c->stream));
  MR_CUDA(c, cudaStreamSynchronize(c->stream));
  memcpy(&c->rho, &rb, sizeof rb);
  c->stats.irregular_rows = nrows;
  c->stats.irregular_nnz = c->hc.irr_nnz;
  c->stats.rock_rho = c->rho;
  c->tables_valid = true;
  return MR_OK;
}

mr_status mass(mr_ctx* c, double* out_host) {
  mr_status s = build_tables(c);  // leaf levels
  if (s) return s;
  TreeBuf& t = c->tb[c->cur];
  const int nb = 152;
  k_mass_partial<<<nb, kBlock, 0, c->stream>>>(t.U, c->leaf_lvl, t.nleaves, c->m, c->cap_leaves, c->d, c->red);
  k_mass_final<<<1, 32, 0, c->stream>>>(c->red, nb, c->m, c->red_out);
  c->launches += 2;
  MR_CUDA(c, cudaMemcpyAsync(out_host, c->red_out, sizeof(double) * c->m, cudaMemcpyDeviceToHost, c->stream));
  MR_CUDA(c, cudaStreamSynchronize(c->stream));
  return MR_OK;
}

}  // namespace mrg
