// Internal declarations of the GB300 multiresolution Strang library.
//
// Data layout in HBM (one context = one problem on one GPU):
//   * nodes of the graded tree, level-major and Morton-sorted inside a level:
//     code[n] (Morton abscissa at the node's level), lvl[n], first_child[n]
//     (children of an internal node are 2^d consecutive nodes), node_leaf[n];
//   * dense direct maps dmap[doff[j] + code] -> node index or -1, one per
//     level.  With 280 GB of HBM a collision-free map of every cell of every
//     level is affordable for d*J <= 30, so a lookup is one load;
//   * leaves (the adapted grid, Sec. 2.2) in the same level-major Morton
//     order: leaf_node[r], leaf state U[i*cap + r] (one contiguous array per
//     species, Sec. 3.2);
//   * node values V[i*cap_nodes + n] for projection and details;
//   * per-level dense byte flags for the adaptation sweep.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mr.h"

namespace mrg {

constexpr int kMaxL = MR_MAX_LEVEL;
constexpr int kMaxM = MR_MAX_SPECIES;
constexpr int kMaxR = MR_MAX_REACTIONS;

// reactions of a network model as the kernels take them: species of every
// reaction and, per species, the reactions that consume (neg) or produce
// (pos) it as bit masks
struct NetModel {
  int m, nr;
  int8_t sp[kMaxR][4];
  double kf[kMaxR], kb[kMaxR];
  uint32_t neg[kMaxM], pos[kMaxM];
};
constexpr int kBlock = 256;
// merged operator rows at level jumps: entries per row (slot) by dimension
constexpr int kIrrSlot2 = 128, kIrrSlot3 = 640;

// ---------------------------------------------------------------- Morton codes
// x is the most significant digit of each group (Sec. 3.1.1).
__host__ __device__ inline uint32_t spread2(uint32_t v) {
  v &= 0x0000ffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
__host__ __device__ inline uint32_t compact2(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0f0f0f0fu;
  v = (v | (v >> 4)) & 0x00ff00ffu;
  v = (v | (v >> 8)) & 0x0000ffffu;
  return v;
}
__host__ __device__ inline uint32_t spread3(uint32_t v) {
  v &= 0x000003ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ inline uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0x030000ffu;
  v = (v | (v >> 16)) & 0x000003ffu;
  return v;
}
template <int D>
__host__ __device__ inline uint32_t morton(const int* k) {
  if (D == 2) return (spread2(k[0]) << 1) | spread2(k[1]);
  return (spread3(k[0]) << 2) | (spread3(k[1]) << 1) | spread3(k[2]);
}
template <int D>
__host__ __device__ inline void unmorton(uint32_t c, int* k) {
  if (D == 2) {
    k[0] = compact2(c >> 1);
    k[1] = compact2(c);
    k[2] = 0;
  } else {
    k[0] = compact3(c >> 2);
    k[1] = compact3(c >> 1);
    k[2] = compact3(c);
  }
}

// ---------------------------------------------------------------- device counters
struct DevCounters {
  unsigned long long radau[8];  // fev, jac, steps, accept, reject, newton, dec, unused
  unsigned long long scale_bits[kMaxM];  // max |u_i| as ordered bits
  int status;                   // first error (mr_status), 0 if none
  int level_internal[kMaxL + 1];
  int irr_rows;
  long long irr_nnz;
  int nleaves;
  unsigned long long work_next; // Radau5 work queue head (64-bit: every resident thread takes one
                                // ticket past the end, which must not wrap near 2^31 cells)
  int overflow;                 // irregular row exceeded its local capacity
  int nretry;                   // rows left to the full-size row builder
};

// ---------------------------------------------------------------- context
struct mr_ctx_impl;

struct TreeBuf {
  uint32_t* code = nullptr;
  uint8_t* lvl = nullptr;
  int32_t* first_child = nullptr;
  int32_t* node_leaf = nullptr;
  int32_t* dmap = nullptr;
  int32_t* leaf_node = nullptr;
  double* U = nullptr;
  // host mirrors
  int64_t nnodes = 0, nleaves = 0;
  int64_t noff[kMaxL + 2] = {0};
  int64_t loff[kMaxL + 2] = {0};
};

}  // namespace mrg

struct mr_ctx {
  mr_problem prob;
  mrg::NetModel net;                 // MR_MODEL_NETWORK reactions
  bool net_set = false;
  int d, J, jmin, m;
  cudaStream_t stream;
  int64_t n_level[mrg::kMaxL + 1];   // 2^(d j)
  int64_t doff[mrg::kMaxL + 2];      // dense offsets, all levels
  int64_t cap_dense, cap_dense_int;  // all levels, levels < J
  int64_t cap_nodes, cap_leaves;
  mrg::TreeBuf tb[2];
  int cur;
  double* V = nullptr;               // node values [m][cap_nodes]
  double* Vnew = nullptr;
  uint8_t* fl_state = nullptr;       // dense flags, levels < J
  uint8_t* fl_forced = nullptr;
  uint8_t* fl_final = nullptr;
  int32_t* grank = nullptr;          // dense exclusive ranks of refined cells
  int32_t* smap = nullptr;           // [cap_dense] per cell of every level: leaf index, -2 internal, -1 absent
  uint8_t* tag = nullptr;            // per node tag of the last detail pass
  int32_t* scan_tmp = nullptr;       // block partials for scans
  int32_t* itmp = nullptr;           // int scratch [cap_nodes]
  int32_t* level_new = nullptr;      // [kMaxL + 2] per level: nodes an adaptation created
  // leaf operator tables
  int32_t* nbr = nullptr;            // [2d][cap_leaves]
  uint8_t* leaf_lvl = nullptr;
  int32_t* irr_leaf = nullptr;       // [cap_leaves]
  int4* reg_tab = nullptr;           // [2 cap_leaves]: per regular leaf (r, 2d neighbours, level)
  int32_t* irr_cnt = nullptr;        // [cap_leaves + 1]
  int64_t* irr_ptr = nullptr;        // [cap_leaves + 1]
  int32_t* irr_col = nullptr;
  double* irr_w = nullptr;
  float* irr_wf = nullptr;           // the merged-row weights in FP32 (exact, dyadic)
  double* e2buf = nullptr;           // [m][cap_leaves] per-leaf error terms of the joint diffusion (lazy)
  int64_t irr_cap = 0;
  int irr_slot = 0;                  // row stride of irr_col / irr_w
  double* rock_tab = nullptr;        // ROCK4-type coefficients of every stage count
  void* rock_ctl = nullptr;          // device control block of the persistent ROCK4 driver
  double rho = 0.0;                  // Gershgorin bound of L
  unsigned long long* rho_bits = nullptr;
  bool tables_valid = false;
  // ROCK4 / reductions
  double* work[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* red = nullptr;             // reduction partials
  double* red_out = nullptr;
  int32_t* complexity = nullptr;
  mrg::DevCounters* dc = nullptr;
  mrg::DevCounters hc;               // host copy
  cudaEvent_t ev[8];
  cudaEvent_t tev[2 * 256];           // per-launch timing pairs of the ROCK4 sweeps
  mr_stats stats;
  int radau_schedule = MR_RADAU_THREAD;  // Radau5 schedule of BZ and NAGUMO contexts
  void* radau_pool = nullptr;          // slot data of the pooled Radau5 kernel (lazy)
  size_t radau_pool_bytes = 0;
  int64_t launches = 0;
  std::string last_error;
  // radau constants (host-computed, passed by value to kernels)
  double rc[64];
  // grow-only device staging for host-pointer arguments
  void* stage[2] = {nullptr, nullptr};
  size_t stage_bytes[2] = {0, 0};
};

namespace mrg {

// launch accounting
inline int grid_for(int64_t n, int block = kBlock) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

mr_status cuda_fail(mr_ctx* c, cudaError_t e, const char* where);
mr_status fp64_probe(double* tflops, double* mhz);
#define MR_CUDA(ctx, call)                                       \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return mrg::cuda_fail(ctx, _e, #call); \
  } while (0)

#define MR_TRY(expr)           \
  do {                         \
    mr_status _s = (expr);     \
    if (_s != MR_OK) return _s; \
  } while (0)

// scan.cu
void scan_u8(mr_ctx* c, const uint8_t* in, int32_t* out, int64_t n, int32_t* total_dev);
void scan_i32(mr_ctx* c, const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev);
void scan_i32_to_i64(mr_ctx* c, const int32_t* in, int64_t* out, int64_t n, long long* total_dev);

// mr.cu
mr_status tree_from_final(mr_ctx* c, int dst, bool keep_values);
mr_status adapt(mr_ctx* c, double eta);
mr_status build_full(mr_ctx* c, const double* u0_dev);
mr_status set_leaves(mr_ctx* c, int64_t n, const uint64_t* keys_dev, const double* vals_dev);
mr_status build_tables(mr_ctx* c);
mr_status apply_operator(mr_ctx* c, const double* in, double* out);
mr_status mass(mr_ctx* c, double* out_host);
mr_status sync_counts(mr_ctx* c);

// radau5.cu
void radau_constants(double* rc);
mr_status react(mr_ctx* c, double dt, double rtol, double atol);

// Reaction sub-step of several contexts (same model kind and precision, one
// thread per cell models) as one persistent launch over the union of their
// leaves, on `stream`.  The caller owns the scratch; counters[7] receives the
// summed Radau5 counters, *kernel_ms the launch's device time.
struct BatchReactScratch {
  DevCounters* dc = nullptr;
  void* inst = nullptr;     // per-instance model, state and complexity arrays (device)
  int64_t* offs = nullptr;  // prefix offsets of the instances' leaf counts (device)
  int cap = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  void* pool = nullptr;     // slot data of the pooled Radau5 kernel (lazy)
  size_t pool_bytes = 0;
};
// launch shape of the joint Radau5 launch (the batch's autotuner picks it):
// threads per block (64 or 128) and the queue order (rev: the finest levels
// first, else leaf order); neither changes a cell's arithmetic
struct RadauShape {
  int block = 128;
  int rev = 1;
  int pool = 0;  // 1: the pooled kernel (4 warps per block; block ignored)
};
mr_status react_batch(mr_ctx* const* cs, int n, double dt, double rtol, double atol, cudaStream_t stream,
                      BatchReactScratch& S, double* kernel_ms, unsigned long long* counters,
                      const RadauShape& shape);
void free_batch_scratch(BatchReactScratch& S);

// opforms.cu
mr_status operator_forms(mr_ctx* c, int reps, double* ms_compact, double* ms_csr, int64_t* csr_nnz,
                         double* max_rel_diff);

// rock4.cu
int rock4_coeffs(int s, double* mu, double* nu, double* kap, double* w, double* errc);
double rock4_ell(int s);
mr_status diffuse(mr_ctx* c, double dt, double tol);

// Diffusion sub-step of several 2D contexts (same species count, one or three,
// and precision) as one cooperative launch; the caller owns the scratch.
struct BatchRockScratch {
  void* inst = nullptr;
  int64_t* off = nullptr;
  void* ctl = nullptr;
  int* ptr = nullptr;
  double* part = nullptr;
  int* flags = nullptr;
  int cap = 0;
  int64_t part_cap = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};
// per_sm: blocks per SM of the cooperative grid (1 or 2; the joint kernel's
// results do not depend on it: its error norms are summed in fixed chunks)
mr_status diffuse_batch(mr_ctx* const* cs, int n, double dt, double tol, cudaStream_t stream, BatchRockScratch& S,
                        double* kernel_ms, int per_sm = 2);
void free_batch_rock(BatchRockScratch& S);

}  // namespace mrg
