// C-ABI entry points (include/mr.h): context lifetime, capacity, host/device
// marshalling, and the Strang composition U_{n+1} = R_{dt/2} D_dt R_{dt/2} U_n
// with the grid adapted first (Sec. 2.1; Sec. 4.2: the adapted grid is
// updated at every time step and the details belong to the adaptation).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "mr_internal.cuh"
#include "radau_common.cuh"

namespace mrg {

mr_status cuda_fail(mr_ctx* c, cudaError_t e, const char* where) {
  if (c) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    c->last_error = buf;
  }
  return e == cudaErrorMemoryAllocation ? MR_ENOMEM : MR_ECUDA;
}

namespace {

// independent FMA chains: 8 per thread, all SMs busy
__global__ void k_fma_probe(double* out, int iters, double a, double b) {
  double x[8];
  for (int q = 0; q < 8; q++) x[q] = threadIdx.x * 1e-9 + q;
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int q = 0; q < 8; q++) x[q] = fma(x[q], a, b);
  double s = 0.0;
  for (int q = 0; q < 8; q++) s += x[q];
  if (s == 1.2345) out[0] = s;  // keeps the chains live
}

__global__ void k_export_keys(const int32_t* __restrict__ leaf_node, const uint32_t* __restrict__ code,
                              const uint8_t* __restrict__ lvl, int64_t N, uint64_t* __restrict__ keys) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    int32_t n = leaf_node[r];
    keys[r] = (uint64_t)code[n] | ((uint64_t)lvl[n] << 48);
  }
}

template <typename T>
mr_status dalloc(mr_ctx* c, T** p, int64_t count) {
  if (count < 1) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
  return MR_OK;
}

mr_status alloc_all(mr_ctx* c) {
  const int m = c->m, d = c->d;
  mr_status s;
#define A(p, n)                       \
  do {                                \
    if ((s = dalloc(c, &(p), (n)))) return s; \
  } while (0)
  for (int b = 0; b < 2; b++) {
    TreeBuf& t = c->tb[b];
    A(t.code, c->cap_nodes);
    A(t.lvl, c->cap_nodes);
    A(t.first_child, c->cap_nodes);
    A(t.node_leaf, c->cap_nodes);
    A(t.dmap, c->cap_dense);
    A(t.leaf_node, c->cap_leaves);
    A(t.U, (int64_t)m * c->cap_leaves);
  }
  A(c->V, (int64_t)m * c->cap_nodes);
  A(c->Vnew, (int64_t)m * c->cap_nodes);
  A(c->fl_state, c->cap_dense_int);
  A(c->fl_forced, c->cap_dense_int);
  A(c->fl_final, c->cap_dense_int);
  A(c->grank, c->cap_dense_int);
  A(c->smap, c->cap_dense);
  A(c->tag, c->cap_nodes);
  int64_t big = std::max(std::max(c->cap_dense_int, c->cap_nodes), c->cap_leaves);
  A(c->scan_tmp, 2 * (big / 2048 + 4));
  A(c->itmp, std::max(c->cap_nodes, 2 * c->cap_leaves + 2));
  A(c->level_new, mrg::kMaxL + 2);
  A(c->nbr, (int64_t)2 * d * c->cap_leaves);
  A(c->leaf_lvl, c->cap_leaves);
  A(c->irr_leaf, c->cap_leaves);
  A(c->reg_tab, 2 * c->cap_leaves);
  A(c->irr_cnt, c->cap_leaves + 1);
  A(c->irr_ptr, c->cap_leaves + 1);
  c->irr_cap = 1 << 16;
  A(c->irr_col, c->irr_cap);
  A(c->irr_w, c->irr_cap);
  A(c->irr_wf, c->irr_cap);
  for (int q = 0; q < 6; q++) A(c->work[q], (int64_t)m * c->cap_leaves);
  A(c->red, (int64_t)152 * 16 * kMaxM);
  A(c->red_out, 128);
  A(c->complexity, c->cap_leaves);
  A(c->dc, 1);
  A(c->rho_bits, 1);
  {
    double* ctl = nullptr;
    A(ctl, 1024);  // holds the ROCK4 control block
    c->rock_ctl = ctl;
  }
#undef A
  MR_CUDA(c, cudaMemset(c->dc, 0, sizeof(DevCounters)));
  MR_CUDA(c, cudaMemset(c->complexity, 0, sizeof(int32_t) * c->cap_leaves));
  return MR_OK;
}

void free_all(mr_ctx* c) {
  for (int b = 0; b < 2; b++) {
    TreeBuf& t = c->tb[b];
    cudaFree(t.code); cudaFree(t.lvl); cudaFree(t.first_child); cudaFree(t.node_leaf);
    cudaFree(t.dmap); cudaFree(t.leaf_node); cudaFree(t.U);
  }
  cudaFree(c->V); cudaFree(c->Vnew); cudaFree(c->fl_state); cudaFree(c->fl_forced);
  cudaFree(c->fl_final); cudaFree(c->grank); cudaFree(c->tag); cudaFree(c->smap); cudaFree(c->scan_tmp);
  cudaFree(c->itmp); cudaFree(c->level_new); cudaFree(c->nbr); cudaFree(c->leaf_lvl); cudaFree(c->irr_leaf); cudaFree(c->reg_tab);
  cudaFree(c->irr_cnt); cudaFree(c->irr_ptr); cudaFree(c->irr_col); cudaFree(c->irr_w); cudaFree(c->irr_wf); cudaFree(c->e2buf);
  cudaFree(c->radau_pool);
  for (int q = 0; q < 6; q++) cudaFree(c->work[q]);
  cudaFree(c->red); cudaFree(c->red_out); cudaFree(c->complexity); cudaFree(c->dc);
  cudaFree(c->rho_bits);
  cudaFree(c->stage[0]);
  cudaFree(c->stage[1]);
  cudaFree(c->rock_tab);
  cudaFree(c->rock_ctl);
}

void refresh_tree_stats(mr_ctx* c) {
  TreeBuf& t = c->tb[c->cur];
  mr_stats& s = c->stats;
  s.leaves = t.nleaves;
  s.nodes = t.nnodes;
  for (int j = 0; j <= kMaxL; j++) s.leaves_per_level[j] = j <= c->J ? t.loff[j + 1] - t.loff[j] : 0;
  s.compression_ratio = (1.0 - (double)t.nleaves / (double)c->n_level[c->J]) * 100.0;
}

mr_status check_ctx(const mr_ctx* c) { return c ? MR_OK : MR_EINVAL; }

// device view of a host or device array: host data is copied into the
// context's grow-only staging buffer `slot` (no allocation once it is large
// enough); *owned is always false
template <typename T>
mr_status to_device(mr_ctx* c, const T* src, int64_t count, int on_device, T** dst, bool* owned, int slot = 0) {
  *owned = false;
  if (on_device) {
    *dst = const_cast<T*>(src);
    return MR_OK;
  }
  size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
  if (c->stage_bytes[slot] < bytes) {
    MR_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->stage[slot]);
    c->stage[slot] = nullptr;
    c->stage_bytes[slot] = 0;
    MR_CUDA(c, cudaMalloc(&c->stage[slot], bytes));
    c->stage_bytes[slot] = bytes;
  }
  *dst = static_cast<T*>(c->stage[slot]);
  MR_CUDA(c, cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
  return MR_OK;
}

}  // namespace

mr_status fp64_probe(double* tflops, double* mhz) {
  int dev = 0, nsm = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return MR_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = nsm * 8, threads = 256, iters = 4096;
  k_fma_probe<<<blocks, threads>>>(out, 64, 0.999999, 1e-7);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; rep++) {
    cudaEventRecord(e0);
    k_fma_probe<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return MR_ECUDA;
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  if (mhz) {
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    *mhz = clk / 1000.0;
  }
  return MR_OK;
}

}  // namespace mrg

using namespace mrg;

extern "C" {

const char* mr_status_str(mr_status s) {
  switch (s) {
    case MR_OK: return "ok";
    case MR_EINVAL: return "invalid argument";
    case MR_ENOMEM: return "out of memory or capacity";
    case MR_ECUDA: return "CUDA runtime error";
    case MR_ESTATE: return "inconsistent state";
    case MR_ERADAU_HMIN: return "Radau5 step size too small";
    case MR_ERADAU_MAXSTEPS: return "Radau5 too many steps";
    case MR_ERADAU_SINGULAR: return "Radau5 singular iteration matrix";
    case MR_EROCK_STEP: return "ROCK4 step size underflow";
    case MR_ENONFINITE: return "non-finite value";
    case MR_ETIMEOUT: return "device wait timed out";
    case MR_EIO: return "checkpoint file error";
  }
  return "unknown status";
}

mr_status mr_last_error(const mr_ctx* c, char* buf, size_t n) {
  if (!c || !buf || n == 0) return MR_EINVAL;
  snprintf(buf, n, "%s", c->last_error.c_str());
  return MR_OK;
}

mr_status mr_create(const mr_problem* p, void* stream, mr_ctx** out) {
  if (!p || !out) return MR_EINVAL;
  *out = nullptr;
  if (p->dim < 2 || p->dim > 3 || p->J < 1 || p->J > kMaxL || p->dim * p->J > 30) return MR_EINVAL;
  if (p->jmin < 1 || p->jmin > p->J) return MR_EINVAL;
  if (p->precision != MR_FP64 && p->precision != MR_MIXED && p->precision != MR_MIXED_F32_DETAILS)
    return MR_EINVAL;
  if (p->model == MR_MODEL_BZ) {
    if (p->m != 3 || p->nparams < 4) return MR_EINVAL;
    if (!(p->params[0] > 0) || !(p->params[1] > 0)) return MR_EINVAL;
  } else if (p->model == MR_MODEL_NAGUMO) {
    if (p->m != 1 || p->nparams < 1) return MR_EINVAL;
  } else if (p->model == MR_MODEL_NETWORK) {
    if (p->m < 2 || p->m > 16) return MR_EINVAL;
  } else if (p->model == MR_MODEL_IONIC) {
    if (p->m != MR_IONIC_SPECIES) return MR_EINVAL;
  } else {
    return MR_EINVAL;
  }
  for (int i = 0; i < p->m; i++)
    if (!(p->D[i] >= 0.0) || !isfinite(p->D[i])) return MR_EINVAL;
  mr_ctx* c = new (std::nothrow) mr_ctx();
  if (!c) return MR_ENOMEM;
  c->prob = *p;
  c->d = p->dim;
  c->J = p->J;
  c->jmin = p->jmin;
  c->m = p->m;
  c->stream = (cudaStream_t)stream;
  c->cur = 0;
  memset(&c->stats, 0, sizeof c->stats);
  memset(&c->hc, 0, sizeof c->hc);
  c->doff[0] = 0;
  for (int j = 0; j <= kMaxL; j++) {
    c->n_level[j] = j <= c->J ? (int64_t)1 << (c->d * j) : 0;
    c->doff[j + 1] = c->doff[j] + c->n_level[j];
  }
  c->cap_dense = c->doff[c->J + 1];
  c->cap_dense_int = c->doff[c->J];
  const int64_t full = c->n_level[c->J];
  c->cap_leaves = p->max_leaves > 0 ? std::min<int64_t>(p->max_leaves, full) : full;
  const int64_t nc = (int64_t)1 << c->d;
  c->cap_nodes = std::min<int64_t>(c->cap_dense, c->cap_leaves + (c->cap_leaves - 1) / (nc - 1) + 1);
  radau_constants(c->rc);
  mr_status s = alloc_all(c);
  if (s == MR_OK) {
    for (int q = 0; q < 8; q++)
      if (cudaEventCreate(&c->ev[q]) != cudaSuccess) s = MR_ECUDA;
    for (int q = 0; q < 2 * 256; q++)
      if (cudaEventCreate(&c->tev[q]) != cudaSuccess) s = MR_ECUDA;
  }
  if (s) {
    free_all(c);
    delete c;
    return s;
  }
  *out = c;
  return MR_OK;
}

void mr_destroy(mr_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int q = 0; q < 8; q++) cudaEventDestroy(c->ev[q]);
  for (int q = 0; q < 2 * 256; q++) cudaEventDestroy(c->tev[q]);
  free_all(c);
  delete c;
}

mr_status mr_build(mr_ctx* c, const double* u0, int on_device, double eta) {
  if (check_ctx(c) || !u0 || !(eta >= 0.0)) return MR_EINVAL;
  if (c->cap_leaves < c->n_level[c->J]) return MR_ENOMEM;
  double* d0;
  bool owned;
  mr_status s = to_device(c, u0, (int64_t)c->m * c->n_level[c->J], on_device, &d0, &owned);
  if (s) return s;
  s = build_full(c, d0);
  if (!s) s = adapt(c, eta);
  if (owned) {
    cudaStreamSynchronize(c->stream);
    cudaFree(d0);
  }
  if (!s) refresh_tree_stats(c);
  return s;
}

mr_status mr_set_network(mr_ctx* c, int nr, const int32_t* species, const double* kf, const double* kb) {
  if (check_ctx(c) || c->prob.model != MR_MODEL_NETWORK || nr < 1 || nr > kMaxR || !species || !kf || !kb)
    return MR_EINVAL;
  NetModel N;
  memset(&N, 0, sizeof N);
  N.m = c->m;
  N.nr = nr;
  for (int r = 0; r < nr; r++) {
    if (!(kf[r] >= 0.0) || !(kb[r] >= 0.0) || !isfinite(kf[r]) || !isfinite(kb[r])) return MR_EINVAL;
    for (int t = 0; t < 4; t++) {
      const int32_t a = species[4 * r + t];
      if (a < 0 || a >= c->m) return MR_EINVAL;
      for (int u = 0; u < t; u++)
        if (species[4 * r + u] == a) return MR_EINVAL;
      N.sp[r][t] = (int8_t)a;
      if (t < 2)
        N.neg[a] |= 1u << r;
      else
        N.pos[a] |= 1u << r;
    }
    N.kf[r] = kf[r];
    N.kb[r] = kb[r];
  }
  c->net = N;
  c->net_set = true;
  return MR_OK;
}

mr_status mr_set_leaves(mr_ctx* c, int64_t n, const uint64_t* keys, const double* values, int on_device) {
  if (check_ctx(c) || n < 1 || !keys || !values || n > c->cap_leaves) return MR_EINVAL;
  uint64_t* dk;
  double* dv;
  bool ok1, ok2;
  mr_status s = to_device(c, keys, n, on_device, &dk, &ok1);
  if (s) return s;
  s = to_device(c, values, (int64_t)c->m * n, on_device, &dv, &ok2, 1);
  if (!s) s = set_leaves(c, n, dk, dv);
  cudaStreamSynchronize(c->stream);
  if (ok1) cudaFree(dk);
  if (ok2) cudaFree(dv);
  if (!s) refresh_tree_stats(c);
  return s;
}

mr_status mr_num_leaves(const mr_ctx* c, int64_t* n) {
  if (check_ctx(c) || !n) return MR_EINVAL;
  *n = c->tb[c->cur].nleaves;
  return MR_OK;
}

mr_status mr_get_leaves(mr_ctx* c, uint64_t* keys, double* values, int64_t cap, int64_t* n, int on_device) {
  if (check_ctx(c) || !n) return MR_EINVAL;
  TreeBuf& t = c->tb[c->cur];
  const int64_t N = t.nleaves;
  *n = N;
  if (cap < N) return MR_ENOMEM;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (keys) {
    uint64_t* dk = on_device ? keys : reinterpret_cast<uint64_t*>(c->work[3]);
    if (!on_device && (int64_t)c->m * c->cap_leaves < N) return MR_ENOMEM;
    k_export_keys<<<grid_for(N), kBlock, 0, c->stream>>>(t.leaf_node, t.code, t.lvl, N, dk);
    c->launches++;
    if (!on_device) MR_CUDA(c, cudaMemcpyAsync(keys, dk, sizeof(uint64_t) * N, kind, c->stream));
  }
  if (values && N > 0)
    MR_CUDA(c, cudaMemcpy2DAsync(values, sizeof(double) * N, t.U, sizeof(double) * c->cap_leaves,
                                 sizeof(double) * N, c->m, kind, c->stream));
  MR_CUDA(c, cudaStreamSynchronize(c->stream));
  return MR_OK;
}

mr_status mr_adapt(mr_ctx* c, double eta) {
  if (check_ctx(c) || !(eta >= 0.0) || !isfinite(eta)) return MR_EINVAL;
  mr_status s = adapt(c, eta);
  if (!s) refresh_tree_stats(c);
  return s;
}

mr_status mr_set_radau_schedule(mr_ctx* c, int schedule) {
  if (check_ctx(c) || (schedule != MR_RADAU_THREAD && schedule != MR_RADAU_POOL)) return MR_EINVAL;
  c->radau_schedule = schedule;
  return MR_OK;
}

mr_status react_radau5(mr_ctx* c, double dt, double rtol, double atol) {
  if (check_ctx(c) || !(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0)) return MR_EINVAL;
  return react(c, dt, rtol, atol);
}

mr_status diffuse_rock4(mr_ctx* c, double dt, double tol) {
  if (check_ctx(c) || !(dt > 0.0) || !(tol > 0.0)) return MR_EINVAL;
  return diffuse(c, dt, tol);
}

mr_status strang_step(mr_ctx* c, double dt, double eta, double rtol, double atol, double rock_tol) {
  if (check_ctx(c) || !(dt > 0.0) || !(eta >= 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !(rock_tol > 0.0))
    return MR_EINVAL;
  MR_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  mr_status s = adapt(c, eta);
  if (s) return s;
  s = build_tables(c);
  if (s) return s;
  MR_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  s = react(c, 0.5 * dt, rtol, atol);
  if (s) return s;
  MR_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
  s = diffuse(c, dt, rock_tol);
  if (s) return s;
  MR_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
  s = react(c, 0.5 * dt, rtol, atol);
  if (s) return s;
  MR_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
  MR_CUDA(c, cudaEventSynchronize(c->ev[4]));
  float a = 0, r1 = 0, d = 0, r2 = 0;
  cudaEventElapsedTime(&a, c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&r1, c->ev[1], c->ev[2]);
  cudaEventElapsedTime(&d, c->ev[2], c->ev[3]);
  cudaEventElapsedTime(&r2, c->ev[3], c->ev[4]);
  c->stats.ms_adapt = a;
  c->stats.ms_react = r1 + r2;
  c->stats.ms_diffuse = d;
  refresh_tree_stats(c);
  return MR_OK;
}

namespace {
struct SaveHeader {
  char magic[8];
  int32_t version, dim, J, jmin, m, model, precision, reserved;
  int64_t n;
  int64_t pad[2];
};
static_assert(sizeof(SaveHeader) == 64, "checkpoint header is 64 bytes");
const char kMagic[8] = {'M', 'R', 'G', 'B', '3', '0', '0', '\0'};
}  // namespace

mr_status mr_save(mr_ctx* c, const char* path) {
  if (check_ctx(c) || !path) return MR_EINVAL;
  const int64_t N = c->tb[c->cur].nleaves;
  std::vector<uint64_t> keys(N);
  std::vector<double> vals((size_t)c->m * N);
  int64_t n = 0;
  mr_status s = mr_get_leaves(c, keys.data(), vals.data(), N, &n, 0);
  if (s) return s;
  SaveHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kMagic, 8);
  h.version = 2;
  h.dim = c->prob.dim;
  h.J = c->prob.J;
  h.jmin = c->prob.jmin;
  h.m = c->m;
  h.model = c->prob.model;
  h.precision = c->prob.precision;
  h.n = n;
  FILE* f = fopen(path, "wb");
  if (!f) {
    c->last_error = "cannot open the checkpoint file for writing";
    return MR_EIO;
  }
  bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(c->prob.params, sizeof(double), 8, f) == 8 &&
            fwrite(c->prob.D, sizeof(double), MR_MAX_SPECIES, f) == MR_MAX_SPECIES &&
            fwrite(keys.data(), sizeof(uint64_t), n, f) == (size_t)n &&
            fwrite(vals.data(), sizeof(double), (size_t)c->m * n, f) == (size_t)c->m * n;
  ok = (fclose(f) == 0) && ok;
  if (!ok) {
    c->last_error = "checkpoint write failed";
    return MR_EIO;
  }
  return MR_OK;
}

mr_status mr_load(mr_ctx* c, const char* path) {
  if (check_ctx(c) || !path) return MR_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) {
    c->last_error = "cannot open the checkpoint file";
    return MR_EIO;
  }
  SaveHeader h;
  double params[8], D[MR_MAX_SPECIES];
  if (fread(&h, sizeof h, 1, f) != 1) {
    fclose(f);
    c->last_error = "checkpoint header truncated";
    return MR_EIO;
  }
  if (memcmp(h.magic, kMagic, 8) != 0 || (h.version != 1 && h.version != 2)) {
    fclose(f);
    c->last_error = "not a checkpoint of this library";
    return MR_EINVAL;
  }
  // version 1 stored 16 diffusion coefficients, version 2 MR_MAX_SPECIES
  const size_t nd = h.version == 1 ? 16 : MR_MAX_SPECIES;
  if (fread(params, sizeof(double), 8, f) != 8 || fread(D, sizeof(double), nd, f) != nd) {
    fclose(f);
    c->last_error = "checkpoint header truncated";
    return MR_EIO;
  }
  if (h.dim != c->prob.dim || h.J != c->prob.J || h.jmin != c->prob.jmin || h.m != c->m ||
      h.model != c->prob.model || h.n < 1 || h.n > c->cap_leaves) {
    fclose(f);
    c->last_error = "checkpoint was written for another problem";
    return MR_EINVAL;
  }
  std::vector<uint64_t> keys(h.n);
  std::vector<double> vals((size_t)c->m * h.n);
  const bool ok = fread(keys.data(), sizeof(uint64_t), h.n, f) == (size_t)h.n &&
                  fread(vals.data(), sizeof(double), (size_t)c->m * h.n, f) == (size_t)c->m * h.n;
  fclose(f);
  if (!ok) {
    c->last_error = "checkpoint data truncated";
    return MR_EIO;
  }
  return mr_set_leaves(c, h.n, keys.data(), vals.data(), 0);
}

mr_status mr_get_stats(const mr_ctx* c, mr_stats* out) {
  if (check_ctx(c) || !out) return MR_EINVAL;
  *out = c->stats;
  out->kernel_launches = c->launches;
  return MR_OK;
}

mr_status mr_get_complexity(mr_ctx* c, int32_t* out, int64_t cap, int on_device) {
  if (check_ctx(c) || !out) return MR_EINVAL;
  const int64_t N = c->tb[c->cur].nleaves;
  if (cap < N) return MR_ENOMEM;
  MR_CUDA(c, cudaMemcpyAsync(out, c->complexity, sizeof(int32_t) * N,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  MR_CUDA(c, cudaStreamSynchronize(c->stream));
  return MR_OK;
}

mr_status mr_mass(mr_ctx* c, double* out) {
  if (check_ctx(c) || !out) return MR_EINVAL;
  return mass(c, out);
}

mr_status mr_apply_operator(mr_ctx* c, const double* u_in, double* out, int on_device, double* rho) {
  if (check_ctx(c) || !u_in || !out) return MR_EINVAL;
  const int64_t N = c->tb[c->cur].nleaves;
  double *din, *dout;
  bool o1, o2;
  mr_status s = to_device(c, u_in, N, on_device, &din, &o1);
  if (s) return s;
  if (on_device) {
    dout = out;
    o2 = false;
  } else {
    s = dalloc(c, &dout, N);
    o2 = true;
  }
  if (!s) s = apply_operator(c, din, dout);
  if (!s && !on_device) {
    cudaError_t e = cudaMemcpy(out, dout, sizeof(double) * N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(c, e, "copy operator result");
  }
  cudaStreamSynchronize(c->stream);
  if (o1) cudaFree(din);
  if (o2) cudaFree(dout);
  if (!s && rho) *rho = c->rho;
  return s;
}

mr_status mr_operator_forms(mr_ctx* c, int reps, double* ms_compact, double* ms_csr, int64_t* csr_nnz,
                            double* max_rel_diff) {
  if (check_ctx(c) || !ms_compact || !ms_csr || !csr_nnz || !max_rel_diff || reps < 1 || reps > 10000)
    return MR_EINVAL;
  return operator_forms(c, reps, ms_compact, ms_csr, csr_nnz, max_rel_diff);
}

mr_status mr_fp64_fma_rate(double* tflops, double* mhz) {
  if (!tflops) return MR_EINVAL;
  return fp64_probe(tflops, mhz);
}

mr_status mr_radau_work(int model, int m, double* out) {
  if (!out || (model != MR_MODEL_BZ && model != MR_MODEL_NAGUMO) || m < 1) return MR_EINVAL;
  const RadauWork w = radau_work(model, m);
  const double v[8] = {w.rhs, w.jac, w.dec, w.newton, w.monitor, w.attempt, w.extrap, w.accept};
  for (int q = 0; q < 8; q++) out[q] = v[q];
  return MR_OK;
}

mr_status mr_rock4_coefficients(int s, double* mu, double* nu, double* kap, double* w, double* errc, double* ell) {
  if (s < 5 || s > 152 || !mu || !nu || !kap || !w || !errc) return MR_EINVAL;
  if (rock4_coeffs(s, mu, nu, kap, w, errc)) return MR_ESTATE;
  if (ell) *ell = rock4_ell(s);
  return MR_OK;
}

}  // extern "C"
