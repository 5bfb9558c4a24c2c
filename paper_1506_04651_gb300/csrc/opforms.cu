// Two storage forms of the finite-volume leaf operator L (Eq. discretise) and
// their cost per application, the comparison of the paper's App. C (Table 5:
// its compact operator against a CSR matrix of the same operator).
//
//   compact  the form the ROCK4 sweeps use: a regular-leaf table (leaf, its
//            2d same-level neighbours, level; the weights 1/h^2 implicit)
//            for every leaf whose faces meet same-level leaves or the
//            boundary, and one merged row of (leaf, weight) pairs for each
//            leaf at a level jump, G lanes per merged row;
//   CSR      every row assembled as (column, weight) pairs in one compressed
//            sparse row matrix in leaf order, G lanes per row.
//
// Both apply L to one FP64 vector; the results agree to rounding (a regular
// row is summed as (sum of neighbours - 2d u) / h^2 in the compact form and
// as a weighted sum in CSR).
#include <string.h>

#include <algorithm>
#include <vector>

#include "mr_internal.cuh"

namespace mrg {
namespace {

__device__ inline double pow4(int j) {  // 4^j = 1/h_j^2, exact
  return __longlong_as_double((long long)(1023 + 2 * j) << 52);
}

template <int D, int G>
__global__ void k_apply_compact(const int4* __restrict__ reg, int64_t nreg, const int32_t* __restrict__ irr_leaf,
                                int64_t nirr, const int32_t* __restrict__ cnt, const int32_t* __restrict__ col,
                                const double* __restrict__ w, int slot, const double* __restrict__ x,
                                double* __restrict__ y) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = tid; q < nreg; q += nth) {
    const int4 e0 = reg[2 * q], e1 = reg[2 * q + 1];
    const int v[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
    double sx = x[v[1]];
#pragma unroll
    for (int f = 1; f < 2 * D; f++) sx += x[v[1 + f]];
    y[v[0]] = (sx - 2.0 * D * x[v[0]]) * pow4(v[1 + 2 * D]);
  }
  const int sub = threadIdx.x & (G - 1);
  const int64_t grp = tid / G, ngrp = nth / G;
  const int64_t rounds = (nirr + ngrp - 1) / ngrp;
  for (int64_t k = 0; k < rounds; k++) {
    const int64_t row = grp + k * ngrp;
    double s = 0.0;
    if (row < nirr) {
      const int n = cnt[row];
      const int32_t* c = col + row * (int64_t)slot;
      const double* wr = w + row * (int64_t)slot;
      for (int e = sub; e < n; e += G) s += wr[e] * x[c[e]];
    }
    for (int sft = G / 2; sft > 0; sft >>= 1) s += __shfl_xor_sync(0xffffffffu, s, sft);
    if (row < nirr && sub == 0) y[irr_leaf[row]] = s;
  }
}

// entries of every row: a regular leaf has itself and its interior faces'
// neighbours (a boundary face folds into its own weight), a merged row its cnt
__global__ void k_csr_count(const int4* __restrict__ reg, int64_t nreg, const int32_t* __restrict__ irr_leaf,
                            int64_t nirr, const int32_t* __restrict__ cnt, int D, int32_t* __restrict__ len) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = tid; q < nreg; q += nth) {
    const int4 e0 = reg[2 * q], e1 = reg[2 * q + 1];
    const int v[7] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z};
    int n = 1;
    for (int f = 0; f < 2 * D; f++) n += v[1 + f] != v[0];
    len[v[0]] = n;
  }
  for (int64_t q = tid; q < nirr; q += nth) len[irr_leaf[q]] = cnt[q];
}

__global__ void k_csr_fill(const int4* __restrict__ reg, int64_t nreg, const int32_t* __restrict__ irr_leaf,
                           int64_t nirr, const int32_t* __restrict__ cnt, const int32_t* __restrict__ col,
                           const double* __restrict__ w, int slot, int D, const int64_t* __restrict__ ptr,
                           int32_t* __restrict__ ccol, double* __restrict__ cw) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = tid; q < nreg; q += nth) {
    const int4 e0 = reg[2 * q], e1 = reg[2 * q + 1];
    const int v[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
    const double ih2 = pow4(v[1 + 2 * D]);
    int64_t p = ptr[v[0]];
    int inner = 0;
    for (int f = 0; f < 2 * D; f++)
      if (v[1 + f] != v[0]) {
        ccol[p] = v[1 + f];
        cw[p++] = ih2;
        inner++;
      }
    ccol[p] = v[0];
    cw[p] = -inner * ih2;
  }
  for (int64_t q = tid; q < nirr; q += nth) {
    const int64_t p = ptr[irr_leaf[q]];
    for (int e = 0; e < cnt[q]; e++) {
      ccol[p + e] = col[q * (int64_t)slot + e];
      cw[p + e] = w[q * (int64_t)slot + e];
    }
  }
}

template <int G>
__global__ void k_apply_csr(const int64_t* __restrict__ ptr, const int32_t* __restrict__ ccol,
                            const double* __restrict__ cw, int64_t N, const double* __restrict__ x,
                            double* __restrict__ y) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const int sub = threadIdx.x & (G - 1);
  const int64_t grp = tid / G, ngrp = nth / G;
  const int64_t rounds = (N + ngrp - 1) / ngrp;
  for (int64_t k = 0; k < rounds; k++) {
    const int64_t r = grp + k * ngrp;
    double s = 0.0;
    if (r < N)
      for (int64_t e = ptr[r] + sub; e < ptr[r + 1]; e += G) s += cw[e] * x[ccol[e]];
    for (int sft = G / 2; sft > 0; sft >>= 1) s += __shfl_xor_sync(0xffffffffu, s, sft);
    if (r < N && sub == 0) y[r] = s;
  }
}

__global__ void k_fill_ramp(double* x, int64_t N) {  // a smooth, non-constant test vector
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x)
    x[r] = 1.0 + 0.5 * sin(1e-3 * (double)r);
}

__global__ void k_max_rel_diff(const double* a, const double* b, int64_t N, unsigned long long* out) {
  double m = 0.0, s = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    m = fmax(m, fabs(a[r] - b[r]));
    s = fmax(s, fabs(b[r]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(s));
  }
}

}  // namespace

mr_status operator_forms(mr_ctx* c, int reps, double* ms_compact, double* ms_csr, int64_t* csr_nnz,
                         double* max_rel_diff) {
  if (reps < 1 || reps > 10000) return MR_EINVAL;
  MR_TRY(build_tables(c));
  TreeBuf& t = c->tb[c->cur];
  const int64_t N = t.nleaves, nirr = c->stats.irregular_rows, nreg = N - nirr;
  const int D = c->d, slot = c->irr_slot;
  int dev = 0, nsm = 152;
  MR_CUDA(c, cudaGetDevice(&dev));
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = nsm * 8, block = 256;
  // scratch: x, two outputs, row lengths, row pointers, the CSR entries
  double *x = nullptr, *y1 = nullptr, *y2 = nullptr, *cw = nullptr;
  int32_t *len = nullptr, *ccol = nullptr;
  int64_t* ptr = nullptr;
  unsigned long long* red = nullptr;
  long long* total = nullptr;
  mr_status st = MR_OK;
  auto fail = [&](cudaError_t e, const char* where) {
    if (st == MR_OK) st = cuda_fail(c, e, where);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  do {
    cudaError_t e;
    if ((e = cudaMalloc(&x, sizeof(double) * N)) || (e = cudaMalloc(&y1, sizeof(double) * N)) ||
        (e = cudaMalloc(&y2, sizeof(double) * N)) || (e = cudaMalloc(&len, sizeof(int32_t) * (N + 1))) ||
        (e = cudaMalloc(&ptr, sizeof(int64_t) * (N + 1))) || (e = cudaMalloc(&red, 2 * sizeof(unsigned long long))) ||
        (e = cudaMalloc(&total, sizeof(long long))) || (e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
      fail(e, "operator_forms scratch");
      break;
    }
    k_fill_ramp<<<grid, block, 0, c->stream>>>(x, N);
    k_csr_count<<<grid, block, 0, c->stream>>>(c->reg_tab, nreg, c->irr_leaf, nirr, c->irr_cnt, D, len);
    scan_i32_to_i64(c, len, ptr, N, total);
    long long nnz = 0;
    if ((e = cudaMemcpyAsync(&nnz, total, sizeof nnz, cudaMemcpyDeviceToHost, c->stream)) ||
        (e = cudaStreamSynchronize(c->stream))) {
      fail(e, "operator_forms count");
      break;
    }
    if ((e = cudaMemcpyAsync(ptr + N, total, sizeof(long long), cudaMemcpyDeviceToDevice, c->stream)) ||
        (e = cudaMalloc(&ccol, sizeof(int32_t) * std::max<long long>(nnz, 1))) ||
        (e = cudaMalloc(&cw, sizeof(double) * std::max<long long>(nnz, 1)))) {
      fail(e, "operator_forms CSR");
      break;
    }
    k_csr_fill<<<grid, block, 0, c->stream>>>(c->reg_tab, nreg, c->irr_leaf, nirr, c->irr_cnt, c->irr_col,
                                               c->irr_w, slot, D, ptr, ccol, cw);
    auto compact = [&]() {
      if (D == 2)
        k_apply_compact<2, 2><<<grid, block, 0, c->stream>>>(c->reg_tab, nreg, c->irr_leaf, nirr, c->irr_cnt,
                                                              c->irr_col, c->irr_w, slot, x, y1);
      else
        k_apply_compact<3, 4><<<grid, block, 0, c->stream>>>(c->reg_tab, nreg, c->irr_leaf, nirr, c->irr_cnt,
                                                              c->irr_col, c->irr_w, slot, x, y1);
    };
    auto csr = [&]() {
      if (D == 2)
        k_apply_csr<2><<<grid, block, 0, c->stream>>>(ptr, ccol, cw, N, x, y2);
      else
        k_apply_csr<4><<<grid, block, 0, c->stream>>>(ptr, ccol, cw, N, x, y2);
    };
    // warm-up, then reps applications of each form back to back
    compact();
    csr();
    float ms = 0.f;
    cudaEventRecord(e0, c->stream);
    for (int q = 0; q < reps; q++) compact();
    cudaEventRecord(e1, c->stream);
    if ((e = cudaEventSynchronize(e1))) {
      fail(e, "operator_forms compact");
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_compact = ms / reps;
    cudaEventRecord(e0, c->stream);
    for (int q = 0; q < reps; q++) csr();
    cudaEventRecord(e1, c->stream);
    if ((e = cudaEventSynchronize(e1))) {
      fail(e, "operator_forms CSR apply");
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_csr = ms / reps;
    c->launches += 5 + 2 * (reps + 1);
    unsigned long long hr[2] = {0, 0};
    if ((e = cudaMemsetAsync(red, 0, 2 * sizeof(unsigned long long), c->stream))) {
      fail(e, "operator_forms compare");
      break;
    }
    k_max_rel_diff<<<grid, block, 0, c->stream>>>(y2, y1, N, red);
    if ((e = cudaMemcpyAsync(hr, red, sizeof hr, cudaMemcpyDeviceToHost, c->stream)) ||
        (e = cudaStreamSynchronize(c->stream)) || (e = cudaGetLastError())) {
      fail(e, "operator_forms compare");
      break;
    }
    double m, sc;
    memcpy(&m, &hr[0], sizeof m);
    memcpy(&sc, &hr[1], sizeof sc);
    *max_rel_diff = sc > 0.0 ? m / sc : m;
    *csr_nnz = nnz;
  } while (false);
  cudaFree(x);
  cudaFree(y1);
  cudaFree(y2);
  cudaFree(len);
  cudaFree(ptr);
  cudaFree(red);
  cudaFree(total);
  cudaFree(ccol);
  cudaFree(cw);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

}  // namespace mrg
