// Device-wide exclusive prefix sums used by the compaction steps of the grid
// adaptation (new node indices, leaf indices, irregular operator rows).
// Three passes over tiles of kTile items: tile sums, a scan of the tile sums
// in one block, then a block scan of every tile with its offset.  Warp scans
// use shuffles; the result is deterministic (integer arithmetic).
#include "mr_internal.cuh"

namespace mrg {
namespace {

constexpr int kItems = 8;
constexpr int kTile = kBlock * kItems;

template <typename T>
__device__ inline T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += t;
  }
  return v;
}

// block exclusive scan of one value per thread; returns the block total in *tot
template <typename T>
__device__ inline T block_excl_scan(T v, T* tot) {
  __shared__ T warp_sums[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = lane < kBlock / 32 ? warp_sums[lane] : T(0);
    s = warp_incl_scan(s);
    if (lane < kBlock / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  T off = wid ? warp_sums[wid - 1] : T(0);
  *tot = warp_sums[kBlock / 32 - 1];
  __syncthreads();
  return off + inc - v;
}

template <typename In, typename Acc>
__global__ void k_tile_sums(const In* __restrict__ in, int64_t n, Acc* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  Acc s = 0;
#pragma unroll
  for (int q = 0; q < kItems; q++)
    if (base + q < n) s += (Acc)in[base + q];
  Acc tot;
  block_excl_scan<Acc>(s, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename Acc>
__global__ void k_scan_parts(Acc* part, int64_t nt, Acc* total) {
  __shared__ Acc carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < nt; b += kBlock) {
    int64_t i = b + threadIdx.x;
    Acc v = i < nt ? part[i] : Acc(0);
    Acc tot;
    Acc ex = block_excl_scan<Acc>(v, &tot);
    if (i < nt) part[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <typename In, typename Acc>
__global__ void k_tile_scan(const In* __restrict__ in, int64_t n, const Acc* __restrict__ part,
                            Acc* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  Acc v[kItems];
  Acc s = 0;
#pragma unroll
  for (int q = 0; q < kItems; q++) {
    v[q] = base + q < n ? (Acc)in[base + q] : Acc(0);
    s += v[q];
  }
  Acc tot;
  Acc ex = block_excl_scan<Acc>(s, &tot) + part[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kItems; q++) {
    if (base + q < n) out[base + q] = ex;
    ex += v[q];
  }
}

template <typename In, typename Acc>
void scan_impl(mr_ctx* c, const In* in, Acc* out, int64_t n, Acc* total_dev) {
  if (n <= 0) {
    if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(Acc), c->stream);
    return;
  }
  int64_t nt = (n + kTile - 1) / kTile;
  Acc* part = reinterpret_cast<Acc*>(c->scan_tmp);
  k_tile_sums<In, Acc><<<(unsigned)nt, kBlock, 0, c->stream>>>(in, n, part);
  k_scan_parts<Acc><<<1, kBlock, 0, c->stream>>>(part, nt, total_dev);
  k_tile_scan<In, Acc><<<(unsigned)nt, kBlock, 0, c->stream>>>(in, n, part, out);
  c->launches += 3;
}

}  // namespace

void scan_u8(mr_ctx* c, const uint8_t* in, int32_t* out, int64_t n, int32_t* total_dev) {
  scan_impl<uint8_t, int32_t>(c, in, out, n, total_dev);
}
void scan_i32(mr_ctx* c, const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev) {
  scan_impl<int32_t, int32_t>(c, in, out, n, total_dev);
}
void scan_i32_to_i64(mr_ctx* c, const int32_t* in, int64_t* out, int64_t n, long long* total_dev) {
  scan_impl<int32_t, long long>(c, in, reinterpret_cast<long long*>(out), n, total_dev);
}

}  // namespace mrg
