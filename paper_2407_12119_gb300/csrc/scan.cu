// Exclusive prefix sum of int32 counts (three passes: block totals, scan of
// the totals in one block, per-block scan with carry-in).  Used to turn
// per-hit edge counts into CSR offsets.
#include "etx_internal.cuh"

namespace etx {
namespace {

constexpr int kThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// exclusive prefix and writes the block total to *total.
__device__ int block_excl_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? sh[lane] : 0;
    int wi = warp_incl_scan(w);
    if (lane < nw) sh[lane] = wi - w;
    if (lane == nw - 1) sh[32] = wi;
  }
  __syncthreads();
  int r = inc - v + sh[wid];
  *total = sh[32];
  __syncthreads();
  return r;
}

__global__ void k_block_totals(const int32_t* in, int64_t n, int32_t* tmp) {
  __shared__ int sh[33];
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i)
    if (base + i < n) s += in[base + i];
  int total;
  block_excl_scan(s, sh, &total);
  if (threadIdx.x == 0) tmp[blockIdx.x] = total;
}

__global__ void k_scan_totals(int32_t* tmp, int nb, int32_t* out_total) {
  __shared__ int sh[33];
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nb ? tmp[i] : 0;
    int total;
    int ex = block_excl_scan(v, sh, &total);
    if (i < nb) tmp[i] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

__global__ void k_block_scan(const int32_t* in, int64_t n, const int32_t* tmp, int32_t* out) {
  __shared__ int sh[33];
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  int v[kItems];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  int total;
  int ex = block_excl_scan(s, sh, &total) + tmp[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
}

}  // namespace

size_t scan_tmp_ints(int64_t n) { return (size_t)((n + kTile - 1) / kTile) + 1; }

cudaError_t exclusive_scan(etx_ctx* ctx, const int32_t* in, int32_t* out, int64_t n,
                           cudaStream_t s) {
  return exclusive_scan_with(ctx, in, out, n, ctx->scan_tmp, ctx->scan_tmp_ints, s);
}

cudaError_t exclusive_scan_with(etx_ctx* ctx, const int32_t* in, int32_t* out, int64_t n,
                                int32_t* tmp, size_t tmp_ints, cudaStream_t s) {
  const int64_t nb = (n + kTile - 1) / kTile;
  if ((size_t)nb + 1 > tmp_ints) return cudaErrorInvalidValue;
  if (nb == 0) {
    return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
  }
  launch(ctx, "scan_block_totals", k_block_totals, (unsigned)nb, kThreads, 0, s, in, n, tmp);
  launch(ctx, "scan_totals", k_scan_totals, 1, 1024, 0, s, tmp, (int)nb, out + n);
  launch(ctx, "scan_blocks", k_block_scan, (unsigned)nb, kThreads, 0, s, in, n, tmp, out);
  return cudaGetLastError();
}

}  // namespace etx
