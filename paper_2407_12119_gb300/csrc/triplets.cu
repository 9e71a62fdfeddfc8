// Triplets of the purified hit graph (paper Sec. 5.3) and their classifiers.
//
// A triplet is a pair of kept edges (logit > cut) sharing a hit C:
// articulations A->C, C->B, left elbows C->A, C->B and right elbows A->C,
// B->C.  Per hit, the kept in-degree a and out-degree b give a*b
// articulations, b(b-1)/2 left and a(a-1)/2 right elbows; three scans give
// every hit its slices, and the lists are written type-major (all
// articulations, then left, then right elbows), by C, then by the first and
// second edge index (the in-edge first for an articulation).  In-edges come
// from the dst-CSC, whose segments are sorted by edge id, out-edges from the
// src-CSR of the sorted edge list.  The two classifiers (one for
// articulations, one for elbows) are FP32 MLPs on [e_first, e_second] of the
// final edge encodings, run by the fused SIMT MLP kernel.
#include <algorithm>
#include <vector>

#include "etx_internal.cuh"

namespace etx {
namespace {

struct TripCtx {
  const int32_t* out_off;  // [n_hits + 1] src-CSR over the edge list
  const int32_t* in_off;   // [n_hits + 1] dst-CSC
  const int32_t* perm_in;  // edge ids of the CSC segments, ascending per segment
  const float* logits;
  float thr;
};

__device__ __forceinline__ void kept_degrees(const TripCtx& c, int64_t h, int* a, int* b) {
  int na = 0, nb = 0;
  for (int q = c.in_off[h]; q < c.in_off[h + 1]; ++q) na += c.logits[c.perm_in[q]] > c.thr;
  for (int q = c.out_off[h]; q < c.out_off[h + 1]; ++q) nb += c.logits[q] > c.thr;
  *a = na;
  *b = nb;
}

__global__ void k_trip_count(TripCtx c, int64_t n_hits, int32_t* __restrict__ n_art,
                             int32_t* __restrict__ n_left, int32_t* __restrict__ n_right) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_hits;
       h += (int64_t)gridDim.x * blockDim.x) {
    int a, b;
    kept_degrees(c, h, &a, &b);
    n_art[h] = a * b;
    n_left[h] = b * (b - 1) / 2;
    n_right[h] = a * (a - 1) / 2;
  }
}

// counts[0..3] = {total, articulations, left elbows, right elbows}; all zero
// when the lists do not fit (flagged by the emit pass).
__global__ void k_trip_total(const int32_t* __restrict__ off_art, const int32_t* __restrict__ off_left,
                             const int32_t* __restrict__ off_right, int64_t n_hits, int64_t capacity,
                             int32_t* __restrict__ counts) {
  const int64_t na = off_art[n_hits], nl = off_left[n_hits], nr = off_right[n_hits];
  const int64_t tot = na + nl + nr;
  const bool fit = tot <= capacity;
  counts[0] = fit ? (int32_t)tot : 0;
  counts[1] = fit ? (int32_t)na : 0;
  counts[2] = fit ? (int32_t)nl : 0;
  counts[3] = fit ? (int32_t)nr : 0;
}

__global__ void k_trip_emit(TripCtx c, int64_t n_hits, const int32_t* __restrict__ off_art,
                            const int32_t* __restrict__ off_left, const int32_t* __restrict__ off_right,
                            int64_t capacity, int32_t* __restrict__ first, int32_t* __restrict__ second,
                            int8_t* __restrict__ kind, int* err) {
  const int64_t na = off_art[n_hits], nl = off_left[n_hits], nr = off_right[n_hits];
  if (na + nl + nr > capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_err(err, DERR_CAPACITY);
    return;
  }
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_hits;
       h += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = c.in_off[h], i1 = c.in_off[h + 1];
    const int o0 = c.out_off[h], o1 = c.out_off[h + 1];
    int64_t w = off_art[h];
    for (int qi = i0; qi < i1; ++qi) {
      const int ei = c.perm_in[qi];
      if (!(c.logits[ei] > c.thr)) continue;
      for (int eo = o0; eo < o1; ++eo) {
        if (!(c.logits[eo] > c.thr)) continue;
        first[w] = ei;
        second[w] = eo;
        kind[w] = 0;
        ++w;
      }
    }
    w = na + off_left[h];
    for (int x = o0; x < o1; ++x) {
      if (!(c.logits[x] > c.thr)) continue;
      for (int y = x + 1; y < o1; ++y) {
        if (!(c.logits[y] > c.thr)) continue;
        first[w] = x;
        second[w] = y;
        kind[w] = 1;
        ++w;
      }
    }
    w = na + nl + off_right[h];
    for (int x = i0; x < i1; ++x) {
      const int ex = c.perm_in[x];
      if (!(c.logits[ex] > c.thr)) continue;
      for (int y = x + 1; y < i1; ++y) {
        const int ey = c.perm_in[y];
        if (!(c.logits[ey] > c.thr)) continue;
        first[w] = ex;
        second[w] = ey;
        kind[w] = 2;
        ++w;
      }
    }
  }
}

}  // namespace

size_t triplets_workspace(int64_t n_hits) { return (size_t)3 * (n_hits + 1) * sizeof(int32_t); }

cudaError_t launch_build_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                  const float* logits, float thr, int64_t n_hits, void* workspace,
                                  int64_t capacity, int32_t* first, int32_t* second, int8_t* kind,
                                  int32_t* counts, cudaStream_t s) {
  cudaError_t e = launch_edge_index(ctx, n_hits, src, dst, ctx->n_edges, s);
  if (e != cudaSuccess) return e;
  int32_t* off_art = static_cast<int32_t*>(workspace);
  int32_t* off_left = off_art + (n_hits + 1);
  int32_t* off_right = off_left + (n_hits + 1);
  TripCtx c{ctx->out_off, ctx->in_off, ctx->perm_in, logits, thr};
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n_hits + 255) / 256, (int64_t)ctx->n_sms * 8));
  if (n_hits > 0)
    launch(ctx, "triplet_count", k_trip_count, grid, 256, 0, s, c, n_hits, off_art, off_left,
           off_right);
  for (int32_t* o : {off_art, off_left, off_right}) {
    e = exclusive_scan(ctx, o, o, n_hits, s);
    if (e != cudaSuccess) return e;
  }
  if (n_hits > 0)
    launch(ctx, "triplet_emit", k_trip_emit, grid, 256, 0, s, c, n_hits, (const int32_t*)off_art,
           (const int32_t*)off_left, (const int32_t*)off_right, capacity, first, second, kind,
           ctx->d_err);
  launch(ctx, "triplet_total", k_trip_total, 1, 1, 0, s, (const int32_t*)off_art,
         (const int32_t*)off_left, (const int32_t*)off_right, n_hits, capacity, counts);
  return cudaGetLastError();
}

// Host: repack the triplet-classifier blob (art then elb, each W1[H][2H] b1 g1
// be1 W2[1][H] b2) into W^T form on the device.
cudaError_t load_triplet_weights(etx_ctx* ctx, const float* blob) {
  const int H = ctx->cfg.hidden;
  std::vector<float> dev;
  const float* p = blob;
  size_t at[2][6];
  auto align4 = [&]() { while (dev.size() % 4) dev.push_back(0.f); };
  for (int t = 0; t < 2; ++t) {
    align4();
    at[t][0] = dev.size();  // W1^T [2H][H]
    dev.resize(dev.size() + (size_t)2 * H * H);
    for (int o = 0; o < H; ++o)
      for (int k = 0; k < 2 * H; ++k) dev[at[t][0] + (size_t)k * H + o] = p[(size_t)o * 2 * H + k];
    p += (size_t)2 * H * H;
    for (int v = 1; v <= 4; ++v) {  // b1, g1, be1, W2 (H each)
      align4();
      at[t][v] = dev.size();
      dev.insert(dev.end(), p, p + H);
      p += H;
    }
    align4();
    at[t][5] = dev.size();  // b2
    dev.push_back(*p++);
  }
  if (ctx->w_trip) cudaFree(ctx->w_trip);
  ctx->w_trip = nullptr;
  cudaError_t e = cudaMalloc(&ctx->w_trip, dev.size() * sizeof(float));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(ctx->w_trip, dev.data(), dev.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  for (int t = 0; t < 2; ++t) {
    ClassifierF32& c = t == 0 ? ctx->trip_art : ctx->trip_elb;
    c.l1.wt = ctx->w_trip + at[t][0];
    c.l1.b = ctx->w_trip + at[t][1];
    c.l1.k_in = c.l1.k_pad = 2 * H;
    c.l1.n = H;
    c.g1 = ctx->w_trip + at[t][2];
    c.be1 = ctx->w_trip + at[t][3];
    c.w2 = ctx->w_trip + at[t][4];
    c.b2 = ctx->w_trip + at[t][5];
  }
  ctx->trip_loaded = true;
  return cudaSuccess;
}

int64_t triplet_weights_size(int H) { return 2 * ((int64_t)2 * H * H + 4 * (int64_t)H + 1); }

}  // namespace etx
