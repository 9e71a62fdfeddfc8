// Rough-graph construction (paper Eq. 1, Sec. 5.1, Sec. 7.2).
//
// Hits arrive plane-sorted per event, so the candidates of every source hit
// on plane p (the hits of planes p+1 and p+2) form one contiguous index range.
// One block (or 2 or 4) per (event, plane): the candidate embeddings are
// staged in shared memory (structure of arrays, so lane j reads candidate j
// bank-conflict free) when they fit the block's stage, else read from global
// memory.  The stage size and the blocks per (event, plane) are launch
// parameters (autotuned): a stage sized for the typical event keeps more
// blocks resident per SM than one sized for the largest.  A warp takes two
// source hits at a time, lanes over candidates: one pass computes both
// sources' FP32 distances from the same candidate loads and ballot-compacts
// the hits inside the radius into a (d2, j) list per source; when more than
// k_max qualify, a listed pair is kept iff fewer than k_max listed pairs are
// smaller, which realises the (d2, j) order.  A source with more than 256
// qualifying hits takes the general path: the k_max-th smallest squared
// distance by a 32-step radix select on the FP32 bit patterns (non-negative
// floats order like their bits), ties at that value in ascending candidate
// index.
//
// Either one pass writes each source's kept edges into k_max fixed slots with
// its count, and a compaction after the scan of the counts forms the edge
// list; or (when the slots do not fit the context) a counting pass, the scan,
// and an emitting pass at the scanned offsets.  The counts' scan is also the
// src-CSR of the edge list; edges come out in (i, j) order.
#include <algorithm>

#include "etx_internal.cuh"

namespace etx {
namespace {

constexpr int kKnnThreads = 128;
constexpr int kStageMaxFloats = 16384;  // largest candidate stage: 64 KB per block
constexpr int kMaxDim = 32;

// register-resident candidate keys per lane: 16 (512 candidates per block) or
// 64 (2048, the shared-memory stage limit for D = 8)

// Squared distance for a compile-time dimension (same operation order).
template <int D>
__device__ __forceinline__ float d2_fixed(const float (&ei)[D], const float* cand, int stride) {
  float s = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float t = __fsub_rn(ei[d], cand[d * stride]);
    s = __fadd_rn(s, __fmul_rn(t, t));
  }
  return s;
}

// Squared distance, FP32, one rounding per operation, dimensions in order.
__device__ __forceinline__ float d2_ordered(const float* __restrict__ ei, const float* cand,
                                            int stride, int D) {
  float s = 0.f;
  for (int d = 0; d < D; ++d) {
    const float t = __fsub_rn(ei[d], cand[d * stride]);
    s = __fadd_rn(s, __fmul_rn(t, t));
  }
  return s;
}

__global__ void k_check_hits(const int8_t* __restrict__ plane, const int32_t* __restrict__ hoff,
                             int32_t n_events, int64_t n_hits, int n_planes, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n_events) {
    const int v = hoff[i];
    if ((i == 0 && v != 0) || (i == n_events && v != n_hits) || (i > 0 && v < hoff[i - 1]))
      set_err(err, DERR_UNSORTED);
  }
  if (i >= n_hits) return;
  const int p = plane[i];
  if (p < 0 || p >= n_planes) {
    set_err(err, DERR_UNSORTED);
    return;
  }
  if (i > 0 && plane[i - 1] > p) {
    // allowed only at an event boundary
    int lo = 0, hi = n_events;  // find b with hoff[b] <= i < hoff[b+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (hoff[mid] <= i) lo = mid; else hi = mid;
    }
    if (hoff[lo] != i) set_err(err, DERR_UNSORTED);
  }
}

// plane_off[b*(P+1) + p] = first hit of event b with plane >= p (p = 0..P).
__global__ void k_plane_bins(const int8_t* __restrict__ plane, const int32_t* __restrict__ hoff,
                             int32_t n_events, int n_hits, int n_planes,
                             int32_t* __restrict__ plane_off) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)n_events * (n_planes + 1);
  if (t >= total) return;
  const int b = (int)(t / (n_planes + 1)), p = (int)(t % (n_planes + 1));
  // clamp so malformed offsets (flagged by k_check_hits) cannot index out of range
  int lo = min(max(hoff[b], 0), n_hits), hi = min(max(hoff[b + 1], 0), n_hits);
  if (hi < lo) hi = lo;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (plane[mid] < p) lo = mid + 1; else hi = mid;
  }
  plane_off[t] = lo;
}

// Fast path (compile-time D; candidate j's dimension d at
// cand[j * cstep + d * cstride], staged or in global memory), two source hits
// per warp: one pass over the candidates computes both sources' distances
// from the same candidate loads (two independent chains) and lists each
// source's qualifying candidates (d2 < r2) in its own per-warp scratch as
// (key, j) pairs, key = the FP32 bit pattern of d2 (order-preserving for
// d2 >= 0), in ascending j (ballot compaction).  Then per source: if more than
// k_max qualify, a pair is kept iff fewer than k_max listed pairs are smaller
// than it ((key, j) pairs are distinct, so this keeps exactly the k_max
// smallest by (d2, j)); kept pairs are written in list order, i.e. ascending j.
// A source with more than kListCap qualifying candidates is left to the
// general path.  The loops run over runtime trip counts so that the code stays
// small (instruction-cache misses dominated the unrolled version).
constexpr int kListCap = 256;  // (key, j) pairs per list: 2 KB of shared memory

// KM: 0 counts min(#inside, k_max) into cnt_or_off[i]; 1 writes (src, dst) at
// offset cnt_or_off[i]; 2 writes dst at the fixed slot i * k_max and the count
// into cnt_or_off[i] (a compaction pass forms the edge list).
// The listing pass for sources i0 and (if two) i1: n0, n1 = qualifying counts.
template <int KM, int D>
__device__ __forceinline__ void knn_scan2(const float* __restrict__ emb, int i0, int i1, bool two,
                                          const float* cand, int cstride, int cstep, int n_cand,
                                          float r2, int lane, uint64_t* list0, uint64_t* list1,
                                          int& n0, int& n1) {
  const unsigned full = 0xffffffffu, lt_mask = (1u << lane) - 1u;
  float e0[D], e1[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    e0[d] = emb[(int64_t)i0 * D + d];
    e1[d] = two ? emb[(int64_t)i1 * D + d] : 0.f;
  }
  n0 = n1 = 0;
#pragma unroll 1
  for (int j0 = 0; j0 < n_cand; j0 += 32) {
    const int j = j0 + lane;
    bool in0 = false, in1 = false;
    uint32_t k0 = 0, k1 = 0;
    if (j < n_cand) {
      const float* cj = cand + (int64_t)j * cstep;
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float c = cj[d * cstride];
        const float t0 = __fsub_rn(e0[d], c), t1 = __fsub_rn(e1[d], c);
        s0 = __fadd_rn(s0, __fmul_rn(t0, t0));
        s1 = __fadd_rn(s1, __fmul_rn(t1, t1));
      }
      in0 = s0 < r2;
      in1 = two && s1 < r2;
      k0 = __float_as_uint(s0);
      k1 = __float_as_uint(s1);
    }
    const unsigned m0 = __ballot_sync(full, in0), m1 = __ballot_sync(full, in1);
    if (KM != 0) {
      if (in0) {
        const int pos = n0 + __popc(m0 & lt_mask);
        if (pos < kListCap) list0[pos] = (static_cast<uint64_t>(k0) << 32) | static_cast<uint32_t>(j);
      }
      if (in1) {
        const int pos = n1 + __popc(m1 & lt_mask);
        if (pos < kListCap) list1[pos] = (static_cast<uint64_t>(k1) << 32) | static_cast<uint32_t>(j);
      }
    }
    n0 += __popc(m0);
    n1 += __popc(m1);
  }
  __syncwarp();
}

// The selection and output of one listed source; false (nothing written) when
// its list overflowed.
template <int KM>
__device__ __forceinline__ bool knn_emit(int i, int n, const uint64_t* list, int c_lo, int k_max,
                                         int32_t* cnt_or_off, int32_t* __restrict__ src,
                                         int32_t* __restrict__ dst, int lane) {
  const unsigned full = 0xffffffffu, lt_mask = (1u << lane) - 1u;
  if (KM == 0) {
    if (lane == 0) cnt_or_off[i] = min(n, k_max);
    return true;
  }
  if (n > kListCap) return false;
  const int64_t base = KM == 2 ? (int64_t)i * k_max : (int64_t)cnt_or_off[i];
  constexpr int R = kListCap / 32;  // list entries per lane: q = 32 r + lane
  bool keep[R];
#pragma unroll
  for (int r = 0; r < R; ++r) keep[r] = 32 * r + lane < n;
  if (n > k_max) {
    uint64_t mine[R];
    int rank[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      mine[r] = keep[r] ? list[32 * r + lane] : ~0ull;
      rank[r] = 0;
    }
    const int nr = (n + 31) >> 5;  // lanes' entries in use
#pragma unroll 1
    for (int q = 0; q < n; ++q) {
      const uint64_t x = list[q];
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r < nr) rank[r] += x < mine[r];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) keep[r] = keep[r] && rank[r] < k_max;
  }
  int written = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (32 * r >= n) break;
    const unsigned m = __ballot_sync(full, keep[r]);
    if (keep[r]) {
      const int64_t pos = base + written + __popc(m & lt_mask);
      if (KM == 1) src[pos] = i;
      dst[pos] = c_lo + static_cast<int>(static_cast<uint32_t>(list[32 * r + lane]));
    }
    written += __popc(m);
  }
  if (KM == 2 && lane == 0) cnt_or_off[i] = written;
  __syncwarp();
  return true;
}

template <int KM, int DT>
__global__ void __launch_bounds__(kKnnThreads)
k_knn(const float* __restrict__ emb, int D, const int32_t* __restrict__ plane_off, int n_planes,
      float radius, int k_max, int32_t* __restrict__ cnt_or_off, int64_t n_hits,
      int32_t* __restrict__ src, int32_t* __restrict__ dst, int64_t capacity, int* err,
      int split, int stage_floats) {
  // [D][n_cand] within the first stage_floats, then two lists of kListCap (key, j) pairs per warp
  extern __shared__ float cand_s[];
  uint64_t* list_s = reinterpret_cast<uint64_t*>(cand_s + stage_floats);  // per-warp pair lists
  // `split` blocks share the sources of one (event, plane): block `part` takes
  // every split-th group of warps' sources (each stages the candidates itself)
  const int bp = blockIdx.x / split, part = blockIdx.x % split;
  const int b = bp / (n_planes - 1);
  const int p = bp % (n_planes - 1);
  const int32_t* po = plane_off + (int64_t)b * (n_planes + 1);
  const int s_lo = po[p], s_hi = po[p + 1];
  const int c_lo = po[p + 1], c_hi = po[min(p + 3, n_planes)];
  const int n_cand = c_hi - c_lo;
  if (KM == 1 && cnt_or_off[n_hits] > capacity) {
    if (threadIdx.x == 0) set_err(err, DERR_CAPACITY);
    return;
  }
  if (s_hi <= s_lo) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  if (n_cand <= 0) {
    if (KM != 1)
      for (int i = s_lo + part * blockDim.x + threadIdx.x; i < s_hi; i += blockDim.x * split)
        cnt_or_off[i] = 0;
    return;
  }
  constexpr int WPB = kKnnThreads / 32;  // warps per block
  if (s_lo + part * WPB >= s_hi) return;  // no source for this part
  // candidate storage: shared (SoA, stride n_cand) or global (AoS, stride 1)
  const bool staged = n_cand * D <= stage_floats;
  if (staged) {
    for (int t = threadIdx.x; t < n_cand * D; t += blockDim.x) {
      const int j = t / D, d = t - j * D;
      cand_s[d * n_cand + j] = emb[(int64_t)(c_lo + j) * D + d];
    }
    __syncthreads();
  }
  const float* cbase = staged ? cand_s : emb + (int64_t)c_lo * D;
  const int cstride = staged ? n_cand : 1;       // stride between dimensions
  const int cstep = staged ? 1 : D;              // stride between candidates
  const float r2 = __fmul_rn(radius, radius);

  // The general path for one source (any D, candidates anywhere, any count).
  auto general = [&](int i) {
    float ei[kMaxDim];
    for (int d = 0; d < D; ++d) ei[d] = emb[(int64_t)i * D + d];
    // pass A: count the hits inside the radius
    int cnt = 0;
    for (int j0 = 0; j0 < n_cand; j0 += 32) {
      const int j = j0 + lane;
      bool ok = false;
      if (j < n_cand) ok = d2_ordered(ei, cbase + (int64_t)j * cstep, cstride, D) < r2;
      cnt += __popc(__ballot_sync(0xffffffffu, ok));
    }
    if (KM == 0) {
      if (lane == 0) cnt_or_off[i] = min(cnt, k_max);
      return;
    }
    const int64_t base = KM == 2 ? (int64_t)i * k_max : (int64_t)cnt_or_off[i];
    uint32_t kth = 0xffffffffu;  // keep keys < kth, plus `take_eq` keys == kth
    int take_eq = 0;
    if (cnt > k_max) {
      // radix select: largest v with #{key < v} < k_max is the k_max-th smallest key
      uint32_t prefix = 0;
      for (int bit = 31; bit >= 0; --bit) {
        const uint32_t trial = prefix | (1u << bit);
        int c = 0;
        for (int j0 = 0; j0 < n_cand; j0 += 32) {
          const int j = j0 + lane;
          bool lt = false;
          if (j < n_cand) {
            const float d2 = d2_ordered(ei, cbase + (int64_t)j * cstep, cstride, D);
            lt = d2 < r2 && __float_as_uint(d2) < trial;
          }
          c += __popc(__ballot_sync(0xffffffffu, lt));
        }
        if (c < k_max) prefix = trial;
      }
      kth = prefix;
      int less = 0;
      for (int j0 = 0; j0 < n_cand; j0 += 32) {
        const int j = j0 + lane;
        bool lt = false;
        if (j < n_cand) {
          const float d2 = d2_ordered(ei, cbase + (int64_t)j * cstep, cstride, D);
          lt = d2 < r2 && __float_as_uint(d2) < kth;
        }
        less += __popc(__ballot_sync(0xffffffffu, lt));
      }
      take_eq = k_max - less;
    }
    // pass B: write the kept edges in ascending j
    int written = 0, eq_seen = 0;
    for (int j0 = 0; j0 < n_cand; j0 += 32) {
      const int j = j0 + lane;
      bool in = false, eq = false;
      if (j < n_cand) {
        const float d2 = d2_ordered(ei, cbase + (int64_t)j * cstep, cstride, D);
        if (d2 < r2) {
          const uint32_t key = __float_as_uint(d2);
          in = key < kth;
          eq = key == kth;
        }
      }
      const unsigned eqm = __ballot_sync(0xffffffffu, eq);
      if (eq) in = eq_seen + __popc(eqm & lt_mask) < take_eq;
      eq_seen += __popc(eqm);
      const unsigned inm = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int64_t pos = base + written + __popc(inm & lt_mask);
        if (KM == 1) src[pos] = i;
        dst[pos] = c_lo + j;
      }
      written += __popc(inm);
    }
    if (KM == 2 && lane == 0) cnt_or_off[i] = written;
  };
  // Sources in pairs per warp: i and i + WPB * split
  const int stride = WPB * split;
  for (int i = s_lo + part * WPB + warp; i < s_hi; i += 2 * stride) {
    const int i2 = i + stride;
    const bool two = i2 < s_hi;
    bool done0 = false, done1 = !two;
    if constexpr (DT > 0) {
      uint64_t* l0 = list_s + 2 * kListCap * warp;
      int n0, n1;
      knn_scan2<KM, DT>(emb, i, i2, two, cbase, cstride, cstep, n_cand, r2, lane, l0,
                        l0 + kListCap, n0, n1);
      done0 = knn_emit<KM>(i, n0, l0, c_lo, k_max, cnt_or_off, src, dst, lane);
      if (two) done1 = knn_emit<KM>(i2, n1, l0 + kListCap, c_lo, k_max, cnt_or_off, src, dst, lane);
    }
    if (!done0) general(i);
    if (!done1) general(i2);
  }
}

// Fixed-stride slots (k_max per source) -> the compact edge list at the
// scanned offsets, a warp per source.  Nothing is written when the edges do
// not fit (ETX_ERR_CAPACITY).
__global__ void k_knn_compact(const int32_t* __restrict__ slots, int k_max,
                              const int32_t* __restrict__ off, int64_t n_hits,
                              int32_t* __restrict__ src, int32_t* __restrict__ dst,
                              int64_t capacity, int* err) {
  if (off[n_hits] > capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_err(err, DERR_CAPACITY);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_hits;
       i += warps) {
    const int o = off[i], n = off[i + 1] - o;
    for (int t = lane; t < n; t += 32) {
      dst[o + t] = slots[i * k_max + t];
      src[o + t] = (int32_t)i;
    }
  }
}

__global__ void k_edge_offsets(const int32_t* __restrict__ off, const int32_t* __restrict__ hoff,
                               int32_t n_events, int n_hits, int32_t* __restrict__ edge_offsets) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b <= n_events) edge_offsets[b] = off[min(max(hoff[b], 0), n_hits)];
}

}  // namespace

cudaError_t launch_build_graph(etx_ctx* ctx, const float* emb, const int8_t* plane,
                               const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                               float radius, int32_t k_max, int32_t* src, int32_t* dst,
                               int64_t edge_capacity, int32_t* edge_offsets, cudaStream_t s) {
  const int P = ctx->cfg.n_planes;
  const int D = ctx->cfg.emb_widths[ctx->cfg.emb_depth];
  const int64_t nchk = (n_hits > n_events ? n_hits : n_events + 1);
  launch(ctx, "graph_check_hits", k_check_hits, (unsigned)((nchk + 255) / 256), 256, 0, s, plane,
         hit_offsets, n_events, n_hits, P, ctx->d_err);
  const int64_t nb = (int64_t)n_events * (P + 1);
  if (nb > 0)
    launch(ctx, "graph_plane_bins", k_plane_bins, (unsigned)((nb + 255) / 256), 256, 0, s, plane,
           hit_offsets, n_events, (int)n_hits, P, ctx->plane_off);
  int32_t* cnt = ctx->hit_cnt;  // counts, then (in place) offsets; [n_hits + 1]
  const int split = ctx->knn_split;
  const int stage = ctx->knn_stage;  // a multiple of 4 in [1024, kStageMaxFloats]
  const unsigned blocks = (unsigned)n_events * (unsigned)(P - 1) * (unsigned)split;
  const size_t smem = (size_t)stage * sizeof(float) + kKnnThreads / 32 * 2 * kListCap * sizeof(uint64_t);
  // hits of the last plane get no block: start from zero counts
  cudaError_t e0 = cudaMemsetAsync(cnt, 0, (size_t)(n_hits + 1) * sizeof(int32_t), s);
  if (e0 != cudaSuccess) return e0;
  auto knn = [&](auto kernel, const char* name, int32_t* sp, int32_t* dp, int64_t cap) {
    launch(ctx, name, kernel, blocks, kKnnThreads, smem, s, emb, D, (const int32_t*)ctx->plane_off,
           P, radius, k_max, cnt, n_hits, sp, dp, cap, ctx->d_err, split, stage);
  };
  // One distance pass into fixed-stride slots when the context's in-edge
  // permutation (rebuilt by every consumer of the edge index) can hold them;
  // otherwise count, scan, then emit at the offsets.
  const int64_t n_slots = n_hits * (int64_t)k_max;
  const bool single = n_slots <= ctx->cfg.max_edges;
  if (single) {
    int32_t* slots = ctx->perm_in;
    ctx->fwd_saved = false;  // the slots overwrite the edge index a backward pass would read
    if (n_hits > 0 && blocks > 0) {
      if (D == 8) knn(k_knn<2, 8>, "graph_knn_slots", nullptr, slots, n_slots);
      else if (D == 4) knn(k_knn<2, 4>, "graph_knn_slots", nullptr, slots, n_slots);
      else knn(k_knn<2, 0>, "graph_knn_slots", nullptr, slots, n_slots);
    }
    cudaError_t e = exclusive_scan(ctx, cnt, cnt, n_hits, s);
    if (e != cudaSuccess) return e;
    if (n_hits > 0) {
      const int64_t wanted = (n_hits + 7) / 8;  // 8 warps per block
      const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(wanted, (int64_t)ctx->n_sms * 16));
      launch(ctx, "graph_knn_compact", k_knn_compact, grid, 256, 0, s, (const int32_t*)slots, k_max,
             (const int32_t*)cnt, n_hits, src, dst, edge_capacity, ctx->d_err);
    }
  } else {
    if (n_hits > 0 && blocks > 0) {
      if (D == 8) knn(k_knn<0, 8>, "graph_knn_count", nullptr, nullptr, 0);
      else if (D == 4) knn(k_knn<0, 4>, "graph_knn_count", nullptr, nullptr, 0);
      else knn(k_knn<0, 0>, "graph_knn_count", nullptr, nullptr, 0);
    }
    cudaError_t e = exclusive_scan(ctx, cnt, cnt, n_hits, s);
    if (e != cudaSuccess) return e;
    if (n_hits > 0 && blocks > 0) {
      if (D == 8) knn(k_knn<1, 8>, "graph_knn_emit", src, dst, edge_capacity);
      else if (D == 4) knn(k_knn<1, 4>, "graph_knn_emit", src, dst, edge_capacity);
      else knn(k_knn<1, 0>, "graph_knn_emit", src, dst, edge_capacity);
    }
  }
  launch(ctx, "graph_edge_offsets", k_edge_offsets, (unsigned)((n_events + 1 + 255) / 256), 256, 0,
         s, cnt, hit_offsets, n_events, (int)n_hits, edge_offsets);
  return cudaGetLastError();
}

cudaError_t launch_plane_bins(etx_ctx* ctx, const int8_t* plane, const int32_t* hit_offsets,
                              int32_t n_events, int64_t n_hits, cudaStream_t s) {
  const int P = ctx->cfg.n_planes;
  const int64_t nchk = (n_hits > n_events ? n_hits : n_events + 1);
  launch(ctx, "graph_check_hits", k_check_hits, (unsigned)((nchk + 255) / 256), 256, 0, s, plane,
         hit_offsets, n_events, n_hits, P, ctx->d_err);
  const int64_t nb = (int64_t)n_events * (P + 1);
  if (nb > 0)
    launch(ctx, "graph_plane_bins", k_plane_bins, (unsigned)((nb + 255) / 256), 256, 0, s, plane,
           hit_offsets, n_events, (int)n_hits, P, ctx->plane_off);
  return cudaGetLastError();
}

cudaError_t knn_set_smem_attr() {
  const int smem = (int)(kStageMaxFloats * sizeof(float) + kKnnThreads / 32 * 2 * kListCap * sizeof(uint64_t));
  const void* ks[] = {(const void*)k_knn<0, 0>, (const void*)k_knn<1, 0>, (const void*)k_knn<2, 0>,
                      (const void*)k_knn<0, 4>, (const void*)k_knn<1, 4>, (const void*)k_knn<2, 4>,
                      (const void*)k_knn<0, 8>, (const void*)k_knn<1, 8>, (const void*)k_knn<2, 8>};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace etx
