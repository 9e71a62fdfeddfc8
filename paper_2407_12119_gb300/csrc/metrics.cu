// Track-finding performance against truth (paper Sec. 6, Table 1).
//
// One block per event.  Global scratch (six int32 arrays of n_hits, used at
// the event's own hit range, so blocks never touch each other's slots):
//   tsize  hits per label value        pcnt   hits per particle id
//   pstart exclusive scan of pcnt      pfill  fill counters
//   plab   labels of each particle's hits, grouped by particle
//   tmatch 1 if the track (label value) has a matching particle
// A track is a set of hits sharing a label; it counts if it has at least
// min_hits hits.  A particle counts (reconstructible, Sec. 3) if it has at
// least min_hits hits.  A (track, particle) pair is a matching candidate when
// match_num / match_den of the track's hits belong to the particle; with a
// fraction above one half a track has at most one such particle.  The
// candidates are found from the particle side: each thread owns particles
// and walks the distinct labels of a particle's hits in ascending order, so
// the FP64 sums are formed in a fixed order.  Block and batch sums use fixed
// reduction trees: the same inputs give the same bits.
#include "etx_internal.cuh"

namespace etx {
namespace {

constexpr int kMT = 256;
constexpr int kCounts = 6;  // particles, matched particles, candidates, candidate particles,
                            // tracks, unmatched tracks

struct EventTally {
  long long c[kCounts];
  double s[2];  // sums over candidates of matched/particle hits, matched/track hits
};
static_assert(sizeof(EventTally) == 64, "tally layout");

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read by the previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = red[0];
  for (int w = 1; w < kMT / 32; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(kMT) k_track_tally(
    const int32_t* __restrict__ labels, const int32_t* __restrict__ pid,
    const int32_t* __restrict__ hoff, int64_t n_hits, int32_t min_hits, int32_t num, int32_t den,
    int32_t* __restrict__ ws, EventTally* __restrict__ tally, int* err) {
  __shared__ long long red_i[kMT / 32];
  __shared__ double red_d[kMT / 32];
  __shared__ int scan_w[kMT / 32];
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t h0 = hoff[b], h1 = hoff[b + 1];
  if (h0 < 0 || h1 < h0 || h1 > n_hits) {  // uniform over the block
    if (t == 0) set_err(err, DERR_RANGE);
    if (t < kCounts) tally[b].c[t] = 0;
    if (t < 2) tally[b].s[t] = 0.0;
    return;
  }
  const int n = (int)(h1 - h0);
  int* tsize = ws + h0;
  int* pcnt = ws + n_hits + h0;
  int* pstart = ws + 2 * n_hits + h0;
  int* pfill = ws + 3 * n_hits + h0;
  int* plab = ws + 4 * n_hits + h0;
  int* tmatch = ws + 5 * n_hits + h0;
  const int32_t* lab = labels + h0;
  const int32_t* pp = pid + h0;

  for (int i = t; i < n; i += kMT) tsize[i] = pcnt[i] = pfill[i] = tmatch[i] = 0;
  __syncthreads();
  for (int i = t; i < n; i += kMT) {
    const int l = lab[i], p = pp[i];
    if (l < 0 || l >= n || p < -1 || p >= n) {
      set_err(err, DERR_RANGE);
      continue;
    }
    atomicAdd(tsize + l, 1);
    if (p >= 0) atomicAdd(pcnt + p, 1);
  }
  __syncthreads();
  {  // exclusive scan of pcnt: a contiguous chunk per thread
    const int per = (n + kMT - 1) / kMT;
    const int lo = min(n, t * per), hi = min(n, lo + per);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += pcnt[i];
    int x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((t & 31) >= o) x += y;
    }
    if ((t & 31) == 31) scan_w[t >> 5] = x;
    __syncthreads();
    int run = x - sum;
    for (int w = 0; w < (t >> 5); ++w) run += scan_w[w];
    for (int i = lo; i < hi; ++i) {
      pstart[i] = run;
      run += pcnt[i];
    }
  }
  __syncthreads();
  for (int i = t; i < n; i += kMT) {
    const int l = lab[i], p = pp[i];
    if (l < 0 || l >= n || p < 0 || p >= n) continue;
    plab[pstart[p] + atomicAdd(pfill + p, 1)] = l;
  }
  __syncthreads();

  long long n_part = 0, n_mpart = 0, n_cand = 0, n_cpart = 0;
  double s_eff = 0.0, s_pur = 0.0;
  for (int p = t; p < n; p += kMT) {
    const int m = pcnt[p];
    if (m == 0) continue;
    const int* L = plab + pstart[p];
    bool any = false;
    int prev = -1;
    for (;;) {  // distinct labels of the particle's hits, ascending
      int cur = INT32_MAX, c = 0;
      for (int k = 0; k < m; ++k) {
        const int l = L[k];
        if (l > prev && l < cur) {
          cur = l;
          c = 1;
        } else if (l == cur) {
          ++c;
        }
      }
      if (cur == INT32_MAX) break;
      const int sz = tsize[cur];
      if (sz >= min_hits && (long long)c * den >= (long long)num * sz) {
        any = true;
        ++n_cand;
        s_eff += (double)c / (double)m;
        s_pur += (double)c / (double)sz;
        tmatch[cur] = 1;
      }
      prev = cur;
    }
    if (m >= min_hits) {
      ++n_part;
      if (any) ++n_mpart;
    }
    if (any) ++n_cpart;
  }
  __syncthreads();
  long long n_trk = 0, n_unm = 0;
  for (int l = t; l < n; l += kMT) {
    if (tsize[l] >= min_hits) {
      ++n_trk;
      if (!tmatch[l]) ++n_unm;
    }
  }
  const long long c[kCounts] = {n_part, n_mpart, n_cand, n_cpart, n_trk, n_unm};
#pragma unroll
  for (int k = 0; k < kCounts; ++k) {
    const long long v = block_sum(c[k], red_i);
    if (t == 0) tally[b].c[k] = v;
  }
  const double e = block_sum(s_eff, red_d);
  const double u = block_sum(s_pur, red_d);
  if (t == 0) {
    tally[b].s[0] = e;
    tally[b].s[1] = u;
  }
}

__device__ __forceinline__ double ratio(double a, double b) {
  return b > 0.0 ? a / b : __longlong_as_double(0x7ff8000000000000LL);  // NaN for 0/0
}

// Batch totals in a fixed order and the Table 1 ratios.
__global__ void __launch_bounds__(kMT) k_tally_total(const EventTally* __restrict__ tally,
                                                     int32_t n_events, int64_t* __restrict__ counts,
                                                     double* __restrict__ values) {
  __shared__ long long red_i[kMT / 32];
  __shared__ double red_d[kMT / 32];
  const int t = threadIdx.x;
  long long c[kCounts] = {0, 0, 0, 0, 0, 0};
  double s0 = 0.0, s1 = 0.0;
  for (int b = t; b < n_events; b += kMT) {
#pragma unroll
    for (int k = 0; k < kCounts; ++k) c[k] += tally[b].c[k];
    s0 += tally[b].s[0];
    s1 += tally[b].s[1];
  }
  long long tot[kCounts];
#pragma unroll
  for (int k = 0; k < kCounts; ++k) tot[k] = block_sum(c[k], red_i);
  const double e = block_sum(s0, red_d);
  const double u = block_sum(s1, red_d);
  if (t == 0) {
    for (int k = 0; k < kCounts; ++k) counts[k] = tot[k];
    const double part = (double)tot[0], mpart = (double)tot[1], cand = (double)tot[2];
    const double cpart = (double)tot[3], trk = (double)tot[4], unm = (double)tot[5];
    values[0] = e;
    values[1] = u;
    values[2] = ratio(mpart, part);          // efficiency
    values[3] = ratio(cand - cpart, cand);   // clone rate
    values[4] = ratio(unm, trk);             // fake rate
    values[5] = ratio(e, cand);              // hit efficiency
    values[6] = ratio(u, cand);              // hit purity
  }
}

}  // namespace

size_t track_metrics_workspace(int32_t n_events, int64_t n_hits) {
  return (size_t)n_events * sizeof(EventTally) + (size_t)n_hits * 6 * sizeof(int32_t);
}

cudaError_t launch_track_metrics(etx_ctx* ctx, const int32_t* labels, const int32_t* particle_id,
                                 const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                                 int32_t min_hits, int32_t num, int32_t den, void* workspace,
                                 int64_t* counts, double* values, cudaStream_t s) {
  EventTally* tally = static_cast<EventTally*>(workspace);
  int32_t* ws = reinterpret_cast<int32_t*>(tally + n_events);
  if (n_events > 0)
    launch(ctx, "metrics_tally", k_track_tally, (unsigned)n_events, kMT, 0, s, labels, particle_id,
           hit_offsets, n_hits, min_hits, num, den, ws, tally, ctx->d_err);
  launch(ctx, "metrics_total", k_tally_total, 1, kMT, 0, s, (const EventTally*)tally, n_events,
         counts, values);
  return cudaGetLastError();
}

}  // namespace etx
