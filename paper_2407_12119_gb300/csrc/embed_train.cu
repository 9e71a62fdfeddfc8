// Training of the hit embedding (paper Sec. 5.1, Eq. 2-3): the training set
// of (query, partner) pairs and the pairwise hinge loss.
//
// Training set, per query q (a hit of a particle with at least min_hits hits;
// the caller removes noise hits first) on plane p, partners on planes p+1
// and p+2 of its event:
//   * hard negatives: the graph rule itself (the k-NN graph build with the
//     training radius and k_max), whose per-source lists come out sorted;
//   * one random partner: the (rand[q] mod c)-th of the c hits on p+1, p+2
//     (they are contiguous because hits are plane-sorted);
//   * the genuine edge: q -> the next hit of q's particle, if on p+1 or p+2.
// The union is written per query in ascending partner order, a pair flagged
// genuine iff the partner is the next hit of q's particle.  Two passes (count,
// emit) around an exclusive scan give every query its output slice.
//
// Loss (Eq. 2-3): L = L_fake + w * L_genuine, L_genuine = mean d2 over the
// genuine pairs, L_fake = mean max(0, m - d2) over the fake pairs; the
// gradient with respect to the embedding is gathered per hit over its pairs
// (as query, then as partner, each in ascending pair index): no atomics, a
// fixed summation order, so a step is bit-reproducible.
#include <algorithm>

#include "etx_internal.cuh"

namespace etx {
namespace {

constexpr int kPT = 256;

// Per event: query flags and next hit of each hit's particle.  Scratch (event
// slice of n_hits-long arrays): pcnt, pstart, pfill, plist.
__global__ void __launch_bounds__(kPT) k_pair_prep(const int32_t* __restrict__ pid,
                                                   const int32_t* __restrict__ hoff, int64_t n_hits,
                                                   int32_t min_hits, int32_t* __restrict__ scratch,
                                                   int32_t* __restrict__ is_q,
                                                   int32_t* __restrict__ nxt, int* err) {
  __shared__ int scan_w[kPT / 32];
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t h0 = hoff[b], h1 = hoff[b + 1];
  if (h0 < 0 || h1 < h0 || h1 > n_hits) {  // uniform over the block; flagged by the graph check too
    if (t == 0) set_err(err, DERR_RANGE);
    return;
  }
  const int n = (int)(h1 - h0);
  int* pcnt = scratch + h0;
  int* pstart = scratch + n_hits + h0;
  int* pfill = scratch + 2 * n_hits + h0;
  int* plist = scratch + 3 * n_hits + h0;
  const int32_t* pp = pid + h0;
  for (int i = t; i < n; i += kPT) {
    pcnt[i] = pfill[i] = 0;
    is_q[h0 + i] = 0;
    nxt[h0 + i] = -1;
  }
  __syncthreads();
  for (int i = t; i < n; i += kPT) {
    const int p = pp[i];
    if (p < 0 || p >= n) {
      set_err(err, DERR_RANGE);  // noise must be removed; ids are event-local
      continue;
    }
    atomicAdd(pcnt + p, 1);
  }
  __syncthreads();
  {  // exclusive scan of pcnt, a contiguous chunk per thread
    const int per = (n + kPT - 1) / kPT;
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
  for (int i = t; i < n; i += kPT) {
    const int p = pp[i];
    if (p < 0 || p >= n) continue;
    plist[pstart[p] + atomicAdd(pfill + p, 1)] = i;
  }
  __syncthreads();
  for (int p = t; p < n; p += kPT) {
    const int m = pcnt[p];
    if (m == 0) continue;
    int* L = plist + pstart[p];
    for (int k = 1; k < m; ++k) {  // insertion sort: hit order = plane order
      const int v = L[k];
      int j = k - 1;
      while (j >= 0 && L[j] > v) {
        L[j + 1] = L[j];
        --j;
      }
      L[j + 1] = v;
    }
    const int q = m >= min_hits ? 1 : 0;
    for (int k = 0; k < m; ++k) {
      is_q[h0 + L[k]] = q;
      nxt[h0 + L[k]] = k + 1 < m ? (int)h0 + L[k + 1] : -1;
    }
  }
}

__device__ __forceinline__ int event_of(const int32_t* __restrict__ hoff, int n_events, int64_t i) {
  int lo = 0, hi = n_events;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (hoff[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

struct PairCtx {
  const int32_t* hoff;
  const int8_t* plane;
  const int32_t* plane_off;  // [n_events][P + 1], global hit indices
  const int32_t* knn_off;    // [n_hits + 1] per-source slice of the k-NN lists
  const int32_t* kdst;
  int64_t kcap;              // entries of kdst actually written
  const uint32_t* rand;
  const int32_t* is_q;
  const int32_t* nxt;
  int n_events, n_planes;
};

// The random and the genuine partner of query q (-1 if none).
__device__ __forceinline__ void extra_partners(const PairCtx& c, int64_t q, int* r, int* g) {
  const int b = event_of(c.hoff, c.n_events, q);
  const int p = c.plane[q];
  if (p < 0 || p >= c.n_planes) {  // flagged by the graph build's input check
    *r = *g = -1;
    return;
  }
  const int32_t* po = c.plane_off + (int64_t)b * (c.n_planes + 1);
  const int lo = po[p + 1];
  const int hi = po[min(p + 3, c.n_planes)];
  *r = hi > lo ? lo + (int)(c.rand[q] % (uint32_t)(hi - lo)) : -1;
  const int nx = c.nxt[q];
  *g = (nx >= 0 && c.plane[nx] - p <= 2) ? nx : -1;
}

__device__ __forceinline__ bool in_sorted(const int32_t* a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < n && a[lo] == v;
}

__device__ __forceinline__ void knn_slice(const PairCtx& c, int64_t q, int64_t* lo, int* n) {
  const int64_t a = min((int64_t)c.knn_off[q], c.kcap), b = min((int64_t)c.knn_off[q + 1], c.kcap);
  *lo = a;
  *n = (int)(b - a);
}

__global__ void k_pair_count(PairCtx c, int64_t n_hits, int32_t* __restrict__ cnt) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_hits;
       q += (int64_t)gridDim.x * blockDim.x) {
    if (!c.is_q[q]) {
      cnt[q] = 0;
      continue;
    }
    int64_t klo;
    int kn;
    knn_slice(c, q, &klo, &kn);
    int r, g;
    extra_partners(c, q, &r, &g);
    const int32_t* K = c.kdst + klo;
    int n = kn;
    if (r >= 0 && !in_sorted(K, kn, r)) ++n;
    if (g >= 0 && g != r && !in_sorted(K, kn, g)) ++n;
    cnt[q] = n;
  }
}

__global__ void k_pair_emit(PairCtx c, int64_t n_hits, const int32_t* __restrict__ off,
                            int64_t capacity, int32_t* __restrict__ pq, int32_t* __restrict__ pa,
                            uint8_t* __restrict__ pg, int* err) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_hits;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o0 = off[q], o1 = off[q + 1];
    if (o1 == o0) continue;
    if (o1 > capacity) {
      set_err(err, DERR_CAPACITY);
      continue;
    }
    int64_t klo;
    int kn;
    knn_slice(c, q, &klo, &kn);
    int r, g;
    extra_partners(c, q, &r, &g);
    // the (at most two) extra partners in ascending order, duplicates dropped
    int ex[2], ne = 0;
    const int32_t* K = c.kdst + klo;
    if (r >= 0 && !in_sorted(K, kn, r)) ex[ne++] = r;
    if (g >= 0 && g != r && !in_sorted(K, kn, g)) ex[ne++] = g;
    if (ne == 2 && ex[0] > ex[1]) {
      const int tmp = ex[0];
      ex[0] = ex[1];
      ex[1] = tmp;
    }
    const int nx = c.nxt[q];
    int64_t o = o0;
    int i = 0, e = 0;
    while ((i < kn || e < ne) && o < o1) {
      int v;
      if (e >= ne || (i < kn && K[i] < ex[e])) v = K[i++];
      else v = ex[e++];
      pq[o] = (int32_t)q;
      pa[o] = v;
      pg[o] = v == nx ? 1 : 0;
      ++o;
    }
  }
}

__global__ void k_pair_total(const int32_t* __restrict__ off, int64_t n_hits, int64_t capacity,
                             int32_t* __restrict__ n_pairs) {
  // on overflow (flagged by the emit pass) no pair is exposed
  const int64_t tot = off[n_hits];
  *n_pairs = tot <= capacity ? (int32_t)tot : 0;
}

// ---- hinge loss -------------------------------------------------------------
__global__ void k_hinge_count(const uint8_t* __restrict__ pg, const int32_t* __restrict__ n_pairs,
                              unsigned long long* __restrict__ counts) {
  __shared__ unsigned long long red[kPT / 32];
  const int64_t n = *n_pairs;
  unsigned long long g = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    g += pg[i] ? 1ull : 0ull;
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kPT / 32; ++w) s += red[w];
    atomicAdd(counts, s);
  }
}

// Per pair p: the gradient coefficient c_p of d2 in L (w / n_genuine for a
// genuine pair, -1 / n_fake for a fake pair inside the margin, else 0; 0 for a
// pair with an index out of range, which is reported), and this block's sums
// of d2 over the genuine pairs and of (margin - d2)+ over the fake ones
// (FP64, a fixed reduction order) in part[2 block], part[2 block + 1].
template <int D>
__global__ void __launch_bounds__(kPT) k_hinge_pairs(const float* __restrict__ emb, int dim,
                                                     const int32_t* __restrict__ pq,
                                                     const int32_t* __restrict__ pa,
                                                     const uint8_t* __restrict__ pg,
                                                     const int32_t* __restrict__ n_pairs,
                                                     const unsigned long long* __restrict__ counts,
                                                     float margin, float w_gen,
                                                     float* __restrict__ coef,
                                                     double* __restrict__ part, int64_t n_hits,
                                                     int* err) {
  __shared__ double red[2][kPT / 32];
  const int Dn = D > 0 ? D : dim;
  const int64_t n = *n_pairs;
  const unsigned long long ng = counts[0], nf = (unsigned long long)n - counts[0];
  const float cg = ng ? (float)((double)w_gen / (double)ng) : 0.f;
  const float cf = nf ? (float)(-1.0 / (double)nf) : 0.f;
  double sg = 0.0, sf = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = pq[i], a = pa[i];
    if (q < 0 || q >= n_hits || a < 0 || a >= n_hits) {
      set_err(err, DERR_RANGE);
      coef[i] = 0.f;
      continue;
    }
    const float* eq = emb + q * Dn;
    const float* ea = emb + a * Dn;
    float d2 = 0.f;
    for (int k = 0; k < Dn; ++k) {
      const float t = eq[k] - ea[k];
      d2 += t * t;
    }
    float c;
    if (pg[i]) {
      sg += d2;
      c = cg;
    } else {
      const bool active = d2 < margin;
      sf += active ? (double)(margin - d2) : 0.0;
      c = active ? cf : 0.f;
    }
    coef[i] = c;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sg += __shfl_xor_sync(0xffffffffu, sg, o);
    sf += __shfl_xor_sync(0xffffffffu, sf, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sg;
    red[1][threadIdx.x >> 5] = sf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kPT / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// dL/d emb of hit h (a thread per hit): 2 c_p (e_h - e_a) over the pairs p
// where h is the query, then -2 c_p (e_q - e_h) over those where h is the
// partner, each list in ascending pair index (the key indices), so the sum
// has a fixed order.  Every row [0, n_hits) is written.
template <int D>
__global__ void __launch_bounds__(kPT) k_hinge_grad(const float* __restrict__ emb, int dim,
                                                    const int32_t* __restrict__ pq,
                                                    const int32_t* __restrict__ pa,
                                                    const float* __restrict__ coef,
                                                    const int32_t* __restrict__ off_q,
                                                    const int32_t* __restrict__ perm_q,
                                                    const int32_t* __restrict__ off_a,
                                                    const int32_t* __restrict__ perm_a,
                                                    int64_t n_hits, float* __restrict__ d_emb) {
  const int Dn = D > 0 ? D : dim;
  constexpr int DM = D > 0 ? D : 16;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_hits;
       h += (int64_t)gridDim.x * blockDim.x) {
    float eh[DM], acc[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) {
      eh[k] = k < Dn ? emb[h * Dn + k] : 0.f;
      acc[k] = 0.f;
    }
    for (int t = off_q[h]; t < off_q[h + 1]; ++t) {
      const int p = perm_q[t];
      const float c = coef[p];
      if (c == 0.f) continue;
      const float* ea = emb + (int64_t)pa[p] * Dn;
#pragma unroll
      for (int k = 0; k < DM; ++k)
        if (k < Dn) acc[k] += 2.f * c * (eh[k] - ea[k]);
    }
    for (int t = off_a[h]; t < off_a[h + 1]; ++t) {
      const int p = perm_a[t];
      const float c = coef[p];
      if (c == 0.f) continue;
      const float* eq = emb + (int64_t)pq[p] * Dn;
#pragma unroll
      for (int k = 0; k < DM; ++k)
        if (k < Dn) acc[k] -= 2.f * c * (eq[k] - eh[k]);
    }
#pragma unroll
    for (int k = 0; k < DM; ++k)
      if (k < Dn) d_emb[h * Dn + k] = acc[k];
  }
}

// The pair count the other kernels use: *n_pairs, or 0 (and ETX_ERR_CAPACITY)
// when it lies outside [0, capacity].
__global__ void k_hinge_clamp(const int32_t* __restrict__ n_pairs, int64_t capacity,
                              int32_t* __restrict__ n_eff, int* err) {
  const int32_t n = *n_pairs;
  const bool ok = n >= 0 && (int64_t)n <= capacity;
  if (!ok) set_err(err, DERR_CAPACITY);
  *n_eff = ok ? n : 0;
}

// The blocks' sums added in a fixed order (thread t: blocks t, t + kPT, ...;
// then a fixed tree over the threads), then the loss.  One block of kPT.
__global__ void __launch_bounds__(kPT) k_hinge_final(const double* __restrict__ part, int n_part,
                                                     const unsigned long long* __restrict__ counts,
                                                     const int32_t* __restrict__ n_pairs,
                                                     float w_gen, float* __restrict__ loss) {
  __shared__ double red[2][kPT / 32];
  double sg = 0.0, sf = 0.0;
  for (int b = threadIdx.x; b < n_part; b += kPT) {
    sg += part[2 * b];
    sf += part[2 * b + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sg += __shfl_xor_sync(0xffffffffu, sg, o);
    sf += __shfl_xor_sync(0xffffffffu, sf, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sg;
    red[1][threadIdx.x >> 5] = sf;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  sg = sf = 0.0;
  for (int w = 0; w < kPT / 32; ++w) {
    sg += red[0][w];
    sf += red[1][w];
  }
  const unsigned long long ng = counts[0], nf = (unsigned long long)*n_pairs - counts[0];
  const double lg = ng ? sg / (double)ng : 0.0;
  const double lf = nf ? sf / (double)nf : 0.0;
  loss[0] = (float)(lf + (double)w_gen * lg);
  loss[1] = (float)lg;
  loss[2] = (float)lf;
}

}  // namespace

size_t embedding_pairs_workspace(int32_t n_events, int64_t n_hits, int32_t k_max) {
  // k-NN src, dst [n_hits * k_max], edge offsets [n_events + 1], prep scratch
  // [4 n_hits], is_q, nxt [n_hits], pair counts / offsets [n_hits + 1]
  const int64_t ints = 2 * n_hits * (int64_t)k_max + (n_events + 1) + 6 * n_hits + (n_hits + 1);
  return (size_t)ints * sizeof(int32_t);
}

cudaError_t launch_embedding_pairs(etx_ctx* ctx, const float* emb, const int8_t* plane,
                                   const int32_t* particle_id, const int32_t* hit_offsets,
                                   int32_t n_events, int64_t n_hits, float radius, int32_t k_max,
                                   const uint32_t* rand, int32_t min_hits, void* workspace,
                                   int32_t* pq, int32_t* pa, uint8_t* pg, int64_t capacity,
                                   int32_t* n_pairs, cudaStream_t s) {
  int32_t* w = static_cast<int32_t*>(workspace);
  const int64_t kcap = n_hits * (int64_t)k_max;
  int32_t* ksrc = w;
  int32_t* kdst = ksrc + kcap;
  int32_t* keoff = kdst + kcap;
  int32_t* prep = keoff + (n_events + 1);
  int32_t* is_q = prep + 4 * n_hits;
  int32_t* nxt = is_q + n_hits;
  int32_t* cnt = nxt + n_hits;  // [n_hits + 1]: counts, then offsets
  cudaError_t e = launch_build_graph(ctx, emb, plane, hit_offsets, n_events, n_hits, radius, k_max,
                                     ksrc, kdst, kcap, keoff, s);
  if (e != cudaSuccess) return e;
  if (n_events > 0)
    launch(ctx, "embtrain_prep", k_pair_prep, (unsigned)n_events, kPT, 0, s, particle_id,
           hit_offsets, n_hits, min_hits, prep, is_q, nxt, ctx->d_err);
  PairCtx c{hit_offsets, plane, ctx->plane_off, ctx->hit_cnt, kdst, kcap, rand, is_q, nxt,
            n_events, ctx->cfg.n_planes};
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_hits + 255) / 256,
                                                                         (int64_t)ctx->n_sms * 8));
  if (n_hits > 0) launch(ctx, "embtrain_pair_count", k_pair_count, grid, 256, 0, s, c, n_hits, cnt);
  e = exclusive_scan(ctx, cnt, cnt, n_hits, s);
  if (e != cudaSuccess) return e;
  if (n_hits > 0)
    launch(ctx, "embtrain_pair_emit", k_pair_emit, grid, 256, 0, s, c, n_hits,
           (const int32_t*)cnt, capacity, pq, pa, pg, ctx->d_err);
  launch(ctx, "embtrain_pair_total", k_pair_total, 1, 1, 0, s, (const int32_t*)cnt, n_hits,
         capacity, n_pairs);
  return cudaGetLastError();
}

namespace {
constexpr int kHingeMaxBlocks = 2048;  // per-block loss sums in the workspace

struct HingeWs {
  double* part;                 // [2 kHingeMaxBlocks]
  unsigned long long* counts;   // [2]
  int32_t* n_eff;               // the pair count in use
  float* coef;                  // [cap]
  int32_t *cnt, *off_q, *off_a; // [n_hits + 1] each
  int32_t *perm_q, *perm_a;     // [cap] each
  size_t bytes;
};

HingeWs hinge_ws(void* base, int64_t n_hits, int64_t cap) {
  HingeWs w{};
  uint8_t* b = static_cast<uint8_t*>(base);
  size_t o = 0;
  auto take = [&](size_t n) {
    uint8_t* r = b ? b + o : nullptr;
    o += (n + 15) & ~static_cast<size_t>(15);
    return r;
  };
  w.part = reinterpret_cast<double*>(take(2 * kHingeMaxBlocks * sizeof(double)));
  w.counts = reinterpret_cast<unsigned long long*>(take(2 * sizeof(unsigned long long)));
  w.n_eff = reinterpret_cast<int32_t*>(take(sizeof(int32_t)));
  w.coef = reinterpret_cast<float*>(take((size_t)cap * sizeof(float)));
  w.cnt = reinterpret_cast<int32_t*>(take((size_t)(n_hits + 1) * sizeof(int32_t)));
  w.off_q = reinterpret_cast<int32_t*>(take((size_t)(n_hits + 1) * sizeof(int32_t)));
  w.off_a = reinterpret_cast<int32_t*>(take((size_t)(n_hits + 1) * sizeof(int32_t)));
  w.perm_q = reinterpret_cast<int32_t*>(take((size_t)cap * sizeof(int32_t)));
  w.perm_a = reinterpret_cast<int32_t*>(take((size_t)cap * sizeof(int32_t)));
  w.bytes = o;
  return w;
}
}  // namespace

size_t hinge_loss_workspace(int64_t n_hits, int64_t pair_capacity) {
  return hinge_ws(nullptr, n_hits, pair_capacity).bytes;
}

cudaError_t launch_hinge_loss(etx_ctx* ctx, const float* emb, int64_t n_hits, const int32_t* pq,
                              const int32_t* pa, const uint8_t* pg, const int32_t* n_pairs,
                              int64_t pair_capacity, float margin, float w_genuine, float* loss,
                              float* d_emb, void* workspace, cudaStream_t s) {
  const int D = ctx->cfg.emb_widths[ctx->cfg.emb_depth];
  const HingeWs w = hinge_ws(workspace, n_hits, pair_capacity);
  cudaError_t e = cudaMemsetAsync(w.counts, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  launch(ctx, "embtrain_hinge_clamp", k_hinge_clamp, 1, 1, 0, s, n_pairs, pair_capacity, w.n_eff,
         ctx->d_err);
  n_pairs = w.n_eff;
  // a grid fixed by the context and the capacity: the loss sums' order with it
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>((pair_capacity + kPT - 1) / kPT, (int64_t)ctx->n_sms * 8),
                           kHingeMaxBlocks));
  launch(ctx, "embtrain_hinge_count", k_hinge_count, grid, kPT, 0, s, pg, n_pairs, w.counts);
  const auto* cnts = (const unsigned long long*)w.counts;
  if (D == 8)
    launch(ctx, "embtrain_hinge_pairs", k_hinge_pairs<8>, grid, kPT, 0, s, emb, D, pq, pa, pg,
           n_pairs, cnts, margin, w_genuine, w.coef, w.part, n_hits, ctx->d_err);
  else if (D == 4)
    launch(ctx, "embtrain_hinge_pairs", k_hinge_pairs<4>, grid, kPT, 0, s, emb, D, pq, pa, pg,
           n_pairs, cnts, margin, w_genuine, w.coef, w.part, n_hits, ctx->d_err);
  else
    launch(ctx, "embtrain_hinge_pairs", k_hinge_pairs<0>, grid, kPT, 0, s, emb, D, pq, pa, pg,
           n_pairs, cnts, margin, w_genuine, w.coef, w.part, n_hits, ctx->d_err);
  // each hit's pairs as query and as partner, in ascending pair index
  static const char* const kQNames[3] = {"embtrain_hinge_index_count", "embtrain_hinge_index_fill",
                                         "embtrain_hinge_index_sort"};
  e = launch_key_index(ctx, pq, n_pairs, pair_capacity, n_hits, w.cnt, w.off_q, w.perm_q, kQNames, s);
  if (e == cudaSuccess)
    e = launch_key_index(ctx, pa, n_pairs, pair_capacity, n_hits, w.cnt, w.off_a, w.perm_a, kQNames, s);
  if (e != cudaSuccess) return e;
  if (n_hits > 0) {
    const int64_t want = (n_hits + kPT - 1) / kPT;
    const void* kg = D == 8 ? (const void*)k_hinge_grad<8>
                   : D == 4 ? (const void*)k_hinge_grad<4> : (const void*)k_hinge_grad<0>;
    const int gg = grid_for(ctx, kg, kPT, 0, want);
    if (D == 8)
      launch(ctx, "embtrain_hinge_grad", k_hinge_grad<8>, gg, kPT, 0, s, emb, D, pq, pa,
             (const float*)w.coef, (const int32_t*)w.off_q, (const int32_t*)w.perm_q,
             (const int32_t*)w.off_a, (const int32_t*)w.perm_a, n_hits, d_emb);
    else if (D == 4)
      launch(ctx, "embtrain_hinge_grad", k_hinge_grad<4>, gg, kPT, 0, s, emb, D, pq, pa,
             (const float*)w.coef, (const int32_t*)w.off_q, (const int32_t*)w.perm_q,
             (const int32_t*)w.off_a, (const int32_t*)w.perm_a, n_hits, d_emb);
    else
      launch(ctx, "embtrain_hinge_grad", k_hinge_grad<0>, gg, kPT, 0, s, emb, D, pq, pa,
             (const float*)w.coef, (const int32_t*)w.off_q, (const int32_t*)w.perm_q,
             (const int32_t*)w.off_a, (const int32_t*)w.perm_a, n_hits, d_emb);
  }
  launch(ctx, "embtrain_hinge_final", k_hinge_final, 1, kPT, 0, s, (const double*)w.part, (int)grid,
         cnts, n_pairs, w_genuine, loss);
  return cudaGetLastError();
}

}  // namespace etx
