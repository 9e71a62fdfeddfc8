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

// ---------------------------------------------------------------------------
// Track building on the purified edge graph (Sec. 5.4).  Nodes are the kept
// edges, links the kept triplets (triplet logit > cut) of the list that
// k_trip_emit wrote for the same edges and edge cut.  Four steps:
//  1. at each hit C, the kept in-edges joined by kept right elbows form
//     groups, and the kept out-edges joined by kept left elbows; an
//     articulation (i, o) at C is present when a kept articulation links i's
//     group to o's group (an elbow's two edges share their continuations);
//  2. a present articulation is shared when i has two or more present
//     articulations at C, or o has; the unshared ones link edges in a
//     union-find over edge indices;
//  3. tracks: every component no shared articulation touches, then every
//     shared articulation (i, o) as the union of i's and o's components;
//  4. a track's hits are the end points of its edges (each component's
//     distinct hits, merged for two components), at least min_hits of them.
// At most kTbMaxDeg kept edges may enter or leave one hit (the group masks
// are 64-bit); a hit above that is skipped and reported as a capacity error.
// ---------------------------------------------------------------------------
constexpr int kTbMaxDeg = 64;
constexpr int kTbFindCap = 1 << 22;
constexpr int kTbUnionCap = 1 << 20;

__device__ __forceinline__ int tb_find(int* parent, int x, int* err) {
  volatile int* par = parent;
  for (int it = 0; it < kTbFindCap; ++it) {
    const int p = par[x];
    if (p == x) return x;
    const int gp = par[p];
    if (gp != p) par[x] = gp;  // path halving
    x = gp;
  }
  set_err(err, DERR_TIMEOUT);
  return x;
}

// Lock-free union by index (the root of a component is its smallest edge).
__device__ __forceinline__ void tb_union(int* parent, int a, int b, int* err) {
  for (int it = 0; it < kTbUnionCap; ++it) {
    a = tb_find(parent, a, err);
    b = tb_find(parent, b, err);
    if (a == b) return;
    if (a < b) { const int t = a; a = b; b = t; }
    const int old = atomicCAS(parent + a, a, b);
    if (old == a) return;
    a = old;
  }
  set_err(err, DERR_TIMEOUT);
}

// local representative of x in a tiny union-find over 32 slots
__device__ __forceinline__ int tb_rep(const int8_t* g, int x) {
  for (int it = 0; it < kTbMaxDeg && g[x] != x; ++it) x = g[x];
  return x;
}

__device__ __forceinline__ void tb_join(int8_t* g, int x, int y) {
  x = tb_rep(g, x);
  y = tb_rep(g, y);
  if (x != y) g[x > y ? x : y] = (int8_t)(x < y ? x : y);
}

// index of pair (x, y), x < y, in the enumeration x = 0..n-1, y = x+1..n-1
__device__ __forceinline__ int64_t tb_pair(int x, int y, int n) {
  return (int64_t)x * (2 * n - x - 1) / 2 + (y - x - 1);
}

struct TbArgs {
  TripCtx c;
  const int32_t* first;
  const int32_t* second;
  const float* tlogits;
  float tthr;
  const int32_t* counts;     // etx_build_triplets' {total, art, left, right}
  const int32_t* off_art;    // recomputed slices, [n_hits + 1] each
  const int32_t* off_left;
  const int32_t* off_right;
  int32_t* art_flag;         // [art count]: 0 absent, 1 link, 2 shared
  int* err;
};

// Steps 1-2 at every hit: one thread per hit.
__global__ void k_tb_hits(TbArgs a, int64_t n_hits) {
  const int64_t na = a.off_art[n_hits], nl = a.off_left[n_hits], nr = a.off_right[n_hits];
  if (na != a.counts[1] || nl != a.counts[2] || nr != a.counts[3]) {
    // not the triplet list of these edges and this edge cut
    if (blockIdx.x == 0 && threadIdx.x == 0) set_err(a.err, DERR_RANGE);
    return;
  }
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_hits;
       h += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a0 = a.off_art[h];
    const int nA = a.off_art[h + 1] - (int)a0;
    if (nA == 0) continue;
    int I[kTbMaxDeg], O[kTbMaxDeg];
    int ni = 0, no = 0;
    bool over = false;
    for (int q = a.c.in_off[h]; q < a.c.in_off[h + 1]; ++q) {
      const int e = a.c.perm_in[q];
      if (!(a.c.logits[e] > a.c.thr)) continue;
      if (ni == kTbMaxDeg) { over = true; break; }
      I[ni++] = e;
    }
    for (int e = a.c.out_off[h]; e < a.c.out_off[h + 1]; ++e) {
      if (!(a.c.logits[e] > a.c.thr)) continue;
      if (no == kTbMaxDeg) { over = true; break; }
      O[no++] = e;
    }
    if (over || ni * no != nA) {
      set_err(a.err, DERR_CAPACITY);
      for (int k = 0; k < nA; ++k) a.art_flag[a0 + k] = 0;
      continue;
    }
    int8_t gi[kTbMaxDeg], go[kTbMaxDeg];
    for (int k = 0; k < ni; ++k) gi[k] = (int8_t)k;
    for (int k = 0; k < no; ++k) go[k] = (int8_t)k;
    bool bad = false;
    // step 1: right elbows join in-edges, left elbows join out-edges
    const int64_t r0 = na + nl + a.off_right[h], l0 = na + a.off_left[h];
    for (int x = 0; x < ni; ++x)
      for (int y = x + 1; y < ni; ++y) {
        const int64_t t = r0 + tb_pair(x, y, ni);
        bad |= a.first[t] != I[x] || a.second[t] != I[y];
        if (a.tlogits[t] > a.tthr) tb_join(gi, x, y);
      }
    for (int x = 0; x < no; ++x)
      for (int y = x + 1; y < no; ++y) {
        const int64_t t = l0 + tb_pair(x, y, no);
        bad |= a.first[t] != O[x] || a.second[t] != O[y];
        if (a.tlogits[t] > a.tthr) tb_join(go, x, y);
      }
    // group pairs linked by a kept articulation (bit g_out of act[g_in])
    uint64_t act[kTbMaxDeg];
    for (int k = 0; k < ni; ++k) act[k] = 0ull;
    for (int x = 0; x < ni; ++x)
      for (int y = 0; y < no; ++y) {
        const int64_t t = a0 + (int64_t)x * no + y;
        bad |= a.first[t] != I[x] || a.second[t] != O[y];
        if (a.tlogits[t] > a.tthr) act[tb_rep(gi, x)] |= 1ull << tb_rep(go, y);
      }
    if (bad) {
      set_err(a.err, DERR_RANGE);
      for (int k = 0; k < nA; ++k) a.art_flag[a0 + k] = 0;
      continue;
    }
    // present (x, y) iff bit rep(y) of act[rep(x)]; step 2: shared or link
    int8_t rx[kTbMaxDeg], ry[kTbMaxDeg];
    for (int x = 0; x < ni; ++x) rx[x] = (int8_t)tb_rep(gi, x);
    for (int y = 0; y < no; ++y) ry[y] = (int8_t)tb_rep(go, y);
    int n_in_of[kTbMaxDeg];
    for (int y = 0; y < no; ++y) n_in_of[y] = 0;
    for (int x = 0; x < ni; ++x)
      for (int y = 0; y < no; ++y) n_in_of[y] += (int)((act[rx[x]] >> ry[y]) & 1ull);
    for (int x = 0; x < ni; ++x) {
      int n_out = 0;
      for (int y = 0; y < no; ++y) n_out += (int)((act[rx[x]] >> ry[y]) & 1ull);
      for (int y = 0; y < no; ++y) {
        const bool present = (act[rx[x]] >> ry[y]) & 1ull;
        a.art_flag[a0 + (int64_t)x * no + y] = !present ? 0 : (n_out >= 2 || n_in_of[y] >= 2 ? 2 : 1);
      }
    }
  }
}

__global__ void k_tb_init(int32_t* __restrict__ parent, const int32_t* __restrict__ n_edges_dev) {
  const int E = *n_edges_dev;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    parent[e] = (int)e;
}

// unshared present articulations link their two edges
__global__ void k_tb_union(const int32_t* __restrict__ first, const int32_t* __restrict__ second,
                           const int32_t* __restrict__ art_flag, const int32_t* __restrict__ counts,
                           int32_t* parent, int* err) {
  const int n = counts[1];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    if (art_flag[t] == 1) tb_union(parent, first[t], second[t], err);
}

// root[e] for kept edges (-1 for dropped ones), and which roots a shared
// articulation touches (touched[r] = 1); standalone[r] = 1 for untouched roots
__global__ void k_tb_roots(const float* __restrict__ logits, float thr,
                           const int32_t* __restrict__ n_edges_dev, int32_t* parent,
                           int32_t* __restrict__ root, int* err) {
  const int E = *n_edges_dev;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    root[e] = logits[e] > thr ? tb_find(parent, (int)e, err) : -1;
}

__global__ void k_tb_touch(const int32_t* __restrict__ first, const int32_t* __restrict__ second,
                           const int32_t* __restrict__ art_flag, const int32_t* __restrict__ counts,
                           const int32_t* __restrict__ root, int32_t* __restrict__ touched) {
  const int n = counts[1];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    if (art_flag[t] == 2) {
      touched[root[first[t]]] = 1;
      touched[root[second[t]]] = 1;
    }
}

// standalone[e] = 1 iff e is the root of a component no shared articulation touches
__global__ void k_tb_standalone(const int32_t* __restrict__ root, const int32_t* __restrict__ touched,
                                const int32_t* __restrict__ n_edges_dev, int64_t e_cap,
                                int32_t* __restrict__ standalone) {
  const int E = *n_edges_dev;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e_cap;
       e += (int64_t)gridDim.x * blockDim.x)
    standalone[e] = e < E && root[e] == (int)e && !touched[e];
}

// The distinct components among a hit's kept edges: for each, the hit is one
// of the component's hits.  EMIT 0 counts (comp_cnt[r] += 1), EMIT 1 writes
// the hit at comp_off[r] + fill[r]++ (order within a component fixed later).
template <int EMIT>
__global__ void k_tb_comp_hits(TripCtx c, const int32_t* __restrict__ root, int64_t n_hits,
                               int32_t* __restrict__ comp_cnt, const int32_t* __restrict__ comp_off,
                               int32_t* __restrict__ fill, int32_t* __restrict__ comp_hits) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_hits;
       h += (int64_t)gridDim.x * blockDim.x) {
    int seen[2 * kTbMaxDeg];
    int ns = 0;
    auto visit = [&](int e) {
      if (!(c.logits[e] > c.thr)) return;
      const int r = root[e];
      for (int k = 0; k < ns; ++k)
        if (seen[k] == r) return;
      if (ns < 2 * kTbMaxDeg) seen[ns++] = r;
      if constexpr (EMIT == 0) {
        atomicAdd(comp_cnt + r, 1);
      } else {
        comp_hits[comp_off[r] + atomicAdd(fill + r, 1)] = (int)h;
      }
    };
    for (int q = c.in_off[h]; q < c.in_off[h + 1]; ++q) visit(c.perm_in[q]);
    for (int e = c.out_off[h]; e < c.out_off[h + 1]; ++e) visit(e);
  }
}

// Sort each component's hit list.  A component lies inside one event, so
// its length is at most the event's hit count.  Lists of up to kTbShort hits:
// one thread, insertion sort (k_tb_sort_short); longer ones: one block,
// bitonic sort in shared memory (k_tb_sort_long), up to kTbLong hits; a
// longer list is left unsorted and reported as a capacity error.
constexpr int kTbShort = 64;
constexpr int kTbLong = 8192;

__global__ void k_tb_sort_short(const int32_t* __restrict__ comp_off,
                                const int32_t* __restrict__ n_edges_dev, int32_t* __restrict__ comp_hits) {
  const int E = *n_edges_dev;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < E;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int lo = comp_off[r], hi = comp_off[r + 1];
    if (hi - lo > kTbShort) continue;
    for (int i = lo + 1; i < hi; ++i) {
      const int v = comp_hits[i];
      int j = i - 1;
      while (j >= lo && comp_hits[j] > v) {
        comp_hits[j + 1] = comp_hits[j];
        --j;
      }
      comp_hits[j + 1] = v;
    }
  }
}

__global__ void __launch_bounds__(1024) k_tb_sort_long(const int32_t* __restrict__ comp_off,
                                                       const int32_t* __restrict__ n_edges_dev,
                                                       int32_t* __restrict__ comp_hits, int* err) {
  __shared__ int32_t v[kTbLong];
  const int E = *n_edges_dev;
  for (int64_t r = blockIdx.x; r < E; r += gridDim.x) {
    const int lo = comp_off[r], n = comp_off[r + 1] - lo;
    if (n <= kTbShort) continue;  // uniform across the block: every thread reads the same r
    if (n > kTbLong) {
      if (threadIdx.x == 0) set_err(err, DERR_CAPACITY);
      continue;
    }
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = i < n ? comp_hits[lo + i] : INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          const int p = i ^ j;
          if (p > i) {
            const bool up = (i & k) == 0;
            const int a = v[i], b = v[p];
            if ((a > b) == up) {
              v[i] = b;
              v[p] = a;
            }
          }
        }
        __syncthreads();
      }
    for (int i = threadIdx.x; i < n; i += blockDim.x) comp_hits[lo + i] = v[i];
    __syncthreads();
  }
}

// number of distinct values in the union of two sorted lists
__device__ __forceinline__ int tb_union_count(const int32_t* a, int na, const int32_t* b, int nb) {
  int i = 0, j = 0, n = 0;
  while (i < na || j < nb) {
    if (j == nb || (i < na && a[i] < b[j])) ++i;
    else if (i == na || b[j] < a[i]) ++j;
    else { ++i; ++j; }
    ++n;
  }
  return n;
}

// Track t (standalone components first, in root order, then the shared
// articulations in list order): its pair of components (ra, rb; rb = -1 for
// one component).
struct TbTracks {
  const int32_t* standalone_off;  // exclusive scan of standalone flags, [e_cap + 1]
  const int32_t* shared_off;      // exclusive scan of (art_flag == 2), [art_cap + 1]
  const int32_t* art_flag;
  const int32_t* first;
  const int32_t* second;
  const int32_t* root;
  const int32_t* comp_off;
  const int32_t* comp_hits;
  int64_t e_cap, art_cap;
};

// Counting pass over the tracks: hit count of each, 1 if kept (>= min_hits)
__global__ void k_tb_track_count(TbTracks tk, const int32_t* __restrict__ n_edges_dev,
                                 const int32_t* __restrict__ counts, int min_hits,
                                 int32_t* __restrict__ keep, int32_t* __restrict__ nhit) {
  const int E = *n_edges_dev, nA = counts[1];
  const int64_t n_std = tk.standalone_off[tk.e_cap];
  // standalone components: one thread per edge root
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (tk.standalone_off[e + 1] == tk.standalone_off[e]) continue;
    const int t = tk.standalone_off[e];
    const int n = tk.comp_off[e + 1] - tk.comp_off[e];
    nhit[t] = n;
    keep[t] = n >= min_hits;
  }
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nA;
       a += (int64_t)gridDim.x * blockDim.x) {
    if (tk.art_flag[a] != 2) continue;
    const int64_t t = n_std + tk.shared_off[a];
    const int ra = tk.root[tk.first[a]], rb = tk.root[tk.second[a]];
    int n;
    if (ra == rb) {
      n = tk.comp_off[ra + 1] - tk.comp_off[ra];
    } else {
      n = tb_union_count(tk.comp_hits + tk.comp_off[ra], tk.comp_off[ra + 1] - tk.comp_off[ra],
                         tk.comp_hits + tk.comp_off[rb], tk.comp_off[rb + 1] - tk.comp_off[rb]);
    }
    nhit[t] = n;
    keep[t] = n >= min_hits;
  }
}

// Kept tracks: sizes into the hit-offset scan input (0 for dropped ones)
__global__ void k_tb_kept_sizes(const int32_t* __restrict__ keep, const int32_t* __restrict__ nhit,
                                int64_t n_tracks_cap, int32_t* __restrict__ size) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tracks_cap;
       t += (int64_t)gridDim.x * blockDim.x)
    size[t] = keep[t] ? nhit[t] : 0;
}

// Emit: kept track t goes to slot keep_off[t] with hits at hit_off[t]
__global__ void k_tb_emit(TbTracks tk, const int32_t* __restrict__ n_edges_dev,
                          const int32_t* __restrict__ counts, const int32_t* __restrict__ keep_off,
                          const int32_t* __restrict__ hit_off, int64_t n_tracks_cap,
                          int64_t track_capacity, int64_t hit_capacity,
                          int32_t* __restrict__ track_offsets, int32_t* __restrict__ track_hits,
                          int32_t* __restrict__ n_out, int* err) {
  const int E = *n_edges_dev, nA = counts[1];
  const int64_t n_std = tk.standalone_off[tk.e_cap];
  const int64_t n_keep = keep_off[n_tracks_cap], n_h = hit_off[n_tracks_cap];
  if (n_keep > track_capacity || n_h > hit_capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      set_err(err, DERR_CAPACITY);
      n_out[0] = n_out[1] = 0;
      if (track_capacity >= 0) track_offsets[0] = 0;
    }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    n_out[0] = (int32_t)n_keep;
    n_out[1] = (int32_t)n_h;
    track_offsets[n_keep] = (int32_t)n_h;
  }
  auto put = [&](int64_t t, int ra, int rb) {
    if (keep_off[t + 1] == keep_off[t]) return;
    const int64_t slot = keep_off[t];
    int64_t w = hit_off[t];
    track_offsets[slot] = (int32_t)w;
    const int32_t* A = tk.comp_hits + tk.comp_off[ra];
    const int na = tk.comp_off[ra + 1] - tk.comp_off[ra];
    if (rb < 0 || rb == ra) {
      for (int i = 0; i < na; ++i) track_hits[w++] = A[i];
      return;
    }
    const int32_t* B = tk.comp_hits + tk.comp_off[rb];
    const int nb = tk.comp_off[rb + 1] - tk.comp_off[rb];
    int i = 0, j = 0;
    while (i < na || j < nb) {
      int v;
      if (j == nb || (i < na && A[i] < B[j])) v = A[i++];
      else if (i == na || B[j] < A[i]) v = B[j++];
      else { v = A[i]; ++i; ++j; }
      track_hits[w++] = v;
    }
  };
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    if (tk.standalone_off[e + 1] != tk.standalone_off[e]) put(tk.standalone_off[e], (int)e, -1);
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nA;
       a += (int64_t)gridDim.x * blockDim.x)
    if (tk.art_flag[a] == 2)
      put(n_std + tk.shared_off[a], tk.root[tk.first[a]], tk.root[tk.second[a]]);
}

__global__ void k_tb_is_shared(const int32_t* __restrict__ art_flag, const int32_t* __restrict__ counts,
                               int64_t art_cap, int32_t* __restrict__ out) {
  const int n = counts[1];
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < art_cap;
       a += (int64_t)gridDim.x * blockDim.x)
    out[a] = a < n && art_flag[a] == 2;
}

}  // namespace

size_t triplets_workspace(int64_t n_hits) { return (size_t)3 * (n_hits + 1) * sizeof(int32_t); }

// Workspace of launch_tracks_from_triplets, in int32 units, laid out as:
// off_art, off_left, off_right [n+1 each], art_flag [A], parent [E], root [E],
// touched [E+1], standalone_off [E+1], comp_off [E+1], fill [E], comp_hits [2E],
// shared_off [A+1], keep [T+1], nhit [T+1], keep_off [T+1], hit_off [T+1]
// with A = articulation capacity (the triplet capacity), T = E + A.
size_t tracks_workspace(int64_t n_hits, int64_t e_cap, int64_t trip_cap) {
  const int64_t T = e_cap + trip_cap;
  const int64_t big = std::max<int64_t>(std::max<int64_t>(n_hits, e_cap), std::max<int64_t>(trip_cap, T));
  const int64_t ints = 3 * (n_hits + 1) + trip_cap + 2 * e_cap + 3 * (e_cap + 1) + e_cap +
                       2 * e_cap + (trip_cap + 1) + 4 * (T + 1) + (int64_t)scan_tmp_ints(big + 1) + 8;
  return (size_t)ints * sizeof(int32_t);
}

cudaError_t launch_tracks_from_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                        const float* logits, float thr, int64_t n_hits,
                                        const int32_t* first, const int32_t* second,
                                        const float* tlogits, float tthr, const int32_t* counts,
                                        int64_t trip_cap, int32_t min_hits, void* workspace,
                                        int32_t* track_offsets, int32_t* track_hits,
                                        int64_t track_capacity, int64_t hit_capacity,
                                        int32_t* n_out, cudaStream_t s) {
  const int64_t E = ctx->cfg.max_edges, A = trip_cap, T = E + A;
  int32_t* w = static_cast<int32_t*>(workspace);
  auto take = [&](int64_t n) { int32_t* p = w; w += n; return p; };
  int32_t* off_art = take(n_hits + 1);
  int32_t* off_left = take(n_hits + 1);
  int32_t* off_right = take(n_hits + 1);
  int32_t* art_flag = take(A);
  int32_t* parent = take(E);
  int32_t* root = take(E);
  int32_t* touched = take(E + 1);
  int32_t* standalone_off = take(E + 1);
  int32_t* comp_off = take(E + 1);
  int32_t* fill = take(E);
  int32_t* comp_hits = take(2 * E);
  int32_t* shared_off = take(A + 1);
  int32_t* keep = take(T + 1);
  int32_t* nhit = take(T + 1);
  int32_t* keep_off = take(T + 1);
  int32_t* hit_off = take(T + 1);
  const int64_t big = std::max<int64_t>(std::max<int64_t>(n_hits, E), std::max<int64_t>(A, T));
  const size_t tmp_ints = scan_tmp_ints(big + 1) + 8;
  int32_t* scan_tmp = take((int64_t)tmp_ints);
  auto scan = [&](const int32_t* in, int32_t* out, int64_t n) {
    return exclusive_scan_with(ctx, in, out, n, scan_tmp, tmp_ints, s);
  };

  cudaError_t e = launch_edge_index(ctx, n_hits, src, dst, ctx->n_edges, s);
  if (e != cudaSuccess) return e;
  TripCtx c{ctx->out_off, ctx->in_off, ctx->perm_in, logits, thr};
  auto grid = [&](int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->n_sms * 8));
  };
  // per-hit slices of the triplet list, as k_trip_emit laid it out
  if (n_hits > 0)
    launch(ctx, "tracks_slices", k_trip_count, grid(n_hits), 256, 0, s, c, n_hits, off_art,
           off_left, off_right);
  for (int32_t* o : {off_art, off_left, off_right})
    if ((e = scan(o, o, n_hits)) != cudaSuccess) return e;
  if (A > 0 && (e = cudaMemsetAsync(art_flag, 0, (size_t)A * 4, s)) != cudaSuccess) return e;
  TbArgs ta{c, first, second, tlogits, tthr, counts, off_art, off_left, off_right, art_flag,
            ctx->d_err};
  if (n_hits > 0) launch(ctx, "tracks_hits", k_tb_hits, grid(n_hits), 128, 0, s, ta, n_hits);
  // step 2: components over the unshared articulations
  launch(ctx, "tracks_uf_init", k_tb_init, grid(E), 256, 0, s, parent, (const int32_t*)ctx->n_edges);
  launch(ctx, "tracks_uf_union", k_tb_union, grid(A), 256, 0, s, first, second,
         (const int32_t*)art_flag, counts, parent, ctx->d_err);
  launch(ctx, "tracks_roots", k_tb_roots, grid(E), 256, 0, s, logits, thr,
         (const int32_t*)ctx->n_edges, parent, root, ctx->d_err);
  // step 3: which components stand alone
  if ((e = cudaMemsetAsync(touched, 0, (size_t)(E + 1) * 4, s)) != cudaSuccess) return e;
  launch(ctx, "tracks_touch", k_tb_touch, grid(A), 256, 0, s, first, second,
         (const int32_t*)art_flag, counts, (const int32_t*)root, touched);
  launch(ctx, "tracks_standalone", k_tb_standalone, grid(E), 256, 0, s, (const int32_t*)root,
         (const int32_t*)touched, (const int32_t*)ctx->n_edges, E, standalone_off);
  if ((e = scan(standalone_off, standalone_off, E)) != cudaSuccess) return e;
  launch(ctx, "tracks_is_shared", k_tb_is_shared, grid(A), 256, 0, s, (const int32_t*)art_flag,
         counts, A, shared_off);
  if ((e = scan(shared_off, shared_off, A)) != cudaSuccess) return e;
  // step 4: each component's distinct hits, sorted
  if ((e = cudaMemsetAsync(comp_off, 0, (size_t)(E + 1) * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(fill, 0, (size_t)E * 4, s)) != cudaSuccess) return e;
  if (n_hits > 0)
    launch(ctx, "tracks_comp_count", k_tb_comp_hits<0>, grid(n_hits), 256, 0, s, c,
           (const int32_t*)root, n_hits, comp_off, (const int32_t*)nullptr, fill, comp_hits);
  if ((e = scan(comp_off, comp_off, E)) != cudaSuccess) return e;
  if (n_hits > 0)
    launch(ctx, "tracks_comp_emit", k_tb_comp_hits<1>, grid(n_hits), 256, 0, s, c,
           (const int32_t*)root, n_hits, (int32_t*)nullptr, (const int32_t*)comp_off, fill,
           comp_hits);
  launch(ctx, "tracks_sort_short", k_tb_sort_short, grid(E), 256, 0, s, (const int32_t*)comp_off,
         (const int32_t*)ctx->n_edges, comp_hits);
  launch(ctx, "tracks_sort_long", k_tb_sort_long, (unsigned)ctx->n_sms * 2, 1024, 0, s,
         (const int32_t*)comp_off, (const int32_t*)ctx->n_edges, comp_hits, ctx->d_err);
  // tracks: sizes, the min_hits filter, offsets, hits
  TbTracks tk{standalone_off, shared_off, art_flag, first, second, root, comp_off, comp_hits, E, A};
  if ((e = cudaMemsetAsync(keep, 0, (size_t)(T + 1) * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(nhit, 0, (size_t)(T + 1) * 4, s)) != cudaSuccess) return e;
  launch(ctx, "tracks_count", k_tb_track_count, grid(std::max(E, A)), 256, 0, s, tk,
         (const int32_t*)ctx->n_edges, counts, (int)min_hits, keep, nhit);
  launch(ctx, "tracks_sizes", k_tb_kept_sizes, grid(T), 256, 0, s, (const int32_t*)keep,
         (const int32_t*)nhit, T, hit_off);
  if ((e = scan(keep, keep_off, T)) != cudaSuccess) return e;
  if ((e = scan(hit_off, hit_off, T)) != cudaSuccess) return e;
  launch(ctx, "tracks_emit", k_tb_emit, grid(std::max(E, A)), 256, 0, s, tk,
         (const int32_t*)ctx->n_edges, counts, (const int32_t*)keep_off, (const int32_t*)hit_off, T,
         track_capacity, hit_capacity, track_offsets, track_hits, n_out, ctx->d_err);
  return cudaGetLastError();
}

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
