// Purified hit graph -> track labels (paper Sec. 5 overview and Sec. 7.3).
//
// Weakly connected components by a lock-free union-find over the kept edges:
// every hit starts as its own root; an edge hooks the larger of its two roots
// under the smaller with atomicCAS (retrying if another thread hooked it
// first), and finds use path halving.  Because a parent always has a smaller
// index than its child, the root of a component is its smallest hit index,
// so the label is exact and independent of scheduling; it is written
// event-local.  Every loop carries an iteration cap: hitting it records
// ETX_ERR_TIMEOUT in the context's error word instead of spinning.
//
// The paper's own kernel instead sweeps the planes forward and backward
// taking minimum neighbour labels; that is not an exact connected-components
// algorithm in general, so it is not the track builder here.  It is provided
// as a variant (k_plane_sweep) for comparison.
#include "etx_internal.cuh"

namespace etx {
namespace {

constexpr int kFindCap = 1 << 22;
constexpr int kUnionCap = 1 << 20;

// Iteration caps of the union-find loops: a find follows at most find_cap
// parent links, an edge makes at most union_cap hook attempts.
struct UfCaps {
  int find_cap, union_cap;
};

__host__ __device__ inline UfCaps uf_caps(int32_t cfg_cap) {
  return cfg_cap > 0 ? UfCaps{cfg_cap, cfg_cap} : UfCaps{kFindCap, kUnionCap};
}

__device__ __forceinline__ int find_root(int* parent, int x, int* err, int cap) {
  volatile int* par = parent;
  for (int it = 0; it < cap; ++it) {
    const int p = par[x];
    if (p == x) return x;
    const int gp = par[p];
    if (gp != p) par[x] = gp;  // halving: gp is an ancestor of x
    x = gp;
  }
  set_err(err, DERR_TIMEOUT);
  return x;
}

// The paper's plane-ordered propagation (Sec. 7.3), one block per event.  Every
// hit starts with its own index; forward, for planes 1 .. P-1 in turn, every
// kept edge i -> j with j on the plane lowers lab[j] to lab[i] (i lies on one of
// the two previous planes, whose labels are final); backward, for planes
// P-2 .. 0, every kept edge i -> j with i on the plane lowers lab[i] to lab[j].
// Edges are sorted by src and hits by plane, so the edges leaving planes
// [a, b) are the contiguous range out_off[first hit of a] .. out_off[first hit
// of b].  The result is independent of thread order (minimum of fixed values).
__global__ void k_plane_sweep(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                              const float* __restrict__ logits, float thr,
                              const int32_t* __restrict__ plane_off, int n_planes,
                              const int32_t* __restrict__ out_off,
                              const int32_t* __restrict__ hit_offsets, int32_t* lab,
                              int32_t* __restrict__ labels) {
  const int b = blockIdx.x;
  const int32_t* po = plane_off + (int64_t)b * (n_planes + 1);
  const int h0 = po[0], h1 = po[n_planes];
  for (int i = h0 + threadIdx.x; i < h1; i += blockDim.x) lab[i] = i;
  __syncthreads();
  for (int p = 1; p < n_planes; ++p) {
    const int j0 = po[p], j1 = po[p + 1];  // hits of plane p
    const int e0 = out_off[po[p >= 2 ? p - 2 : 0]], e1 = out_off[po[p]];
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int i = src[e], j = dst[e];
      if (j >= j0 && j < j1 && i >= h0 && i < h1 && logits[e] > thr) atomicMin(&lab[j], lab[i]);
    }
    __syncthreads();
  }
  for (int p = n_planes - 2; p >= 0; --p) {
    const int e0 = out_off[po[p]], e1 = out_off[po[p + 1]];
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int i = src[e], j = dst[e];
      if (i >= h0 && i < h1 && j >= h0 && j < h1 && logits[e] > thr) atomicMin(&lab[i], lab[j]);
    }
    __syncthreads();
  }
  const int base = hit_offsets[b];
  for (int i = h0 + threadIdx.x; i < h1; i += blockDim.x) labels[i] = lab[i] - base;
}

__global__ void k_init(int32_t* __restrict__ parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (int)i;
}

__global__ void k_union(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                        const float* __restrict__ logits, float thr,
                        const int32_t* __restrict__ n_edges_dev, int n_hits,
                        int32_t* parent, int* err, UfCaps caps) {
  const int E = *n_edges_dev;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!(logits[e] > thr)) continue;
    int a = src[e], b = dst[e];
    if (a < 0 || a >= n_hits || b < 0 || b >= n_hits) {
      set_err(err, DERR_RANGE);
      continue;
    }
    int it = 0;
    for (; it < caps.union_cap; ++it) {
      a = find_root(parent, a, err, caps.find_cap);
      b = find_root(parent, b, err, caps.find_cap);
      if (a == b) break;
      if (a < b) { const int t = a; a = b; b = t; }  // hook larger root a under b
      const int old = atomicCAS(parent + a, a, b);
      if (old == a) break;
      a = old;  // a was hooked meanwhile: continue from its new parent
    }
    if (it == caps.union_cap) set_err(err, DERR_TIMEOUT);
  }
}

__global__ void k_labels(int32_t* parent, const int32_t* __restrict__ hoff, int32_t n_events,
                         int64_t n_hits, int32_t* __restrict__ labels, int* err, UfCaps caps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_hits;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = find_root(parent, (int)i, err, caps.find_cap);
    int lo = 0, hi = n_events;  // event b with hoff[b] <= i < hoff[b+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (hoff[mid] <= i) lo = mid; else hi = mid;
    }
    labels[i] = r - hoff[lo];
  }
}

__global__ void k_count_tracks(const int32_t* __restrict__ labels, const int32_t* __restrict__ hoff,
                               int32_t n_events, int64_t n_hits, int32_t min_hits,
                               int32_t* __restrict__ size_tmp, int32_t* __restrict__ n_tracks) {
  // size_tmp[i] = size of the component whose root is hit i (filled by atomics)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_hits;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_events;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (hoff[mid] <= i) lo = mid; else hi = mid;
    }
    const int root = hoff[lo] + labels[i];
    const int sz = atomicAdd(size_tmp + root, 1) + 1;
    if (sz == min_hits) atomicAdd(n_tracks + lo, 1);
  }
}

}  // namespace

cudaError_t launch_plane_sweep(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                               const float* logits, float thr, const int32_t* hit_offsets,
                               int32_t n_events, int64_t n_hits, int32_t* labels, cudaStream_t s) {
  if (n_events == 0 || n_hits == 0) return cudaSuccess;
  launch(ctx, "cc_plane_sweep", k_plane_sweep, (unsigned)n_events, 256, 0, s, src, dst, logits, thr,
         (const int32_t*)ctx->plane_off, ctx->cfg.n_planes, (const int32_t*)ctx->out_off,
         hit_offsets, ctx->parent, labels);
  return cudaGetLastError();
}

cudaError_t launch_edges_to_tracks(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                   const float* logits, float thr, const int32_t* n_edges_dev,
                                   const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                                   int32_t min_hits, int32_t* labels, int32_t* n_tracks,
                                   cudaStream_t s) {
  if (n_hits == 0) {
    if (n_tracks && n_events > 0)
      return cudaMemsetAsync(n_tracks, 0, (size_t)n_events * sizeof(int32_t), s);
    return cudaSuccess;
  }
  const int gn = grid_for(ctx, (const void*)k_init, 256, 0, (n_hits + 255) / 256);
  launch(ctx, "cc_init", k_init, gn, 256, 0, s, ctx->parent, n_hits);
  const int ge = grid_for(ctx, (const void*)k_union, 256, 0, (ctx->cfg.max_edges + 255) / 256);
  const UfCaps caps = uf_caps(ctx->cfg.uf_iter_cap);
  launch(ctx, "cc_union", k_union, ge, 256, 0, s, src, dst, logits, thr, n_edges_dev, (int)n_hits,
         ctx->parent, ctx->d_err, caps);
  const int gl = grid_for(ctx, (const void*)k_labels, 256, 0, (n_hits + 255) / 256);
  launch(ctx, "cc_labels", k_labels, gl, 256, 0, s, ctx->parent, hit_offsets, n_events, n_hits,
         labels, ctx->d_err, caps);
  if (n_tracks) {
    cudaError_t e = cudaMemsetAsync(n_tracks, 0, (size_t)n_events * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    // reuse the parent array as the per-root size counter
    e = cudaMemsetAsync(ctx->parent, 0, (size_t)n_hits * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int mh = min_hits < 1 ? 1 : min_hits;
    launch(ctx, "cc_count_tracks", k_count_tracks, gl, 256, 0, s, labels, hit_offsets, n_events,
           n_hits, mh, ctx->parent, n_tracks);
  }
  return cudaGetLastError();
}

}  // namespace etx

// ---------------------------------------------------------------------------
// Allocation-free variant of etx_edges_to_tracks (see include/etx.h).
//
// Its scratch (the union-find parents, reused as per-root size counters, plus
// an error word) is the file-scope array below: every GPU that loads the
// library holds it until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress (that device current) and caches
// it; later calls only launch kernels.  Calls that overlap on the GPU share
// the array and race.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {
constexpr int64_t kNoAllocMaxHits = int64_t(1) << 21;  // 2,097,152 hits, 8 MiB of scratch
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
int32_t* g_noalloc_ptr[kNoAllocMaxDevices] = {};
int g_noalloc_sms[kNoAllocMaxDevices] = {};

// Error bits of the union-find kernels -> etx_status, for the caller's status word.
__global__ void k_noalloc_status(const int* __restrict__ err, int32_t* __restrict__ status) {
  const int w = *err;
  *status = (w & etx::DERR_TIMEOUT) ? ETX_ERR_TIMEOUT : (w & etx::DERR_RANGE) ? ETX_ERR_UNSORTED : ETX_OK;
}

// Launch one kernel and return that launch's own error (cudaLaunchKernel reports
// the launch it made; the process-wide last-error state is not consulted, so a
// failure left there by unrelated earlier work is not charged to this call).
template <typename... KArgs, typename... Args>
cudaError_t launch_checked(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s,
                           Args... args) {
  void* argv[] = {static_cast<void*>(&args)...};
  return cudaLaunchKernel(reinterpret_cast<const void*>(kernel), dim3(grid), dim3(block), argv, 0, s);
}
}  // namespace

static __device__ __align__(256) int32_t g_cc_scratch[kNoAllocMaxHits + 64];

extern "C" etx_status etx_edges_to_tracks_noalloc(const int32_t* src, const int32_t* dst,
                                                  const float* logits, float threshold_logit,
                                                  const int32_t* edge_offsets,
                                                  const int32_t* hit_offsets, int32_t n_events,
                                                  int64_t n_hits, int32_t min_hits,
                                                  int32_t* labels, int32_t* n_tracks,
                                                  int32_t* status, void* stream) {
  using namespace etx;
  if (n_events < 0 || n_hits < 0) return ETX_ERR_ARG;
  if (n_hits > kNoAllocMaxHits) return ETX_ERR_CAPACITY;
  if (!edge_offsets || !hit_offsets || !src || !dst || !logits) return ETX_ERR_ARG;
  if (n_hits > 0 && (!labels || n_events == 0)) return ETX_ERR_ARG;
  if (threshold_logit != threshold_logit) return ETX_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return ETX_ERR_CUDA;
  int32_t* scratch;
  int sms;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_cc_scratch) != cudaSuccess || !p) return ETX_ERR_CUDA;
      int n = 0;
      if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ETX_ERR_CUDA;
      g_noalloc_sms[dev] = n > 0 ? n : 1;
      g_noalloc_ptr[dev] = static_cast<int32_t*>(p);
    }
    scratch = g_noalloc_ptr[dev];
    sms = g_noalloc_sms[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* parent = scratch;
  int* err = scratch + kNoAllocMaxHits;
  // this call's error bits start from zero (a memset allocates nothing)
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return ETX_ERR_CUDA;
  if (n_hits == 0) {
    if (n_tracks && n_events > 0 &&
        cudaMemsetAsync(n_tracks, 0, (size_t)n_events * sizeof(int32_t), s) != cudaSuccess)
      return ETX_ERR_CUDA;
  } else {
    const UfCaps caps = uf_caps(0);
    const int64_t cap = (int64_t)sms * 8;
    const int64_t hb = (n_hits + 255) / 256;
    const unsigned gh = (unsigned)(hb < cap ? hb : cap);
    if (launch_checked(k_init, gh, 256, s, parent, n_hits) != cudaSuccess) return ETX_ERR_CUDA;
    // the edge count is read on the device from edge_offsets[n_events]
    if (launch_checked(k_union, (unsigned)cap, 256, s, src, dst, logits, threshold_logit,
                       edge_offsets + n_events, (int)n_hits, parent, err, caps) != cudaSuccess)
      return ETX_ERR_CUDA;
    if (launch_checked(k_labels, gh, 256, s, parent, hit_offsets, n_events, n_hits, labels, err,
                       caps) != cudaSuccess)
      return ETX_ERR_CUDA;
    if (n_tracks) {
      if (cudaMemsetAsync(n_tracks, 0, (size_t)n_events * sizeof(int32_t), s) != cudaSuccess)
        return ETX_ERR_CUDA;
      if (cudaMemsetAsync(parent, 0, (size_t)n_hits * sizeof(int32_t), s) != cudaSuccess)
        return ETX_ERR_CUDA;
      if (launch_checked(k_count_tracks, gh, 256, s, labels, hit_offsets, n_events, n_hits,
                         min_hits < 1 ? 1 : min_hits, parent, n_tracks) != cudaSuccess)
        return ETX_ERR_CUDA;
    }
  }
  if (status && launch_checked(k_noalloc_status, 1, 1, s, (const int*)err, status) != cudaSuccess)
    return ETX_ERR_CUDA;
  return ETX_OK;
}
