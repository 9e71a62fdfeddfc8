// Hit embedding MLP (paper Sec. 5.1), FP32 on the SIMT pipes.
//
// Each 256-thread block owns 64 hits at a time (persistent grid-stride loop):
// the features (r, phi, z) are built and normalised in registers, every
// hidden layer is a 64 x EW register tile (simt_tile.cuh) fed from shared
// memory, and the last layer (EW -> D) is a per-(hit, output) dot product.
// The output is FP32 because the graph cut is taken on it.
#include "simt_tile.cuh"

namespace etx {
namespace {

constexpr int kKC = 16;  // k-chunk of the streamed weights

struct EmbArgs {
  const float* norm;  // mu[3], sigma[3]
  LinF32 lin[ETX_MAX_EMB_LAYERS];
  int depth;
  int dim;  // D
};

// Copy a 64-row activation tile from shared memory to rows [row0, n) of a
// row-major [n][EW] array (the training forward keeps them for the reverse pass).
template <int EW>
__device__ __forceinline__ void save_tile(const float* Act, int lda, float* __restrict__ out,
                                          int64_t row0, int64_t n, int tid) {
  for (int idx = tid; idx < kTileM * EW / 4; idx += kTileThreads) {
    const int r = idx / (EW / 4), c4 = idx - r * (EW / 4);
    if (row0 + r < n)
      *reinterpret_cast<float4*>(out + (row0 + r) * EW + c4 * 4) =
          *reinterpret_cast<const float4*>(Act + r * lda + c4 * 4);
  }
}

// SAVE: also write the normalised inputs ([n][4], last column 0) and every
// hidden layer's activations ([n][EW] each, after ReLU) to `saved`.
template <int EW, bool SAVE>
__global__ void __launch_bounds__(kTileThreads) k_embed(const float* __restrict__ x,
                                                        const float* __restrict__ y,
                                                        const float* __restrict__ z, int64_t n,
                                                        EmbArgs a, float* __restrict__ emb,
                                                        float* __restrict__ saved) {
  constexpr int LDA = EW + 4;
  __shared__ __align__(16) float In[kTileM * 4];
  __shared__ __align__(16) float Act[kTileM * LDA];
  __shared__ __align__(16) float Ws[kKC * EW];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const float mu0 = __ldg(a.norm + 0), mu1 = __ldg(a.norm + 1), mu2 = __ldg(a.norm + 2);
  const float is0 = 1.0f / __ldg(a.norm + 3), is1 = 1.0f / __ldg(a.norm + 4),
              is2 = 1.0f / __ldg(a.norm + 5);
  const int64_t n_tiles = (n + kTileM - 1) / kTileM;

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTileM;
    __syncthreads();
    if (tid < kTileM) {
      const int64_t i = row0 + tid;
      float f0 = 0.f, f1 = 0.f, f2 = 0.f;
      if (i < n) {
        const float xv = x[i], yv = y[i], zv = z[i];
        f0 = (sqrtf(xv * xv + yv * yv) - mu0) * is0;
        f1 = (atan2f(yv, xv) - mu1) * is1;
        f2 = (zv - mu2) * is2;
      }
      *reinterpret_cast<float4*>(In + tid * 4) = make_float4(f0, f1, f2, 0.f);
      if constexpr (SAVE) {
        if (i < n) *reinterpret_cast<float4*>(saved + i * 4) = make_float4(f0, f1, f2, 0.f);
      }
    }
    if (tid < 4 * EW / 4) {
      // layer 0 weights: W^T [4][EW] (k padded 3 -> 4 with a zero row)
      reinterpret_cast<float4*>(Ws)[tid] = __ldg(reinterpret_cast<const float4*>(a.lin[0].wt) + tid);
    }
    __syncthreads();
    TileAcc<EW> acc;
    acc.zero();
    acc.template mma<4>(In, 4, 0, Ws, ty, tx);
    // bias + ReLU, to shared memory
#pragma unroll
    for (int j = 0; j < EW / 16; ++j) {
      const float bj = __ldg(a.lin[0].b + ColMap<EW>::col(tx, j));
#pragma unroll
      for (int r = 0; r < 4; ++r) acc.v[r][j] = fmaxf(acc.v[r][j] + bj, 0.f);
    }
    store_tile_smem<EW>(acc, Act, LDA, ty, tx);
    if constexpr (SAVE) {
      __syncthreads();
      save_tile<EW>(Act, LDA, saved + n * 4, row0, n, tid);
    }

    for (int l = 1; l < a.depth - 1; ++l) {
      acc.zero();
      for (int k0 = 0; k0 < EW; k0 += kKC) {
        __syncthreads();
        load_w_chunk<kKC, EW>(Ws, a.lin[l].wt + (size_t)k0 * EW, tid);
        __syncthreads();
        acc.template mma<kKC>(Act, LDA, k0, Ws, ty, tx);
      }
#pragma unroll
      for (int j = 0; j < EW / 16; ++j) {
        const float bj = __ldg(a.lin[l].b + ColMap<EW>::col(tx, j));
#pragma unroll
        for (int r = 0; r < 4; ++r) acc.v[r][j] = fmaxf(acc.v[r][j] + bj, 0.f);
      }
      __syncthreads();  // everyone finished reading Act
      store_tile_smem<EW>(acc, Act, LDA, ty, tx);
      if constexpr (SAVE) {
        __syncthreads();
        save_tile<EW>(Act, LDA, saved + n * 4 + (int64_t)l * n * EW, row0, n, tid);
      }
    }
    __syncthreads();
    // last layer: EW -> D, thread = (row, group of outputs)
    const LinF32& lo = a.lin[a.depth - 1];
    const int row = tid & (kTileM - 1);
    const int grp = tid >> 6;                 // 0..3
    const int per = (a.dim + 3) >> 2;
    const int64_t i = row0 + row;
    for (int q = 0; q < per; ++q) {
      const int d = grp * per + q;
      if (d >= a.dim) break;
      float s = __ldg(lo.b + d);
      const float* arow = Act + row * LDA;
#pragma unroll 4
      for (int k = 0; k < EW; k += 4) {
        const float4 av = *reinterpret_cast<const float4*>(arow + k);
        s = fmaf(av.x, __ldg(lo.wt + (size_t)(k + 0) * lo.n + d), s);
        s = fmaf(av.y, __ldg(lo.wt + (size_t)(k + 1) * lo.n + d), s);
        s = fmaf(av.z, __ldg(lo.wt + (size_t)(k + 2) * lo.n + d), s);
        s = fmaf(av.w, __ldg(lo.wt + (size_t)(k + 3) * lo.n + d), s);
      }
      if (i < n) emb[i * a.dim + d] = s;
    }
  }
}

template <int EW>
cudaError_t run(etx_ctx* ctx, const float* x, const float* y, const float* z, int64_t n,
                const EmbArgs& a, float* emb, float* saved, cudaStream_t s) {
  const int64_t tiles = (n + kTileM - 1) / kTileM;
  if (saved) {
    const int grid = grid_for(ctx, (const void*)k_embed<EW, true>, kTileThreads, 0, tiles);
    launch(ctx, "embed_mlp_save", k_embed<EW, true>, grid, kTileThreads, 0, s, x, y, z, n, a, emb,
           saved);
  } else {
    const int grid = grid_for(ctx, (const void*)k_embed<EW, false>, kTileThreads, 0, tiles);
    launch(ctx, "embed_mlp", k_embed<EW, false>, grid, kTileThreads, 0, s, x, y, z, n, a, emb,
           (float*)nullptr);
  }
  return cudaGetLastError();
}

cudaError_t dispatch(etx_ctx* ctx, const float* x, const float* y, const float* z, int64_t n,
                     float* emb, float* saved, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  EmbArgs a{};
  a.norm = ctx->w.norm;
  a.depth = ctx->cfg.emb_depth;
  a.dim = ctx->cfg.emb_widths[a.depth];
  for (int l = 0; l < a.depth; ++l) a.lin[l] = ctx->w.emb[l];
  switch (ctx->cfg.emb_widths[1]) {
    case 16: return run<16>(ctx, x, y, z, n, a, emb, saved, s);
    case 32: return run<32>(ctx, x, y, z, n, a, emb, saved, s);
    case 64: return run<64>(ctx, x, y, z, n, a, emb, saved, s);
    case 128: return run<128>(ctx, x, y, z, n, a, emb, saved, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_embed(etx_ctx* ctx, const float* x, const float* y, const float* z,
                         int64_t n, float* emb, cudaStream_t s) {
  return dispatch(ctx, x, y, z, n, emb, nullptr, s);
}

cudaError_t launch_embed_save(etx_ctx* ctx, const float* x, const float* y, const float* z,
                              int64_t n, float* emb, float* saved, cudaStream_t s) {
  return dispatch(ctx, x, y, z, n, emb, saved, s);
}

}  // namespace etx
