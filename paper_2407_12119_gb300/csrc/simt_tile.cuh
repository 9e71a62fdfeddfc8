// FP32 SIMT building blocks for row-wise MLPs: a 64-row x N-column register
// tile computed by 256 threads from a shared-memory A tile and a shared-memory
// W^T chunk, and the bias + LayerNorm + ReLU epilogue on that tile.
//
// Thread layout: ty = tid / 16 owns rows 4*ty .. 4*ty+3; tx = tid % 16 owns
// columns g*64 + 4*tx + c (N >= 64, g < N/64, c < 4) or j*16 + tx (N < 64).
// The 16 threads that share a row sit in one half-warp, so row reductions
// are four xor-shuffles.
#pragma once

#include "etx_internal.cuh"

namespace etx {

constexpr int kTileM = 64;
constexpr int kTileThreads = 256;

template <int N>
struct ColMap {
  static constexpr int CPT = N / 16;  // columns per thread
  __device__ __forceinline__ static int col(int tx, int j) {
    if constexpr (N >= 64) {
      return (j >> 2) * 64 + tx * 4 + (j & 3);
    } else {
      return j * 16 + tx;
    }
  }
};

template <int N>
struct TileAcc {
  static constexpr int CPT = N / 16;
  float v[4][CPT];

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < CPT; ++j) v[r][j] = 0.f;
  }

  // acc += A[rows, k0:k0+KC] * Ws[0:KC, :]; A row-major with leading dim lda
  // (floats, multiple of 4), Ws row-major [KC][N].
  template <int KC>
  __device__ __forceinline__ void mma(const float* __restrict__ A, int lda, int k0,
                                      const float* __restrict__ Ws, int ty, int tx) {
#pragma unroll
    for (int kk = 0; kk < KC; kk += 4) {
      float4 a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        a[r] = *reinterpret_cast<const float4*>(A + (ty * 4 + r) * lda + k0 + kk);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float w[CPT];
        const float* wrow = Ws + (kk + c) * N;
        if constexpr (N >= 64) {
#pragma unroll
          for (int g = 0; g < N / 64; ++g) {
            float4 t = *reinterpret_cast<const float4*>(wrow + g * 64 + tx * 4);
            w[g * 4 + 0] = t.x;
            w[g * 4 + 1] = t.y;
            w[g * 4 + 2] = t.z;
            w[g * 4 + 3] = t.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < CPT; ++j) w[j] = wrow[j * 16 + tx];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float av = c == 0 ? a[r].x : c == 1 ? a[r].y : c == 2 ? a[r].z : a[r].w;
          if constexpr (CPT % 2 == 0) {
            // packed FP32x2 FMAs (each lane the same IEEE fma as fmaf)
            const float2 a2 = make_float2(av, av);
#pragma unroll
            for (int j = 0; j < CPT; j += 2) {
              const float2 p = __ffma2_rn(a2, make_float2(w[j], w[j + 1]),
                                          make_float2(v[r][j], v[r][j + 1]));
              v[r][j] = p.x;
              v[r][j + 1] = p.y;
            }
          } else {
#pragma unroll
            for (int j = 0; j < CPT; ++j) v[r][j] = fmaf(av, w[j], v[r][j]);
          }
        }
      }
    }
  }
};

__device__ __forceinline__ float halfwarp_sum(float s) {
  s += __shfl_xor_sync(0xffffffffu, s, 8);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}

// v[r][j] <- ReLU(LN(v + b) * g + be) over the N columns of each row.
template <int N>
__device__ __forceinline__ void bias_ln_relu(TileAcc<N>& t, const float* __restrict__ b,
                                             const float* __restrict__ g,
                                             const float* __restrict__ be, int tx) {
  constexpr int CPT = N / 16;
  float bb[CPT], gg[CPT], ee[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int c = ColMap<N>::col(tx, j);
    bb[j] = __ldg(b + c);
    gg[j] = __ldg(g + c);
    ee[j] = __ldg(be + c);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      t.v[r][j] += bb[j];
      s += t.v[r][j];
    }
    const float mean = halfwarp_sum(s) * (1.0f / N);
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const float d = t.v[r][j] - mean;
      q += d * d;
    }
    const float var = halfwarp_sum(q) * (1.0f / N);
    const float rstd = 1.0f / sqrtf(var + kLnEps);
#pragma unroll
    for (int j = 0; j < CPT; ++j)
      t.v[r][j] = fmaxf((t.v[r][j] - mean) * rstd * gg[j] + ee[j], 0.f);
  }
}

// Copy a contiguous [KC][N] chunk of W^T from global memory into shared memory.
template <int KC, int N>
__device__ __forceinline__ void load_w_chunk(float* __restrict__ Ws,
                                             const float* __restrict__ wt, int tid) {
  constexpr int NV = KC * N / 4;
  const float4* src = reinterpret_cast<const float4*>(wt);
  float4* dst = reinterpret_cast<float4*>(Ws);
#pragma unroll
  for (int i = tid; i < NV; i += kTileThreads) dst[i] = __ldg(src + i);
}

// Store the tile's values as rows of a row-major shared array (lda floats).
template <int N>
__device__ __forceinline__ void store_tile_smem(const TileAcc<N>& t, float* A, int lda, int ty,
                                                int tx) {
  constexpr int CPT = N / 16;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float* row = A + (ty * 4 + r) * lda;
    if constexpr (N >= 64) {
#pragma unroll
      for (int g = 0; g < N / 64; ++g)
        *reinterpret_cast<float4*>(row + g * 64 + tx * 4) =
            make_float4(t.v[r][g * 4], t.v[r][g * 4 + 1], t.v[r][g * 4 + 2], t.v[r][g * 4 + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < CPT; ++j) row[j * 16 + tx] = t.v[r][j];
    }
  }
}

}  // namespace etx
