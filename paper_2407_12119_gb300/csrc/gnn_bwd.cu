// Reverse pass of the interaction network (training), FP32 SIMT.
//
// Forward (paper Sec. 5.2, Eq. 4), per message-passing step k:
//     m^k = [sum_{l->j} e^k_lj, sum_{i->l} e^k_il]
//     h^{k+1} = h^k + f_node,k([h^k, m^k])
//     e^{k+1} = e^k + f_edge,k([e^k, h^{k+1}_i, h^{k+1}_j])
// with f = Lin -> LN -> ReLU -> Lin -> LN -> ReLU, then the classifier
// logit = w . ReLU(LN(Lin(e^L))) + b.  A training forward keeps h^k and e^k
// (checkpoints); this pass walks the steps backwards and, for each block,
// recomputes its forward from the checkpoint inside one fused tile kernel
// (k_block_bwd) that also runs the block's backward: LayerNorm / ReLU
// derivatives, dr1 = da2 W2 and dX = da1 W1.  The per-row factors are written
// out so that the weight gradients reduce over rows afterwards
// (dW = da^T X by k_gemm_tn, bias / LayerNorm terms by column sums).  The
// gradient of the gathers h_i, h_j is a segment sum over the src-sorted and
// dst-permuted edge lists; the gradient of the message sums is a gather.
// No global atomics on the per-row data; weight-gradient partials of each
// CTA are added with atomics (a few per weight).
#include <algorithm>

#include "simt_tile.cuh"

namespace etx {
namespace {

constexpr int kKC = 16;
constexpr int kLdaChunk = kKC + 4;

enum BMode { B_NODE_ENC = 0, B_EDGE_ENC = 1, B_NODE_UPD = 2, B_EDGE_UPD = 3, B_CLS = 4 };

struct BwdArgs {
  int64_t n_nodes;
  const int32_t* n_edges_dev;
  const float *x, *y, *z;
  const float* norm;         // gnn mu[3], sigma[3]
  const int32_t *src, *dst;
  const float* hg;           // node rows gathered by this block
  const float* ein;          // edge rows (edge update input / classifier input)
  const float* m;            // messages (node update)
  const float* gout;         // incoming gradient rows [R][H] (blocks)
  const float* dlogit;       // incoming gradient [E] (classifier)
  LinF32 l1, l2;             // forward layouts (W^T)
  const float* W1;           // original [H][K]
  const float* W2;           // original [H][H]
  const float *g1, *be1, *g2, *be2;
  const float* wcls;         // classifier last Linear [H]
  int K;                     // row width of the block input (4 for the node encoder)
  // per-row outputs
  float *X, *R1, *DA1, *DY1, *DY1N1, *DA2, *DY2, *DY2N2, *DX;
};

template <int H, int MODE>
__device__ __forceinline__ float4 gather4_bwd(const BwdArgs& a, int64_t row, bool valid, int k,
                                              int s, int d) {
  if (!valid) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float* p;
  if constexpr (MODE == B_EDGE_ENC) {
    p = k < H ? a.hg + (int64_t)s * H + k : a.hg + (int64_t)d * H + (k - H);
  } else if constexpr (MODE == B_NODE_UPD) {
    p = k < H ? a.hg + row * H + k : a.m + row * 2 * H + (k - H);
  } else if constexpr (MODE == B_EDGE_UPD) {
    p = k < H ? a.ein + row * H + k
              : (k < 2 * H ? a.hg + (int64_t)s * H + (k - H) : a.hg + (int64_t)d * H + (k - 2 * H));
  } else {  // B_CLS
    p = a.ein + row * H + k;
  }
  return *reinterpret_cast<const float4*>(p);
}

// Load Ws[kk][n] = B[(k0 + kk) * ldb + n0 + n] for kk < KC, n < N (zero outside nmax).
template <int KC, int N>
__device__ __forceinline__ void load_b_strided(float* __restrict__ Ws, const float* __restrict__ B,
                                               int64_t ldb, int k0, int kmax, int n0, int nmax,
                                               int tid) {
  for (int i = tid; i < KC * N; i += kTileThreads) {
    const int kk = i / N, n = i - kk * N;
    const int kr = k0 + kk, nc = n0 + n;
    Ws[i] = (kr < kmax && nc < nmax) ? __ldg(B + (int64_t)kr * ldb + nc) : 0.f;
  }
}

// Per-row mean over H of t (4 rows x CPT columns per thread, 16 threads per row).
template <int H>
__device__ __forceinline__ void row_means(const TileAcc<H>& t, float (&mean)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < H / 16; ++j) s += t.v[r][j];
    mean[r] = halfwarp_sum(s) * (1.0f / H);
  }
}

template <int H>
__device__ __forceinline__ void store_rows_global(const TileAcc<H>& t, float* __restrict__ out,
                                                  int64_t ld, int64_t row0, int64_t n_rows, int ty,
                                                  int tx, int coff = 0) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t row = row0 + ty * 4 + r;
    if (row >= n_rows) continue;
#pragma unroll
    for (int j = 0; j < H / 16; ++j) out[row * ld + coff + ColMap<H>::col(tx, j)] = t.v[r][j];
  }
}

template <int H, int MODE>
__global__ void __launch_bounds__(kTileThreads) k_block_bwd(BwdArgs a) {
  constexpr int LDS = H + 4;
  constexpr int CPT = H / 16;
  extern __shared__ __align__(16) float sm[];
  float* As = sm;                        // [64][20]
  float* Ws = As + kTileM * kLdaChunk;   // [16][H]
  float* S1 = Ws + kKC * H;              // n1   [64][H+4]
  float* S2 = S1 + kTileM * LDS;         // r1
  float* S3 = S2 + kTileM * LDS;         // da2, then da1
  __shared__ int s_src[kTileM], s_dst[kTileM];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t n_rows = (MODE == B_NODE_ENC || MODE == B_NODE_UPD) ? a.n_nodes : (int64_t)*a.n_edges_dev;
  const int64_t n_tiles = (n_rows + kTileM - 1) / kTileM;
  const int K = a.K;
  const int nn = (int)a.n_nodes;

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTileM;
    __syncthreads();
    if constexpr (MODE == B_EDGE_ENC || MODE == B_EDGE_UPD) {
      if (tid < kTileM) {
        const int64_t r = row0 + tid;
        s_src[tid] = r < n_rows ? min(max(a.src[r], 0), max(nn - 1, 0)) : 0;
        s_dst[tid] = r < n_rows ? min(max(a.dst[r], 0), max(nn - 1, 0)) : 0;
      }
    }
    // ---- forward recompute: GEMM 1 -------------------------------------------
    TileAcc<H> acc;
    acc.zero();
    if constexpr (MODE == B_NODE_ENC) {
      if (tid < kTileM) {
        const int64_t r = row0 + tid;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < n_rows) {
          f.x = (a.x[r] - __ldg(a.norm + 0)) / __ldg(a.norm + 3);
          f.y = (a.y[r] - __ldg(a.norm + 1)) / __ldg(a.norm + 4);
          f.z = (a.z[r] - __ldg(a.norm + 2)) / __ldg(a.norm + 5);
          *reinterpret_cast<float4*>(a.X + r * 4) = f;
        }
        *reinterpret_cast<float4*>(As + tid * 4) = f;
      }
      if (tid < H) reinterpret_cast<float4*>(Ws)[tid] = __ldg(reinterpret_cast<const float4*>(a.l1.wt) + tid);
      __syncthreads();
      acc.template mma<4>(As, 4, 0, Ws, ty, tx);
    } else {
      const int qrow = tid >> 2, qk = (tid & 3) * 4;
      const int64_t grow = row0 + qrow;
      const bool valid = grow < n_rows;
      for (int k0 = 0; k0 < K; k0 += kKC) {
        __syncthreads();
        const float4 f = (MODE == B_EDGE_ENC || MODE == B_EDGE_UPD)
                             ? gather4_bwd<H, MODE>(a, grow, valid, k0 + qk, s_src[qrow], s_dst[qrow])
                             : gather4_bwd<H, MODE>(a, grow, valid, k0 + qk, 0, 0);
        *reinterpret_cast<float4*>(As + qrow * kLdaChunk + qk) = f;
        if (valid) *reinterpret_cast<float4*>(a.X + grow * K + k0 + qk) = f;
        load_w_chunk<kKC, H>(Ws, a.l1.wt + (size_t)k0 * H, tid);
        __syncthreads();
        acc.template mma<kKC>(As, kLdaChunk, 0, Ws, ty, tx);
      }
    }
    // v1 = acc + b1; n1 = LN-normalised; r1 = ReLU(n1 g1 + be1)
    float rstd1[4];
    {
      float b[CPT];
#pragma unroll
      for (int j = 0; j < CPT; ++j) b[j] = __ldg(a.l1.b + ColMap<H>::col(tx, j));
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc.v[r][j] += b[j];
      float mean[4];
      row_means<H>(acc, mean);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          acc.v[r][j] -= mean[r];
          q += acc.v[r][j] * acc.v[r][j];
        }
        rstd1[r] = 1.0f / sqrtf(halfwarp_sum(q) * (1.0f / H) + kLnEps);
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc.v[r][j] *= rstd1[r];
      }
    }
    store_tile_smem<H>(acc, S1, LDS, ty, tx);  // n1
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int c = ColMap<H>::col(tx, j);
      const float g = __ldg(a.g1 + c), be = __ldg(a.be1 + c);
#pragma unroll
      for (int r = 0; r < 4; ++r) acc.v[r][j] = fmaxf(acc.v[r][j] * g + be, 0.f);
    }
    store_tile_smem<H>(acc, S2, LDS, ty, tx);  // r1
    store_rows_global<H>(acc, a.R1, H, row0, n_rows, ty, tx);

    TileAcc<H> dy;  // gradient at y1 = n1 g1 + be1 (after the ReLU mask)
    if constexpr (MODE == B_CLS) {
      // logit = wcls . r1 + b: dr1 = dlogit * wcls
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t row = row0 + ty * 4 + r;
        const float dl = row < n_rows ? a.dlogit[row] : 0.f;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int c = ColMap<H>::col(tx, j);
          dy.v[r][j] = acc.v[r][j] > 0.f ? dl * __ldg(a.wcls + c) : 0.f;
        }
      }
    } else {
      // ---- forward recompute: GEMM 2 -----------------------------------------
      TileAcc<H> t2;
      t2.zero();
      for (int k0 = 0; k0 < H; k0 += kKC) {
        __syncthreads();
        load_w_chunk<kKC, H>(Ws, a.l2.wt + (size_t)k0 * H, tid);
        __syncthreads();
        t2.template mma<kKC>(S2, LDS, k0, Ws, ty, tx);
      }
      float rstd2[4];
      {
        float b[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) b[j] = __ldg(a.l2.b + ColMap<H>::col(tx, j));
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int j = 0; j < CPT; ++j) t2.v[r][j] += b[j];
        float mean[4];
        row_means<H>(t2, mean);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float q = 0.f;
#pragma unroll
          for (int j = 0; j < CPT; ++j) {
            t2.v[r][j] -= mean[r];
            q += t2.v[r][j] * t2.v[r][j];
          }
          rstd2[r] = 1.0f / sqrtf(halfwarp_sum(q) * (1.0f / H) + kLnEps);
#pragma unroll
          for (int j = 0; j < CPT; ++j) t2.v[r][j] *= rstd2[r];  // n2
        }
      }
      // ---- backward through LN2 / ReLU ---------------------------------------
      TileAcc<H> tg;  // t = dy2 * g2
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t row = row0 + ty * 4 + r;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int c = ColMap<H>::col(tx, j);
          const float g2 = __ldg(a.g2 + c), be2 = __ldg(a.be2 + c);
          const float y2 = t2.v[r][j] * g2 + be2;
          const float go = row < n_rows ? a.gout[row * H + c] : 0.f;
          const float d = y2 > 0.f ? go : 0.f;
          dy.v[r][j] = d;
          tg.v[r][j] = d * g2;
        }
      }
      store_rows_global<H>(dy, a.DY2, H, row0, n_rows, ty, tx);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < CPT; ++j) dy.v[r][j] *= t2.v[r][j];
      store_rows_global<H>(dy, a.DY2N2, H, row0, n_rows, ty, tx);
      {
        float m1[4], m2[4];
        row_means<H>(tg, m1);
        TileAcc<H> tn;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int j = 0; j < CPT; ++j) tn.v[r][j] = tg.v[r][j] * t2.v[r][j];
        row_means<H>(tn, m2);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int j = 0; j < CPT; ++j)
            tg.v[r][j] = rstd2[r] * (tg.v[r][j] - m1[r] - t2.v[r][j] * m2[r]);  // da2
      }
      store_rows_global<H>(tg, a.DA2, H, row0, n_rows, ty, tx);
      __syncthreads();
      store_tile_smem<H>(tg, S3, LDS, ty, tx);
      // dr1 = da2 W2 (W2 original [out][in]: rows out are the reduction index)
      TileAcc<H> t3;
      t3.zero();
      for (int k0 = 0; k0 < H; k0 += kKC) {
        __syncthreads();
        load_w_chunk<kKC, H>(Ws, a.W2 + (size_t)k0 * H, tid);
        __syncthreads();
        t3.template mma<kKC>(S3, LDS, k0, Ws, ty, tx);
      }
      // dy1 = dr1 where r1 > 0
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const float r1 = S2[(ty * 4 + r) * LDS + ColMap<H>::col(tx, j)];
          dy.v[r][j] = r1 > 0.f ? t3.v[r][j] : 0.f;
        }
    }
    // ---- backward through LN1 --------------------------------------------------
    {
      TileAcc<H> tg, n1;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int c = ColMap<H>::col(tx, j);
          n1.v[r][j] = S1[(ty * 4 + r) * LDS + c];
          tg.v[r][j] = dy.v[r][j] * __ldg(a.g1 + c);
        }
      store_rows_global<H>(dy, a.DY1, H, row0, n_rows, ty, tx);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < CPT; ++j) dy.v[r][j] *= n1.v[r][j];
      store_rows_global<H>(dy, a.DY1N1, H, row0, n_rows, ty, tx);
      float m1[4], m2[4];
      row_means<H>(tg, m1);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < CPT; ++j) dy.v[r][j] = tg.v[r][j] * n1.v[r][j];
      row_means<H>(dy, m2);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < CPT; ++j)
          tg.v[r][j] = rstd1[r] * (tg.v[r][j] - m1[r] - n1.v[r][j] * m2[r]);  // da1
      store_rows_global<H>(tg, a.DA1, H, row0, n_rows, ty, tx);
      if constexpr (MODE != B_NODE_ENC) {
        __syncthreads();
        store_tile_smem<H>(tg, S3, LDS, ty, tx);
      }
    }
    // ---- dX = da1 W1 (W1 original [H][K]), column blocks of H -------------------
    if constexpr (MODE != B_NODE_ENC) {
      for (int n0 = 0; n0 < K; n0 += H) {
        TileAcc<H> t4;
        t4.zero();
        for (int k0 = 0; k0 < H; k0 += kKC) {
          __syncthreads();
          load_b_strided<kKC, H>(Ws, a.W1, K, k0, H, n0, K, tid);
          __syncthreads();
          t4.template mma<kKC>(S3, LDS, k0, Ws, ty, tx);
        }
        store_rows_global<H>(t4, a.DX, K, row0, n_rows, ty, tx, n0);
      }
    }
  }
}

// C[M][N] (+)= sum_r A[r][m] * B[r][n], r < R (device count or host count).
// Grid: (M / 64) x ceil(N / 128) x splits over r; each CTA adds its partial.
__global__ void __launch_bounds__(kTileThreads)
k_gemm_tn(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb, int M, int N,
          int64_t R_host, const int32_t* __restrict__ R_dev, float* __restrict__ C,
          float* __restrict__ P) {
  constexpr int NT = 128;
  __shared__ __align__(16) float As[kTileM * kLdaChunk];
  __shared__ __align__(16) float Ws[kKC * NT];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * NT;
  const int64_t R = R_dev ? (int64_t)*R_dev : R_host;
  const int64_t chunks = (R + kKC - 1) / kKC;
  const int64_t per = (chunks + gridDim.z - 1) / gridDim.z;
  const int64_t c_lo = blockIdx.z * per, c_hi = min(chunks, c_lo + per);
  TileAcc<NT> acc;
  acc.zero();
  for (int64_t ch = c_lo; ch < c_hi; ++ch) {
    const int64_t r0 = ch * kKC;
    __syncthreads();
    for (int i = tid; i < kTileM * kKC; i += kTileThreads) {
      const int rr = i / kTileM, mm = i - rr * kTileM;  // consecutive threads: consecutive m
      const int64_t r = r0 + rr;
      As[mm * kLdaChunk + rr] = (r < R && m0 + mm < M) ? A[r * lda + m0 + mm] : 0.f;
    }
    for (int i = tid; i < kKC * NT; i += kTileThreads) {
      const int rr = i / NT, n = i - rr * NT;
      const int64_t r = r0 + rr;
      Ws[i] = (r < R && n0 + n < N) ? B[r * ldb + n0 + n] : 0.f;
    }
    __syncthreads();
    acc.template mma<kKC>(As, kLdaChunk, 0, Ws, ty, tx);
  }
  // P != NULL: this split's partial tile (zeros if it had no rows) goes to
  // P[z][M][N] and k_reduce_parts adds the splits in order (fixed summation
  // order: the same inputs give the same bits); otherwise atomics into C.
  if (!P && c_lo >= c_hi) return;
  float* Pz = P ? P + (int64_t)blockIdx.z * M * N : nullptr;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int m = m0 + ty * 4 + r;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < NT / 16; ++j) {
      const int n = n0 + ColMap<NT>::col(tx, j);
      if (n >= N) continue;
      if (Pz) Pz[(int64_t)m * N + n] = c_lo < c_hi ? acc.v[r][j] : 0.f;
      else atomicAdd(C + (int64_t)m * N + n, acc.v[r][j]);
    }
  }
}

// C[i] += sum over z = 0 .. splits-1, in that order, of P[z][i], i < MN.
__global__ void k_reduce_parts(const float* __restrict__ P, int splits, int64_t MN,
                               float* __restrict__ C) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN;
       i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
#pragma unroll 8
    for (int z = 0; z < splits; ++z) acc += P[(int64_t)z * MN + i];  // loads in flight, adds in order
    C[i] += acc;
  }
}

// The same sum for a short vector over many partials (column sums): a block
// takes 32 outputs; warp y adds the partials z = y, y + 8, ... (consecutive
// lanes read consecutive outputs), and the 8 warp sums are added in warp order.
__global__ void __launch_bounds__(256) k_reduce_parts_narrow(const float* __restrict__ P, int splits,
                                                             int64_t MN, float* __restrict__ C) {
  __shared__ float sh[8][32];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + x;
  float acc = 0.f;
  if (i < MN)
    for (int z = y; z < splits; z += 8) acc += P[(int64_t)z * MN + i];
  sh[y][x] = acc;
  __syncthreads();
  if (y == 0 && i < MN) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sh[w][x];
    C[i] += t;
  }
}

// Sum of the threads' values of a block in a fixed order (warp trees, then
// the warp totals in warp order); the result is valid in thread 0.
__device__ __forceinline__ float block_sum_fixed(float v, float* sh) {
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;
}

// *out = scale * sum of part[0 .. n-1] in a fixed order (one block).
__global__ void k_finish_sum(const float* __restrict__ part, int n, float scale,
                             float* __restrict__ out) {
  __shared__ float sh[32];
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  const float t = block_sum_fixed(acc, sh);
  if (threadIdx.x == 0) *out = t * scale;
}

// out[c] += sum_r A[r][c] * (w ? w[r] : 1), c < H; blocks split the rows.
// part != NULL: block b writes its column sums to part[b][H] (summed later in
// block order by k_reduce_parts); otherwise atomics into out.
__global__ void k_colsum(const float* __restrict__ A, int H, const float* __restrict__ w,
                         int64_t R_host, const int32_t* __restrict__ R_dev, float* __restrict__ out,
                         float* __restrict__ part) {
  const int64_t R = R_dev ? (int64_t)*R_dev : R_host;
  const int c = threadIdx.x;
  if (c >= H) return;
  float s = 0.f;
  for (int64_t r = blockIdx.x; r < R; r += gridDim.x) s += A[r * H + c] * (w ? w[r] : 1.f);
  if (part) part[(int64_t)blockIdx.x * H + c] = s;
  else atomicAdd(out + c, s);
}

// Column sums of three [R][H] arrays at once (a layer's bias, LayerNorm-gain and
// LayerNorm-shift gradients): block b writes part[b][3][H].
__global__ void k_colsum3(const float* __restrict__ A0, const float* __restrict__ A1,
                          const float* __restrict__ A2, int H, int64_t R_host,
                          const int32_t* __restrict__ R_dev, float* __restrict__ part) {
  const int64_t R = R_dev ? (int64_t)*R_dev : R_host;
  const int c = threadIdx.x;
  if (c >= H) return;
  // four rows in flight per array (independent partial sums, fixed order)
  float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f};
  const int64_t G = gridDim.x;
  int64_t r = blockIdx.x;
  for (; r + 3 * G < R; r += 4 * G) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = (r + u * G) * H + c;
      s0[u] += A0[i];
      s1[u] += A1[i];
      s2[u] += A2[i];
    }
  }
  for (int u = 0; r < R; r += G, ++u) {
    const int64_t i = r * H + c;
    s0[u] += A0[i];
    s1[u] += A1[i];
    s2[u] += A2[i];
  }
  float* o = part + (int64_t)blockIdx.x * 3 * H;
  o[c] = (s0[0] + s0[1]) + (s0[2] + s0[3]);
  o[H + c] = (s1[0] + s1[1]) + (s1[2] + s1[3]);
  o[2 * H + c] = (s2[0] + s2[1]) + (s2[2] + s2[3]);
}

// part[blockIdx.x] = this block's sum (fixed order); k_finish_sum adds the blocks.
__global__ void k_sum(const float* __restrict__ a, int64_t R_host, const int32_t* __restrict__ R_dev,
                      float* __restrict__ part) {
  __shared__ float sh[32];
  const int64_t R = R_dev ? (int64_t)*R_dev : R_host;
  float s = 0.f;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x)
    s += a[r];
  const float t = block_sum_fixed(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Y[r][c] = (accumulate ? Y[r][c] : 0) + X[r][c0 + c] for c < H.
__global__ void k_add_cols(float* __restrict__ Y, int H, const float* __restrict__ X, int ldx, int c0,
                           int accumulate, int64_t R_host, const int32_t* __restrict__ R_dev) {
  const int64_t R = R_dev ? (int64_t)*R_dev : R_host;
  const int64_t n = R * H;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / H;
    const int c = (int)(i - r * H);
    const float v = X[r * ldx + c0 + c];
    Y[i] = accumulate ? Y[i] + v : v;
  }
}

// dh[l] += sum_{e: src(e)=l} G[e][cs..cs+H) + sum_{e: dst(e)=l} G[e][cd..cd+H)
// (gradient of the h_i / h_j gathers; segments of the sorted edge lists).
template <int H>
__global__ void k_scatter_bwd(const float* __restrict__ G, int ldg, int cs, int cd,
                              const int32_t* __restrict__ out_off, const int32_t* __restrict__ in_off,
                              const int32_t* __restrict__ perm, const int32_t* __restrict__ n_edges_dev,
                              int n_hits, float* __restrict__ dh) {
  constexpr int GL = H / 4;
  constexpr int PER_WARP = 32 / GL;
  const int E = *n_edges_dev;
  const int lane = threadIdx.x & 31, sub = lane / GL, c = (lane % GL) * 4;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t l0 = warp0 * PER_WARP; l0 < n_hits; l0 += nwarps * PER_WARP) {
    const int64_t l = l0 + sub;
    if (l >= n_hits) continue;
    const int o0 = min(max(out_off[l], 0), E), o1 = min(max(out_off[l + 1], 0), E);
    const int i0 = min(max(in_off[l], 0), E), i1 = min(max(in_off[l + 1], 0), E);
    float4 s = *reinterpret_cast<const float4*>(dh + l * H + c);
    for (int q = o0; q < o1; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(G + (int64_t)q * ldg + cs + c);
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
    for (int q = i0; q < i1; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(G + (int64_t)perm[q] * ldg + cd + c);
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
    *reinterpret_cast<float4*>(dh + l * H + c) = s;
  }
}

// de[e] += G[src(e)][cs..cs+H) + G[dst(e)][cd..cd+H)  (gradient of the message sums)
template <int H>
__global__ void k_gather_bwd(const float* __restrict__ G, int ldg, int cs, int cd,
                             const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                             const int32_t* __restrict__ n_edges_dev, int n_hits, float* __restrict__ de) {
  const int64_t E = *n_edges_dev;
  const int64_t n = E * (H / 4);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / (H / 4);
    const int c = (int)(i - e * (H / 4)) * 4;
    const int s = min(max(src[e], 0), n_hits - 1), d = min(max(dst[e], 0), n_hits - 1);
    const float4 a = *reinterpret_cast<const float4*>(G + (int64_t)s * ldg + cs + c);
    const float4 b = *reinterpret_cast<const float4*>(G + (int64_t)d * ldg + cd + c);
    float4 o = *reinterpret_cast<const float4*>(de + e * H + c);
    o.x += a.x + b.x; o.y += a.y + b.y; o.z += a.z + b.z; o.w += a.w + b.w;
    *reinterpret_cast<float4*>(de + e * H + c) = o;
  }
}

// Offsets (floats) of one block's parameters in the flat gradient buffer.
struct BlockGrad {
  float *W1, *b1, *g1, *be1, *W2, *b2, *g2, *be2;
};

// Splits over rows of a weight-gradient GEMM and blocks of a column sum; the
// context's partial buffer is sized for the largest of them.
// (about 4,096 rows per split, so the partials stay a small fraction of the
// rows read).
inline int grad_splits(const etx_ctx* ctx, int64_t rows) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ctx->n_sms, (rows + 4095) / 4096));
}
inline int colsum_blocks(const etx_ctx* ctx, int64_t rows) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ctx->n_sms * 4, (rows + 127) / 128));
}

template <int H>
struct Bwd {
  etx_ctx* ctx;
  cudaStream_t s;
  const int32_t* n_edges;
  int64_t N;
  int64_t Ecap;

  size_t smem_block() const { return (size_t)(kTileM * kLdaChunk + kKC * H + 3 * kTileM * (H + 4)) * 4; }

  template <int MODE>
  void block_pass(BwdArgs a, int64_t max_rows) {
    static bool attr[8] = {false};
    if (!attr[ctx->device & 7]) {
      cudaFuncSetAttribute(k_block_bwd<H, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_block());
      attr[ctx->device & 7] = true;
    }
    const int64_t tiles = (max_rows + kTileM - 1) / kTileM;
    if (tiles == 0) return;
    const int grid = grid_for(ctx, (const void*)k_block_bwd<H, MODE>, kTileThreads, smem_block(), tiles);
    launch(ctx, "gnn_block_backward_f32", k_block_bwd<H, MODE>, grid, kTileThreads, smem_block(), s, a);
  }

  // dW (M x N, split over rows into partial tiles) or column sums, each added
  // to its gradient in a fixed order (ctx->bw_part holds the partials).
  // H = 128 with 128, 256 or 384 input columns: TF32 tensor cores, one split
  // per SM; otherwise the FP32 SIMT GEMM.
  void weight_grad(const float* A, int lda, const float* B, int ldb, int M, int Ncols, int64_t Rh,
                   const int32_t* Rd, int splits, float* out) {
    if (wgrad_tc_supported(M, Ncols)) {
      const int64_t Rcap = Rd ? Ecap : Rh;
      const int sp = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->n_sms, (Rcap + 255) / 256));
      launch_wgrad_tc(ctx, A, lda, B, ldb, Ncols, Rh, Rd, Rcap, sp, ctx->bw_part, s);
      reduce(sp, (int64_t)M * Ncols, out);
      return;
    }
    // a narrow dW (the node encoder's 3 inputs) is a few hundred values: split its
    // rows finely (about 128 a CTA) so the row loop is not a serial latency chain
    if (Ncols <= 32) {
      const int64_t Rcap = Rd ? Ecap : Rh;
      const int64_t cap = (int64_t)ctx->n_sms * H * 3 * H / ((int64_t)M * Ncols);  // bw_part size
      splits = (int)std::max<int64_t>(splits, std::min<int64_t>({(int64_t)ctx->n_sms * 4, (Rcap + 127) / 128, cap}));
    }
    launch(ctx, "gnn_weight_grad", k_gemm_tn, dim3((M + kTileM - 1) / kTileM, (Ncols + 127) / 128, splits),
           kTileThreads, 0, s, A, lda, B, ldb, M, Ncols, Rh, Rd, out, ctx->bw_part);
    reduce(splits, (int64_t)M * Ncols, out);
  }
  void colsum(const float* A, const float* w, int64_t Rh, const int32_t* Rd, int cb, float* out) {
    launch(ctx, "gnn_colsum", k_colsum, cb, H, 0, s, A, H, w, Rh, Rd, out, ctx->bw_part);
    reduce(cb, H, out);
  }
  // out[0..3H) = column sums of A0, A1, A2 (a layer's b, g, be gradients, contiguous)
  void colsum3(const float* A0, const float* A1, const float* A2, int64_t Rh, const int32_t* Rd,
               int cb, float* out) {
    launch(ctx, "gnn_colsum", k_colsum3, cb, H, 0, s, A0, A1, A2, H, Rh, Rd, ctx->bw_part);
    reduce(cb, 3 * H, out);
  }
  void reduce(int parts, int64_t n, float* out, const float* src = nullptr) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ctx->n_sms * 4));
    const float* P = src ? src : (const float*)ctx->bw_part;
    if (n <= 4096 && parts >= 64)
      launch(ctx, "gnn_grad_reduce", k_reduce_parts_narrow, (int)((n + 31) / 32), 256, 0, s, P, parts, n, out);
    else
      launch(ctx, "gnn_grad_reduce", k_reduce_parts, g, 256, 0, s, P, parts, n, out);
  }

  // Parameter gradients of a block whose reverse pass ran on the tensor cores:
  // the weight gradients from the per-row factors, the b, g, be gradients of
  // both layers from the column-sum partials that pass left.
  void param_grads_tc(const BwdArgs& a, const BlockGrad& g, int K, bool is_edge) {
    const int32_t* Rd = is_edge ? n_edges : nullptr;
    const int64_t Rh = is_edge ? 0 : N;
    const int64_t Rcap = is_edge ? Ecap : N;
    const int splits = grad_splits(ctx, Rcap);
    const int parts = block_bwd_tc_colsum_parts(ctx, Rcap);
    weight_grad(a.DA1, H, a.X, K, H, K, Rh, Rd, splits, g.W1);
    reduce(parts, 3 * H, g.b1, ctx->bw_cs_part + (size_t)ctx->n_sms * 4 * 3 * H);
    weight_grad(a.DA2, H, a.R1, H, H, H, Rh, Rd, splits, g.W2);
    reduce(parts, 3 * H, g.b2, ctx->bw_cs_part);
  }

  // Parameter gradients of one block from the per-row factors.
  void param_grads(const BwdArgs& a, const BlockGrad& g, int K, bool is_edge, bool has_l2) {
    const int32_t* Rd = is_edge ? n_edges : nullptr;
    const int64_t Rh = is_edge ? 0 : N;
    const int64_t Rcap = is_edge ? Ecap : N;
    const int splits = grad_splits(ctx, Rcap);
    const int kreal = K == 4 ? 3 : K;  // the node encoder input is padded 3 -> 4
    weight_grad(a.DA1, H, a.X, K, H, kreal, Rh, Rd, splits, g.W1);
    const int cb = colsum_blocks(ctx, Rcap);
    // b1, g1, be1 (and b2, g2, be2) are contiguous in the blob
    colsum3(a.DA1, a.DY1N1, a.DY1, Rh, Rd, cb, g.b1);
    if (has_l2) {
      weight_grad(a.DA2, H, a.R1, H, H, H, Rh, Rd, splits, g.W2);
      colsum3(a.DA2, a.DY2N2, a.DY2, Rh, Rd, cb, g.b2);
    }
  }
};

}  // namespace

namespace {

template <int H>
cudaError_t backward(etx_ctx* ctx, const float* dlogits, float* dparams, cudaStream_t s) {
  const etx_config& c = ctx->cfg;
  const int L = c.n_iters;
  const int64_t N = ctx->fwd_n_hits;
  const int64_t Ecap = c.max_edges;
  Bwd<H> b{ctx, s, ctx->n_edges, N, Ecap};
  // flat parameter offsets (blob order of the interaction network)
  int64_t off = 0;
  auto take = [&](int64_t n) { float* p = dparams + off; off += n; return p; };
  auto block_grad = [&](int K) {
    BlockGrad g;
    g.W1 = take((int64_t)H * K);
    g.b1 = take(H);
    g.g1 = take(H);
    g.be1 = take(H);
    g.W2 = take((int64_t)H * H);
    g.b2 = take(H);
    g.g2 = take(H);
    g.be2 = take(H);
    return g;
  };
  const int64_t gnn0 = ctx->gnn_blob_offset;
  auto orig = [&](const float* grad_ptr) { return ctx->blob_dev + gnn0 + (grad_ptr - dparams); };
  BlockGrad g_node_enc = block_grad(3), g_edge_enc = block_grad(2 * H);
  std::vector<BlockGrad> g_node, g_edge;
  for (int k = 0; k < L; ++k) {
    g_node.push_back(block_grad(3 * H));
    g_edge.push_back(block_grad(3 * H));
  }
  float* gc_W1 = take((int64_t)H * H);
  float* gc_b1 = take(H);
  float* gc_g1 = take(H);
  float* gc_be1 = take(H);
  float* gc_W2 = take(H);
  float* gc_b2 = take(1);
  cudaError_t e = cudaMemsetAsync(dparams, 0, (size_t)off * sizeof(float), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ctx->dh, 0, (size_t)N * H * sizeof(float), s);
  if (e != cudaSuccess) return e;

  BwdArgs base{};
  base.n_nodes = N;
  base.n_edges_dev = ctx->n_edges;
  base.x = ctx->fwd_x;
  base.y = ctx->fwd_y;
  base.z = ctx->fwd_z;
  base.norm = ctx->w.norm + 6;
  base.src = ctx->fwd_src;
  base.dst = ctx->fwd_dst;
  base.X = ctx->bw_X;
  base.R1 = ctx->bw_R1;
  base.DA1 = ctx->bw_DA1;
  base.DY1 = ctx->bw_DY1;
  base.DY1N1 = ctx->bw_DY1N1;
  base.DA2 = ctx->bw_DA2;
  base.DY2 = ctx->bw_DY2;
  base.DY2N2 = ctx->bw_DY2N2;
  base.DX = ctx->bw_DX;
  auto set_block = [&](BwdArgs& a, const BlockF32& w, const BlockGrad& g) {
    a.l1 = w.l1;
    a.l2 = w.l2;
    a.g1 = w.g1;
    a.be1 = w.be1;
    a.g2 = w.g2;
    a.be2 = w.be2;
    a.W1 = orig(g.W1);
    a.W2 = orig(g.W2);
  };
  // H = 128: the edge encoder, node and edge updates on the tensor cores (TF32),
  // from TF32 images of their weights refreshed here
  const bool tc = H == 128 && ctx->bw_img && block_bwd_tc_supported(ctx);
  struct Img { float *W1n, *W1t, *W2n, *W2t, *W1n_lo, *W2n_lo; };
  std::vector<Img> imgs;  // edge encoder, then node k and edge k for k = 0..L-1
  if (tc) {
    float* q = ctx->bw_img;
    const bool fill = ctx->bw_img_jobs_host.empty();
    if (fill) ctx->bw_img_jobs_host.resize((size_t)ctx->bw_img_n_jobs * tf32_image_job_bytes());
    int j = 0;
    auto add = [&](const BlockF32& w, const BlockGrad& g, int K) {
      const size_t hk = (size_t)H * K, hh = (size_t)H * H;
      Img im{q, q + hk, q + 3 * hk, q + 3 * hk + hh, q + 2 * hk, q + 3 * hk + 2 * hh};
      q += 3 * hk + 3 * hh;
      if (fill) {
        unsigned char* jh = ctx->bw_img_jobs_host.data();
        tf32_image_job(jh, j++, orig(g.W1), im.W1n, (int64_t)hk, false);
        tf32_image_job(jh, j++, w.l1.wt, im.W1t, (int64_t)hk, false);
        tf32_image_job(jh, j++, orig(g.W1), im.W1n_lo, (int64_t)hk, true);
        tf32_image_job(jh, j++, orig(g.W2), im.W2n, (int64_t)hh, false);
        tf32_image_job(jh, j++, w.l2.wt, im.W2t, (int64_t)hh, false);
        tf32_image_job(jh, j++, orig(g.W2), im.W2n_lo, (int64_t)hh, true);
      }
      imgs.push_back(im);
    };
    add(ctx->w.edge_enc, g_edge_enc, 2 * H);
    for (int k = 0; k < L; ++k) {
      add(ctx->w.node[k], g_node[k], 3 * H);
      add(ctx->w.edge[k], g_edge[k], 3 * H);
    }
    if (fill) {
      e = cudaMemcpyAsync(ctx->bw_img_jobs, ctx->bw_img_jobs_host.data(), ctx->bw_img_jobs_host.size(),
                          cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return e;
    }
    e = launch_tf32_images(ctx, ctx->bw_img_jobs, ctx->bw_img_n_jobs, (int64_t)H * 3 * H, s);
    if (e != cudaSuccess) return e;
  }
  // one block's reverse pass on the tensor cores (same stored factors as block_pass)
  auto tc_block = [&](int mode, const BwdArgs& a, const Img& im, int64_t R_host, const int32_t* R_dev) {
    BlockBwdTc p{};
    p.n_nodes = N;
    p.R_host = R_host;
    p.R_dev = R_dev;
    p.hg = a.hg;
    p.ein = a.ein;
    p.m = a.m;
    p.src = a.src;
    p.dst = a.dst;
    p.W1n = im.W1n;
    p.W1t = im.W1t;
    p.W2n = im.W2n;
    p.W2t = im.W2t;
    p.W1n_lo = im.W1n_lo;
    p.W2n_lo = im.W2n_lo;
    p.X_lo = ctx->bw_Xlo;
    p.R1_lo = ctx->bw_R1lo;
    p.cs2 = ctx->bw_cs_part;
    p.cs1 = ctx->bw_cs_part + (size_t)ctx->n_sms * 4 * 3 * H;
    p.b1 = a.l1.b;
    p.g1 = a.g1;
    p.be1 = a.be1;
    p.b2 = a.l2.b;
    p.g2 = a.g2;
    p.be2 = a.be2;
    p.G = a.gout;
    p.X = a.X;
    p.R1 = a.R1;
    p.N1 = ctx->bw_N1;
    p.rstd1 = ctx->bw_rstd1;
    p.DA1 = a.DA1;
    p.DY1 = a.DY1;
    p.DY1N1 = a.DY1N1;
    p.DA2 = a.DA2;
    p.DY2 = a.DY2;
    p.DY2N2 = a.DY2N2;
    p.DX = a.DX;
    return launch_block_bwd_tc(ctx, mode, p, s);
  };
  float* hck = ctx->h_ck;
  float* eck = ctx->e_ck;
  auto hk = [&](int k) { return hck + (size_t)k * N * H; };
  auto ek = [&](int k) { return eck + (size_t)k * Ecap * H; };
  const int ge = grid_for(ctx, (const void*)k_add_cols, 256, 0, (Ecap * H + 255) / 256);
  const int gn = grid_for(ctx, (const void*)k_add_cols, 256, 0, (N * H + 255) / 256);
  const int gs = grid_for(ctx, (const void*)k_scatter_bwd<H>, 256, 0,
                          (N + 8 * (32 / (H / 4)) - 1) / (8 * (32 / (H / 4))));
  const int gg = grid_for(ctx, (const void*)k_gather_bwd<H>, 256, 0, (Ecap * (H / 4) + 255) / 256);

  // ---- classifier ------------------------------------------------------------
  {
    BwdArgs a = base;
    a.ein = ek(L);
    a.dlogit = dlogits;
    a.l1 = ctx->w.cls.l1;
    a.g1 = ctx->w.cls.g1;
    a.be1 = ctx->w.cls.be1;
    a.W1 = orig(gc_W1);
    a.wcls = ctx->w.cls.w2;
    a.K = H;
    b.template block_pass<B_CLS>(a, Ecap);
    BlockGrad g{gc_W1, gc_b1, gc_g1, gc_be1, nullptr, nullptr, nullptr, nullptr};
    b.param_grads(a, g, H, true, false);
    b.colsum(a.R1, dlogits, (int64_t)0, ctx->n_edges, colsum_blocks(ctx, Ecap), gc_W2);
    launch(ctx, "gnn_sum", k_sum, ctx->n_sms, 256, 0, s, dlogits, (int64_t)0,
           (const int32_t*)ctx->n_edges, ctx->bw_part);
    launch(ctx, "gnn_grad_reduce", k_finish_sum, 1, 256, 0, s, (const float*)ctx->bw_part,
           (int)ctx->n_sms, 1.0f, gc_b2);
    launch(ctx, "gnn_add_rows", k_add_cols, ge, 256, 0, s, ctx->de, H, (const float*)ctx->bw_DX, H, 0,
           0, (int64_t)0, (const int32_t*)ctx->n_edges);
  }
  // ---- message-passing steps, last to first -------------------------------------
  for (int k = L - 1; k >= 0; --k) {
    {  // e^{k+1} = e^k + f_edge,k([e^k, h^{k+1}_i, h^{k+1}_j])
      BwdArgs a = base;
      set_block(a, ctx->w.edge[k], g_edge[k]);
      a.ein = ek(k);
      a.hg = hk(k + 1);
      a.gout = ctx->de;
      a.K = 3 * H;
      if (tc) {
        if ((e = tc_block(BWD_EDGE_UPD, a, imgs[2 + 2 * k], 0, ctx->n_edges)) != cudaSuccess) return e;
      } else {
        b.template block_pass<B_EDGE_UPD>(a, Ecap);
      }
      if (tc) b.param_grads_tc(a, g_edge[k], 3 * H, true);
      else b.param_grads(a, g_edge[k], 3 * H, true, true);
      launch(ctx, "gnn_add_rows", k_add_cols, ge, 256, 0, s, ctx->de, H, (const float*)ctx->bw_DX,
             3 * H, 0, 1, (int64_t)0, (const int32_t*)ctx->n_edges);
      if (N > 0)
        launch(ctx, "gnn_scatter_backward", k_scatter_bwd<H>, gs, 256, 0, s, (const float*)ctx->bw_DX,
               3 * H, H, 2 * H, (const int32_t*)ctx->out_off, (const int32_t*)ctx->in_off,
               (const int32_t*)ctx->perm_in, (const int32_t*)ctx->n_edges, (int)N, ctx->dh);
    }
    {  // h^{k+1} = h^k + f_node,k([h^k, m(e^k)])
      e = launch_messages(ctx, ek(k), ctx->m, N, s);
      if (e != cudaSuccess) return e;
      BwdArgs a = base;
      set_block(a, ctx->w.node[k], g_node[k]);
      a.hg = hk(k);
      a.m = ctx->m;
      a.gout = ctx->dh;
      a.K = 3 * H;
      if (tc) {
        if ((e = tc_block(BWD_NODE_UPD, a, imgs[1 + 2 * k], N, nullptr)) != cudaSuccess) return e;
      } else {
        b.template block_pass<B_NODE_UPD>(a, N);
      }
      if (tc) b.param_grads_tc(a, g_node[k], 3 * H, false);
      else b.param_grads(a, g_node[k], 3 * H, false, true);
      launch(ctx, "gnn_add_rows", k_add_cols, gn, 256, 0, s, ctx->dh, H, (const float*)ctx->bw_DX,
             3 * H, 0, 1, N, (const int32_t*)nullptr);
      launch(ctx, "gnn_gather_backward", k_gather_bwd<H>, gg, 256, 0, s, (const float*)ctx->bw_DX,
             3 * H, H, 2 * H, ctx->fwd_src, ctx->fwd_dst, (const int32_t*)ctx->n_edges, (int)N,
             ctx->de);
    }
  }
  // ---- encoders -------------------------------------------------------------------
  {
    BwdArgs a = base;
    set_block(a, ctx->w.edge_enc, g_edge_enc);
    a.hg = hk(0);
    a.gout = ctx->de;
    a.K = 2 * H;
    if (tc) {
      if ((e = tc_block(BWD_EDGE_ENC, a, imgs[0], 0, ctx->n_edges)) != cudaSuccess) return e;
    } else {
      b.template block_pass<B_EDGE_ENC>(a, Ecap);
    }
    if (tc) b.param_grads_tc(a, g_edge_enc, 2 * H, true);
    else b.param_grads(a, g_edge_enc, 2 * H, true, true);
    if (N > 0)
      launch(ctx, "gnn_scatter_backward", k_scatter_bwd<H>, gs, 256, 0, s, (const float*)ctx->bw_DX,
             2 * H, 0, H, (const int32_t*)ctx->out_off, (const int32_t*)ctx->in_off,
             (const int32_t*)ctx->perm_in, (const int32_t*)ctx->n_edges, (int)N, ctx->dh);
  }
  {
    BwdArgs a = base;
    set_block(a, ctx->w.node_enc, g_node_enc);
    a.gout = ctx->dh;
    a.K = 4;
    b.template block_pass<B_NODE_ENC>(a, N);
    b.param_grads(a, g_node_enc, 4, false, true);
  }
  return cudaGetLastError();
}

__global__ void k_copy_rows(float* __restrict__ dst, const float* __restrict__ src, int H,
                            int64_t R_host, const int32_t* __restrict__ R_dev) {
  const int64_t R = R_dev ? (int64_t)*R_dev : R_host;
  const int64_t n = R * H / 4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(src)[i];
}

}  // namespace

cudaError_t launch_checkpoint(etx_ctx* ctx, float* dst, const float* src, int64_t rows_host,
                              const int32_t* rows_dev, int64_t rows_cap, cudaStream_t s) {
  const int H = ctx->cfg.hidden;
  const int g = grid_for(ctx, (const void*)k_copy_rows, 256, 0, (rows_cap * H / 4 + 255) / 256);
  launch(ctx, "gnn_checkpoint", k_copy_rows, g, 256, 0, s, dst, src, H, rows_host, rows_dev);
  return cudaGetLastError();
}

cudaError_t launch_gnn_backward(etx_ctx* ctx, const float* dlogits, float* dparams, cudaStream_t s) {
  switch (ctx->cfg.hidden) {
    case 16: return backward<16>(ctx, dlogits, dparams, s);
    case 32: return backward<32>(ctx, dlogits, dparams, s);
    case 64: return backward<64>(ctx, dlogits, dparams, s);
    case 128: return backward<128>(ctx, dlogits, dparams, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// weighted BCE (the edge term of the training loss) and Adam
// ---------------------------------------------------------------------------
namespace {

// part[blockIdx.x] = the block's share of the loss sum (fixed order); the
// mean is formed by k_finish_sum.
__global__ void k_weighted_bce(const float* __restrict__ z, const float* __restrict__ y,
                               const int32_t* __restrict__ n_edges_dev, float pos_weight,
                               float* __restrict__ part, float* __restrict__ dz) {
  __shared__ float sh[32];
  const int64_t E = *n_edges_dev;
  const float inv = E > 0 ? 1.0f / (float)E : 0.f;
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float zi = z[i], yi = y[i];
    // softplus(t) = max(t, 0) + log1p(exp(-|t|)); sigmoid(t) = 1 / (1 + exp(-t))
    const float sp_pos = fmaxf(zi, 0.f) + log1pf(expf(-fabsf(zi)));   // softplus(z)
    const float sp_neg = sp_pos - zi;                                  // softplus(-z)
    const float sig = 1.0f / (1.0f + expf(-zi));
    acc += pos_weight * yi * sp_neg + (1.0f - yi) * sp_pos;
    dz[i] = inv * (-pos_weight * yi * (1.0f - sig) + (1.0f - yi) * sig);
  }
  const float t = block_sum_fixed(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// The sigmoid focal loss (Sec. 5.2, Eq. 5; the form of Lin et al. 2017): per
// block sums of the loss terms and dz = d loss / d z over E, written directly.
// p and 1 - p are formed separately (no cancellation), log p = -softplus(-z),
// log(1 - p) = -softplus(z).
__global__ void k_focal(const float* __restrict__ z, const float* __restrict__ y,
                        const int32_t* __restrict__ n_edges_dev, float alpha, float gamma,
                        float* __restrict__ part, float* __restrict__ dz) {
  __shared__ float sh[32];
  const int64_t E = *n_edges_dev;
  const float inv = E > 0 ? 1.0f / (float)E : 0.f;
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float zi = z[i], yi = y[i];
    const float sp_pos = fmaxf(zi, 0.f) + log1pf(expf(-fabsf(zi)));  // softplus(z)
    const float sp_neg = sp_pos - zi;                                 // softplus(-z)
    const float p = 1.0f / (1.0f + expf(-zi)), q = 1.0f / (1.0f + expf(zi));
    const float lp = -sp_neg, lq = -sp_pos;                           // log p, log(1 - p)
    const float qg = powf(q, gamma), pg = powf(p, gamma);
    acc += yi * (-alpha * qg * lp) + (1.0f - yi) * (-(1.0f - alpha) * pg * lq);
    const float d1 = alpha * qg * (gamma * p * lp - q);
    const float d0 = (1.0f - alpha) * pg * (p - gamma * q * lq);
    dz[i] = inv * (yi * d1 + (1.0f - yi) * d0);
  }
  const float t = block_sum_fixed(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_bce_mean(const float* __restrict__ part, int n, const int32_t* __restrict__ n_edges_dev,
                           float* __restrict__ loss) {
  __shared__ float sh[32];
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  const float t = block_sum_fixed(acc, sh);
  const int64_t E = *n_edges_dev;
  if (threadIdx.x == 0) *loss = E > 0 ? t * (1.0f / (float)E) : 0.f;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

cudaError_t launch_weighted_bce(etx_ctx* ctx, const float* logits, const float* targets,
                                const int32_t* n_edges_dev, float pos_weight, float* loss,
                                float* dlogits, cudaStream_t s) {
  int g = grid_for(ctx, (const void*)k_weighted_bce, 256, 0, (ctx->cfg.max_edges + 255) / 256);
  if (g > (int)ctx->red_part_n) g = (int)ctx->red_part_n;
  launch(ctx, "loss_weighted_bce", k_weighted_bce, g, 256, 0, s, logits, targets, n_edges_dev,
         pos_weight, ctx->red_part, dlogits);
  launch(ctx, "loss_mean", k_bce_mean, 1, 256, 0, s, (const float*)ctx->red_part, g, n_edges_dev, loss);
  return cudaGetLastError();
}

cudaError_t launch_focal_loss(etx_ctx* ctx, const float* logits, const float* targets,
                              const int32_t* n_edges_dev, float alpha, float gamma, float* loss,
                              float* dlogits, cudaStream_t s) {
  int g = grid_for(ctx, (const void*)k_focal, 256, 0, (ctx->cfg.max_edges + 255) / 256);
  if (g > (int)ctx->red_part_n) g = (int)ctx->red_part_n;
  launch(ctx, "loss_focal", k_focal, g, 256, 0, s, logits, targets, n_edges_dev, alpha, gamma,
         ctx->red_part, dlogits);
  launch(ctx, "loss_mean", k_bce_mean, 1, 256, 0, s, (const float*)ctx->red_part, g, n_edges_dev, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(etx_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n,
                        float lr, float b1, float b2, float eps, int64_t step, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  const int grid = grid_for(ctx, (const void*)k_adam, 256, 0, (n + 255) / 256);
  launch(ctx, "adam_step", k_adam, grid, 256, 0, s, p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

// ---- embedding MLP reverse pass (training of Sec. 5.1) -----------------------

namespace {

// Y[r][:] = (X[r][:K] . W[K][NT]) * (mask[r][:] > 0): the gradient through one
// Linear layer (W in its original [out][in] layout, K = out) and the ReLU of
// the layer below (mask = its saved activations).
template <int NT>
__global__ void __launch_bounds__(kTileThreads)
k_back_rows(const float* __restrict__ X, int K, const float* __restrict__ W,
            const float* __restrict__ mask, float* __restrict__ Y, int64_t n) {
  __shared__ __align__(16) float As[kTileM * kLdaChunk];
  __shared__ __align__(16) float Ws[kKC * NT];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t tiles = (n + kTileM - 1) / kTileM;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTileM;
    TileAcc<NT> acc;
    acc.zero();
    for (int k0 = 0; k0 < K; k0 += kKC) {
      __syncthreads();
      for (int i = tid; i < kTileM * kKC; i += kTileThreads) {
        const int mm = i / kKC, kk = i - mm * kKC;
        const int64_t r = row0 + mm;
        const int k = k0 + kk;
        As[mm * kLdaChunk + kk] = (r < n && k < K) ? X[r * K + k] : 0.f;
      }
      for (int i = tid; i < kKC * NT; i += kTileThreads) {
        const int kk = i / NT, c = i - kk * NT;
        const int k = k0 + kk;
        Ws[i] = k < K ? W[(int64_t)k * NT + c] : 0.f;
      }
      __syncthreads();
      acc.template mma<kKC>(As, kLdaChunk, 0, Ws, ty, tx);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t row = row0 + ty * 4 + r;
      if (row >= n) continue;
#pragma unroll
      for (int j = 0; j < NT / 16; ++j) {
        const int64_t o = row * NT + ColMap<NT>::col(tx, j);
        Y[o] = mask[o] > 0.f ? acc.v[r][j] : 0.f;
      }
    }
  }
}

template <int NT>
void back_rows(etx_ctx* ctx, const float* X, int K, const float* W, const float* mask, float* Y,
               int64_t n, cudaStream_t s) {
  const int64_t tiles = (n + kTileM - 1) / kTileM;
  const int grid = grid_for(ctx, (const void*)k_back_rows<NT>, kTileThreads, 0, tiles);
  launch(ctx, "embtrain_back_rows", k_back_rows<NT>, grid, kTileThreads, 0, s, X, K, W, mask, Y, n);
}

}  // namespace

int64_t embed_param_count(const etx_config& c) {
  int64_t p = 0;
  for (int l = 0; l < c.emb_depth; ++l)
    p += (int64_t)c.emb_widths[l + 1] * c.emb_widths[l] + c.emb_widths[l + 1];
  return p;
}

// Row splits of the embedding's weight gradients and blocks of its column sums
// (upper bounds: the partials live in the caller's workspace).
constexpr int kEmbMaxSplits = 256, kEmbMaxColBlocks = 1024;

// Largest weight-matrix and output widths of the embedding layers.
static void embed_part_sizes(const etx_config& c, int64_t& max_mn, int64_t& max_m) {
  max_mn = 0;
  max_m = 0;
  for (int l = 0; l < c.emb_depth; ++l) {
    max_mn = std::max<int64_t>(max_mn, (int64_t)c.emb_widths[l + 1] * c.emb_widths[l]);
    max_m = std::max<int64_t>(max_m, c.emb_widths[l + 1]);
  }
}

size_t embed_backward_workspace(const etx_config& c, int64_t n) {
  const int64_t EW = c.emb_widths[1];
  int64_t max_mn, max_m;
  embed_part_sizes(c, max_mn, max_m);
  // saved inputs [n][4] and hidden activations [depth-1][n][EW], two gradient buffers [n][EW],
  // and the partial sums of the weight gradients and column sums (added in a fixed order)
  const int64_t part = std::max<int64_t>(kEmbMaxSplits * max_mn, kEmbMaxColBlocks * max_m);
  return (size_t)(n * 4 + (int64_t)(c.emb_depth - 1) * n * EW + 2 * n * EW + part) * sizeof(float);
}

cudaError_t launch_embed_backward(etx_ctx* ctx, int64_t n, const float* saved, const float* d_emb,
                                  float* dz_a, float* dz_b, float* d_params, cudaStream_t s) {
  const etx_config& c = ctx->cfg;
  const int depth = c.emb_depth, EW = c.emb_widths[1];
  int64_t woff[ETX_MAX_EMB_LAYERS], boff[ETX_MAX_EMB_LAYERS], off = 0;
  for (int l = 0; l < depth; ++l) {
    woff[l] = off;
    off += (int64_t)c.emb_widths[l + 1] * c.emb_widths[l];
    boff[l] = off;
    off += c.emb_widths[l + 1];
  }
  cudaError_t e = cudaMemsetAsync(d_params, 0, (size_t)off * sizeof(float), s);
  if (e != cudaSuccess || n == 0) return e;
  const float* Wblob = ctx->blob_dev + 12;  // embedding parameters follow the 12 normalisation values
  auto act = [&](int l) { return saved + n * 4 + (int64_t)l * n * EW; };
  const int splits = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)ctx->n_sms, (n + 1023) / 1024, (int64_t)kEmbMaxSplits}));
  const int cb = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)ctx->n_sms * 4, n, (int64_t)kEmbMaxColBlocks}));
  float* part = dz_b + n * EW;  // partial sums (workspace tail), added in a fixed order
  auto reduce = [&](int parts, int64_t m, float* out) {
    if (m <= 4096 && parts >= 64)
      launch(ctx, "embtrain_grad_reduce", k_reduce_parts_narrow, (int)((m + 31) / 32), 256, 0, s,
             (const float*)part, parts, m, out);
    else
      launch(ctx, "embtrain_grad_reduce", k_reduce_parts,
             (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, ctx->n_sms * 4)), 256, 0, s,
             (const float*)part, parts, m, out);
  };
  const float* dz = d_emb;  // gradient at the output of layer l (before its ReLU, if any)
  for (int l = depth - 1; l >= 0; --l) {
    const int M = c.emb_widths[l + 1], n_in = c.emb_widths[l];
    const float* in = l > 0 ? act(l - 1) : saved;
    const int ld_in = l > 0 ? EW : 4;
    launch(ctx, "embtrain_weight_grad", k_gemm_tn,
           dim3((M + kTileM - 1) / kTileM, (n_in + 127) / 128, splits), kTileThreads, 0, s, dz, M,
           in, ld_in, M, n_in, n, (const int32_t*)nullptr, d_params + woff[l], part);
    reduce(splits, (int64_t)M * n_in, d_params + woff[l]);
    launch(ctx, "embtrain_colsum", k_colsum, cb, M, 0, s, dz, M, (const float*)nullptr, n,
           (const int32_t*)nullptr, d_params + boff[l], part);
    reduce(cb, M, d_params + boff[l]);
    if (l > 0) {
      float* out = dz == dz_a ? dz_b : dz_a;
      switch (EW) {
        case 16: back_rows<16>(ctx, dz, M, Wblob + woff[l], act(l - 1), out, n, s); break;
        case 32: back_rows<32>(ctx, dz, M, Wblob + woff[l], act(l - 1), out, n, s); break;
        case 64: back_rows<64>(ctx, dz, M, Wblob + woff[l], act(l - 1), out, n, s); break;
        case 128: back_rows<128>(ctx, dz, M, Wblob + woff[l], act(l - 1), out, n, s); break;
        default: return cudaErrorInvalidValue;
      }
      dz = out;
    }
  }
  return cudaGetLastError();
}

}  // namespace etx
