// Interaction-network MLP blocks on the 5th-generation tensor cores
// (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// One persistent CTA per SM (256 threads) walks 128-row tiles.  For a tile:
//   1. the block input rows ([h_i, h_j], [h, m_out, m_in], [e, h_i, h_j] or e)
//      are gathered from the FP32 streams, rounded to BF16 and written into
//      shared memory in the K-major 128-byte-swizzle layout, 64 columns at a
//      time through a two-slot ring; one thread issues the tcgen05.mma for a
//      chunk as soon as it lands while the CTA gathers the next one;
//   2. the 128 x 128 FP32 accumulator is read back from tensor memory
//      (tcgen05.ld; warp w owns TMEM lanes 32(w%4).. and half of the columns),
//      bias + LayerNorm + ReLU are applied in registers and the result is
//      written back to shared memory as the BF16 A operand of the second
//      Linear;
//   3. the second GEMM accumulates into another 128 TMEM columns, and its
//      epilogue applies bias + LayerNorm + ReLU, adds the FP32 residual and
//      stores FP32 rows.  The classifier instead ends in a dot product.
// The weights of the block stay resident in shared memory (pre-swizzled BF16
// images copied with one bulk async copy per 16 KB).  All waits are bounded.
#include <cuda_bf16.h>

#include "sm100.cuh"

namespace etx {
namespace {

using namespace sm100;

constexpr int H = 128;
constexpr int TM = 128;                    // rows per tile
constexpr int KCH = 64;                    // K columns per shared-memory chunk
constexpr int CHUNK = TM * KCH * 2;        // 16 KB per BF16 chunk (A or B)
constexpr int THREADS = 256;
constexpr uint32_t IDESC = idesc_bf16_f32<TM, H>();
constexpr uint32_t TMEM_COLS = 256;        // D1 at column 0, D2 at column 128

enum TcMode { TC_EDGE_ENC = 0, TC_NODE_UPD = 1, TC_EDGE_UPD = 2, TC_CLS = 3 };

template <int MODE>
struct Cfg {
  static constexpr int KC1 = MODE == TC_EDGE_ENC ? 4 : (MODE == TC_CLS ? 2 : 6);
  static constexpr bool G2 = MODE != TC_CLS;
  static constexpr int OFF_W1 = 0;
  static constexpr int OFF_W2 = OFF_W1 + KC1 * CHUNK;
  static constexpr int OFF_A = OFF_W2 + (G2 ? 2 * CHUNK : 0);
  static constexpr int OFF_A2 = OFF_A + 2 * CHUNK;
  static constexpr int OFF_BAR = OFF_A2 + (G2 ? 2 * CHUNK : 0);
  static constexpr int OFF_TMEM = OFF_BAR + 64;
  static constexpr int OFF_RED = OFF_TMEM + 16;
  static constexpr int OFF_IDX = OFF_RED + 4 * TM * 4;
  static constexpr int BYTES = OFF_IDX + 2 * TM * 4;
  static constexpr int SMEM = BYTES + 1024;  // slack for 1024-byte alignment
};

struct TcArgs {
  int64_t n_nodes;
  const int32_t* n_edges_dev;
  const int32_t *src, *dst;
  const float* h;
  const float* m;
  float* e;
  float* h_out;
  float* logits;
  const uint8_t* w1;  // BF16 swizzled image, KC1 chunks
  const uint8_t* w2;  // BF16 swizzled image, 2 chunks
  const float *b1, *g1, *be1, *b2, *g2, *be2;
  const float* wcls;  // classifier last Linear [H]
  const float* bcls;  // [1]
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&t);
}

// Byte offset of 16-byte unit u (0..7) of row r in a K-major SW128 chunk.
__device__ __forceinline__ uint32_t sw128(int r, int u) {
  return static_cast<uint32_t>(r * 128 + ((u ^ (r & 7)) << 4));
}

template <int MODE>
__device__ __forceinline__ const float* chunk_src(const TcArgs& a, int c, int64_t g, int s, int d) {
  if constexpr (MODE == TC_EDGE_ENC) {
    return c < 2 ? a.h + (int64_t)s * H + KCH * c : a.h + (int64_t)d * H + KCH * (c - 2);
  } else if constexpr (MODE == TC_NODE_UPD) {
    return c < 2 ? a.h + g * H + KCH * c : a.m + g * 2 * H + KCH * (c - 2);
  } else if constexpr (MODE == TC_EDGE_UPD) {
    return c < 2 ? a.e + g * H + KCH * c
                 : (c < 4 ? a.h + (int64_t)s * H + KCH * (c - 2) : a.h + (int64_t)d * H + KCH * (c - 4));
  } else {
    return a.e + g * H + KCH * c;
  }
}

// Read 64 FP32 accumulator columns [col, col+64) of this thread's TMEM lane.
__device__ __forceinline__ void tmem_row64(uint32_t taddr, float* v) {
  float t[32];
  tmem_ld32_wait(taddr, t);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = t[i];
  tmem_ld32_wait(taddr + 32, t);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[32 + i] = t[i];
}

// v <- ReLU(LN(v + b) * g + be) for a 128-wide row split over two threads
// (column halves hf = 0, 1), statistics exchanged through shared memory.
__device__ __forceinline__ void bias_ln_relu_split(float* v, const float* __restrict__ b,
                                                   const float* __restrict__ g,
                                                   const float* __restrict__ be, int hf, int r,
                                                   float* red) {
  const int c0 = hf * 64;
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    v[j] += __ldg(b + c0 + j);
    s += v[j];
  }
  red[hf * TM + r] = s;
  __syncthreads();
  const float mean = (red[r] + red[TM + r]) * (1.0f / H);
  float q = 0.f;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    const float d = v[j] - mean;
    q += d * d;
  }
  red[2 * TM + hf * TM + r] = q;
  __syncthreads();
  const float var = (red[2 * TM + r] + red[3 * TM + r]) * (1.0f / H);
  const float rstd = 1.0f / sqrtf(var + kLnEps);
#pragma unroll
  for (int j = 0; j < 64; ++j)
    v[j] = fmaxf((v[j] - mean) * rstd * __ldg(g + c0 + j) + __ldg(be + c0 + j), 0.f);
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) k_mlp_tc(TcArgs a) {
  using C = Cfg<MODE>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sW1 = smem + C::OFF_W1;
  uint8_t* sW2 = smem + C::OFF_W2;
  uint8_t* sA = smem + C::OFF_A;
  uint8_t* sA2 = smem + C::OFF_A2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);  // 0 weights, 1-2 ring, 3 gemm2
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_TMEM);
  float* red = reinterpret_cast<float*>(smem + C::OFF_RED);
  int* s_src = reinterpret_cast<int*>(smem + C::OFF_IDX);
  int* s_dst = s_src + TM;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, hf = warp >> 2, r = 32 * q + lane;  // epilogue row / column half

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tD1 = tmem, tD2 = tmem + 128;
  const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;

  if (tid == 0) {
    const uint32_t bytes = (C::KC1 + (C::G2 ? 2 : 0)) * CHUNK;
    mbar_arrive_expect_tx(&bars[0], bytes);
    for (int c = 0; c < C::KC1; ++c) bulk_g2s(sW1 + c * CHUNK, a.w1 + (size_t)c * CHUNK, CHUNK, &bars[0]);
    if (C::G2)
      for (int c = 0; c < 2; ++c) bulk_g2s(sW2 + c * CHUNK, a.w2 + (size_t)c * CHUNK, CHUNK, &bars[0]);
  }
  bool ok = mbar_wait(&bars[0], 0, a.err);
  const bool aborted0 = __syncthreads_or(!ok);

  const int64_t n_rows = MODE == TC_NODE_UPD ? a.n_nodes : (int64_t)*a.n_edges_dev;
  const int64_t n_tiles = (n_rows + TM - 1) / TM;
  const int nn = (int)a.n_nodes;
  uint32_t ring_uses[2] = {0u, 0u};
  uint32_t g2_uses = 0;
  const int grow = tid >> 1, gpart = tid & 1;  // gather: row, which 32-column half of the chunk

  for (int64_t tile = blockIdx.x; !aborted0 && tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * TM;
    if constexpr (MODE == TC_EDGE_ENC || MODE == TC_EDGE_UPD) {
      if (tid < TM) {
        const int64_t gr = row0 + tid;
        s_src[tid] = gr < n_rows ? min(max(a.src[gr], 0), nn - 1) : 0;
        s_dst[tid] = gr < n_rows ? min(max(a.dst[gr], 0), nn - 1) : 0;
      }
      __syncthreads();
    }
    const int64_t g = row0 + grow;
    const bool valid = g < n_rows;
    // ---- GEMM 1: stream the gathered input through the two-slot ring --------
    bool abort = false;
    for (int c = 0; c < C::KC1; ++c) {
      const int slot = c & 1;
      if (ring_uses[slot] > 0) ok = mbar_wait(&bars[1 + slot], (ring_uses[slot] - 1) & 1, a.err);
      float4 f[8];
      if (valid) {
        const float* p = chunk_src<MODE>(a, c, g, s_src[grow], s_dst[grow]) + 32 * gpart;
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = *reinterpret_cast<const float4*>(p + 4 * i);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      uint8_t* dstc = sA + slot * CHUNK;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint4 u;
        u.x = pack_bf16(f[2 * i].x, f[2 * i].y);
        u.y = pack_bf16(f[2 * i].z, f[2 * i].w);
        u.z = pack_bf16(f[2 * i + 1].x, f[2 * i + 1].y);
        u.w = pack_bf16(f[2 * i + 1].z, f[2 * i + 1].w);
        *reinterpret_cast<uint4*>(dstc + sw128(grow, 4 * gpart + i)) = u;
      }
      fence_proxy_async();
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(dstc), b0 = smem_u32(sW1 + c * CHUNK);
#pragma unroll
        for (int k = 0; k < KCH / 16; ++k)
          mma_f16(tD1, sdesc_k_sw128(a0 + 32 * k), sdesc_k_sw128(b0 + 32 * k), IDESC,
                  (c > 0 || k > 0) ? 1u : 0u);
        mma_commit(&bars[1 + slot]);
      }
      ++ring_uses[slot];
    }
    if (abort) break;
    const int last = (C::KC1 - 1) & 1;
    ok = mbar_wait(&bars[1 + last], (ring_uses[last] - 1) & 1, a.err);
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();

    // ---- epilogue 1 ---------------------------------------------------------
    float v[64];
    tmem_row64(tD1 + lane_off + 64 * hf, v);
    const int64_t grr = row0 + r;
    if constexpr (MODE == TC_CLS) {
      bias_ln_relu_split(v, a.b1, a.g1, a.be1, hf, r, red);
      float p = 0.f;
#pragma unroll
      for (int j = 0; j < 64; ++j) p = fmaf(v[j], __ldg(a.wcls + 64 * hf + j), p);
      red[hf * TM + r] = p;
      __syncthreads();
      if (hf == 0 && grr < n_rows) a.logits[grr] = red[r] + red[TM + r] + __ldg(a.bcls);
      tc_fence_before();
      __syncthreads();
      continue;
    } else {
      bias_ln_relu_split(v, a.b1, a.g1, a.be1, hf, r, red);
      uint8_t* dst2 = sA2 + hf * CHUNK;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        uint4 w;
        w.x = pack_bf16(v[8 * u + 0], v[8 * u + 1]);
        w.y = pack_bf16(v[8 * u + 2], v[8 * u + 3]);
        w.z = pack_bf16(v[8 * u + 4], v[8 * u + 5]);
        w.w = pack_bf16(v[8 * u + 6], v[8 * u + 7]);
        *reinterpret_cast<uint4*>(dst2 + sw128(r, u)) = w;
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      // ---- GEMM 2 -----------------------------------------------------------
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint32_t a0 = smem_u32(sA2 + c * CHUNK), b0 = smem_u32(sW2 + c * CHUNK);
#pragma unroll
          for (int k = 0; k < KCH / 16; ++k)
            mma_f16(tD2, sdesc_k_sw128(a0 + 32 * k), sdesc_k_sw128(b0 + 32 * k), IDESC,
                    (c > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&bars[3]);
      }
      ok = mbar_wait(&bars[3], g2_uses & 1, a.err);
      ++g2_uses;
      if (__syncthreads_or(!ok)) break;
      tc_fence_after();
      // ---- epilogue 2 ---------------------------------------------------------
      tmem_row64(tD2 + lane_off + 64 * hf, v);
      bias_ln_relu_split(v, a.b2, a.g2, a.be2, hf, r, red);
      if (grr < n_rows) {
        float* out;
        const float* res = nullptr;
        if constexpr (MODE == TC_NODE_UPD) {
          out = a.h_out + grr * H + 64 * hf;
          res = a.h + grr * H + 64 * hf;
        } else if constexpr (MODE == TC_EDGE_UPD) {
          out = a.e + grr * H + 64 * hf;
          res = out;
        } else {
          out = a.e + grr * H + 64 * hf;
        }
#pragma unroll
        for (int j = 0; j < 64; j += 4) {
          float4 o = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          if (res) {
            const float4 t = *reinterpret_cast<const float4*>(res + j);
            o.x += t.x; o.y += t.y; o.z += t.z; o.w += t.w;
          }
          *reinterpret_cast<float4*>(out + j) = o;
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <int MODE>
cudaError_t launch_tc(etx_ctx* ctx, const char* name, const TcArgs& a, int64_t max_rows,
                      cudaStream_t s) {
  using C = Cfg<MODE>;
  static bool attr_set[8] = {false};
  if (!attr_set[ctx->device & 7]) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[ctx->device & 7] = true;
  }
  const int64_t tiles = (max_rows + TM - 1) / TM;
  if (tiles == 0) return cudaSuccess;
  const int grid = (int)(tiles < ctx->n_sms ? tiles : ctx->n_sms);
  launch(ctx, name, k_mlp_tc<MODE>, grid, THREADS, C::SMEM, s, a);
  return cudaGetLastError();
}

TcArgs base_args(etx_ctx* ctx, int64_t N, const int32_t* src, const int32_t* dst,
                 const int32_t* n_edges_dev, float* logits) {
  TcArgs a{};
  a.n_nodes = N;
  a.n_edges_dev = n_edges_dev;
  a.src = src;
  a.dst = dst;
  a.h = ctx->h;
  a.m = ctx->m;
  a.e = ctx->e;
  a.h_out = ctx->h;
  a.logits = logits;
  a.err = ctx->d_err;
  return a;
}

void set_block(TcArgs& a, const BlockF32& f, const BlockTC& t) {
  a.w1 = t.w1;
  a.w2 = t.w2;
  a.b1 = f.l1.b;
  a.g1 = f.g1;
  a.be1 = f.be1;
  a.b2 = f.l2.b;
  a.g2 = f.g2;
  a.be2 = f.be2;
}

}  // namespace

cudaError_t launch_edge_encoder_tc(etx_ctx* ctx, int64_t N, const int32_t* src, const int32_t* dst,
                                   const int32_t* n_edges_dev, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, src, dst, n_edges_dev, nullptr);
  set_block(a, ctx->w.edge_enc, ctx->w.edge_enc_tc);
  return launch_tc<TC_EDGE_ENC>(ctx, "gnn_edge_encoder_bf16", a, ctx->cfg.max_edges, s);
}

cudaError_t launch_node_update_tc(etx_ctx* ctx, int k, int64_t N, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, nullptr, nullptr, nullptr, nullptr);
  set_block(a, ctx->w.node[k], ctx->w.node_tc[k]);
  return launch_tc<TC_NODE_UPD>(ctx, "gnn_node_update_bf16", a, N, s);
}

cudaError_t launch_edge_update_tc(etx_ctx* ctx, int k, int64_t N, const int32_t* src,
                                  const int32_t* dst, const int32_t* n_edges_dev, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, src, dst, n_edges_dev, nullptr);
  set_block(a, ctx->w.edge[k], ctx->w.edge_tc[k]);
  return launch_tc<TC_EDGE_UPD>(ctx, "gnn_edge_update_bf16", a, ctx->cfg.max_edges, s);
}

cudaError_t launch_classifier_tc(etx_ctx* ctx, int64_t N, const int32_t* n_edges_dev, float* logits,
                                 cudaStream_t s) {
  TcArgs a = base_args(ctx, N, nullptr, nullptr, n_edges_dev, logits);
  a.w1 = ctx->w.cls_tc.w1;
  a.b1 = ctx->w.cls.l1.b;
  a.g1 = ctx->w.cls.g1;
  a.be1 = ctx->w.cls.be1;
  a.wcls = ctx->w.cls.w2;
  a.bcls = ctx->w.cls.b2;
  return launch_tc<TC_CLS>(ctx, "gnn_classifier_bf16", a, ctx->cfg.max_edges, s);
}

}  // namespace etx
