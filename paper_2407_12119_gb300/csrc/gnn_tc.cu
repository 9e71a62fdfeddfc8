// Interaction-network MLP blocks on the 5th-generation tensor cores
// (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// Persistent kernel, one CTA per SM, 416 threads in three roles that run
// concurrently over the CTA's 128-row tiles:
//   warps 4-11 producers: gather the block's input rows ([h_i, h_j],
//              [h, m_out, m_in], [e, h_i, h_j] or e) from the FP32 streams,
//              round them to BF16 and write them, 64 columns at a time, into a
//              3-slot ring in the K-major 128-byte-swizzle layout; coalesced
//              (8 threads per 256-byte row segment) and two chunks prefetched
//              in registers;
//   warp 12    MMA issuer (one thread): tcgen05.mma of each ring slot into the
//              tile's first accumulator (two TMEM buffers, so the next tile's
//              first GEMM runs while the epilogue reads this one), then the
//              second GEMM of the previous tile from the epilogue's BF16
//              activations;
//   warps 0-3  epilogue, one row per thread (TMEM lane = row): bias +
//              LayerNorm + ReLU of the first GEMM into the BF16 operand of the
//              second, then bias + LayerNorm + ReLU + FP32 residual and the
//              row store (or the classifier's dot product).
// Stages hand over through mbarriers (transaction-counted bulk copies for
// the resident BF16 weights, tcgen05.commit for MMA completion, thread
// arrivals otherwise).  Every wait is bounded; a timeout records
// ETX_ERR_TIMEOUT, raises a shared abort flag and every role stops.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "sm100.cuh"

namespace etx {
namespace {

using namespace sm100;

constexpr int H = 128;
constexpr int TM = 128;                  // rows per tile
constexpr int CHUNK = TM * 128;          // 16 KB operand chunk: 128 rows x 128 bytes
constexpr int SUB = 64;                  // K columns a producer fetches per step (256 B FP32)
constexpr int KSTEPS = 4;                // MMAs per chunk (32 bytes of K each)
constexpr int NSTAGE = 3;                // A-operand ring slots
constexpr int EPI_WARPS = 4, PROD_WARPS = 8;
constexpr int MMA_WARP = EPI_WARPS + PROD_WARPS;
constexpr int THREADS = 32 * (MMA_WARP + 1);  // 416
constexpr int PROD_THREADS = 32 * PROD_WARPS;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;      // D1 buffers at columns 0 and 128, D2 at 256

enum TcMode { TC_EDGE_ENC = 0, TC_NODE_UPD = 1, TC_EDGE_UPD = 2, TC_CLS = 3 };

// barrier indices
enum { B_W = 0, B_FULL = 1, B_EMPTY = B_FULL + NSTAGE, B_D1FULL = B_EMPTY + NSTAGE,
       B_D1EMPTY = B_D1FULL + 2, B_A2FULL = B_D1EMPTY + 2, B_D2FULL = B_A2FULL + 1,
       N_BARS = B_D2FULL + 1 };

// Operand type: BF16 (2 bytes, 64 K columns per 128-byte row) or FP8 e4m3
// (1 byte, 128 K columns per row).
template <bool F8>
struct Elt {
  static constexpr int KCH = F8 ? 128 : 64;   // K columns per chunk
  static constexpr int SUBS = KCH / SUB;       // producer steps per chunk
  static constexpr uint32_t IDESC = F8 ? idesc_e4m3_f32<TM, H>() : idesc_bf16_f32<TM, H>();
};

template <int MODE, bool F8>
struct Cfg {
  static constexpr int KIN = MODE == TC_EDGE_ENC ? 2 * H : (MODE == TC_CLS ? H : 3 * H);
  static constexpr int KC1 = KIN / Elt<F8>::KCH;     // chunks of the first GEMM
  static constexpr int KS = KIN / SUB;               // producer steps per tile
  static constexpr int C2 = H / Elt<F8>::KCH;        // chunks of the second GEMM
  static constexpr bool G2 = MODE != TC_CLS;
  static constexpr int OFF_W1 = 0;
  static constexpr int OFF_W2 = OFF_W1 + KC1 * CHUNK;
  static constexpr int OFF_A = OFF_W2 + (G2 ? C2 * CHUNK : 0);
  static constexpr int OFF_A2 = OFF_A + NSTAGE * CHUNK;
  // A2 holds the second GEMM's operand, then stages 128 x 64 FP32 outputs (32 KB)
  static constexpr int OFF_PAR = OFF_A2 + (G2 ? 2 * CHUNK : 0);     // 7 x 128 floats
  static constexpr int OFF_BAR = OFF_PAR + 7 * H * 4;
  static constexpr int OFF_MISC = OFF_BAR + 8 * N_BARS;              // tmem addr, abort flag
  static constexpr int BYTES = OFF_MISC + 16;
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
  const uint8_t* w1;  // swizzled operand image of W1 (KC1 chunks)
  const uint8_t* w2;  // swizzled operand image of W2 (C2 chunks)
  float ws1, ws2;     // per-tensor weight scales (1 for BF16)
  const float *b1, *g1, *be1, *b2, *g2, *be2;
  const float* wcls;  // classifier last Linear [H]
  const float* bcls;  // [1]
  int* err;
};

// Four values to e4m3 (saturating), first value in the lowest byte.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&t);
}

// Byte offset of 16-byte unit u (0..7) of row r in a K-major SW128 chunk.
__device__ __forceinline__ uint32_t sw128(int r, int u) {
  return static_cast<uint32_t>(r * 128 + ((u ^ (r & 7)) << 4));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up when another role raised the abort flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, int* err,
                                              volatile int* abort) {
  for (uint32_t i = 0; i < kWaitCap; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  set_err(err, DERR_TIMEOUT);
  *abort = 1;
  return false;
}

// Source of columns [col0, col0 + 64) of block-input row g.
template <int MODE>
__device__ __forceinline__ const float* chunk_src(const TcArgs& a, int col0, int64_t g, int s, int d) {
  if constexpr (MODE == TC_EDGE_ENC) {
    return col0 < H ? a.h + (int64_t)s * H + col0 : a.h + (int64_t)d * H + (col0 - H);
  } else if constexpr (MODE == TC_NODE_UPD) {
    return col0 < H ? a.h + g * H + col0 : a.m + g * 2 * H + (col0 - H);
  } else if constexpr (MODE == TC_EDGE_UPD) {
    return col0 < H ? a.e + g * H + col0
                    : (col0 < 2 * H ? a.h + (int64_t)s * H + (col0 - H)
                                    : a.h + (int64_t)d * H + (col0 - 2 * H));
  } else {
    return a.e + g * H + col0;
  }
}

// Row statistics of x_j = sc * acc_j + b_j over the 128 accumulator columns
// of this thread's TMEM lane (shifted sums: shift = first value).
__device__ __forceinline__ void row_stats(uint32_t taddr, const float* __restrict__ b, float sc,
                                          float& mean, float& rstd) {
  float v[32];
  float shift = 0.f;
  float s4[4] = {0.f, 0.f, 0.f, 0.f}, q4[4] = {0.f, 0.f, 0.f, 0.f};  // independent chains
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    tmem_ld32_wait(taddr + 32 * cc, v);
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      const float4 bb = *reinterpret_cast<const float4*>(b + 32 * cc + j);
      const float x0 = fmaf(v[j], sc, bb.x), x1 = fmaf(v[j + 1], sc, bb.y),
                  x2 = fmaf(v[j + 2], sc, bb.z), x3 = fmaf(v[j + 3], sc, bb.w);
      if (cc == 0 && j == 0) shift = x0;
      const float d0 = x0 - shift, d1 = x1 - shift, d2 = x2 - shift, d3 = x3 - shift;
      s4[0] += d0; s4[1] += d1; s4[2] += d2; s4[3] += d3;
      q4[0] = fmaf(d0, d0, q4[0]); q4[1] = fmaf(d1, d1, q4[1]);
      q4[2] = fmaf(d2, d2, q4[2]); q4[3] = fmaf(d3, d3, q4[3]);
    }
  }
  const float s = (s4[0] + s4[1]) + (s4[2] + s4[3]), ss = (q4[0] + q4[1]) + (q4[2] + q4[3]);
  const float ms = s * (1.0f / H);
  mean = shift + ms;
  const float var = fmaxf(ss * (1.0f / H) - ms * ms, 0.f);
  rstd = 1.0f / sqrtf(var + kLnEps);
}

// 32 normalised, ReLU'd values of columns [32 cc, 32 cc + 32).
__device__ __forceinline__ void row_norm32(uint32_t taddr, int cc, const float* __restrict__ b,
                                           const float* __restrict__ g, const float* __restrict__ be,
                                           float sc, float mean, float rstd, float (&y)[32]) {
  tmem_ld32_wait(taddr + 32 * cc, y);
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 bb = *reinterpret_cast<const float4*>(b + 32 * cc + j);
    const float4 gg = *reinterpret_cast<const float4*>(g + 32 * cc + j);
    const float4 ee = *reinterpret_cast<const float4*>(be + 32 * cc + j);
    y[j] = fmaxf((fmaf(y[j], sc, bb.x) - mean) * rstd * gg.x + ee.x, 0.f);
    y[j + 1] = fmaxf((fmaf(y[j + 1], sc, bb.y) - mean) * rstd * gg.y + ee.y, 0.f);
    y[j + 2] = fmaxf((fmaf(y[j + 2], sc, bb.z) - mean) * rstd * gg.z + ee.z, 0.f);
    y[j + 3] = fmaxf((fmaf(y[j + 3], sc, bb.w) - mean) * rstd * gg.w + ee.w, 0.f);
  }
}

template <int MODE, bool F8>
__global__ void __launch_bounds__(THREADS, 1) k_mlp_tc(TcArgs a) {
  using C = Cfg<MODE, F8>;
  using EL = Elt<F8>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sW1 = smem + C::OFF_W1;
  uint8_t* sW2 = smem + C::OFF_W2;
  uint8_t* sA = smem + C::OFF_A;
  uint8_t* sA2 = smem + C::OFF_A2;
  float* par = reinterpret_cast<float*>(smem + C::OFF_PAR);  // b1 g1 be1 b2 g2 be2 wcls
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + C::OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- set-up -------------------------------------------------------------
  if (tid == 0) {
    mbar_init(&bars[B_W], 1);
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&bars[B_FULL + s], PROD_WARPS);  // one arrival per producer warp
      mbar_init(&bars[B_EMPTY + s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars[B_D1FULL + b], 1);
      mbar_init(&bars[B_D1EMPTY + b], EPI_WARPS);
    }
    mbar_init(&bars[B_A2FULL], EPI_WARPS);
    mbar_init(&bars[B_D2FULL], 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (tid < H) {
    par[tid] = __ldg(a.b1 + tid);
    par[H + tid] = __ldg(a.g1 + tid);
    par[2 * H + tid] = __ldg(a.be1 + tid);
    if (C::G2) {
      par[3 * H + tid] = __ldg(a.b2 + tid);
      par[4 * H + tid] = __ldg(a.g2 + tid);
      par[5 * H + tid] = __ldg(a.be2 + tid);
    } else {
      par[6 * H + tid] = __ldg(a.wcls + tid);
    }
  }
  if (warp == MMA_WARP) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n_rows = MODE == TC_NODE_UPD ? a.n_nodes : (int64_t)*a.n_edges_dev;
  const int64_t n_tiles = (n_rows + TM - 1) / TM;
  const int nn = (int)a.n_nodes;

  if (warp >= EPI_WARPS && warp < MMA_WARP) {
    // =========================== producers =================================
    // Flattened stream of this CTA's (tile, chunk) pairs, prefetched two chunks
    // ahead in a three-deep register ring so that loads of the next chunks
    // (also across tile boundaries) are in flight while one chunk is stored.
    // Thread t8 = pt % 8 of a row group reads bytes [16 t8, 16 t8 + 16) of each
    // 128-byte line of a 256-byte FP32 row segment (two fully coalesced loads)
    // and writes the two resulting 8-byte BF16 halves.  Row groups sharing a
    // half-warp own rows 4 apart, so those 8-byte shared stores never collide.
    const int pt = tid - EPI_THREADS;
    const int t8 = pt & 7, rg = pt >> 3, wg = rg & 3, wi = rg >> 2;
    const int rbase = 8 * (wi >> 1) + 4 * (wg & 1) + 2 * (wi & 1) + (wg >> 1);  // 0..31
    constexpr int RPT = TM / (PROD_THREADS / 8);  // rows per producer thread
    const int64_t my_tiles =
        n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_tiles * C::KS;  // 64-column steps
    // gather indices of the tile being fetched, read when its first chunk is
    // fetched (chunks reach the same tile in order, two ahead of the stores)
    int sidx[RPT], didx[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) sidx[i] = didx[i] = 0;
    auto fetch = [&](int64_t q, float4 (&f)[2 * RPT]) {
      if (q >= total) return;
      const int64_t row0 = (blockIdx.x + (q / C::KS) * gridDim.x) * TM;
      const int c = (int)(q % C::KS);
      if constexpr (MODE == TC_EDGE_ENC || MODE == TC_EDGE_UPD) {
        if (c == 0) {
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const int64_t gr = row0 + rbase + 32 * i;
            sidx[i] = gr < n_rows ? min(max(a.src[gr], 0), nn - 1) : 0;
            didx[i] = gr < n_rows ? min(max(a.dst[gr], 0), nn - 1) : 0;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int64_t gr = row0 + rbase + 32 * i;
        if (gr < n_rows) {
          const float* p = chunk_src<MODE>(a, SUB * c, gr, sidx[i], didx[i]) + 4 * t8;
          f[2 * i] = *reinterpret_cast<const float4*>(p);
          f[2 * i + 1] = *reinterpret_cast<const float4*>(p + 32);
        } else {
          f[2 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
          f[2 * i + 1] = f[2 * i];
        }
      }
    };
    auto store = [&](int64_t q, const float4 (&f)[2 * RPT]) {
      const int64_t j = q / EL::SUBS;            // ring chunk
      const int hpart = (int)(q % EL::SUBS);     // which 64 columns of it
      const int slot = (int)(j % NSTAGE);
      const uint32_t round = (uint32_t)(j / NSTAGE);
      if (hpart == 0 && round > 0 &&
          !wait_or_abort(&bars[B_EMPTY + slot], (round - 1) & 1, a.err, abort))
        return false;
      const uint32_t dstc = smem_u32(sA + slot * CHUNK);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = rbase + 32 * i;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const float4 v = f[2 * i + hh];
          if constexpr (F8) {
            // columns 64 hpart + 32 hh + 4 t8 .. +3: 16 values per 16-byte unit
            const uint32_t addr = dstc + sw128(r, 4 * hpart + 2 * hh + (t8 >> 2)) + 4 * (t8 & 3);
            asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(pack_e4m3x4(v.x, v.y, v.z, v.w))
                         : "memory");
          } else {
            const uint32_t addr = dstc + sw128(r, 4 * hh + (t8 >> 1)) + 8 * (t8 & 1);
            asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(pack_bf16(v.x, v.y)),
                         "r"(pack_bf16(v.z, v.w))
                         : "memory");
          }
        }
      }
      if (hpart == EL::SUBS - 1) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[B_FULL + slot]);
      }
      return true;
    };
    float4 b0[2 * RPT], b1[2 * RPT], b2[2 * RPT];
    fetch(0, b0);
    fetch(1, b1);
    for (int64_t q = 0; q < total; q += 3) {
      fetch(q + 2, b2);
      if (!store(q, b0)) break;
      if (q + 1 >= total) break;
      fetch(q + 3, b0);
      if (!store(q + 1, b1)) break;
      if (q + 2 >= total) break;
      fetch(q + 4, b1);
      if (!store(q + 2, b2)) break;
    }
  } else if (warp == MMA_WARP) {
    // =========================== MMA issuer ================================
    if (lane == 0) {
      const uint32_t wbytes = (C::KC1 + (C::G2 ? C::C2 : 0)) * CHUNK;
      mbar_arrive_expect_tx(&bars[B_W], wbytes);
      for (int c = 0; c < C::KC1; ++c)
        bulk_g2s(sW1 + c * CHUNK, a.w1 + (size_t)c * CHUNK, CHUNK, &bars[B_W]);
      if (C::G2)
        for (int c = 0; c < C::C2; ++c)
          bulk_g2s(sW2 + c * CHUNK, a.w2 + (size_t)c * CHUNK, CHUNK, &bars[B_W]);
      bool live = wait_or_abort(&bars[B_W], 0, a.err, abort);
      uint32_t gchunk = 0;
      int i = 0;
      int pending = -1;  // local tile whose second GEMM waits for the epilogue's A2
      auto issue_gemm2 = [&]() {
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < C::C2; ++c) {
          const uint32_t a0 = smem_u32(sA2 + c * CHUNK), b0 = smem_u32(sW2 + c * CHUNK);
#pragma unroll
          for (int k = 0; k < KSTEPS; ++k)
            mma_tc<F8>(tmem + 256, sdesc_k_sw128(a0 + 32 * k), sdesc_k_sw128(b0 + 32 * k),
                       EL::IDESC, (c > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&bars[B_D2FULL]);
        pending = -1;
      };
      // Wait for `bar`; meanwhile issue the pending second GEMM as soon as its
      // operand is ready, so it never queues behind the next tile's gather.
      auto wait_poll = [&](uint64_t* bar, uint32_t parity) {
        for (uint32_t it = 0; it < kWaitCap; ++it) {
          if (mbar_try_wait(bar, parity)) return true;
          if (C::G2 && pending >= 0 && mbar_try_wait(&bars[B_A2FULL], pending & 1)) issue_gemm2();
          if ((it & 255) == 255 && *abort) return false;
        }
        set_err(a.err, DERR_TIMEOUT);
        *abort = 1;
        return false;
      };
      for (int64_t tile = blockIdx.x; live && tile < n_tiles; tile += gridDim.x, ++i) {
        const int b = i & 1;
        const uint32_t use = i >> 1;
        if (use > 0 && !wait_poll(&bars[B_D1EMPTY + b], (use - 1) & 1)) break;
        tc_fence_after();
        const uint32_t d1 = tmem + 128 * b;
        for (int c = 0; c < C::KC1; ++c) {
          const int slot = gchunk % NSTAGE;
          if (!wait_poll(&bars[B_FULL + slot], (gchunk / NSTAGE) & 1)) {
            live = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + slot * CHUNK), b0 = smem_u32(sW1 + c * CHUNK);
#pragma unroll
          for (int k = 0; k < KSTEPS; ++k)
            mma_tc<F8>(d1, sdesc_k_sw128(a0 + 32 * k), sdesc_k_sw128(b0 + 32 * k), EL::IDESC,
                       (c > 0 || k > 0) ? 1u : 0u);
          mma_commit(&bars[B_EMPTY + slot]);
          ++gchunk;
        }
        if (!live) break;
        mma_commit(&bars[B_D1FULL + b]);
        if (C::G2) {
          if (pending >= 0) {
            if (!wait_or_abort(&bars[B_A2FULL], pending & 1, a.err, abort)) break;
            issue_gemm2();
          }
          pending = i;
        }
      }
      if (C::G2 && pending >= 0 && !*abort &&
          wait_or_abort(&bars[B_A2FULL], pending & 1, a.err, abort))
        issue_gemm2();
    }
  } else {
    // =========================== epilogue ==================================
    const int r = tid;  // TMEM lane == tile row
    const uint32_t lane_off = static_cast<uint32_t>(32 * warp) << 16;
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
      const int b = i & 1;
      const int64_t gr = tile * TM + r;
      const bool valid = gr < n_rows;
      if (!wait_or_abort(&bars[B_D1FULL + b], (i >> 1) & 1, a.err, abort)) break;
      tc_fence_after();
      const uint32_t t1 = tmem + 128 * b + lane_off;
      float mean, rstd;
      row_stats(t1, par, a.ws1, mean, rstd);
      float y[32];
      if constexpr (MODE == TC_CLS) {
        float p = 0.f;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          row_norm32(t1, cc, par, par + H, par + 2 * H, a.ws1, mean, rstd, y);
#pragma unroll
          for (int j = 0; j < 32; ++j) p = fmaf(y[j], par[6 * H + 32 * cc + j], p);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[B_D1EMPTY + b]);
        if (valid) a.logits[gr] = p + __ldg(a.bcls);
      } else {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          row_norm32(t1, cc, par, par + H, par + 2 * H, a.ws1, mean, rstd, y);
          if constexpr (F8) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              uint4 w;
              w.x = pack_e4m3x4(y[16 * q + 0], y[16 * q + 1], y[16 * q + 2], y[16 * q + 3]);
              w.y = pack_e4m3x4(y[16 * q + 4], y[16 * q + 5], y[16 * q + 6], y[16 * q + 7]);
              w.z = pack_e4m3x4(y[16 * q + 8], y[16 * q + 9], y[16 * q + 10], y[16 * q + 11]);
              w.w = pack_e4m3x4(y[16 * q + 12], y[16 * q + 13], y[16 * q + 14], y[16 * q + 15]);
              *reinterpret_cast<uint4*>(sA2 + sw128(r, 2 * cc + q)) = w;
            }
          } else {
            uint8_t* dst2 = sA2 + (cc >> 1) * CHUNK;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint4 w;
              w.x = pack_bf16(y[8 * q + 0], y[8 * q + 1]);
              w.y = pack_bf16(y[8 * q + 2], y[8 * q + 3]);
              w.z = pack_bf16(y[8 * q + 4], y[8 * q + 5]);
              w.w = pack_bf16(y[8 * q + 6], y[8 * q + 7]);
              *reinterpret_cast<uint4*>(dst2 + sw128(r, 4 * (cc & 1) + q)) = w;
            }
          }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&bars[B_D1EMPTY + b]);
          mbar_arrive(&bars[B_A2FULL]);
        }
        if (!wait_or_abort(&bars[B_D2FULL], i & 1, a.err, abort)) break;
        tc_fence_after();
        const uint32_t t2 = tmem + 256 + lane_off;
        row_stats(t2, par + 3 * H, a.ws2, mean, rstd);
        // The second GEMM has consumed A2, so its 32 KB stage the FP32 output:
        // 64 columns at a time, row-per-thread writes with 16-byte units
        // XOR-swizzled by (row % 8), then coalesced residual loads and stores
        // (16 lanes cover one 256-byte row segment).
        float* stg = reinterpret_cast<float*>(sA2);
        const int64_t row0 = tile * TM;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          // residual of the rows this thread stores in the coalesced pass, in two
          // batches fetched ahead of their use so the latency hides behind the
          // normalisation (batch a) and behind batch a's stores (batch b)
          const int l16 = lane & 15;
          constexpr int NIT = TM / (2 * EPI_WARPS);
          constexpr int NB = 4;
          float4 ra[NB], rb[NB];
          auto fetch_res = [&](int it0, float4 (&rr4)[NB]) {
#pragma unroll
            for (int k = 0; k < NB; ++k) {
              const int rr = ((it0 + k) * EPI_WARPS + warp) * 2 + (lane >> 4);
              const int64_t g2 = row0 + rr;
              rr4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
              if (g2 < n_rows) {
                const int64_t off = g2 * H + 64 * half + 4 * l16;
                if constexpr (MODE == TC_NODE_UPD) rr4[k] = *reinterpret_cast<const float4*>(a.h + off);
                if constexpr (MODE == TC_EDGE_UPD) rr4[k] = *reinterpret_cast<const float4*>(a.e + off);
              }
            }
          };
          auto store_rows = [&](int it0, const float4 (&rr4)[NB]) {
#pragma unroll
            for (int k = 0; k < NB; ++k) {
              const int rr = ((it0 + k) * EPI_WARPS + warp) * 2 + (lane >> 4);
              const int64_t g2 = row0 + rr;
              const float4 v = *reinterpret_cast<const float4*>(stg + rr * 64 + 4 * (l16 ^ (rr & 7)));
              if (g2 < n_rows) {
                const float4 o = make_float4(v.x + rr4[k].x, v.y + rr4[k].y, v.z + rr4[k].z,
                                             v.w + rr4[k].w);
                float* outp = MODE == TC_NODE_UPD ? a.h_out : a.e;
                *reinterpret_cast<float4*>(outp + g2 * H + 64 * half + 4 * l16) = o;
              }
            }
          };
          fetch_res(0, ra);
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            row_norm32(t2, 2 * half + cc, par + 3 * H, par + 4 * H, par + 5 * H, a.ws2, mean, rstd, y);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int un = (8 * cc + q) ^ (r & 7);
              *reinterpret_cast<float4*>(stg + r * 64 + 4 * un) =
                  make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
            }
          }
          fetch_res(NB, rb);
          asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
#pragma unroll
          for (int it0 = 0; it0 < NIT; it0 += 2 * NB) {
            store_rows(it0, ra);
            if (it0 + 2 * NB < NIT) fetch_res(it0 + 2 * NB, ra);
            store_rows(it0 + NB, rb);
            if (it0 + 3 * NB < NIT) fetch_res(it0 + 3 * NB, rb);
          }
          asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
        }
        tc_fence_before();
      }
    }
  }
  // ---- teardown -------------------------------------------------------------
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <int MODE, bool F8>
cudaError_t launch_tc(etx_ctx* ctx, const char* name, const TcArgs& a, int64_t max_rows,
                      cudaStream_t s) {
  using C = Cfg<MODE, F8>;
  static bool attr_set[8] = {false};
  if (!attr_set[ctx->device & 7]) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<MODE, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[ctx->device & 7] = true;
  }
  const int64_t tiles = (max_rows + TM - 1) / TM;
  if (tiles == 0) return cudaSuccess;
  const int grid = (int)(tiles < ctx->n_sms ? tiles : ctx->n_sms);
  launch(ctx, name, k_mlp_tc<MODE, F8>, grid, THREADS, C::SMEM, s, a);
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

void set_block(TcArgs& a, const BlockF32& f, const BlockTC& t, bool f8) {
  a.w1 = f8 ? t.w1f8 : t.w1;
  a.w2 = f8 ? t.w2f8 : t.w2;
  a.ws1 = f8 ? t.s1 : 1.f;
  a.ws2 = f8 ? t.s2 : 1.f;
  a.b1 = f.l1.b;
  a.g1 = f.g1;
  a.be1 = f.be1;
  a.b2 = f.l2.b;
  a.g2 = f.g2;
  a.be2 = f.be2;
}

template <int MODE>
cudaError_t launch_any(etx_ctx* ctx, bool f8, const char* n16, const char* n8, const TcArgs& a,
                       int64_t max_rows, cudaStream_t s) {
  return f8 ? launch_tc<MODE, true>(ctx, n8, a, max_rows, s)
            : launch_tc<MODE, false>(ctx, n16, a, max_rows, s);
}

}  // namespace

cudaError_t launch_edge_encoder_tc(etx_ctx* ctx, int64_t N, const int32_t* src, const int32_t* dst,
                                   const int32_t* n_edges_dev, bool f8, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, src, dst, n_edges_dev, nullptr);
  set_block(a, ctx->w.edge_enc, ctx->w.edge_enc_tc, f8);
  return launch_any<TC_EDGE_ENC>(ctx, f8, "gnn_edge_encoder_bf16", "gnn_edge_encoder_fp8", a,
                                 ctx->cfg.max_edges, s);
}

cudaError_t launch_node_update_tc(etx_ctx* ctx, int k, int64_t N, bool f8, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, nullptr, nullptr, nullptr, nullptr);
  set_block(a, ctx->w.node[k], ctx->w.node_tc[k], f8);
  return launch_any<TC_NODE_UPD>(ctx, f8, "gnn_node_update_bf16", "gnn_node_update_fp8", a, N, s);
}

cudaError_t launch_edge_update_tc(etx_ctx* ctx, int k, int64_t N, const int32_t* src,
                                  const int32_t* dst, const int32_t* n_edges_dev, bool f8,
                                  cudaStream_t s) {
  TcArgs a = base_args(ctx, N, src, dst, n_edges_dev, nullptr);
  set_block(a, ctx->w.edge[k], ctx->w.edge_tc[k], f8);
  return launch_any<TC_EDGE_UPD>(ctx, f8, "gnn_edge_update_bf16", "gnn_edge_update_fp8", a,
                                 ctx->cfg.max_edges, s);
}

cudaError_t launch_classifier_tc(etx_ctx* ctx, int64_t N, const int32_t* n_edges_dev, float* logits,
                                 bool f8, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, nullptr, nullptr, n_edges_dev, logits);
  const BlockTC& t = ctx->w.cls_tc;
  a.w1 = f8 ? t.w1f8 : t.w1;
  a.ws1 = f8 ? t.s1 : 1.f;
  a.ws2 = 1.f;
  a.b1 = ctx->w.cls.l1.b;
  a.g1 = ctx->w.cls.g1;
  a.be1 = ctx->w.cls.be1;
  a.wcls = ctx->w.cls.w2;
  a.bcls = ctx->w.cls.b2;
  return launch_any<TC_CLS>(ctx, f8, "gnn_classifier_bf16", "gnn_classifier_fp8", a,
                            ctx->cfg.max_edges, s);
}

}  // namespace etx
