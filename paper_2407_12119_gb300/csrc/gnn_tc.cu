// Interaction-network MLP blocks on the 5th-generation tensor cores
// (tcgen05, BF16 or e4m3 operands, FP32 accumulation in tensor memory).
//
// Persistent kernel, one CTA per SM, 512 threads (16 warps, so 128 registers
// a thread) in three roles that run concurrently over the CTA's 128-row tiles:
//   warps 8-14 producers: fill a 3-slot ring of A-operand chunks (128 rows x
//              128 bytes, K-major 128-byte swizzle).  Columns that come from
//              the FP32 streams (e, [h, m_out, m_in]) are loaded coalesced,
//              rounded to the operand type and stored, one step of loads in
//              flight in registers; gathered node rows ([h_i, h_j] of the edge
//              blocks) are copied without conversion from a low-precision copy
//              of h by asynchronous 16-byte copies that the ring's mbarrier
//              counts;
//   warp 15    MMA issuer (one thread), an event loop over two queues: the
//              first GEMM of the next tile, one ring slot at a time, and the
//              second GEMM of the oldest tile whose activations are ready;
//   warps 0-7  epilogue, two groups of four warps that take alternate tiles, so
//              that one group's second epilogue overlaps the other's first.
//              Warp w reads TMEM lanes 32 (w % 4) .. +31, one row per thread,
//              64 columns per wait.  Bias + LayerNorm (one pass of shifted
//              sums) + ReLU of the first GEMM are written back to tensor memory,
//              over the accumulator columns already consumed, as the A operand
//              of the second GEMM; bias + LayerNorm + ReLU + FP32 residual of
//              the second are staged per warp in shared memory and stored
//              coalesced (or, for the classifier, reduced to the logit); the
//              node update also writes the low-precision copy of h.
//              Elementwise math uses the packed FP32x2 instructions.
// Tensor memory (512 columns): group g owns D1 at column 128 g (first GEMM,
// then its activations in the first 64 columns) and D2 at 256 + 128 g.
// Stages hand over through mbarriers (transaction-counted bulk copies for
// the resident weights, tcgen05.commit for MMA completion, warp arrivals
// otherwise).  Every wait is bounded; a timeout records ETX_ERR_TIMEOUT,
// raises a shared abort flag and every role stops.
#include <cuda_bf16.h>

#include <cstring>

#include "sm100.cuh"

namespace etx {
namespace {

using namespace sm100;

constexpr int H = 128;
constexpr int TM = 128;                  // rows per tile
constexpr int CHUNK = TM * 128;          // 16 KB operand chunk: 128 rows x 128 bytes
constexpr int SUB = 64;                  // K columns a producer fetches per step (256 B FP32)
constexpr int KSTEPS = 4;                // MMAs per chunk (32 bytes of K each)
// 16 warps: an SM sub-partition then holds four, and each thread 128 registers
constexpr int EPI_WARPS = 8, PROD_WARPS = 7;  // two epilogue groups of four warps
constexpr int MMA_WARP = EPI_WARPS + PROD_WARPS;
constexpr int THREADS = 32 * (MMA_WARP + 1);  // 512
constexpr int NCH = H / 64;              // 64-column chunks of a row (two TMEM loads, one wait)
constexpr int PROD_THREADS = 32 * PROD_WARPS;
constexpr uint32_t TMEM_COLS = 512;

enum TcMode { TC_EDGE_ENC = 0, TC_NODE_UPD = 1, TC_EDGE_UPD = 2, TC_CLS = 3 };


// Operand type: BF16 (2 bytes, 64 K columns per 128-byte row) or FP8 e4m3
// (1 byte, 128 K columns per row).  Either way one MMA consumes 32 bytes of K,
// which is 8 columns of an A operand held in tensor memory.
template <bool F8>
struct Elt {
  static constexpr int KCH = F8 ? 128 : 64;   // K columns per chunk
  static constexpr int SUBS = KCH / SUB;       // producer steps per chunk
  static constexpr uint32_t IDESC = F8 ? idesc_e4m3_f32<TM, H>() : idesc_bf16_f32<TM, H>();
};

constexpr int SMEM_MAX = 232448;         // opt-in shared memory per CTA
template <int MODE, bool F8, int NS>
struct Cfg {
  static constexpr int KIN = MODE == TC_EDGE_ENC ? 2 * H : (MODE == TC_CLS ? H : 3 * H);
  static constexpr int KC1 = KIN / Elt<F8>::KCH;     // chunks of the first GEMM
  static constexpr int KS = KIN / SUB;               // producer steps per tile
  static constexpr int C2 = H / Elt<F8>::KCH;        // chunks of the second GEMM
  static constexpr bool G2 = MODE != TC_CLS;
  // LayerNorm parameters: read from the kernel's parameter space at compile-time
  // offsets (column loops unrolled), except in the e4m3 node and edge updates,
  // which ran 5% and 15% slower that way and keep a shared-memory copy read in
  // rolled loops.
  static constexpr bool SP = F8 && (MODE == TC_NODE_UPD || MODE == TC_EDGE_UPD);
  static constexpr int PAR_BYTES = SP ? 7 * H * 4 : 0;
  static constexpr int OFF_W1 = 0;
  static constexpr int OFF_W2 = OFF_W1 + KC1 * CHUNK;
  static constexpr int OFF_A = OFF_W2 + (G2 ? C2 * CHUNK : 0);
  static constexpr int FIXED = OFF_A + (G2 ? EPI_WARPS * 2048 : 0) + PAR_BYTES + 8 * 64 + 16 + 1024;
  // NS A-operand ring slots (as far as shared memory holds them).  A deeper ring
  // lets the first GEMM of later tiles queue in the (in-order) tensor pipe
  // ahead of the second GEMM the epilogue waits for; the autotuner picks NS.
  static constexpr int NST = (SMEM_MAX - FIXED) / CHUNK > NS ? NS : (SMEM_MAX - FIXED) / CHUNK;
  static_assert(NST >= 2, "shared memory too small for the ring");
  // barrier indices (the per-group ones come in pairs, index + group)
  static constexpr int B_W = 0, B_FULL = 1, B_EMPTY = B_FULL + NST, B_D1FULL = B_EMPTY + NST,
                       B_D1EMPTY = B_D1FULL + 2, B_A2FULL = B_D1EMPTY + 2, B_D2FULL = B_A2FULL + 2,
                       B_D2EMPTY = B_D2FULL + 2, N_BARS = B_D2EMPTY + 2;
  static_assert(N_BARS <= 64, "barrier area");
  static constexpr int OFF_STG = OFF_A + NST * CHUNK;               // 8 per-warp 2 KB output stages
  static constexpr int OFF_PAR = OFF_STG + (G2 ? EPI_WARPS * 2048 : 0);  // SP: 7 x 128 floats
  static constexpr int OFF_BAR = OFF_PAR + PAR_BYTES;
  static constexpr int OFF_MISC = OFF_BAR + 8 * 64;                  // tmem addr, abort flag
  static constexpr int BYTES = OFF_MISC + 16;
  static constexpr int SMEM = BYTES + 1024;  // slack for 1024-byte alignment
  static_assert(SMEM <= SMEM_MAX, "shared memory");
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
  float ws1, ws2;     // accumulator scales: weight scale x activation scale (1 for BF16)
  // e4m3 only: reciprocal power-of-two activation scales applied before rounding:
  // the block input (FP32 stream columns), the second product's operand, and the
  // low-precision h copy the node update writes for the next edge block
  float in_inv, mid_inv, hlp_inv;
  const float* bcls;  // [1]
  uint8_t* h_lp;      // h rounded to the operand type (node update writes it)
  uint8_t* e_lp;      // edge stream stored in BF16 (ES kernels): rows of H values, 2H bytes
  const uint8_t* m_lp;  // node update: [m_out, m_in] rounded to the operand type, rows of 2H
  int* err;
  // b1 g1 be1 b2 g2 be2 of the block (or b1 g1 be1, -, -, -, w2 of the classifier), by
  // value: the epilogue reads them at compile-time offsets from the kernel's
  // parameter space (constant bank), not through the load/store pipe.
  alignas(16) float prm[7][H];
};

// Four values to e4m3 (round to nearest even, saturating to +-448), first value
// in the lowest byte.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  uint32_t r;
  asm("{\n\t.reg .b16 lo, hi;\n\t"
      "cvt.rn.satfinite.e4m3x2.f32 lo, %2, %1;\n\t"
      "cvt.rn.satfinite.e4m3x2.f32 hi, %4, %3;\n\t"
      "mov.b32 %0, {lo, hi};\n\t}"
      : "=r"(r)
      : "f"(a), "f"(b), "f"(c), "f"(d));
  return r;
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

// Bounded wait (2 s of device time, or an iteration cap) that also gives up
// when another role raised the abort flag.  A waiting thread sleeps in
// try_wait for up to 256 ns per poll.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, int* err,
                                              volatile int* abort) {
  uint64_t t0 = 0;
  for (uint32_t i = 0; i < (kWaitCap << 4); ++i) {
    if (mbar_try_wait_sleep(bar, parity, 256)) return true;
    if ((i & 15) == 15) {
      if (*abort) return false;
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kWaitNs) break;
    }
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

// Two values to BF16 with ReLU, first value in the low half.
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Four LayerNorm parameters: from shared memory (SP, a load kept in program
// order, which limits how many the compiler hoists ahead of their use and so
// the registers they hold) or from the kernel's parameter space (compile-time
// offsets once the loops are unrolled).
template <bool SP>
__device__ __forceinline__ float4 lds4(const float* p) {
  if constexpr (SP) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(smem_u32(p)));
    return v;
  } else {
    return make_float4(p[0], p[1], p[2], p[3]);
  }
}

// t -= mean in place over N values; returns the sum of squares of the centred values.
template <int N>
__device__ __forceinline__ float centre_sq(float* __restrict__ t, float mean) {
  float2 acc[4] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
  const float2 nm = f2(-mean, -mean);
#pragma unroll
  for (int j = 0; j < N; j += 2) {
    const float2 d = __fadd2_rn(f2(t[j], t[j + 1]), nm);
    t[j] = d.x; t[j + 1] = d.y;
    acc[(j >> 1) & 3] = __ffma2_rn(d, d, acc[(j >> 1) & 3]);
  }
  const float2 s01 = __fadd2_rn(acc[0], acc[1]), s23 = __fadd2_rn(acc[2], acc[3]);
  const float2 s = __fadd2_rn(s01, s23);
  return s.x + s.y;
}

// t = sc * acc + b over N columns, in place; adds the sums of d = t - shift and
// of d^2 to s and q (four interleaved pair chains, fixed order).
template <int N, bool SP>
__device__ __forceinline__ void shifted_sums(float* __restrict__ t, const float* __restrict__ b,
                                             float sc, float shift, float& s, float& q) {
  float2 as[2] = {f2(0.f, 0.f), f2(0.f, 0.f)}, aq[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
  const float2 sc2 = f2(sc, sc), ns = f2(-shift, -shift);
#pragma unroll
  for (int j = 0; j < N; j += 4) {
    const float4 bb = lds4<SP>(b + j);
    const float2 x0 = __ffma2_rn(f2(t[j], t[j + 1]), sc2, f2(bb.x, bb.y));
    const float2 x1 = __ffma2_rn(f2(t[j + 2], t[j + 3]), sc2, f2(bb.z, bb.w));
    t[j] = x0.x; t[j + 1] = x0.y; t[j + 2] = x1.x; t[j + 3] = x1.y;
    const float2 d0 = __fadd2_rn(x0, ns), d1 = __fadd2_rn(x1, ns);
    as[0] = __fadd2_rn(as[0], d0);
    as[1] = __fadd2_rn(as[1], d1);
    aq[0] = __ffma2_rn(d0, d0, aq[0]);
    aq[1] = __ffma2_rn(d1, d1, aq[1]);
  }
  const float2 ss = __fadd2_rn(as[0], as[1]), qq = __fadd2_rn(aq[0], aq[1]);
  s += ss.x + ss.y;
  q += qq.x + qq.y;
}

// t -= mean over N values.
template <int N>
__device__ __forceinline__ void centre(float* __restrict__ t, float mean) {
  const float2 nm = f2(-mean, -mean);
#pragma unroll
  for (int j = 0; j < N; j += 2) {
    const float2 d = __fadd2_rn(f2(t[j], t[j + 1]), nm);
    t[j] = d.x; t[j + 1] = d.y;
  }
}

// y = (d * rstd) * g + be for N centred values d (ReLU left to the caller).
template <int N, bool SP>
__device__ __forceinline__ void affine(float* __restrict__ d, const float* __restrict__ g,
                                       const float* __restrict__ be, float rstd) {
  const float2 rs = f2(rstd, rstd);
#pragma unroll
  for (int j = 0; j < N; j += 4) {
    const float4 gg = lds4<SP>(g + j);
    const float4 ee = lds4<SP>(be + j);
    const float2 y0 = __ffma2_rn(__fmul2_rn(f2(d[j], d[j + 1]), rs), f2(gg.x, gg.y), f2(ee.x, ee.y));
    const float2 y1 =
        __ffma2_rn(__fmul2_rn(f2(d[j + 2], d[j + 3]), rs), f2(gg.z, gg.w), f2(ee.z, ee.w));
    d[j] = y0.x; d[j + 1] = y0.y; d[j + 2] = y1.x; d[j + 3] = y1.y;
  }
}

// ES (BF16 only; edge encoder, edge update, classifier): the edge stream e is
// stored in BF16 (a.e_lp) instead of FP32: the producers copy its rows into
// the ring like the gathered node rows, the epilogue adds the BF16 residual
// and writes the sum rounded to BF16.
template <int MODE, bool F8, int NS, bool ES = false>
__global__ void __launch_bounds__(THREADS, 1) k_mlp_tc(const __grid_constant__ TcArgs a) {
  static_assert(!ES || (!F8 && MODE != TC_NODE_UPD), "BF16 edge storage: BF16 edge blocks only");
  using C = Cfg<MODE, F8, NS>;
  using EL = Elt<F8>;
  constexpr int NSTAGE = C::NST;
  constexpr int B_W = C::B_W, B_FULL = C::B_FULL, B_EMPTY = C::B_EMPTY, B_D1FULL = C::B_D1FULL,
                B_D1EMPTY = C::B_D1EMPTY, B_A2FULL = C::B_A2FULL, B_D2FULL = C::B_D2FULL,
                B_D2EMPTY = C::B_D2EMPTY;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sW1 = smem + C::OFF_W1;
  uint8_t* sW2 = smem + C::OFF_W2;
  uint8_t* sA = smem + C::OFF_A;
  // b1 g1 be1 b2 g2 be2 wcls: parameter space, or (SP) a shared-memory copy
  const float* par = C::SP ? reinterpret_cast<const float*>(smem + C::OFF_PAR) : &a.prm[0][0];
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
    for (int g = 0; g < 2; ++g) {
      mbar_init(&bars[B_D1FULL + g], 1);
      // D1 is free again once the second GEMM has read the activations in it
      // (or, for the classifier, once the epilogue group has read it)
      mbar_init(&bars[B_D1EMPTY + g], C::G2 ? 1 : 4);
      mbar_init(&bars[B_A2FULL + g], 4);
      mbar_init(&bars[B_D2FULL + g], 1);
      mbar_init(&bars[B_D2EMPTY + g], 4);
    }
    *abort = 0;
    fence_mbar_init();
  }
  if constexpr (C::SP) {
    float* sp = reinterpret_cast<float*>(smem + C::OFF_PAR);
    for (int i = tid; i < 7 * H; i += THREADS) sp[i] = a.prm[i / H][i % H];
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
  const int64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nn = (int)a.n_nodes;

  if (warp >= EPI_WARPS && warp < MMA_WARP) {
    // =========================== producers =================================
    // Ring chunks are filled in order.  Chunks of FP32 stream columns are
    // converted by the producer threads: a 64-column step of the tile is 2048
    // float4 pieces, piece f = pt + PROD_THREADS k is row f / 16, columns
    // 4 (f % 16) .. +3, so consecutive threads read consecutive 16 bytes of a
    // row (coalesced) and write 8 (BF16) or 4 (e4m3) bytes of its swizzled
    // operand row.  Chunks of gathered node rows ([h_i, h_j] of the edge
    // blocks) are copied from the low-precision copy of h with asynchronous
    // 16-byte copies: piece f is row f / 8, 16-byte unit f % 8, no conversion.
    const int pt = tid - 32 * EPI_WARPS;
    constexpr int NF = (TM * SUB / 4 + PROD_THREADS - 1) / PROD_THREADS;  // float4 pieces per thread
    constexpr int NG = (TM * 8 + PROD_THREADS - 1) / PROD_THREADS;        // 16-byte copies per thread
    // edge blocks copy [h_i, h_j] from the low-precision h; the node update
    // copies [m_out, m_in] from the low-precision messages (its own row)
    constexpr bool GATHER = MODE != TC_CLS || ES;
    // 64-column FP32 steps per tile done by the threads (the copies do the rest)
    constexpr int SE = GATHER ? ((MODE == TC_EDGE_ENC || ES) ? 0 : H / SUB) : C::KS;
    // ES: the first H / KCH chunks of the edge blocks are the tile's own e rows
    constexpr int KOWN = (ES && MODE != TC_EDGE_ENC) ? H / EL::KCH : 0;
    // Loads of step c (64 columns of the FP32 block input) of local tile t.
    auto fetch = [&](int64_t t, int c, float4 (&f)[NF]) {
      if (t >= my_tiles) return;
      const int64_t row0 = (blockIdx.x + t * gridDim.x) * TM;
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int fi = pt + PROD_THREADS * k;
        const int64_t gr = row0 + (fi >> 4);
        f[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (fi < TM * SUB / 4 && gr < n_rows)
          // L2 only: the epilogue re-reads these rows (the residual) from L2
          f[k] = __ldcg(reinterpret_cast<const float4*>(chunk_src<MODE>(a, SUB * c, gr, 0, 0) + 4 * (fi & 15)));
      }
    };
    // Wait until ring chunk j's slot is free again (its previous round consumed).
    auto slot_free = [&](int64_t j) {
      const uint32_t round = (uint32_t)(j / NSTAGE);
      return round == 0 ||
             wait_or_abort(&bars[B_EMPTY + (int)(j % NSTAGE)], (round - 1) & 1, a.err, abort);
    };
    // Convert and store step c of local tile t.
    auto store = [&](int64_t t, int c, const float4 (&f)[NF]) {
      const int64_t j = t * C::KC1 + c / EL::SUBS;  // ring chunk
      const int hpart = c % EL::SUBS;              // which 64 columns of it
      const int slot = (int)(j % NSTAGE);
      if (hpart == 0 && !slot_free(j)) return false;
      uint8_t* dstc = sA + slot * CHUNK;
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int fi = pt + PROD_THREADS * k;
        if (fi < TM * SUB / 4) {
          const int r = fi >> 4, u = fi & 15;
          const float4 v = f[k];
          if constexpr (F8)
            *reinterpret_cast<uint32_t*>(dstc + sw128(r, 4 * hpart + (u >> 2)) + 4 * (u & 3)) =
                pack_e4m3x4(v.x * a.in_inv, v.y * a.in_inv, v.z * a.in_inv, v.w * a.in_inv);
          else
            *reinterpret_cast<uint2*>(dstc + sw128(r, u >> 1) + 8 * (u & 1)) =
                make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
        }
      }
      if (hpart == EL::SUBS - 1) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[B_FULL + slot]);
      }
      return true;
    };
    // The edge rows e of a later local tile (contiguous, H floats a row) are
    // prefetched into L2 by one thread, so the register loads of the
    // producers hit L2 and DRAM streams independently of them: the classifier
    // two tiles ahead (1.14 -> 0.94 ms), the BF16 edge update one tile ahead
    // (3.13 -> 2.9 ms; two and three tiles ahead were 2% and 9% slower than
    // one).  The FP8 edge update, which moves fewer operand bytes per tile,
    // ran 7% slower with it and goes without.
    auto prefetch_tile = [&](int64_t t) {
      if (pt != 0 || t >= my_tiles) return;
      const int64_t row0 = (blockIdx.x + t * gridDim.x) * TM;
      const int64_t rows = n_rows - row0 < TM ? n_rows - row0 : TM;
      if (rows <= 0) return;
      if constexpr (ES)
        prefetch_l2_bulk(a.e_lp + row0 * 2 * H, (uint32_t)(rows * H * 2));
      else
        prefetch_l2_bulk(a.e + row0 * H, (uint32_t)(rows * H * sizeof(float)));
    };
    float4 b0[NF], b1[NF];
    if constexpr (GATHER) {
      constexpr int KE = (SE * SUB) / EL::KCH;  // chunks of FP32 stream columns
      constexpr int KH = H / EL::KCH;           // chunks per gathered node row
      // node indices of this thread's copy rows, loaded one tile ahead of use
      int gs[NG], gd[NG], ns[NG], nd[NG], go[NG], no[NG];
      auto load_idx = [&](int64_t t, int (&xs)[NG], int (&xd)[NG], int (&xo)[NG]) {
        const int64_t r0 = (blockIdx.x + t * gridDim.x) * TM;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          const int fi = pt + PROD_THREADS * k;
          const int64_t gr = r0 + (fi >> 3);
          const bool ok = t < my_tiles && fi < TM * 8 && gr < n_rows;
          xo[k] = ok ? (int)gr : 0;  // the tile's own row (rows past the end read row 0)
          if constexpr (MODE == TC_NODE_UPD || MODE == TC_CLS) {
            xs[k] = xd[k] = xo[k];
          } else {
            // raw indices: clamped where they are used, a tile later, so these
            // loads stay in flight instead of stalling the producers here
            xs[k] = ok ? a.src[gr] : 0;
            xd[k] = ok ? a.dst[gr] : 0;
          }
        }
      };
      load_idx(0, gs, gd, go);
      if constexpr (SE > 0) {
        fetch(0, 0, b0);
        fetch(0, 1, b1);
      }
      for (int64_t t = 0; t < my_tiles; ++t) {
        if constexpr (MODE == TC_EDGE_UPD && !F8) prefetch_tile(t + 1);
        if constexpr (MODE == TC_CLS) prefetch_tile(t + 2);
        load_idx(t + 1, ns, nd, no);
        if constexpr (SE > 0) {
          if (!store(t, 0, b0)) break;
          if (!store(t, 1, b1)) break;
        }
        bool ok = true;
        for (int c = KE; c < C::KC1; ++c) {
          // The next tile's FP32 loads go out before this tile's last gather
          // chunk: issued earlier, they queue ahead of the gathers the MMA
          // waits for next (measured 5% slower), issued later, they land late.
          if (SE > 0 && c == C::KC1 - 1) {
            fetch(t + 1, 0, b0);
            fetch(t + 1, 1, b1);
          }
          const int64_t j = t * C::KC1 + c;
          const int slot = (int)(j % NSTAGE);
          if (!slot_free(j)) {
            ok = false;
            break;
          }
          // source rows: the tile's own e rows (ES, first KOWN chunks), node rows of h
          // (H values) or message rows (2H values)
          const bool own = c < KOWN;
          const int hc = own ? c : c - KE - KOWN;
          const int rowbytes = (MODE == TC_NODE_UPD ? 2 : 1) * (F8 ? H : 2 * H);
          const int cbase = (MODE == TC_NODE_UPD || own ? hc : hc % KH) * 128;  // byte offset in the row
          const uint8_t* srcb = own ? a.e_lp : (MODE == TC_NODE_UPD ? a.m_lp : a.h_lp);
#pragma unroll
          for (int k = 0; k < NG; ++k) {
            const int fi = pt + PROD_THREADS * k;
            const int row = own ? go[k] : min(max(hc < KH ? gs[k] : gd[k], 0), max(nn - 1, 0));
            if (fi < TM * 8)
              cp_async16(sA + slot * CHUNK + sw128(fi >> 3, fi & 7),
                         srcb + (int64_t)row * rowbytes + cbase + 16 * (fi & 7));
          }
          cp_async_arrive(&bars[B_FULL + slot]);
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars[B_FULL + slot]);
        }
        if (!ok) break;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          gs[k] = ns[k];
          gd[k] = nd[k];
          go[k] = no[k];
        }
      }
    } else {
      // every chunk from the FP32 streams: a flattened stream of steps with the
      // next step's loads in flight while one is stored
      const int64_t total = my_tiles * C::KS;
      prefetch_tile(1);
      fetch(0, 0, b0);
      for (int64_t q = 0; q < total; q += 2) {
        if (q % C::KS == 0) prefetch_tile(q / C::KS + 2);
        fetch((q + 1) / C::KS, (int)((q + 1) % C::KS), b1);
        if (!store(q / C::KS, (int)(q % C::KS), b0)) break;
        if (q + 1 >= total) break;
        fetch((q + 2) / C::KS, (int)((q + 2) % C::KS), b0);
        if (!store((q + 1) / C::KS, (int)((q + 1) % C::KS), b1)) break;
      }
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
      if (wait_or_abort(&bars[B_W], 0, a.err, abort)) {
        int64_t g1 = 0, g2 = 0;  // next local tile of the first / second GEMM
        int c1 = 0;              // next chunk of tile g1
        bool d1_free = false;    // D1 of tile g1 may be written
        uint32_t gchunk = 0, idle = 0;
        uint64_t t0 = 0;
        while (C::G2 ? g2 < my_tiles : g1 < my_tiles) {
          bool progress = false;
          // second GEMM of tile g2, A = its activations in D1, into D2
          if (C::G2 && g2 < g1) {
            const int b = (int)(g2 & 1);
            const uint32_t u = (uint32_t)(g2 >> 1);
            if (mbar_try_wait(&bars[B_A2FULL + b], u & 1) &&
                (u == 0 || mbar_try_wait(&bars[B_D2EMPTY + b], (u - 1) & 1))) {
              tc_fence_after();
              const uint32_t a2 = tmem + 128 * b, d2 = tmem + 256 + 128 * b;
#pragma unroll
              for (int c = 0; c < C::C2; ++c)
#pragma unroll
                for (int k = 0; k < KSTEPS; ++k)
                  mma_tc_ts<F8>(d2, a2 + 8 * (c * KSTEPS + k),
                                sdesc_k_sw128(smem_u32(sW2 + c * CHUNK) + 32 * k), EL::IDESC,
                                (c > 0 || k > 0) ? 1u : 0u);
              mma_commit(&bars[B_D2FULL + b]);
              mma_commit(&bars[B_D1EMPTY + b]);
              ++g2;
              progress = true;
            }
          }
          // next ring slot of the first GEMM of tile g1, into D1
          if (g1 < my_tiles) {
            const int b = (int)(g1 & 1);
            const uint32_t u = (uint32_t)(g1 >> 1);
            if (!d1_free) d1_free = u == 0 || mbar_try_wait(&bars[B_D1EMPTY + b], (u - 1) & 1);
            const int slot = (int)(gchunk % NSTAGE);
            if (d1_free && mbar_try_wait(&bars[B_FULL + slot], (gchunk / NSTAGE) & 1)) {
              tc_fence_after();
              fence_proxy_async();  // ring data written by asynchronous copies
              const uint32_t a0 = smem_u32(sA + slot * CHUNK), w0 = smem_u32(sW1 + c1 * CHUNK);
#pragma unroll
              for (int k = 0; k < KSTEPS; ++k)
                mma_tc<F8>(tmem + 128 * b, sdesc_k_sw128(a0 + 32 * k), sdesc_k_sw128(w0 + 32 * k),
                           EL::IDESC, (c1 > 0 || k > 0) ? 1u : 0u);
              mma_commit(&bars[B_EMPTY + slot]);
              ++gchunk;
              if (++c1 == C::KC1) {
                mma_commit(&bars[B_D1FULL + b]);
                c1 = 0;
                ++g1;
                d1_free = false;
              }
              progress = true;
            }
          }
          if (progress) {
            idle = 0;
            t0 = 0;
          } else if ((++idle & 63) == 0) {
            if (*abort) break;
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) {
              t0 = now;
            } else if (now - t0 > kWaitNs || idle > (kWaitCap << 4)) {
              set_err(a.err, DERR_TIMEOUT);
              *abort = 1;
              break;
            }
          }
        }
      }
    }
  } else {
    // =========================== epilogue ==================================
    const int grp = warp >> 2, qr = warp & 3;  // group, TMEM lane quarter
    const int r = 32 * qr + lane;              // TMEM lane == tile row
    const uint32_t lane_off = static_cast<uint32_t>(32 * qr) << 16;
    const uint32_t t1 = tmem + 128 * grp + lane_off;        // D1, then the activations
    const uint32_t t2 = tmem + 256 + 128 * grp + lane_off;  // D2
    float* stg = reinterpret_cast<float*>(smem + C::OFF_STG + 2048 * warp);  // 32 rows x 16 FP32
    // LayerNorm statistics of t = sc * acc + b over the row's 128 columns, in one
    // pass over two 64-column chunks read from TMEM: sums of d = t - t_0 and of
    // d^2 (shifted by the row's first value, so the variance does not cancel).
    auto layer_stats = [&](uint32_t tb, float (&t)[64], const float* b, float sc, float& mean,
                           float& rstd) {
      float s = 0.f, q = 0.f, shift = 0.f;
#pragma unroll (C::SP ? 1 : NCH)
      for (int ch = 0; ch < NCH; ++ch) {
        tmem_ld64_wait(tb + 64 * ch, t);
        if (ch == 0) shift = fmaf(t[0], sc, b[0]);
        shifted_sums<64, C::SP>(t, b + 64 * ch, sc, shift, s, q);
      }
      const float ms = s * (1.0f / H);
      mean = shift + ms;
      rstd = 1.0f / sqrtf(fmaxf(q * (1.0f / H) - ms * ms, 0.f) + kLnEps);
    };
    // Chunk ch (64 columns) of the row, normalised (ReLU left to the caller).
    auto norm_chunk = [&](uint32_t tb, float (&t)[64], int ch, const float* p3, float sc,
                          float mean, float rstd) {
      tmem_ld64_wait(tb + 64 * ch, t);
      float s_unused = 0.f, q_unused = 0.f;
      shifted_sums<64, C::SP>(t, p3 + 64 * ch, sc, 0.f, s_unused, q_unused);
      centre<64>(t, mean);
      affine<64, C::SP>(t, p3 + H + 64 * ch, p3 + 2 * H + 64 * ch, rstd);
    };
    const float* resid = MODE == TC_NODE_UPD ? a.h : a.e;
    float* outp = MODE == TC_NODE_UPD ? a.h_out : a.e;
    for (int64_t i = grp; i < my_tiles; i += 2) {
      const uint32_t ph = (uint32_t)(i >> 1) & 1;
      const int64_t row0 = (blockIdx.x + i * gridDim.x) * TM;
      const int64_t gr = row0 + r;
      if (!wait_or_abort(&bars[B_D1FULL + grp], ph, a.err, abort)) break;
      tc_fence_after();
      float t[64];
      float mean, rstd;
      layer_stats(t1, t, par, a.ws1, mean, rstd);
      if constexpr (MODE == TC_CLS) {
        float2 acc[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll (C::SP ? 1 : NCH)
        for (int ch = 0; ch < NCH; ++ch) {
          norm_chunk(t1, t, ch, par, a.ws1, mean, rstd);
          const float* wc = par + 6 * H + 64 * ch;
#pragma unroll
          for (int j = 0; j < 64; j += 4) {
            const float4 ww = lds4<C::SP>(wc + j);
            acc[0] = __ffma2_rn(f2(fmaxf(t[j], 0.f), fmaxf(t[j + 1], 0.f)), f2(ww.x, ww.y), acc[0]);
            acc[1] = __ffma2_rn(f2(fmaxf(t[j + 2], 0.f), fmaxf(t[j + 3], 0.f)), f2(ww.z, ww.w), acc[1]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[B_D1EMPTY + grp]);
        const float2 pp = __fadd2_rn(acc[0], acc[1]);
        if (gr < n_rows) a.logits[gr] = (pp.x + pp.y) + __ldg(a.bcls);
      } else {
        // Activations of chunk ch (64 columns) go to TMEM columns [32 ch, 32 ch + 32)
        // as BF16 pairs (or [16 ch, 16 ch + 16) as e4m3 quads): accumulator
        // columns this warp has already read, as chunks run in order.
#pragma unroll (C::SP ? 1 : NCH)
        for (int ch = 0; ch < NCH; ++ch) {
          norm_chunk(t1, t, ch, par, a.ws1, mean, rstd);
          if constexpr (F8) {
            uint32_t v[16];
            const float mi = a.mid_inv;  // a power of two: the scaling is exact
#pragma unroll
            for (int q = 0; q < 16; ++q)
              v[q] = pack_e4m3x4(fmaxf(t[4 * q], 0.f) * mi, fmaxf(t[4 * q + 1], 0.f) * mi,
                                 fmaxf(t[4 * q + 2], 0.f) * mi, fmaxf(t[4 * q + 3], 0.f) * mi);
            tmem_st16(t1 + 16 * ch, v);
          } else {
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              uint32_t v[16];
#pragma unroll
              for (int q = 0; q < 16; ++q) v[q] = pack_bf16_relu(t[32 * h2 + 2 * q], t[32 * h2 + 2 * q + 1]);
              tmem_st16(t1 + 32 * ch + 16 * h2, v);
            }
          }
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[B_A2FULL + grp]);
        // Output: each 64-column chunk goes out as four 16-column quarters.  A
        // quarter is staged row per thread (64 bytes a row, 16-byte units
        // XOR-swizzled by (row / 2) % 4) in the warp's 2 KB buffer, read back in
        // the coalesced layout (4 lanes per 64-byte row segment, 8 rows per
        // instruction), added to the residual and stored; no barrier waits on
        // the global stores.  One buffer instead of two alternating ones costs a
        // second warp barrier per quarter and leaves 16 KB more for L1 (node
        // update 8% faster, the others unchanged).
        const int u4 = lane & 3;
        const int64_t crow = row0 + 32 * qr + (lane >> 2);  // rows crow + 8 it, it < 4
        const int nval = (int)(n_rows - crow < 32 ? (n_rows - crow > 0 ? n_rows - crow : 0) : 32);
        const int64_t coff = crow * H + 4 * u4;
        if (!wait_or_abort(&bars[B_D2FULL + grp], ph, a.err, abort)) break;
        tc_fence_after();
        layer_stats(t2, t, par + 3 * H, a.ws2, mean, rstd);
#pragma unroll (C::SP ? 1 : NCH)
        for (int ch = 0; ch < NCH; ++ch) {
          norm_chunk(t2, t, ch, par + 3 * H, a.ws2, mean, rstd);
          if (ch == NCH - 1) {  // D2 fully read: the group's next second GEMM may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[B_D2EMPTY + grp]);
          }
#pragma unroll
          for (int hh = 0; hh < 4; ++hh) {
            const int col = 64 * ch + 16 * hh;  // first column of the quarter
            float* buf = stg;  // 2 KB: 32 rows x 16 FP32
            __syncwarp();      // the previous quarter's reads are done
            float4 res[4];
#pragma unroll
            for (int it = 0; it < 4; ++it) {
              res[it] = make_float4(0.f, 0.f, 0.f, 0.f);
              if (MODE != TC_EDGE_ENC && 8 * it < nval) {
                if constexpr (ES) {
                  const uint2 u = *reinterpret_cast<const uint2*>(a.e_lp + 2 * (coff + 8 * it * H + col));
                  res[it] = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                        __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
                } else {
                  res[it] = *reinterpret_cast<const float4*>(resid + coff + 8 * it * H + col);
                }
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              *reinterpret_cast<float4*>(buf + 16 * lane + 4 * (u ^ ((lane >> 1) & 3))) =
                  make_float4(fmaxf(t[16 * hh + 4 * u], 0.f), fmaxf(t[16 * hh + 4 * u + 1], 0.f),
                              fmaxf(t[16 * hh + 4 * u + 2], 0.f), fmaxf(t[16 * hh + 4 * u + 3], 0.f));
            __syncwarp();
#pragma unroll
            for (int it = 0; it < 4; ++it) {
              const int lr = 8 * it + (lane >> 2);
              const float4 v = *reinterpret_cast<const float4*>(buf + 16 * lr + 4 * (u4 ^ ((lr >> 1) & 3)));
              if (8 * it < nval) {
                const float2 o0 = __fadd2_rn(f2(v.x, v.y), f2(res[it].x, res[it].y));
                const float2 o1 = __fadd2_rn(f2(v.z, v.w), f2(res[it].z, res[it].w));
                const int64_t el = coff + 8 * it * H + col;  // element index in the stream
                // streaming store: the row is not read again in this launch
                if constexpr (ES)
                  __stcs(reinterpret_cast<uint2*>(a.e_lp + 2 * el),
                         make_uint2(pack_bf16(o0.x, o0.y), pack_bf16(o1.x, o1.y)));
                else
                  __stcs(reinterpret_cast<float4*>(outp + el), make_float4(o0.x, o0.y, o1.x, o1.y));
                if constexpr (MODE == TC_NODE_UPD) {  // the copy the edge blocks gather
                  if constexpr (F8)
                    *reinterpret_cast<uint32_t*>(a.h_lp + el) =
                        pack_e4m3x4(o0.x * a.hlp_inv, o0.y * a.hlp_inv, o1.x * a.hlp_inv,
                                    o1.y * a.hlp_inv);
                  else
                    *reinterpret_cast<uint2*>(a.h_lp + 2 * el) =
                        make_uint2(pack_bf16(o0.x, o0.y), pack_bf16(o1.x, o1.y));
                }
              }
            }
          }
        }
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

template <int MODE, bool F8, int NS, bool ES>
cudaError_t launch_tc_ns(etx_ctx* ctx, const char* name, const TcArgs& a, int64_t max_rows,
                         cudaStream_t s) {
  using C = Cfg<MODE, F8, NS>;
  static bool attr_set[8] = {false};
  if (!attr_set[ctx->device & 7]) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<MODE, F8, NS, ES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[ctx->device & 7] = true;
  }
  const int64_t tiles = (max_rows + TM - 1) / TM;
  if (tiles == 0) return cudaSuccess;
  const int grid = (int)(tiles < ctx->n_sms ? tiles : ctx->n_sms);
  launch(ctx, name, k_mlp_tc<MODE, F8, NS, ES>, grid, THREADS, C::SMEM, s, a);
  return cudaGetLastError();
}

// ring depth from the context's tuning (2 to 5 slots; capped by shared memory)
template <int MODE, bool F8, bool ES = false>
cudaError_t launch_tc(etx_ctx* ctx, const char* name, const TcArgs& a, int64_t max_rows,
                      cudaStream_t s) {
  switch (ctx->tc_stages[MODE][F8 ? 1 : 0]) {
    case 2: return launch_tc_ns<MODE, F8, 2, ES>(ctx, name, a, max_rows, s);
    case 4: return launch_tc_ns<MODE, F8, 4, ES>(ctx, name, a, max_rows, s);
    case 5: return launch_tc_ns<MODE, F8, 5, ES>(ctx, name, a, max_rows, s);
    default: return launch_tc_ns<MODE, F8, 3, ES>(ctx, name, a, max_rows, s);
  }
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
  a.h_lp = ctx->h_lp;
  a.e_lp = reinterpret_cast<uint8_t*>(ctx->e);
  a.err = ctx->d_err;
  a.in_inv = a.mid_inv = a.hlp_inv = 1.f;
  return a;
}

// e4m3 activation scale i (etx_set_fp8_scales order) of the context: 1 unless set.
float act_scale(const etx_ctx* ctx, int i) {
  return i < (int)ctx->fp8_act.size() ? ctx->fp8_act[i] : 1.f;
}

// Copy H parameters of a device weight array (inside ctx->w_dev) from the
// host copy of the repacked weights.
void host_params(const etx_ctx* ctx, const float* dev_ptr, float* out) {
  const size_t off = static_cast<size_t>(dev_ptr - ctx->w_dev);
  std::memcpy(out, ctx->w_host.data() + off, H * sizeof(float));
}

// s_in, s_mid: the block's e4m3 activation scales (powers of two; ignored for BF16)
void set_block(etx_ctx* ctx, TcArgs& a, const BlockF32& f, const BlockTC& t, bool f8, float s_in,
               float s_mid) {
  a.w1 = f8 ? t.w1f8 : t.w1;
  a.w2 = f8 ? t.w2f8 : t.w2;
  a.ws1 = f8 ? t.s1 * s_in : 1.f;
  a.ws2 = f8 ? t.s2 * s_mid : 1.f;
  a.in_inv = f8 ? 1.f / s_in : 1.f;
  a.mid_inv = f8 ? 1.f / s_mid : 1.f;
  const float* src[6] = {f.l1.b, f.g1, f.be1, f.l2.b, f.g2, f.be2};
  for (int i = 0; i < 6; ++i) host_params(ctx, src[i], a.prm[i]);
}

// es: the edge stream is stored in BF16 (BF16 edge blocks only)
template <int MODE>
cudaError_t launch_any(etx_ctx* ctx, bool f8, const char* n16, const char* n8, const TcArgs& a,
                       int64_t max_rows, cudaStream_t s, bool es = false, const char* n16s = nullptr) {
  if constexpr (MODE != TC_NODE_UPD) {
    if (es) return launch_tc<MODE, false, true>(ctx, n16s, a, max_rows, s);
  }
  return f8 ? launch_tc<MODE, true>(ctx, n8, a, max_rows, s)
            : launch_tc<MODE, false>(ctx, n16, a, max_rows, s);
}

}  // namespace

cudaError_t launch_edge_encoder_tc(etx_ctx* ctx, int64_t N, const int32_t* src, const int32_t* dst,
                                   const int32_t* n_edges_dev, bool f8, bool es, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, src, dst, n_edges_dev, nullptr);
  set_block(ctx, a, ctx->w.edge_enc, ctx->w.edge_enc_tc, f8, act_scale(ctx, 0), act_scale(ctx, 1));
  return launch_any<TC_EDGE_ENC>(ctx, f8, "gnn_edge_encoder_bf16", "gnn_edge_encoder_fp8", a,
                                 ctx->cfg.max_edges, s, es, "gnn_edge_encoder_bf16s");
}

cudaError_t launch_node_update_tc(etx_ctx* ctx, int k, int64_t N, bool f8, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, nullptr, nullptr, nullptr, nullptr);
  a.m_lp = reinterpret_cast<const uint8_t*>(ctx->m);  // written by the messages kernel
  set_block(ctx, a, ctx->w.node[k], ctx->w.node_tc[k], f8, act_scale(ctx, 2 + 4 * k),
            act_scale(ctx, 3 + 4 * k));
  // the h copy it writes feeds edge network k
  a.hlp_inv = f8 ? 1.f / act_scale(ctx, 4 + 4 * k) : 1.f;
  return launch_any<TC_NODE_UPD>(ctx, f8, "gnn_node_update_bf16", "gnn_node_update_fp8", a, N, s);
}

cudaError_t launch_edge_update_tc(etx_ctx* ctx, int k, int64_t N, const int32_t* src,
                                  const int32_t* dst, const int32_t* n_edges_dev, bool f8, bool es,
                                  cudaStream_t s) {
  TcArgs a = base_args(ctx, N, src, dst, n_edges_dev, nullptr);
  set_block(ctx, a, ctx->w.edge[k], ctx->w.edge_tc[k], f8, act_scale(ctx, 4 + 4 * k),
            act_scale(ctx, 5 + 4 * k));
  return launch_any<TC_EDGE_UPD>(ctx, f8, "gnn_edge_update_bf16", "gnn_edge_update_fp8", a,
                                 ctx->cfg.max_edges, s, es, "gnn_edge_update_bf16s");
}

cudaError_t launch_classifier_tc(etx_ctx* ctx, int64_t N, const int32_t* n_edges_dev, float* logits,
                                 bool f8, bool es, cudaStream_t s) {
  TcArgs a = base_args(ctx, N, nullptr, nullptr, n_edges_dev, logits);
  const BlockTC& t = ctx->w.cls_tc;
  const float s_in = act_scale(ctx, 4 * ctx->cfg.n_iters + 2);
  a.w1 = f8 ? t.w1f8 : t.w1;
  a.ws1 = f8 ? t.s1 * s_in : 1.f;
  a.in_inv = f8 ? 1.f / s_in : 1.f;
  a.ws2 = 1.f;
  host_params(ctx, ctx->w.cls.l1.b, a.prm[0]);
  host_params(ctx, ctx->w.cls.g1, a.prm[1]);
  host_params(ctx, ctx->w.cls.be1, a.prm[2]);
  host_params(ctx, ctx->w.cls.w2, a.prm[6]);
  a.bcls = ctx->w.cls.b2;
  return launch_any<TC_CLS>(ctx, f8, "gnn_classifier_bf16", "gnn_classifier_fp8", a,
                            ctx->cfg.max_edges, s, es, "gnn_classifier_bf16s");
}

}  // namespace etx
