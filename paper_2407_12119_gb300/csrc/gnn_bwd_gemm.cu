// Reverse pass of the interaction network's hidden-width MLP blocks (edge
// encoder, node and edge updates; H = 128) on the 5th-generation tensor cores,
// with TF32 operands (FP32 values rounded to 10 mantissa bits) and FP32
// accumulation in tensor memory.
//
// A block out = in + ReLU(LN2(W2 ReLU(LN1(W1 X + b1)) + b2)) (Sec. 5.2) needs
// four matrix products per row in its reverse pass: the two of the forward,
// recomputed from the checkpointed block input X, and the two input gradients.
// Each is one launch of k_bwd_gemm (C = A B^T over 128-row tiles, A and B
// K-major, both brought in by TMA tensor copies with the 128-byte swizzle the
// MMA descriptors expect; persistent, one CTA per SM, two accumulators in
// tensor memory where they fit so one tile's epilogue overlaps the next tile's
// products), and the row-wise work between them runs in that launch's
// epilogue, one row (one TMEM lane) per thread, its global reads and writes
// made coalesced through a per-warp shared-memory transpose:
//   1  X W1^T   -> LN1 forward: R1 = ReLU(n1 g1 + be1), n1, rstd1
//   2  R1 W2^T  -> LN2 forward and backward against the incoming gradient G:
//                  DY2, DY2 n2, DA2
//   3  DA2 W2   -> ReLU mask and LN1 backward: DY1, DY1 n1, DA1
//   4  DA1 W1   -> DX, the gradient of the block input
// The per-row factors are the ones the FP32 block backward stores, so the
// weight gradients, column sums and scatters that follow are shared with it.
// Every GEMM operand is rounded to TF32 (cvt.rna) where it is written (X, R1,
// DA2, DA1 and the weight images), so the tensor core multiplies exact TF32
// values; LayerNorm statistics and the factors stay FP32.  The two recomputed
// forward products decide ReLU masks and LayerNorm inputs, and one TF32
// rounding there moves the gradients by up to ~2e-2 (measured against the
// FP64 reverse pass); they run split (a = hi + lo, both TF32; A B^T =
// Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T, three MMAs), which is within FP32 rounding
// of the exact products.  The two gradient products stay single TF32 (~5e-4).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "sm100.cuh"

namespace etx {
namespace {

using namespace sm100;

constexpr int BG_H = 128;                 // hidden width (the tile's TMEM lanes)
constexpr int BG_TM = 128;                // rows per tile
constexpr int BG_KC = 32;                 // K columns per stage (128 bytes of TF32)
constexpr int BG_STAGES = 3;
constexpr int BG_THREADS = 192;           // warps 0-3 epilogue, 4 TMA, 5 MMA
constexpr float kBgLnEps = 1e-5f;

enum BgEpi { EPI_LN1F = 0, EPI_LN2 = 1, EPI_LN1B = 2, EPI_STORE = 3 };

// SPLIT: each stage holds A hi, A lo, B hi, B lo.  ACC accumulators in tensor
// memory (two where they fit, so the epilogue of one tile overlaps the products
// of the next); a 4 KB staging buffer per epilogue warp (32 rows x 32 columns)
// turns its row-per-thread values into coalesced 128-byte row segments.
// ROWS: the epilogue reads a [R][H] array row by row (G or n1): each warp's 32
// rows of a tile come into a 16 KB block by asynchronous copies, all in flight
// at once, issued before the accumulator wait.  These epilogues (LN2, LN1B) also
// sum the columns of the three factors they write (the layer's bias, gain and
// shift gradients), per warp in shared memory (3 x H floats).
template <int NB, bool SPLIT = false, bool ROWS = false>
struct BgCfg {
  static constexpr int NST = SPLIT && ROWS ? 2 : BG_STAGES;  // ring stages
  static constexpr int NH = NB == 384 ? 192 : NB;  // N per MMA instruction (at most 256)
  static constexpr int NHALF = NB / NH;
  static constexpr int ACC = 2 * NB <= 512 ? 2 : 1;
  static constexpr int A_BYTES = BG_TM * 128;
  static constexpr int B_BYTES = NB * 128;
  static constexpr int STAGE = (SPLIT ? 2 : 1) * (A_BYTES + B_BYTES);
  static constexpr int OFF_STG = NST * STAGE;
  static constexpr int OFF_ROWS = OFF_STG + 4 * 4096;
  static constexpr int OFF_CS = OFF_ROWS + (ROWS ? 4 * 16384 : 0);
  static constexpr int OFF_BAR = OFF_CS + (ROWS ? 4 * 3 * BG_H * 4 : 0);
  static constexpr int SMEM = OFF_BAR + 16 * 8 + 16 + 1024;
  static constexpr uint32_t TMEM_COLS = ACC * NB <= 128 ? 128 : (ACC * NB <= 256 ? 256 : 512);
  static constexpr uint32_t IDESC = idesc_tf32_f32<BG_TM, NH>();
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(NB % 128 == 0, "B is copied in boxes of 128 rows");
};

// Staging of a warp's 32 rows x 32 columns: row r's 16-byte unit q sits at
// unit q ^ (r % 8) of its 128-byte line, so both the row-per-lane side and the
// coalesced side (8 lanes per row, 4 rows per instruction) are conflict-free.
__device__ __forceinline__ void stage_put(float* buf, int lane, const float (&v)[32]) {
  __syncwarp();  // earlier reads of the buffer are done
#pragma unroll
  for (int q = 0; q < 8; ++q)
    *reinterpret_cast<float4*>(buf + lane * 32 + 4 * (q ^ (lane & 7))) =
        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  __syncwarp();
}

// Store the staged block to rows g + r * ld (r < nvalid), coalesced.
__device__ __forceinline__ void stage_flush(const float* buf, int lane, float* g, int64_t ld,
                                            int nvalid) {
  const int u = lane & 7;
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int r = 4 * it + (lane >> 3);
    const float4 x = *reinterpret_cast<const float4*>(buf + r * 32 + 4 * (u ^ (r & 7)));
    if (r < nvalid) *reinterpret_cast<float4*>(g + r * ld + 4 * u) = x;
  }
}

struct BgArgs {
  CUtensorMap ta;        // A [rows][K] FP32 (TF32 values), boxes of 32 columns x 128 rows
  CUtensorMap tb;        // B [NB][K] FP32 (TF32 values), same boxes
  CUtensorMap ta2, tb2;  // SPLIT: the low parts of A and B
  int K;                 // reduction length, a multiple of 32
  int64_t R_host;        // rows (R_dev == NULL)
  const int32_t* R_dev;  // row count on the device (edges)
  const float *b, *g, *be;  // the layer's bias, gain and shift [H]
  const float* G;        // EPI_LN2: incoming gradient rows [R][H]
  const float* N1;       // EPI_LN1B: n1 rows [R][H]
  const float* rs_in;    // EPI_LN1B: rstd1 [R]
  float* rs_out;         // EPI_LN1F: rstd1 [R]
  float *o0, *o1, *o2;   // outputs (see the modes)
  float* o3;             // EPI_LN1F: the low part of R1 (R1 - tf32(R1), rounded), or NULL
  int ldo;               // EPI_STORE: row stride of o0
  // EPI_LN2 / EPI_LN1B: column sums of o2, o1, o0 (a layer's b, g, be gradients)
  // per (CTA, epilogue warp): [gridDim.x * 4][3 H], added in a fixed order later
  float* cs_part;
  int* err;
};

__device__ __forceinline__ bool bg_wait(uint64_t* bar, uint32_t parity, int* err, volatile int* abort) {
  uint64_t t0 = 0;
  for (uint32_t i = 0; i < (kWaitCap << 4); ++i) {
    if (mbar_try_wait_sleep(bar, parity, 128)) return true;
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

__device__ __forceinline__ void bg_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ float tf32r(float f) { return __uint_as_float(to_tf32(f)); }

// Lane j adds column j of the staged block's first nvalid rows to *acc (its
// own shared-memory word: no other lane touches it).
__device__ __forceinline__ void stage_colsum(const float* buf, int lane, int nvalid, float* acc) {
  float t = 0.f;
#pragma unroll 8
  for (int r = 0; r < 32; ++r)
    if (r < nvalid) t += buf[r * 32 + 4 * ((lane >> 2) ^ (r & 7)) + (lane & 3)];
  *acc += t;
}

// The warp's 32 rows g + r * H (r < nvalid; zeros after) into its row block:
// row r's 16-byte unit u at unit u ^ (r % 8), one row per copy instruction.
__device__ __forceinline__ void rows_fetch(float* blk, int lane, const float* g, int nvalid) {
#pragma unroll 4
  for (int r = 0; r < 32; ++r) {
    float* d = blk + r * BG_H + 4 * (lane ^ (r & 7));
    if (r < nvalid)
      cp_async16(d, g + (int64_t)r * BG_H + 4 * lane);
    else
      *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__device__ __forceinline__ void rows_ready() {
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();
}

// Columns c0 .. c0 + 31 of the lane's own row from the row block.
__device__ __forceinline__ void rows_get(const float* blk, int lane, int c0, float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 x = *reinterpret_cast<const float4*>(blk + lane * BG_H + 4 * (((c0 >> 2) + q) ^ (lane & 7)));
    v[4 * q] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
}

template <int NB, int EPI, bool SPLIT>
__global__ void __launch_bounds__(BG_THREADS, 1) k_bwd_gemm(const __grid_constant__ BgArgs a) {
  using C = BgCfg<NB, SPLIT, EPI == EPI_LN2 || EPI == EPI_LN1B>;
  static_assert(EPI == EPI_STORE || NB == BG_H, "row-wise epilogues take H columns");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // FULL[3], EMPTY[3], TFULL[2], TEMPTY[2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + C::NST;
  uint64_t* tfull = bars + 2 * C::NST;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 16 * 8);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + C::OFF_BAR + 16 * 8 + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // persistent: tiles blockIdx.x, blockIdx.x + gridDim.x, ... below R
  const int64_t R = a.R_dev ? (int64_t)*a.R_dev : a.R_host;
  const int64_t n_tiles = (R + BG_TM - 1) / BG_TM;
  if ((int64_t)blockIdx.x >= n_tiles) {  // the whole CTA: no barrier or TMEM use yet
    if (a.cs_part)  // an empty partial
      for (int i = tid; i < 4 * 3 * BG_H; i += BG_THREADS) a.cs_part[(int64_t)blockIdx.x * 4 * 3 * BG_H + i] = 0.f;
    return;
  }
  const int64_t my_tiles = (n_tiles - 1 - blockIdx.x) / gridDim.x + 1;
  const int nk = a.K / BG_KC;

  if (tid == 0) {
    for (int s = 0; s < C::NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);  // every epilogue warp has read the accumulator
    }
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    // ---- TMA producer: chunk q (tile q / nk, K columns 32 (q % nk) ..) into stage q % 3
    if (lane == 0) {
      int64_t issued = 0;
      const int64_t total = my_tiles * nk;
      for (int64_t q = 0; q < total; ++q) {
        const int st = (int)(q % C::NST);
        const uint32_t round = (uint32_t)(q / C::NST);
        if (round > 0 && !bg_wait(&empty[st], (round - 1) & 1, a.err, abort)) break;
        const int64_t row0 = (blockIdx.x + (q / nk) * gridDim.x) * BG_TM;
        const int c = (int)(q % nk);
        uint8_t* sa = smem + st * C::STAGE;
        mbar_arrive_expect_tx(&full[st], C::STAGE);
        tma_load_2d(sa, &a.ta, BG_KC * c, (int)row0, &full[st]);
#pragma unroll
        for (int b = 0; b < NB / 128; ++b)
          tma_load_2d(sa + C::A_BYTES + b * 128 * 128, &a.tb, BG_KC * c, 128 * b, &full[st]);
        if constexpr (SPLIT) {
          uint8_t* sl = sa + C::A_BYTES + C::B_BYTES;  // A lo, then B lo
          tma_load_2d(sl, &a.ta2, BG_KC * c, (int)row0, &full[st]);
#pragma unroll
          for (int b = 0; b < NB / 128; ++b)
            tma_load_2d(sl + C::A_BYTES + b * 128 * 128, &a.tb2, BG_KC * c, 128 * b, &full[st]);
        }
        ++issued;
      }
      if (*abort) {
        // let the copies still in flight land before the CTA exits (bounded)
        for (int64_t q = issued > C::NST ? issued - C::NST : 0; q < issued; ++q)
          for (int i = 0; i < (1 << 20) &&
                          !mbar_try_wait(&full[q % C::NST], (uint32_t)(q / C::NST) & 1);
               ++i) {
          }
      }
    }
  } else if (warp == 5) {
    // ---- MMA issuer: tile i into accumulator i % ACC --------------------------------
    if (lane == 0) {
      bool ok = true;
      int64_t q = 0;
      for (int64_t i = 0; i < my_tiles && ok; ++i) {
        const int b = (int)(i % C::ACC);
        const uint32_t u = (uint32_t)(i / C::ACC);
        if (u > 0 && !(ok = bg_wait(&tempty[b], (u - 1) & 1, a.err, abort))) break;
        tc_fence_after();
        const uint32_t d0 = tmem + b * NB;
        for (int c = 0; c < nk; ++c, ++q) {
          const int st = (int)(q % C::NST);
          if (!(ok = bg_wait(&full[st], (uint32_t)(q / C::NST) & 1, a.err, abort))) break;
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + st * C::STAGE);
          const uint32_t sb = sa + C::A_BYTES;
          const uint32_t sal = sb + C::B_BYTES, sbl = sal + C::A_BYTES;  // SPLIT: low parts
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int h = 0; h < C::NHALF; ++h) {
              const uint32_t d = d0 + h * C::NH, bo = h * C::NH * 128 + 32 * k;
              if constexpr (SPLIT) {  // the small cross terms first
                mma_tf32(d, sdesc_k_sw128(sal + 32 * k), sdesc_k_sw128(sb + bo), C::IDESC,
                         (c > 0 || k > 0) ? 1u : 0u);
                mma_tf32(d, sdesc_k_sw128(sa + 32 * k), sdesc_k_sw128(sbl + bo), C::IDESC, 1u);
                mma_tf32(d, sdesc_k_sw128(sa + 32 * k), sdesc_k_sw128(sb + bo), C::IDESC, 1u);
              } else {
                mma_tf32(d, sdesc_k_sw128(sa + 32 * k), sdesc_k_sw128(sb + bo), C::IDESC,
                         (c > 0 || k > 0) ? 1u : 0u);
              }
            }
          mma_commit(&empty[st]);
        }
        if (ok) mma_commit(&tfull[b]);
      }
    }
  } else {
    // ---- epilogue: warp w owns TMEM lanes (tile rows) 32 w .. 32 w + 31 ----------
    float* buf = reinterpret_cast<float*>(smem + C::OFF_STG + 4096 * warp);
    float* blk = reinterpret_cast<float*>(smem + C::OFF_ROWS + 16384 * warp);  // ROWS only
    float* csm = reinterpret_cast<float*>(smem + C::OFF_CS + 3 * BG_H * 4 * warp);  // ROWS only
    constexpr bool CS = EPI == EPI_LN2 || EPI == EPI_LN1B;
    if constexpr (CS)
      for (int j = lane; j < 3 * BG_H; j += 32) csm[j] = 0.f;
    const uint32_t lane_off = static_cast<uint32_t>(32 * warp) << 16;
    for (int64_t i = 0; i < my_tiles; ++i) {
      const int b = (int)(i % C::ACC);
      const int64_t r0w = (blockIdx.x + i * gridDim.x) * BG_TM + 32 * warp;  // the warp's first row
      const int nvalid = (int)(R - r0w < 32 ? (R - r0w > 0 ? R - r0w : 0) : 32);
      if constexpr (EPI == EPI_LN2) rows_fetch(blk, lane, a.G + r0w * BG_H, nvalid);
      if constexpr (EPI == EPI_LN1B) rows_fetch(blk, lane, a.N1 + r0w * BG_H, nvalid);
      if (!bg_wait(&tfull[b], (uint32_t)(i / C::ACC) & 1, a.err, abort)) break;
      tc_fence_after();
      if constexpr (EPI == EPI_LN2 || EPI == EPI_LN1B) rows_ready();
      const uint32_t tl = tmem + b * NB + lane_off;
      const int64_t gr = r0w + lane;
      const bool valid = lane < nvalid;
      if constexpr (EPI == EPI_STORE) {
        for (int c0 = 0; c0 < NB; c0 += 32) {
          float v[32];
          tmem_ld32_wait(tl + c0, v);
          stage_put(buf, lane, v);
          stage_flush(buf, lane, a.o0 + r0w * a.ldo + c0, a.ldo, nvalid);
        }
      } else if constexpr (EPI == EPI_LN1F || EPI == EPI_LN2) {
        // v = acc + b, read from TMEM 32 columns at a time (again for every pass,
        // which keeps the row out of registers); LayerNorm statistics in two passes
        auto ldc = [&](int c0, float (&v)[32]) {
          tmem_ld32_wait(tl + c0, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += __ldg(a.b + c0 + j);
        };
        float s = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < BG_H; c0 += 32) {
          float v[32];
          ldc(c0, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) s += v[j];
        }
        const float mean = s * (1.0f / BG_H);
        float q = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < BG_H; c0 += 32) {
          float v[32];
          ldc(c0, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float d = v[j] - mean;
            q += d * d;
          }
        }
        const float rstd = 1.0f / sqrtf(q * (1.0f / BG_H) + kBgLnEps);
        if constexpr (EPI == EPI_LN1F) {
          if (valid) a.rs_out[gr] = rstd;
#pragma unroll 1
          for (int c0 = 0; c0 < BG_H; c0 += 32) {
            float v[32], y[32];
            ldc(c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              v[j] = (v[j] - mean) * rstd;  // n1
              y[j] = fmaxf(fmaf(v[j], __ldg(a.g + c0 + j), __ldg(a.be + c0 + j)), 0.f);  // r1
            }
            stage_put(buf, lane, v);
            stage_flush(buf, lane, a.o1 + r0w * BG_H + c0, BG_H, nvalid);
            if (a.o3) {
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] = tf32r(y[j] - tf32r(y[j]));  // low part
              stage_put(buf, lane, v);
              stage_flush(buf, lane, a.o3 + r0w * BG_H + c0, BG_H, nvalid);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) y[j] = tf32r(y[j]);
            stage_put(buf, lane, y);
            stage_flush(buf, lane, a.o0 + r0w * BG_H + c0, BG_H, nvalid);
          }
        } else {  // EPI_LN2
          // pass 1: d = G where y2 = n2 g2 + be2 > 0; DY2, DY2 n2; the means of
          // dn = d g2 and of dn n2
          float m1 = 0.f, m2 = 0.f;
#pragma unroll 1
          for (int c0 = 0; c0 < BG_H; c0 += 32) {
            float v[32], gv[32];
            ldc(c0, v);
            rows_get(blk, lane, c0, gv);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float gg = __ldg(a.g + c0 + j);
              const float n = (v[j] - mean) * rstd;
              const float d = fmaf(n, gg, __ldg(a.be + c0 + j)) > 0.f ? gv[j] : 0.f;
              const float dn = d * gg;
              m1 += dn;
              m2 += dn * n;
              gv[j] = d;
              v[j] = d * n;
            }
            stage_put(buf, lane, gv);
            stage_colsum(buf, lane, nvalid, csm + 2 * BG_H + c0 + lane);
            stage_flush(buf, lane, a.o0 + r0w * BG_H + c0, BG_H, nvalid);
            stage_put(buf, lane, v);
            stage_colsum(buf, lane, nvalid, csm + BG_H + c0 + lane);
            stage_flush(buf, lane, a.o1 + r0w * BG_H + c0, BG_H, nvalid);
          }
          m1 *= 1.0f / BG_H;
          m2 *= 1.0f / BG_H;
          // pass 2: DA2 = rstd2 (dn - m1 - n2 m2), the incoming rows read again
#pragma unroll 1
          for (int c0 = 0; c0 < BG_H; c0 += 32) {
            float v[32], gv[32];
            ldc(c0, v);
            rows_get(blk, lane, c0, gv);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float gg = __ldg(a.g + c0 + j);
              const float n = (v[j] - mean) * rstd;
              const float d = fmaf(n, gg, __ldg(a.be + c0 + j)) > 0.f ? gv[j] : 0.f;
              v[j] = tf32r(rstd * (d * gg - m1 - n * m2));
            }
            stage_put(buf, lane, v);
            stage_colsum(buf, lane, nvalid, csm + c0 + lane);
            stage_flush(buf, lane, a.o2 + r0w * BG_H + c0, BG_H, nvalid);
          }
        }
      } else {  // EPI_LN1B: acc = dr1
        const float rstd = valid ? a.rs_in[gr] : 0.f;
        float m1 = 0.f, m2 = 0.f;
        // pass 1: d = dr1 where n1 g1 + be1 > 0; DY1, DY1 n1; the means
#pragma unroll 1
        for (int c0 = 0; c0 < BG_H; c0 += 32) {
          float v[32], nv[32];
          tmem_ld32_wait(tl + c0, v);
          rows_get(blk, lane, c0, nv);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float gg = __ldg(a.g + c0 + j);
            const float d = fmaf(nv[j], gg, __ldg(a.be + c0 + j)) > 0.f ? v[j] : 0.f;
            const float dn = d * gg;
            m1 += dn;
            m2 += dn * nv[j];
            v[j] = d;
            nv[j] = d * nv[j];
          }
          stage_put(buf, lane, v);
          stage_colsum(buf, lane, nvalid, csm + 2 * BG_H + c0 + lane);
          stage_flush(buf, lane, a.o0 + r0w * BG_H + c0, BG_H, nvalid);
          stage_put(buf, lane, nv);
          stage_colsum(buf, lane, nvalid, csm + BG_H + c0 + lane);
          stage_flush(buf, lane, a.o1 + r0w * BG_H + c0, BG_H, nvalid);
        }
        m1 *= 1.0f / BG_H;
        m2 *= 1.0f / BG_H;
        // pass 2: DA1 = rstd1 (dn - m1 - n1 m2)
#pragma unroll 1
        for (int c0 = 0; c0 < BG_H; c0 += 32) {
          float v[32], nv[32];
          tmem_ld32_wait(tl + c0, v);
          rows_get(blk, lane, c0, nv);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float gg = __ldg(a.g + c0 + j);
            const float d = fmaf(nv[j], gg, __ldg(a.be + c0 + j)) > 0.f ? v[j] : 0.f;
            v[j] = tf32r(rstd * (d * gg - m1 - nv[j] * m2));
          }
          stage_put(buf, lane, v);
          stage_colsum(buf, lane, nvalid, csm + c0 + lane);
          stage_flush(buf, lane, a.o2 + r0w * BG_H + c0, BG_H, nvalid);
        }
      }
      // the accumulator (and the row block) is read: the MMA may reuse it for
      // tile i + ACC, the next fetch may overwrite the block
      tc_fence_before();
      __syncwarp();
      if (lane == 0) bg_arrive(&tempty[b]);
    }
    if constexpr (CS) {
      if (a.cs_part) {
        __syncwarp();
        float* P = a.cs_part + ((int64_t)blockIdx.x * 4 + warp) * 3 * BG_H;
        for (int j = lane; j < 3 * BG_H; j += 32) P[j] = csm[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// Weight images for the reverse pass: `n` floats of `src` rounded to TF32, for
// a list of (src, dst, n) jobs (blockIdx.y = job).
struct ImgJob {
  const float* src;
  float* dst;
  int64_t n;
  int lo;  // 1: the low part v - tf32(v), rounded to TF32
};

__global__ void k_tf32_images(const ImgJob* __restrict__ jobs) {
  const ImgJob j = jobs[blockIdx.y];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < j.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = j.src[i], hi = tf32r(v);
    j.dst[i] = j.lo ? tf32r(v - hi) : hi;
  }
}

// The block input X [R][K] of an edge encoder, node update or edge update,
// rounded to TF32: [h_src, h_dst] (K = 2H), [h, m] (K = 3H, m = [m_out, m_in])
// or [e, h_src, h_dst] (K = 3H); one float4 per thread and step.
template <int MODE>
__global__ void k_gather_x(const float* __restrict__ hg, const float* __restrict__ ein,
                           const float* __restrict__ m, const int32_t* __restrict__ src,
                           const int32_t* __restrict__ dst, int nn, int64_t R_host,
                           const int32_t* __restrict__ R_dev, float* __restrict__ X,
                           float* __restrict__ Xlo) {
  constexpr int H = BG_H;
  constexpr int K = MODE == BWD_EDGE_ENC ? 2 * H : 3 * H;
  constexpr int Q = K / 4;  // float4 pieces of a row
  const int64_t R = R_dev ? (int64_t)*R_dev : R_host;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R * Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / Q;
    const int k = 4 * (int)(i - row * Q);
    const float* p;
    if constexpr (MODE == BWD_NODE_UPD) {
      p = k < H ? hg + row * H + k : m + row * 2 * H + (k - H);
    } else {
      const int s = min(max(src[row], 0), max(nn - 1, 0));
      const int d = min(max(dst[row], 0), max(nn - 1, 0));
      if constexpr (MODE == BWD_EDGE_ENC)
        p = k < H ? hg + (int64_t)s * H + k : hg + (int64_t)d * H + (k - H);
      else
        p = k < H ? ein + row * H + k
                  : (k < 2 * H ? hg + (int64_t)s * H + (k - H) : hg + (int64_t)d * H + (k - 2 * H));
    }
    const float4 f = *reinterpret_cast<const float4*>(p);
    const float4 hi = make_float4(tf32r(f.x), tf32r(f.y), tf32r(f.z), tf32r(f.w));
    *reinterpret_cast<float4*>(X + row * K + k) = hi;
    *reinterpret_cast<float4*>(Xlo + row * K + k) =
        make_float4(tf32r(f.x - hi.x), tf32r(f.y - hi.y), tf32r(f.z - hi.z), tf32r(f.w - hi.w));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

// Tensor map of a row-major FP32 matrix [rows][cols] (cols a multiple of 32,
// base 16-byte aligned): boxes of 32 columns x 128 rows with the 128-byte
// swizzle, rows past the end read as zeros.
bool encode_rows(CUtensorMap* m, const float* base, int64_t rows, int cols) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode || rows < 1 || cols % BG_KC != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)BG_KC, (cuuint32_t)BG_TM};
  const cuuint32_t elem[2] = {1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
                elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

const char* kBgName[4] = {"gnn_block_backward_tc_ln1", "gnn_block_backward_tc_ln2",
                          "gnn_block_backward_tc_ln1b", "gnn_block_backward_tc_dx"};

// A_lo / B_lo non-NULL: the split (three-product) form
template <int NB, int EPI, bool SPLIT = false>
cudaError_t launch_bg(etx_ctx* ctx, BgArgs& a, const float* A, int64_t Rcap, const float* B,
                      cudaStream_t s, const float* A_lo = nullptr, const float* B_lo = nullptr) {
  using C = BgCfg<NB, SPLIT, EPI == EPI_LN2 || EPI == EPI_LN1B>;
  if (!encode_rows(&a.ta, A, Rcap, a.K) || !encode_rows(&a.tb, B, NB, a.K))
    return cudaErrorInvalidValue;
  if (SPLIT && (!encode_rows(&a.ta2, A_lo, Rcap, a.K) || !encode_rows(&a.tb2, B_lo, NB, a.K)))
    return cudaErrorInvalidValue;
  static bool attr_set[8] = {false};
  if (!attr_set[ctx->device & 7]) {
    cudaError_t e = cudaFuncSetAttribute(k_bwd_gemm<NB, EPI, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[ctx->device & 7] = true;
  }
  const int64_t tiles = (Rcap + BG_TM - 1) / BG_TM;
  if (tiles == 0) return cudaSuccess;
  // persistent: one CTA per SM (shared memory holds one), tiles strided over them
  const int grid = (int)(tiles < ctx->n_sms ? tiles : ctx->n_sms);
  launch(ctx, kBgName[EPI], k_bwd_gemm<NB, EPI, SPLIT>, grid, BG_THREADS, C::SMEM, s, a);
  return cudaGetLastError();
}

}  // namespace

int block_bwd_tc_colsum_parts(const etx_ctx* ctx, int64_t rows_cap) {
  const int64_t tiles = (rows_cap + BG_TM - 1) / BG_TM;
  return 4 * (int)(tiles < ctx->n_sms ? tiles : ctx->n_sms);
}

bool block_bwd_tc_supported(const etx_ctx* ctx) {
  return ctx->cfg.hidden == BG_H && tensor_map_encoder() != nullptr;
}

cudaError_t launch_tf32_images(etx_ctx* ctx, const void* jobs_dev, int n_jobs, int64_t max_n,
                               cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  const int gx = (int)std::min<int64_t>((max_n + 255) / 256, 64);
  launch(ctx, "gnn_tf32_images", k_tf32_images, dim3(gx, n_jobs), 256, 0, s,
         reinterpret_cast<const ImgJob*>(jobs_dev));
  return cudaGetLastError();
}

size_t tf32_image_job_bytes() { return sizeof(ImgJob); }

void tf32_image_job(void* jobs_host, int i, const float* src, float* dst, int64_t n, bool lo) {
  reinterpret_cast<ImgJob*>(jobs_host)[i] = ImgJob{src, dst, n, lo ? 1 : 0};
}

cudaError_t launch_block_bwd_tc(etx_ctx* ctx, int mode, const BlockBwdTc& p, cudaStream_t s) {
  constexpr int H = BG_H;
  const int K = mode == BWD_EDGE_ENC ? 2 * H : 3 * H;
  const int64_t Rcap = p.R_dev ? ctx->cfg.max_edges : p.R_host;
  if (Rcap == 0) return cudaSuccess;
  // 1: the block input, rounded to TF32
  {
    const int64_t work = Rcap * (K / 4);
    const int g = (int)std::min<int64_t>((work + 255) / 256, (int64_t)ctx->n_sms * 16);
    if (mode == BWD_EDGE_ENC)
      launch(ctx, "gnn_gather_x", k_gather_x<BWD_EDGE_ENC>, g, 256, 0, s, p.hg, p.ein, p.m, p.src, p.dst,
             (int)p.n_nodes, p.R_host, p.R_dev, p.X, p.X_lo);
    else if (mode == BWD_NODE_UPD)
      launch(ctx, "gnn_gather_x", k_gather_x<BWD_NODE_UPD>, g, 256, 0, s, p.hg, p.ein, p.m, p.src, p.dst,
             (int)p.n_nodes, p.R_host, p.R_dev, p.X, p.X_lo);
    else
      launch(ctx, "gnn_gather_x", k_gather_x<BWD_EDGE_UPD>, g, 256, 0, s, p.hg, p.ein, p.m, p.src, p.dst,
             (int)p.n_nodes, p.R_host, p.R_dev, p.X, p.X_lo);
  }
  BgArgs a{};
  a.R_host = p.R_host;
  a.R_dev = p.R_dev;
  a.err = ctx->d_err;
  cudaError_t e;
  // 2: GEMM 1 + LN1 forward
  a.K = K;
  a.b = p.b1; a.g = p.g1; a.be = p.be1;
  a.o0 = p.R1; a.o1 = p.N1; a.rs_out = p.rstd1; a.o3 = p.R1_lo;
  if ((e = launch_bg<128, EPI_LN1F, true>(ctx, a, p.X, Rcap, p.W1n, s, p.X_lo, p.W1n_lo)) != cudaSuccess)
    return e;
  // 3: GEMM 2 + LN2 forward and backward
  a.K = H;
  a.b = p.b2; a.g = p.g2; a.be = p.be2;
  a.G = p.G;
  a.o0 = p.DY2; a.o1 = p.DY2N2; a.o2 = p.DA2; a.o3 = nullptr;
  a.cs_part = p.cs2;
  if ((e = launch_bg<128, EPI_LN2, true>(ctx, a, p.R1, Rcap, p.W2n, s, p.R1_lo, p.W2n_lo)) != cudaSuccess)
    return e;
  // 4: GEMM 3 + LN1 backward
  a.g = p.g1; a.be = p.be1;
  a.N1 = p.N1; a.rs_in = p.rstd1;
  a.o0 = p.DY1; a.o1 = p.DY1N1; a.o2 = p.DA1;
  a.cs_part = p.cs1;
  if ((e = launch_bg<128, EPI_LN1B>(ctx, a, p.DA2, Rcap, p.W2t, s)) != cudaSuccess) return e;
  // 5: GEMM 4, the input gradient
  a.o0 = p.DX; a.ldo = K;
  a.cs_part = nullptr;
  return K == 2 * H ? launch_bg<256, EPI_STORE>(ctx, a, p.DA1, Rcap, p.W1t, s)
                    : launch_bg<384, EPI_STORE>(ctx, a, p.DA1, Rcap, p.W1t, s);
}

}  // namespace etx
