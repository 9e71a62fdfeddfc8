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
// MMA descriptors expect), and the row-wise work between them runs in that
// launch's epilogue, one row (one TMEM lane) per thread:
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

// SPLIT: each stage holds A hi, A lo, B hi, B lo
template <int NB, bool SPLIT = false>
struct BgCfg {
  static constexpr int NH = NB == 384 ? 192 : NB;  // N per MMA instruction (at most 256)
  static constexpr int NHALF = NB / NH;
  static constexpr int A_BYTES = BG_TM * 128;
  static constexpr int B_BYTES = NB * 128;
  static constexpr int STAGE = (SPLIT ? 2 : 1) * (A_BYTES + B_BYTES);
  static constexpr int OFF_BAR = BG_STAGES * STAGE;
  static constexpr int SMEM = OFF_BAR + 8 * 16 + 16 + 1024;
  static constexpr uint32_t TMEM_COLS = NB <= 128 ? 128 : (NB <= 256 ? 256 : 512);
  static constexpr uint32_t IDESC = idesc_tf32_f32<BG_TM, NH>();
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(NB % 128 == 0, "B is copied in boxes of 128 rows");
};

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

__device__ __forceinline__ float tf32r(float f) { return __uint_as_float(to_tf32(f)); }

__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

template <int NB, int EPI, bool SPLIT>
__global__ void __launch_bounds__(BG_THREADS, 1) k_bwd_gemm(const __grid_constant__ BgArgs a) {
  using C = BgCfg<NB, SPLIT>;
  static_assert(EPI == EPI_STORE || NB == BG_H, "row-wise epilogues take H columns");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);  // FULL[3], EMPTY[3], DONE
  uint64_t* full = bars;
  uint64_t* empty = bars + BG_STAGES;
  uint64_t* done = bars + 2 * BG_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 8 * 16);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + C::OFF_BAR + 8 * 16 + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int64_t R = a.R_dev ? (int64_t)*a.R_dev : a.R_host;
  const int64_t row0 = (int64_t)blockIdx.x * BG_TM;
  if (row0 >= R) return;  // the whole CTA: no barrier or TMEM use yet
  const int nk = a.K / BG_KC;

  if (tid == 0) {
    for (int s = 0; s < BG_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
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
    // ---- TMA producer: stage s holds A[row0.., 32 c..] and B[.., 32 c..] -------
    if (lane == 0) {
      int issued = 0;
      for (int c = 0; c < nk; ++c) {
        const int st = c % BG_STAGES;
        const uint32_t round = (uint32_t)(c / BG_STAGES);
        if (round > 0 && !bg_wait(&empty[st], (round - 1) & 1, a.err, abort)) break;
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
        for (int c = issued > BG_STAGES ? issued - BG_STAGES : 0; c < issued; ++c)
          for (int i = 0; i < (1 << 20) && !mbar_try_wait(&full[c % BG_STAGES], (c / BG_STAGES) & 1); ++i) {
          }
      }
    }
  } else if (warp == 5) {
    // ---- MMA issuer ------------------------------------------------------------
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nk && ok; ++c) {
        const int st = c % BG_STAGES;
        ok = bg_wait(&full[st], (uint32_t)(c / BG_STAGES) & 1, a.err, abort);
        if (!ok) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + st * C::STAGE);
        const uint32_t sb = sa + C::A_BYTES;
        const uint32_t sal = sb + C::B_BYTES, sbl = sal + C::A_BYTES;  // SPLIT: low parts
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int h = 0; h < C::NHALF; ++h) {
            const uint32_t d = tmem + h * C::NH, bo = h * C::NH * 128 + 32 * k;
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
      mma_commit(done);  // also after an abort: the epilogue's wait then ends
    }
  } else {
    // ---- epilogue: warp w owns TMEM lanes (tile rows) 32 w .. 32 w + 31 ----------
    const bool ok = bg_wait(done, 0, a.err, abort);
    tc_fence_after();
    const int r = 32 * warp + lane;
    const int64_t gr = row0 + r;
    const bool valid = ok && gr < R;
    const uint32_t tl = tmem + (static_cast<uint32_t>(32 * warp) << 16);
    if constexpr (EPI == EPI_STORE) {
      for (int c0 = 0; c0 < NB; c0 += 32) {
        float v[32];
        tmem_ld32_wait(tl + c0, v);
        if (valid) {
          float* o = a.o0 + gr * a.ldo + c0;
#pragma unroll
          for (int q = 0; q < 8; ++q) st4(o + 4 * q, v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
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
          float v[32];
          ldc(c0, v);
          if (valid) {
            float* o_r1 = a.o0 + gr * BG_H + c0;
            float* o_n1 = a.o1 + gr * BG_H + c0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float n[4], y[4], lo[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                n[u] = (v[j + u] - mean) * rstd;
                const float r1 = fmaxf(fmaf(n[u], __ldg(a.g + c0 + j + u), __ldg(a.be + c0 + j + u)), 0.f);
                y[u] = tf32r(r1);
                lo[u] = tf32r(r1 - y[u]);
              }
              st4(o_r1 + j, y[0], y[1], y[2], y[3]);
              st4(o_n1 + j, n[0], n[1], n[2], n[3]);
              if (a.o3) st4(a.o3 + gr * BG_H + c0 + j, lo[0], lo[1], lo[2], lo[3]);
            }
          }
        }
      } else {  // EPI_LN2
        // pass 1: d = G where y2 = n2 g2 + be2 > 0; DY2, DY2 n2; the means of
        // dn = d g2 and of dn n2
        float m1 = 0.f, m2 = 0.f;
        const float* grow = a.G + (valid ? gr : 0) * BG_H;
#pragma unroll 1
        for (int c0 = 0; c0 < BG_H; c0 += 32) {
          float v[32];
          ldc(c0, v);
          if (valid) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 go = *reinterpret_cast<const float4*>(grow + c0 + j);
              const float gv[4] = {go.x, go.y, go.z, go.w};
              float d[4], n[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float gg = __ldg(a.g + c0 + j + u);
                n[u] = (v[j + u] - mean) * rstd;
                d[u] = fmaf(n[u], gg, __ldg(a.be + c0 + j + u)) > 0.f ? gv[u] : 0.f;
                const float dn = d[u] * gg;
                m1 += dn;
                m2 += dn * n[u];
              }
              st4(a.o0 + gr * BG_H + c0 + j, d[0], d[1], d[2], d[3]);
              st4(a.o1 + gr * BG_H + c0 + j, d[0] * n[0], d[1] * n[1], d[2] * n[2], d[3] * n[3]);
            }
          }
        }
        m1 *= 1.0f / BG_H;
        m2 *= 1.0f / BG_H;
        // pass 2: DA2 = rstd2 (dn - m1 - n2 m2), the incoming rows read again
#pragma unroll 1
        for (int c0 = 0; c0 < BG_H; c0 += 32) {
          float v[32];
          ldc(c0, v);
          if (valid) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 go = *reinterpret_cast<const float4*>(grow + c0 + j);
              const float gv[4] = {go.x, go.y, go.z, go.w};
              float o[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float gg = __ldg(a.g + c0 + j + u);
                const float n = (v[j + u] - mean) * rstd;
                const float d = fmaf(n, gg, __ldg(a.be + c0 + j + u)) > 0.f ? gv[u] : 0.f;
                o[u] = tf32r(rstd * (d * gg - m1 - n * m2));
              }
              st4(a.o2 + gr * BG_H + c0 + j, o[0], o[1], o[2], o[3]);
            }
          }
        }
      }
    } else {  // EPI_LN1B: acc = dr1
      const float* n1row = a.N1 + (valid ? gr : 0) * BG_H;
      const float rstd = valid ? a.rs_in[gr] : 0.f;
      float m1 = 0.f, m2 = 0.f;
      // pass 1: d = dr1 where n1 g1 + be1 > 0; DY1, DY1 n1; the means
      for (int c0 = 0; c0 < BG_H; c0 += 32) {
        float v[32];
        tmem_ld32_wait(tl + c0, v);
        if (valid) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 n4 = *reinterpret_cast<const float4*>(n1row + c0 + j);
            const float nv[4] = {n4.x, n4.y, n4.z, n4.w};
            float d[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float gg = __ldg(a.g + c0 + j + u);
              d[u] = fmaf(nv[u], gg, __ldg(a.be + c0 + j + u)) > 0.f ? v[j + u] : 0.f;
              const float dn = d[u] * gg;
              m1 += dn;
              m2 += dn * nv[u];
            }
            st4(a.o0 + gr * BG_H + c0 + j, d[0], d[1], d[2], d[3]);
            st4(a.o1 + gr * BG_H + c0 + j, d[0] * nv[0], d[1] * nv[1], d[2] * nv[2], d[3] * nv[3]);
          }
        }
      }
      m1 *= 1.0f / BG_H;
      m2 *= 1.0f / BG_H;
      // pass 2: DA1 = rstd1 (dn - m1 - n1 m2)
      for (int c0 = 0; c0 < BG_H; c0 += 32) {
        float v[32];
        tmem_ld32_wait(tl + c0, v);
        if (valid) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 n4 = *reinterpret_cast<const float4*>(n1row + c0 + j);
            const float nv[4] = {n4.x, n4.y, n4.z, n4.w};
            float o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float gg = __ldg(a.g + c0 + j + u);
              const float d = fmaf(nv[u], gg, __ldg(a.be + c0 + j + u)) > 0.f ? v[j + u] : 0.f;
              o[u] = tf32r(rstd * (d * gg - m1 - nv[u] * m2));
            }
            st4(a.o2 + gr * BG_H + c0 + j, o[0], o[1], o[2], o[3]);
          }
        }
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
  using C = BgCfg<NB, SPLIT>;
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
  launch(ctx, kBgName[EPI], k_bwd_gemm<NB, EPI, SPLIT>, (unsigned)tiles, BG_THREADS, C::SMEM, s, a);
  return cudaGetLastError();
}

}  // namespace

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
  if ((e = launch_bg<128, EPI_LN2, true>(ctx, a, p.R1, Rcap, p.W2n, s, p.R1_lo, p.W2n_lo)) != cudaSuccess)
    return e;
  // 4: GEMM 3 + LN1 backward
  a.g = p.g1; a.be = p.be1;
  a.N1 = p.N1; a.rs_in = p.rstd1;
  a.o0 = p.DY1; a.o1 = p.DY1N1; a.o2 = p.DA1;
  if ((e = launch_bg<128, EPI_LN1B>(ctx, a, p.DA2, Rcap, p.W2t, s)) != cudaSuccess) return e;
  // 5: GEMM 4, the input gradient
  a.o0 = p.DX; a.ldo = K;
  return K == 2 * H ? launch_bg<256, EPI_STORE>(ctx, a, p.DA1, Rcap, p.W1t, s)
                    : launch_bg<384, EPI_STORE>(ctx, a, p.DA1, Rcap, p.W1t, s);
}

}  // namespace etx
