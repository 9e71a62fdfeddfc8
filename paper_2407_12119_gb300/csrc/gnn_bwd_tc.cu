// Weight gradients of the interaction network on the 5th-generation tensor
// cores: dW = sum over rows r of A[r]^T B[r] (A = the layer's pre-activation
// gradients [R][128], B = its inputs [R][N]), with TF32 operands (FP32 values
// rounded to 10 mantissa bits) and FP32 accumulation in tensor memory.
//
// The reduction runs over rows (edges or hits), so each operand is needed with
// the row index along K: producer warps load 4 x 4 blocks of the FP32 rows
// (coalesced float4 loads), round them to TF32, transpose them in registers
// and store them into the K-major 128-byte-swizzle operand layout (a 128-byte
// smem row = 32 K values = 32 input rows of one output feature).  One thread
// issues the MMAs (M = 128, N up to 256 per instruction, K = 8 per 32-byte
// step), the accumulator stays in tensor memory until the CTA's rows are done,
// and the CTA writes its 128 x N partial to P[split]; the splits are added in
// a fixed order afterwards (no atomics, the same bits every run).
#include "sm100.cuh"

namespace etx {
namespace {

using namespace sm100;

constexpr int WG_M = 128;               // output features (H)
constexpr int WG_KR = 32;               // input rows per chunk (128 bytes of TF32)
constexpr int WG_PROD_WARPS = 8;
constexpr int WG_THREADS = 32 * (WG_PROD_WARPS + 1);  // + one MMA warp
constexpr int WG_STAGES = 3;

template <int NB>
struct WgCfg {
  static constexpr int NH = NB == 384 ? 192 : (NB == 256 ? 256 : 128);  // N per MMA
  static constexpr int NHALF = NB / NH;
  static constexpr int A_BYTES = WG_M * 128;
  static constexpr int B_BYTES = NB * 128;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int OFF_BAR = WG_STAGES * STAGE;
  static constexpr int SMEM = OFF_BAR + 8 * 16 + 16 + 1024;
  static constexpr uint32_t TMEM_COLS = NB <= 128 ? 128 : (NB <= 256 ? 256 : 512);
  static constexpr uint32_t IDESC = idesc_tf32_f32<WG_M, NH>();
  static_assert(SMEM <= 232448, "shared memory");
};

struct WgArgs {
  const float* A;  // [R][lda], the M = 128 gradient columns
  int lda;
  const float* B;  // [R][ldb], the N input columns
  int ldb;
  int64_t R_host;
  const int32_t* R_dev;  // row count on the device (edges), or NULL: R_host
  int64_t rows_per_split;
  float* P;        // [gridDim.x][128][NB] partials
  int* err;
};

__device__ __forceinline__ void wg_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool wg_wait(uint64_t* bar, uint32_t parity, int* err, volatile int* abort) {
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

// One 4-row x 4-column block of src (rows r0 + 4 rq .. +3 below R, columns c0 ..
// c0 + 3) rounded to TF32 and stored transposed: smem row (c0 + i) gets the
// four rows' values of column c0 + i as its 16-byte unit rq (swizzled).
__device__ __forceinline__ void wg_block(const float* __restrict__ src, int ld, int64_t r0, int rq,
                                         int c0, int64_t R, uint8_t* tile) {
  float4 v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t r = r0 + 4 * rq + j;
    v[j] = r < R ? __ldg(reinterpret_cast<const float4*>(src + r * ld + c0))
                 : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const float* f = reinterpret_cast<const float*>(v);  // f[4 j + i] = row j, column c0 + i
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = c0 + i;
    const uint4 u = make_uint4(to_tf32(f[i]), to_tf32(f[4 + i]), to_tf32(f[8 + i]), to_tf32(f[12 + i]));
    *reinterpret_cast<uint4*>(tile + m * 128 + ((rq ^ (m & 7)) << 4)) = u;
  }
}

template <int NB>
__global__ void __launch_bounds__(WG_THREADS, 1) k_wgrad_tc(const __grid_constant__ WgArgs a) {
  using C = WgCfg<NB>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);  // FULL[3], EMPTY[3], DONE
  uint64_t* full = bars;
  uint64_t* empty = bars + WG_STAGES;
  uint64_t* done = bars + 2 * WG_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + 8 * 16);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + C::OFF_BAR + 8 * 16 + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int64_t R = a.R_dev ? (int64_t)*a.R_dev : a.R_host;
  const int64_t lo = (int64_t)blockIdx.x * a.rows_per_split;
  const int64_t hi = lo + a.rows_per_split < R ? lo + a.rows_per_split : R;
  const int64_t n_chunks = hi > lo ? (hi - lo + WG_KR - 1) / WG_KR : 0;
  float* Pz = a.P + (int64_t)blockIdx.x * WG_M * NB;
  if (n_chunks == 0) {  // no rows: a zero partial
    for (int i = tid; i < WG_M * NB; i += WG_THREADS) Pz[i] = 0.f;
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < WG_STAGES; ++s) {
      mbar_init(&full[s], WG_PROD_WARPS);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == WG_PROD_WARPS) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < WG_PROD_WARPS) {
    // ---- producers: chunk c (rows lo + 32 c ..) into stage c % 3 ----------------
    // thread t: row quad rq = t % 8, column quads cq = t / 8 + 32 k
    const int rq = tid & 7, cq0 = tid >> 3;
    for (int64_t c = 0; c < n_chunks; ++c) {
      const int st = (int)(c % WG_STAGES);
      const uint32_t round = (uint32_t)(c / WG_STAGES);
      if (round > 0 && !wg_wait(&empty[st], (round - 1) & 1, a.err, abort)) break;
      uint8_t* ta = smem + st * C::STAGE;
      uint8_t* tb = ta + C::A_BYTES;
      const int64_t r0 = lo + c * WG_KR;
      const int64_t rend = hi;
      wg_block(a.A, a.lda, r0, rq, 4 * cq0, rend, ta);            // 32 column quads of A
#pragma unroll
      for (int k = 0; k < NB / 128; ++k) wg_block(a.B, a.ldb, r0, rq, 4 * (cq0 + 32 * k), rend, tb);
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) wg_arrive(&full[st]);
    }
  } else if (lane == 0) {
    // ---- MMA issuer ------------------------------------------------------------------
    for (int64_t c = 0; c < n_chunks; ++c) {
      const int st = (int)(c % WG_STAGES);
      if (!wg_wait(&full[st], (uint32_t)(c / WG_STAGES) & 1, a.err, abort)) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + st * C::STAGE);
      const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int h = 0; h < C::NHALF; ++h)
          mma_tf32(tmem + h * C::NH, sdesc_k_sw128(sa + 32 * k),
                   sdesc_k_sw128(sb + h * C::NH * 128 + 32 * k), C::IDESC,
                   (c > 0 || k > 0) ? 1u : 0u);
      mma_commit(&empty[st]);
    }
    mma_commit(done);
  }
  // ---- epilogue: warps 0-3 read their TMEM lanes (one output feature each) ------------
  if (warp < 4) {
    const bool ok = wg_wait(done, 0, a.err, abort);
    tc_fence_after();
    const int m = 32 * warp + lane;
    const uint32_t lane_off = static_cast<uint32_t>(32 * warp) << 16;
    for (int col = 0; col < NB; col += 32) {
      float v[32];
      tmem_ld32_wait(tmem + lane_off + col, v);
      float4* dst = reinterpret_cast<float4*>(Pz + (int64_t)m * NB + col);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        dst[q] = ok ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3])
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == WG_PROD_WARPS) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <int NB>
cudaError_t launch_wgrad(etx_ctx* ctx, const WgArgs& a, int splits, cudaStream_t s) {
  using C = WgCfg<NB>;
  static bool attr_set[8] = {false};
  if (!attr_set[ctx->device & 7]) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[ctx->device & 7] = true;
  }
  launch(ctx, "gnn_weight_grad_tc", k_wgrad_tc<NB>, splits, WG_THREADS, C::SMEM, s, a);
  return cudaGetLastError();
}

}  // namespace

bool wgrad_tc_supported(int M, int N) { return M == WG_M && (N == 128 || N == 256 || N == 384); }

cudaError_t launch_wgrad_tc(etx_ctx* ctx, const float* A, int lda, const float* B, int ldb, int N,
                            int64_t R_host, const int32_t* R_dev, int64_t R_cap, int splits,
                            float* P, cudaStream_t s) {
  if (splits < 1) return cudaErrorInvalidValue;
  WgArgs a{};
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.R_host = R_host;
  a.R_dev = R_dev;
  // rows per split: a multiple of the chunk, covering the row capacity
  a.rows_per_split = ((R_cap + splits - 1) / splits + WG_KR - 1) / WG_KR * WG_KR;
  a.P = P;
  a.err = ctx->d_err;
  switch (N) {
    case 128: return launch_wgrad<128>(ctx, a, splits, s);
    case 256: return launch_wgrad<256>(ctx, a, splits, s);
    case 384: return launch_wgrad<384>(ctx, a, splits, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace etx
