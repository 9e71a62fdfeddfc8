// Internal declarations shared by the CUDA translation units of libetx.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/etx.h"

namespace etx {

// Device error word bits (the context's d_err).
enum : int {
  DERR_UNSORTED = 1,
  DERR_CAPACITY = 2,
  DERR_TIMEOUT = 4,
  DERR_RANGE = 8,
};

__device__ __forceinline__ void set_err(int* err, int bit) { atomicOr(err, bit); }

constexpr int kMaxPlanes = 64;
constexpr float kLnEps = 1e-5f;

// One Linear layer of the FP32 path: W^T stored [k_pad][n] row-major (k-major),
// zero rows for k >= k_in; bias[n].
struct LinF32 {
  const float* wt = nullptr;
  const float* b = nullptr;
  int k_in = 0, k_pad = 0, n = 0;
};

// Lin -> LN -> ReLU -> Lin -> LN -> ReLU block.
struct BlockF32 {
  LinF32 l1, l2;
  const float *g1 = nullptr, *be1 = nullptr, *g2 = nullptr, *be2 = nullptr;
};

struct ClassifierF32 {
  LinF32 l1;
  const float *g1 = nullptr, *be1 = nullptr;
  const float* w2 = nullptr;  // [H]
  const float* b2 = nullptr;  // [1]
};

// Tensor-core copies of a block's two Linear weights: BF16, W[n][k] split in
// 64-column chunks of 128 rows x 128 bytes, each laid out exactly as the
// K-major 128-byte-swizzle shared-memory operand (16 KB per chunk).
// FP8 (e4m3) images use the same layout with 128 K columns per chunk and hold
// W / s rounded to e4m3, s = amax(W) / 448 per tensor (the epilogue rescales).
struct BlockTC {
  const uint8_t* w1 = nullptr;
  const uint8_t* w2 = nullptr;
  const uint8_t* w1f8 = nullptr;
  const uint8_t* w2f8 = nullptr;
  float s1 = 1.f, s2 = 1.f;
};

struct Weights {
  const float* norm = nullptr;  // emb mu[3], sigma[3], gnn mu[3], sigma[3] (device)
  std::vector<LinF32> emb;
  BlockF32 node_enc, edge_enc;
  std::vector<BlockF32> node, edge;
  ClassifierF32 cls;
  bool has_tc = false;          // BF16 images exist (hidden == 128)
  BlockTC edge_enc_tc, cls_tc;
  std::vector<BlockTC> node_tc, edge_tc;
};

}  // namespace etx

namespace etx {
// One step of etx_set_gnn_params' device repack (from the interaction-network
// parameter vector, blob order): k_in > 0: a Linear W [n][k_in] at src to W^T
// at dst of the FP32 weights (and its BF16 operand image at byte img of w_tc
// when img >= 0); k_in <= 0: n values copied from src to dst.
struct RepackJob {
  int64_t src, dst, img;
  int32_t k_in, n;
};

struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
}  // namespace etx

struct etx_ctx {
  etx_config cfg{};
  int device = 0;
  int n_sms = 0;
  std::string err;
  bool weights_loaded = false;

  int* d_err = nullptr;
  int32_t* n_edges = nullptr;    // device: edge count of the current call, clamped
  double* small = nullptr;       // device: 8 doubles of reduction scratch (loss sums, counts)

  // weights
  float* w_dev = nullptr;   // repacked FP32 weights
  size_t w_dev_floats = 0;
  std::vector<float> w_host;  // host copy of w_dev (kernel-parameter copies of small vectors)
  float* blob_dev = nullptr;  // raw blob copy (float32) for the backward pass
  uint8_t* w_tc = nullptr;    // BF16 operand images of the interaction network
  // device-side weight updates (etx_set_gnn_params)
  etx::RepackJob* repack_dev = nullptr;
  int n_repack = 0;
  int64_t n_theta = 0;             // interaction-network parameters
  float* w_host_pinned = nullptr;  // asynchronous host copy of w_dev
  cudaEvent_t w_host_ev = nullptr;
  bool w_host_pending = false;     // w_host must be refreshed from w_host_pinned
  bool f8_stale = false;           // e4m3 images predate the last device update
  etx::Weights w;

  // graph scratch
  int32_t* plane_off = nullptr;  // [max_events * (n_planes + 1)]
  int32_t* hit_cnt = nullptr;    // [max_hits + 1]
  int32_t* scan_tmp = nullptr;   // block partials
  size_t scan_tmp_ints = 0;

  // interaction-network scratch
  int32_t* out_off = nullptr;    // [max_hits + 1]
  int32_t* in_off = nullptr;     // [max_hits + 1]
  int32_t* in_cnt = nullptr;     // [max_hits + 1]
  int32_t* perm_in = nullptr;    // [max_edges]
  float* h = nullptr;            // [max_hits * H]
  float* m = nullptr;            // [max_hits * 2H]
  float* e = nullptr;            // [max_edges * H]

  // tensor-core paths: h rounded to the operand type (BF16 rows of 256 bytes,
  // or e4m3 rows of 128 bytes) for the edge blocks' gathers
  uint8_t* h_lp = nullptr;       // [max_hits * 256 bytes]

  // components
  int32_t* parent = nullptr;     // [max_hits]
  // the last forward stored the edge stream in BF16 (dtype ETX_BF16_EDGE_STORE):
  // ctx->e then holds BF16 rows, which the FP32 readers of e must not use
  bool e_bf16 = false;

  // triplet classifiers (etx_load_triplet_weights): articulations, elbows
  float* w_trip = nullptr;
  etx::ClassifierF32 trip_art, trip_elb;
  bool trip_loaded = false;

  // training (cfg.train): checkpoints of the last forward and backward scratch
  float* h_ck = nullptr;         // [(L+1) * max_hits * H]: h^k
  float* e_ck = nullptr;         // [(L+1) * max_edges * H]: e^k
  float* de = nullptr;           // [max_edges * H]
  float* dh = nullptr;           // [max_hits * H]
  float *bw_X = nullptr, *bw_DX = nullptr;          // [rows * 3H]
  float *bw_R1 = nullptr, *bw_DA1 = nullptr, *bw_DY1 = nullptr, *bw_DY1N1 = nullptr;  // [rows * H]
  float *bw_DA2 = nullptr, *bw_DY2 = nullptr, *bw_DY2N2 = nullptr;
  // per-split partial gradients, added in a fixed order (deterministic reductions):
  // n_sms x H x 3H floats
  float* bw_part = nullptr;
  // tensor-core block backward (H = 128): n1 rows, rstd1, TF32 weight images and
  // the job list that refreshes them (filled at the first backward)
  etx::RepackJob* embed_repack_dev = nullptr;  // the embedding's repack plan (etx_set_embed_params)
  int n_embed_repack = 0;
  float* bw_N1 = nullptr;
  float* bw_Xlo = nullptr;   // low parts of the block inputs [R][3H] and of R1 [R][H]
  float* bw_R1lo = nullptr;
  float* bw_cs_part = nullptr;  // 2 x [4 n_sms][3H]: fused column-sum partials
  float* bw_rstd1 = nullptr;
  float* bw_img = nullptr;
  void* bw_img_jobs = nullptr;
  std::vector<unsigned char> bw_img_jobs_host;
  int bw_img_n_jobs = 0;
  bool bw_img_ready = false;
  // per-block partial sums of the loss, red_part_n floats (every context)
  float* red_part = nullptr;
  int64_t red_part_n = 0;
  bool fwd_saved = false;        // a training forward ran since the weights were loaded
  const float *fwd_x = nullptr, *fwd_y = nullptr, *fwd_z = nullptr;
  const int32_t *fwd_src = nullptr, *fwd_dst = nullptr;
  int64_t fwd_n_hits = 0;
  int64_t gnn_blob_offset = 0;   // first interaction-network value in the weight blob

  // e4m3 activation scales (etx_set_fp8_scales; powers of two, empty = all 1)
  std::vector<float> fp8_act;

  // launch configurations picked by etx_autotune (defaults: measured on the
  // 500-event workload)
  int knn_split = 1;                         // blocks per (event, plane) in the k-NN
  int knn_stage = 4096;                      // floats of staged k-NN candidates per block
  int tc_stages[4][2] = {{3, 2}, {3, 2}, {3, 2}, {3, 2}};  // ring slots [mode][e4m3]

  // launch accounting and optional per-launch CUDA-event timing
  int64_t launches = 0;
  bool prof_on = false;
  std::vector<etx::ProfRec> prof;
  size_t prof_used = 0;
};

namespace etx {

// ---- launch helpers implemented in the .cu files --------------------------
// scan.cu: exclusive scan of n int32 (n host-known); out[n] receives the total.
cudaError_t exclusive_scan(etx_ctx* ctx, const int32_t* in, int32_t* out, int64_t n,
                           cudaStream_t s);
// the same with caller-provided block-total scratch of tmp_ints >= scan_tmp_ints(n) ints
cudaError_t exclusive_scan_with(etx_ctx* ctx, const int32_t* in, int32_t* out, int64_t n,
                                int32_t* tmp, size_t tmp_ints, cudaStream_t s);
size_t scan_tmp_ints(int64_t n);

// embed.cu
cudaError_t launch_embed(etx_ctx* ctx, const float* x, const float* y, const float* z,
                         int64_t n, float* emb, cudaStream_t s);

// graph.cu
cudaError_t launch_build_graph(etx_ctx* ctx, const float* emb, const int8_t* plane,
                               const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                               float radius, int32_t k_max, int32_t* src, int32_t* dst,
                               int64_t edge_capacity, int32_t* edge_offsets, cudaStream_t s);

// gnn_f32.cu
// dtype ETX_BF16 / ETX_FP8E4M3: tensor-core MLP blocks (hidden == 128), ETX_F32: SIMT
cudaError_t launch_gnn_forward(etx_ctx* ctx, const float* x, const float* y, const float* z,
                               int64_t n_hits, const int32_t* src, const int32_t* dst,
                               const int32_t* n_edges_dev, float* logits, etx_dtype dtype,
                               cudaStream_t s);
cudaError_t launch_edge_index(etx_ctx* ctx, int64_t n_hits, const int32_t* src,
                              const int32_t* dst, const int32_t* n_edges_dev, cudaStream_t s);
// CSR of the element ids 0 .. *n_dev - 1 grouped by keys[id] (ids whose key is
// outside [0, n_keys) are left out), each segment in ascending id (so the
// order is fixed): off [n_keys + 1], perm [n_cap]; cnt [n_keys + 1] scratch.
// names: the three launches' profile names (count, fill, sort).
cudaError_t launch_key_index(etx_ctx* ctx, const int32_t* keys, const int32_t* n_dev, int64_t n_cap,
                             int64_t n_keys, int32_t* cnt, int32_t* off, int32_t* perm,
                             const char* const names[3], cudaStream_t s);
// messages of edge features e (uses the context's edge index structures)
cudaError_t launch_messages(etx_ctx* ctx, const float* e, float* m, int64_t n_hits, cudaStream_t s);

// gnn_bwd.cu
cudaError_t launch_checkpoint(etx_ctx* ctx, float* dst, const float* src, int64_t rows_host,
                              const int32_t* rows_dev, int64_t rows_cap, cudaStream_t s);
cudaError_t launch_gnn_backward(etx_ctx* ctx, const float* dlogits, float* dparams, cudaStream_t s);
cudaError_t launch_weighted_bce(etx_ctx* ctx, const float* logits, const float* targets,
                                const int32_t* n_edges_dev, float pos_weight, float* loss,
                                float* dlogits, cudaStream_t s);
cudaError_t launch_focal_loss(etx_ctx* ctx, const float* logits, const float* targets,
                              const int32_t* n_edges_dev, float alpha, float gamma, float* loss,
                              float* dlogits, cudaStream_t s);
cudaError_t launch_adam(etx_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n,
                        float lr, float b1, float b2, float eps, int64_t step, cudaStream_t s);

// gnn_bwd_tc.cu: P[z][128][N] = partial dW = sum over the rows of split z of A[r]^T B[r]
// (TF32 tensor cores, FP32 accumulation); R_cap bounds the rows, splits CTAs
bool wgrad_tc_supported(int M, int N);

// gnn_bwd_gemm.cu: the reverse pass of one hidden-width block (H = 128) on the
// tensor cores (TF32).  Block kinds as in the FP32 block backward.
enum BwdBlockMode { BWD_NODE_ENC = 0, BWD_EDGE_ENC = 1, BWD_NODE_UPD = 2, BWD_EDGE_UPD = 3, BWD_CLS = 4 };
struct BlockBwdTc {
  int64_t n_nodes;
  int64_t R_host;              // rows (hits) when R_dev is NULL
  const int32_t* R_dev;        // rows (edges) on the device; capacity cfg.max_edges
  const float *hg, *ein, *m;   // gathered node rows, edge rows, messages [N][2H]
  const int32_t *src, *dst;
  const float *W1n, *W1t, *W2n, *W2t;  // TF32 images: W1 [H][K], W1^T [K][H], W2, W2^T
  const float *W1n_lo, *W2n_lo;        // low parts of W1, W2 (split products)
  const float *b1, *g1, *be1, *b2, *g2, *be2;
  const float* G;              // incoming gradient rows [R][H]
  float *X, *R1, *N1, *rstd1, *DA1, *DY1, *DY1N1, *DA2, *DY2, *DY2N2, *DX;
  float *X_lo, *R1_lo;                 // low parts of X and R1 (split products)
  // column-sum partials of layer 1 and layer 2 ([parts][3H]: b, g, be gradients)
  float *cs1, *cs2;
};
// partials per column-sum array of a block with rows_cap rows
int block_bwd_tc_colsum_parts(const etx_ctx* ctx, int64_t rows_cap);
bool block_bwd_tc_supported(const etx_ctx* ctx);
cudaError_t launch_block_bwd_tc(etx_ctx* ctx, int mode, const BlockBwdTc& p, cudaStream_t s);
// TF32 images of the weights: a job list (src, dst, n) held on the device
size_t tf32_image_job_bytes();
void tf32_image_job(void* jobs_host, int i, const float* src, float* dst, int64_t n, bool lo);
cudaError_t launch_tf32_images(etx_ctx* ctx, const void* jobs_dev, int n_jobs, int64_t max_n,
                               cudaStream_t s);
cudaError_t launch_wgrad_tc(etx_ctx* ctx, const float* A, int lda, const float* B, int ldb, int N,
                            int64_t R_host, const int32_t* R_dev, int64_t R_cap, int splits,
                            float* P, cudaStream_t s);

// gnn_tc.cu (hidden == 128 only; the edge encoder gathers ctx->h_lp, the copy
// of h that the node encoder writes in the operand type)
// f8: e4m3 operands (kind::f8f6f4), else BF16 (kind::f16)
// es: the edge stream is stored in BF16 (dtype ETX_BF16_EDGE_STORE)
cudaError_t launch_edge_encoder_tc(etx_ctx* ctx, int64_t N, const int32_t* src, const int32_t* dst,
                                   const int32_t* n_edges_dev, bool f8, bool es, cudaStream_t s);
cudaError_t launch_node_update_tc(etx_ctx* ctx, int k, int64_t N, bool f8, cudaStream_t s);
cudaError_t launch_edge_update_tc(etx_ctx* ctx, int k, int64_t N, const int32_t* src,
                                  const int32_t* dst, const int32_t* n_edges_dev, bool f8, bool es,
                                  cudaStream_t s);
cudaError_t launch_classifier_tc(etx_ctx* ctx, int64_t N, const int32_t* n_edges_dev, float* logits,
                                 bool f8, bool es, cudaStream_t s);

// graph.cu: hit checks and ctx->plane_off (first hit of each plane, per event)
cudaError_t launch_plane_bins(etx_ctx* ctx, const int8_t* plane, const int32_t* hit_offsets,
                              int32_t n_events, int64_t n_hits, cudaStream_t s);
// gnn_f32.cu: ctx->out_off, the src-CSR of edges sorted by src (checks order and range)
cudaError_t launch_out_offsets(etx_ctx* ctx, int64_t N, const int32_t* src, const int32_t* dst,
                               const int32_t* n_edges_dev, cudaStream_t s);

// triplets.cu: triplets of the kept edges (Sec. 5.3) and the classifier weights
size_t triplets_workspace(int64_t n_hits);
cudaError_t launch_build_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                  const float* logits, float thr, int64_t n_hits, void* workspace,
                                  int64_t capacity, int32_t* first, int32_t* second, int8_t* kind,
                                  int32_t* counts, cudaStream_t s);
cudaError_t load_triplet_weights(etx_ctx* ctx, const float* blob);
// triplets.cu: tracks on the purified edge graph (Sec. 5.4)
size_t tracks_workspace(int64_t n_hits, int64_t e_cap, int64_t trip_cap);
cudaError_t launch_tracks_from_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                        const float* logits, float thr, int64_t n_hits,
                                        const int32_t* first, const int32_t* second,
                                        const float* tlogits, float tthr, const int32_t* counts,
                                        int64_t trip_cap, int32_t min_hits, void* workspace,
                                        int32_t* track_offsets, int32_t* track_hits,
                                        int64_t track_capacity, int64_t hit_capacity,
                                        int32_t* n_out, cudaStream_t s);
int64_t triplet_weights_size(int H);
// gnn_f32.cu: a triplet classifier over rows [*row_lo_dev (or 0), *row_hi_dev) of first/second
cudaError_t launch_triplet_classifier(etx_ctx* ctx, const int32_t* first, const int32_t* second,
                                      const int32_t* row_lo_dev, const int32_t* row_hi_dev,
                                      int64_t capacity, const ClassifierF32& cls, float* logits,
                                      cudaStream_t s);

// embed_train.cu: the embedding's training set and hinge loss (Sec. 5.1, Eq. 2-3)
size_t embedding_pairs_workspace(int32_t n_events, int64_t n_hits, int32_t k_max);
cudaError_t launch_embedding_pairs(etx_ctx* ctx, const float* emb, const int8_t* plane,
                                   const int32_t* particle_id, const int32_t* hit_offsets,
                                   int32_t n_events, int64_t n_hits, float radius, int32_t k_max,
                                   const uint32_t* rand, int32_t min_hits, void* workspace,
                                   int32_t* pq, int32_t* pa, uint8_t* pg, int64_t capacity,
                                   int32_t* n_pairs, cudaStream_t s);
// scratch: 3 doubles of device memory
size_t hinge_loss_workspace(int64_t n_hits, int64_t pair_capacity);
cudaError_t launch_hinge_loss(etx_ctx* ctx, const float* emb, int64_t n_hits, const int32_t* pq,
                              const int32_t* pa, const uint8_t* pg, const int32_t* n_pairs,
                              int64_t pair_capacity, float margin, float w_genuine, float* loss,
                              float* d_emb, void* workspace, cudaStream_t s);
// embed.cu / gnn_bwd.cu: embedding forward with saved activations, and its reverse pass
size_t embed_backward_workspace(const etx_config& cfg, int64_t n_hits);
int64_t embed_param_count(const etx_config& cfg);
cudaError_t launch_embed_save(etx_ctx* ctx, const float* x, const float* y, const float* z,
                              int64_t n, float* emb, float* saved, cudaStream_t s);
cudaError_t launch_embed_backward(etx_ctx* ctx, int64_t n, const float* saved, const float* d_emb,
                                  float* dz_a, float* dz_b, float* d_params, cudaStream_t s);

// metrics.cu: Table 1 counts; workspace = per-event tallies then six int32 arrays of n_hits
size_t track_metrics_workspace(int32_t n_events, int64_t n_hits);
cudaError_t launch_track_metrics(etx_ctx* ctx, const int32_t* labels, const int32_t* particle_id,
                                 const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                                 int32_t min_hits, int32_t num, int32_t den, void* workspace,
                                 int64_t* counts, double* values, cudaStream_t s);

// cc.cu
// the paper's plane-sweep labels (needs ctx->plane_off and ctx->out_off)
cudaError_t launch_plane_sweep(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                               const float* logits, float thr, const int32_t* hit_offsets,
                               int32_t n_events, int64_t n_hits, int32_t* labels, cudaStream_t s);
cudaError_t launch_edges_to_tracks(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                   const float* logits, float thr, const int32_t* n_edges_dev,
                                   const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                                   int32_t min_hits, int32_t* labels, int32_t* n_tracks,
                                   cudaStream_t s);

int grid_for(const etx_ctx* ctx, const void* kernel, int threads, size_t smem, int64_t max_blocks);

void prof_begin(etx_ctx* ctx, const char* name, cudaStream_t s);
void prof_end(etx_ctx* ctx, cudaStream_t s);

// Launch one of this library's kernels: counted, and timed with a CUDA event
// pair on the launching stream when profiling is on.
template <typename... KArgs, typename... Args>
inline void launch(etx_ctx* ctx, const char* name, void (*kernel)(KArgs...), dim3 grid,
                   dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  prof_begin(ctx, name, s);
  kernel<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
  prof_end(ctx, s);
  ++ctx->launches;
}

}  // namespace etx
