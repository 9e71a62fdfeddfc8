// C ABI of libetx: context lifetime, weight repacking, argument checks and
// the launch sequence of each pipeline step.  See include/etx.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <iterator>
#include <new>

#include <cuda_bf16.h>

#include "etx_internal.cuh"

namespace etx {
cudaError_t knn_set_smem_attr();

int grid_for(const etx_ctx* ctx, const void* kernel, int threads, size_t smem, int64_t max_blocks) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
    per_sm = 1;
  if (per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)per_sm * ctx->n_sms;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return (int)g;
}

void prof_begin(etx_ctx* ctx, const char* name, cudaStream_t s) {
  if (!ctx->prof_on) return;
  if (ctx->prof_used == ctx->prof.size()) {
    ProfRec r{name, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
    ctx->prof.push_back(r);
  }
  ProfRec& r = ctx->prof[ctx->prof_used];
  r.name = name;
  cudaEventRecord(r.a, s);
}

void prof_end(etx_ctx* ctx, cudaStream_t s) {
  if (!ctx->prof_on || ctx->prof_used == ctx->prof.size()) return;
  cudaEventRecord(ctx->prof[ctx->prof_used].b, s);
  ++ctx->prof_used;
}

namespace {

__global__ void k_clamp_edges(const int32_t* __restrict__ edge_offsets, int32_t n_events,
                              int64_t cap, int32_t* __restrict__ n_edges, int* err) {
  int E = edge_offsets[n_events];
  if (E < 0) {
    set_err(err, DERR_RANGE);
    E = 0;
  }
  if (E > cap) {
    set_err(err, DERR_CAPACITY);
    E = (int)cap;
  }
  *n_edges = E;
}

bool valid_width(int w) { return w == 16 || w == 32 || w == 64 || w == 128; }

etx_status fail(etx_ctx* ctx, etx_status st, const char* msg) {
  if (ctx) ctx->err = msg;
  return st;
}

etx_status cuda_fail(etx_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) {
    ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return ETX_ERR_CUDA;
}

const char* config_problem(const etx_config* c) {
  if (!c) return "config is NULL";
  if (c->emb_depth < 2 || c->emb_depth > ETX_MAX_EMB_LAYERS)
    return "emb_depth must be in [2, 8]";
  if (c->emb_widths[0] != 3) return "emb_widths[0] must be 3 (r, phi, z)";
  for (int l = 1; l < c->emb_depth; ++l)
    if (c->emb_widths[l] != c->emb_widths[1]) return "embedding hidden widths must be equal";
  if (!valid_width(c->emb_widths[1])) return "embedding hidden width must be 16, 32, 64 or 128";
  const int D = c->emb_widths[c->emb_depth];
  if (D < 1 || D > 32) return "embedding dimension D must be in [1, 32]";
  if (!valid_width(c->hidden)) return "hidden must be 16, 32, 64 or 128";
  if (c->n_iters < 0 || c->n_iters > 64) return "n_iters must be in [0, 64]";
  if (c->n_planes < 2 || c->n_planes > kMaxPlanes) return "n_planes must be in [2, 64]";
  if (c->max_events < 1) return "max_events must be >= 1";
  if (c->max_hits < 1 || c->max_hits >= (int64_t)1 << 31) return "max_hits must be in [1, 2^31)";
  if (c->max_edges < 1 || c->max_edges >= (int64_t)1 << 31) return "max_edges must be in [1, 2^31)";
  if (c->uf_iter_cap < 0) return "uf_iter_cap must be >= 0 (0 = default caps)";
  return nullptr;
}

// Round to the nearest BF16, ties to even (NaN stays NaN).
uint16_t f32_to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return static_cast<uint16_t>((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}

// Append the tensor-core image of W[n_out][k] (n_out == 128, k % 64 == 0): for
// each 64-column chunk, 128 rows of 128 bytes with the 16-byte unit u of row n
// stored at unit position u ^ (n % 8) -- the K-major 128-byte-swizzle layout.
void append_bf16_image(const float* W, int n_out, int k, std::vector<uint8_t>& img) {
  const size_t at = img.size();
  img.resize(at + (size_t)n_out * k * 2);
  for (int c = 0; c < k / 64; ++c)
    for (int n = 0; n < n_out; ++n)
      for (int u = 0; u < 8; ++u)
        for (int j = 0; j < 8; ++j) {
          const uint16_t b = f32_to_bf16(W[(size_t)n * k + 64 * c + 8 * u + j]);
          const size_t off = at + (size_t)c * n_out * 128 + (size_t)n * 128 + ((u ^ (n & 7)) * 16) + 2 * j;
          img[off] = static_cast<uint8_t>(b & 0xff);
          img[off + 1] = static_cast<uint8_t>(b >> 8);
        }
}

// e4m3: 1 sign bit, 4 exponent bits (bias 7), 3 mantissa bits, no infinities,
// largest finite value 448.  Round to nearest, ties to even; magnitudes that
// round above 448 saturate to 448.
uint8_t f32_to_e4m3(float f) {
  const uint8_t sign = std::signbit(f) ? 0x80 : 0x00;
  if (std::isnan(f)) return 0x7F;
  const float a = std::fabs(f);
  if (a == 0.f) return sign;
  int e = 0;
  (void)std::frexp(a, &e);                 // a in [2^(e-1), 2^e)
  const int ex = std::max(e - 1, -6);      // below 2^-6 the spacing stays 2^-9
  const float step = std::ldexp(1.0f, ex - 3);
  const float r = std::nearbyint(a / step) * step;
  if (r >= 448.f) return sign | 0x7E;
  if (r < std::ldexp(1.0f, -6)) return sign | static_cast<uint8_t>(r / std::ldexp(1.0f, -9));
  int e2 = 0;
  const float m2 = std::frexp(r, &e2);     // r = m2 2^e2, m2 in [0.5, 1)
  const int E = e2 - 1 + 7;
  const int M = static_cast<int>((m2 * 2.f - 1.f) * 8.f);
  return sign | static_cast<uint8_t>((E << 3) | M);
}

// Per-tensor scale amax / 448 (1 for an all-zero tensor).
float e4m3_scale(const float* W, size_t n) {
  float m = 0.f;
  for (size_t i = 0; i < n; ++i) m = std::max(m, std::fabs(W[i]));
  return m > 0.f ? m / 448.0f : 1.0f;
}

// e4m3 image of W[n_out][k] / s: 128-column chunks, 16-byte unit u of row n at
// unit position u ^ (n % 8) (the 128-byte-swizzle K-major operand layout).
void append_e4m3_image(const float* W, int n_out, int k, float s, std::vector<uint8_t>& img) {
  const size_t at = img.size();
  img.resize(at + (size_t)n_out * k);
  for (int c = 0; c < k / 128; ++c)
    for (int n = 0; n < n_out; ++n)
      for (int u = 0; u < 8; ++u)
        for (int j = 0; j < 16; ++j) {
          const float q = W[(size_t)n * k + 128 * c + 16 * u + j] / s;
          img[at + (size_t)c * n_out * 128 + (size_t)n * 128 + ((u ^ (n & 7)) * 16) + j] =
              f32_to_e4m3(q);
        }
}

int64_t block_floats(int H, int K) { return (int64_t)H * K + 3 * H + (int64_t)H * H + 3 * H; }

template <class T>
etx_status dmalloc(etx_ctx* ctx, T** p, size_t count, const char* what) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return ETX_OK;
}

}  // namespace
}  // namespace etx

using namespace etx;

extern "C" {

int64_t etx_gnn_param_count(const etx_config* c) {
  if (config_problem(c)) return -1;
  const int64_t H = c->hidden;
  int64_t n = block_floats(H, 3) + block_floats(H, 2 * H);
  n += (int64_t)c->n_iters * 2 * block_floats(H, 3 * H);
  n += H * H + 3 * H + H + 1;
  return n;
}

int64_t etx_weights_size(const etx_config* c) {
  if (config_problem(c)) return -1;
  int64_t n = 12;
  for (int l = 0; l < c->emb_depth; ++l)
    n += (int64_t)c->emb_widths[l + 1] * c->emb_widths[l] + c->emb_widths[l + 1];
  return n + etx_gnn_param_count(c);
}

const char* etx_last_error(const etx_ctx* ctx) {
  if (!ctx) return "no context";
  return ctx->err.c_str();
}

etx_status etx_ctx_create(const etx_config* cfg, int32_t device, etx_ctx** out) {
  if (!out) return ETX_ERR_ARG;
  *out = nullptr;
  if (config_problem(cfg)) return ETX_ERR_ARG;
  etx_ctx* ctx = new (std::nothrow) etx_ctx();
  if (!ctx) return ETX_ERR_ARG;
  ctx->cfg = *cfg;
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return ETX_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&ctx->n_sms, cudaDevAttrMultiProcessorCount, device);
  if (ctx->n_sms < 1) ctx->n_sms = 1;
  const int64_t N = cfg->max_hits, E = cfg->max_edges, B = cfg->max_events;
  const int64_t H = cfg->hidden;
  etx_status st = ETX_OK;
  auto chk = [&](etx_status s) { if (st == ETX_OK) st = s; };
  chk(dmalloc(ctx, &ctx->d_err, 1, "error word"));
  chk(dmalloc(ctx, &ctx->n_edges, 1, "edge count"));
  chk(dmalloc(ctx, &ctx->small, 8, "reduction scratch"));
  ctx->red_part_n = (int64_t)ctx->n_sms * 16;
  chk(dmalloc(ctx, &ctx->red_part, (size_t)ctx->red_part_n, "loss partial sums"));
  chk(dmalloc(ctx, &ctx->plane_off, (size_t)B * (cfg->n_planes + 1), "plane offsets"));
  chk(dmalloc(ctx, &ctx->hit_cnt, (size_t)N + 1, "hit counts"));
  ctx->scan_tmp_ints = scan_tmp_ints(N + 1) + 8;
  chk(dmalloc(ctx, &ctx->scan_tmp, ctx->scan_tmp_ints, "scan scratch"));
  chk(dmalloc(ctx, &ctx->out_off, (size_t)N + 1, "out offsets"));
  chk(dmalloc(ctx, &ctx->in_off, (size_t)N + 1, "in offsets"));
  chk(dmalloc(ctx, &ctx->in_cnt, (size_t)N + 1, "in counts"));
  chk(dmalloc(ctx, &ctx->perm_in, (size_t)E, "in permutation"));
  chk(dmalloc(ctx, &ctx->h, (size_t)N * H, "node features"));
  chk(dmalloc(ctx, &ctx->m, (size_t)N * 2 * H, "messages"));
  chk(dmalloc(ctx, &ctx->e, (size_t)E * H, "edge features"));
  chk(dmalloc(ctx, &ctx->parent, (size_t)N, "union-find parents"));
  if (H == 128) chk(dmalloc(ctx, &ctx->h_lp, (size_t)N * 2 * H, "low-precision node features"));
  if (cfg->train) {
    const size_t L1 = (size_t)cfg->n_iters + 1, R = (size_t)(N > E ? N : E);
    chk(dmalloc(ctx, &ctx->h_ck, L1 * N * H, "node checkpoints"));
    chk(dmalloc(ctx, &ctx->e_ck, L1 * E * H, "edge checkpoints"));
    chk(dmalloc(ctx, &ctx->de, (size_t)E * H, "edge gradients"));
    chk(dmalloc(ctx, &ctx->dh, (size_t)N * H, "node gradients"));
    chk(dmalloc(ctx, &ctx->bw_X, R * 3 * H, "backward inputs"));
    chk(dmalloc(ctx, &ctx->bw_DX, R * 3 * H, "backward input gradients"));
    float** rows[] = {&ctx->bw_R1, &ctx->bw_DA1, &ctx->bw_DY1, &ctx->bw_DY1N1,
                      &ctx->bw_DA2, &ctx->bw_DY2, &ctx->bw_DY2N2};
    for (float** q : rows) chk(dmalloc(ctx, q, R * H, "backward row factors"));
    const size_t part = std::max<size_t>((size_t)ctx->n_sms * H * 3 * H, (size_t)ctx->n_sms * 4 * H);
    chk(dmalloc(ctx, &ctx->bw_part, part, "partial gradients"));
    if (H == 128) {
      // tensor-core block backward: n1 rows, rstd1, TF32 images of every
      // hidden-width block's W1, W1^T, W2, W2^T, and their job list
      chk(dmalloc(ctx, &ctx->bw_N1, R * H, "backward n1 rows"));
      chk(dmalloc(ctx, &ctx->bw_rstd1, R, "backward rstd1"));
      chk(dmalloc(ctx, &ctx->bw_Xlo, R * 3 * H, "backward input low parts"));
      chk(dmalloc(ctx, &ctx->bw_R1lo, R * H, "backward R1 low parts"));
      chk(dmalloc(ctx, &ctx->bw_cs_part, 2 * (size_t)ctx->n_sms * 4 * 3 * H, "column-sum partials"));
      // per block: W1, W1^T, W1 low [H][K] each, W2, W2^T, W2 low [H][H] each
      const size_t per_upd = 3 * (size_t)H * 3 * H + 3 * (size_t)H * H;
      const size_t per_enc = 3 * (size_t)H * 2 * H + 3 * (size_t)H * H;
      chk(dmalloc(ctx, &ctx->bw_img, per_enc + 2 * (size_t)cfg->n_iters * per_upd, "TF32 weight images"));
      ctx->bw_img_n_jobs = 6 * (1 + 2 * cfg->n_iters);
      unsigned char* jobs = nullptr;
      chk(dmalloc(ctx, &jobs, (size_t)ctx->bw_img_n_jobs * tf32_image_job_bytes(), "image jobs"));
      ctx->bw_img_jobs = jobs;
    }
  }
  if (st == ETX_OK) {
    e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "cudaMemset");
  }
  if (st == ETX_OK) {
    e = knn_set_smem_attr();
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "kNN shared-memory attribute");
  }
  if (st != ETX_OK) {
    etx_ctx_destroy(ctx);
    return st;
  }
  *out = ctx;
  return ETX_OK;
}

etx_status etx_ctx_destroy(etx_ctx* ctx) {
  if (!ctx) return ETX_OK;
  cudaSetDevice(ctx->device);
  void* bufs[] = {ctx->d_err, ctx->n_edges, ctx->w_dev, ctx->blob_dev, ctx->w_tc, ctx->plane_off,
                  ctx->hit_cnt, ctx->scan_tmp, ctx->out_off, ctx->in_off, ctx->in_cnt,
                  ctx->perm_in, ctx->h, ctx->m, ctx->e, ctx->parent, ctx->h_ck, ctx->e_ck,
                  ctx->de, ctx->dh, ctx->bw_X, ctx->bw_DX, ctx->bw_R1, ctx->bw_DA1, ctx->bw_DY1,
                  ctx->bw_DY1N1, ctx->bw_DA2, ctx->bw_DY2, ctx->bw_DY2N2, ctx->h_lp,
                  ctx->small, ctx->w_trip, ctx->bw_part, ctx->red_part, ctx->repack_dev,
                  ctx->embed_repack_dev,
                  ctx->bw_N1, ctx->bw_rstd1, ctx->bw_img, ctx->bw_img_jobs, ctx->bw_Xlo,
                  ctx->bw_R1lo, ctx->bw_cs_part};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (auto& r : ctx->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (ctx->w_host_pinned) {
    cudaEventSynchronize(ctx->w_host_ev);
    cudaEventDestroy(ctx->w_host_ev);
    cudaFreeHost(ctx->w_host_pinned);
  }
  delete ctx;
  return ETX_OK;
}

int64_t etx_launch_count(const etx_ctx* ctx) { return ctx ? ctx->launches : -1; }

etx_status etx_profile_enable(etx_ctx* ctx, int32_t on) {
  if (!ctx) return ETX_ERR_ARG;
  ctx->prof_on = on != 0;
  ctx->prof_used = 0;
  return ETX_OK;
}

int32_t etx_profile_read(etx_ctx* ctx, const char** names, double* total_ms, int64_t* counts,
                         int32_t max_entries) {
  if (!ctx) return -1;
  cudaSetDevice(ctx->device);
  int32_t n = 0;
  for (size_t i = 0; i < ctx->prof_used; ++i) {
    const ProfRec& r = ctx->prof[i];
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return -1;
    int32_t k = 0;
    while (k < n && std::strcmp(names[k], r.name) != 0) ++k;
    if (k == n) {
      if (n == max_entries) continue;
      names[n] = r.name;
      total_ms[n] = 0.0;
      counts[n] = 0;
      ++n;
    }
    total_ms[k] += ms;
    counts[k] += 1;
  }
  ctx->prof_used = 0;
  return n;
}

etx_status etx_load_weights(etx_ctx* ctx, const float* blob, int64_t n_floats) {
  if (!ctx) return ETX_ERR_ARG;
  if (!blob) return fail(ctx, ETX_ERR_ARG, "weight blob is NULL");
  const etx_config& c = ctx->cfg;
  if (n_floats != etx_weights_size(&c)) return fail(ctx, ETX_ERR_ARG, "weight blob size does not match the config");
  cudaSetDevice(ctx->device);
  const int H = c.hidden;
  // --- host-side repack: every Linear to W^T [k_pad][n] ---------------------
  std::vector<float> dev;
  dev.reserve((size_t)n_floats * 2);
  const float* p = blob;
  struct Pending { size_t wt, b; int k_in, k_pad, n; const float* w; };
  // every array starts on a 16-byte boundary (float4 loads of W^T chunks)
  auto align4 = [&]() { while (dev.size() % 4) dev.push_back(0.f); };
  auto push_lin = [&](int n_out, int k_in) {
    align4();
    Pending q;
    q.k_in = k_in;
    q.k_pad = k_in <= 4 ? 4 : k_in;
    q.n = n_out;
    q.w = p;
    q.wt = dev.size();
    dev.resize(dev.size() + (size_t)q.k_pad * n_out, 0.f);
    for (int o = 0; o < n_out; ++o)
      for (int k = 0; k < k_in; ++k) dev[q.wt + (size_t)k * n_out + o] = p[(size_t)o * k_in + k];
    p += (size_t)n_out * k_in;
    align4();
    q.b = dev.size();
    dev.insert(dev.end(), p, p + n_out);
    p += n_out;
    return q;
  };
  std::vector<RepackJob> vec_jobs;  // vectors of the interaction network (for etx_set_gnn_params)
  int64_t gnn_at = -1;               // blob offset of the interaction network once known
  auto push_vec = [&](int n) {
    align4();
    size_t at = dev.size();
    if (gnn_at >= 0) vec_jobs.push_back(RepackJob{(int64_t)(p - blob) - gnn_at, (int64_t)at, -1, 0, n});
    dev.insert(dev.end(), p, p + n);
    p += n;
    return at;
  };
  const size_t norm_at = push_vec(12);
  std::vector<Pending> emb;
  for (int l = 0; l < c.emb_depth; ++l) emb.push_back(push_lin(c.emb_widths[l + 1], c.emb_widths[l]));
  const int64_t gnn_offset = p - blob;
  gnn_at = gnn_offset;
  struct PB { Pending l1, l2; size_t g1, be1, g2, be2; };
  auto push_block = [&](int k_in) {
    PB b;
    b.l1 = push_lin(H, k_in);
    b.g1 = push_vec(H);
    b.be1 = push_vec(H);
    b.l2 = push_lin(H, H);
    b.g2 = push_vec(H);
    b.be2 = push_vec(H);
    return b;
  };
  PB node_enc = push_block(3), edge_enc = push_block(2 * H);
  std::vector<PB> node, edge;
  for (int k = 0; k < c.n_iters; ++k) {
    node.push_back(push_block(3 * H));
    edge.push_back(push_block(3 * H));
  }
  Pending cl1 = push_lin(H, H);
  size_t cg1 = push_vec(H), cbe1 = push_vec(H), cw2 = push_vec(H), cb2 = push_vec(1);
  if (p != blob + n_floats) return fail(ctx, ETX_ERR_ARG, "internal: blob walk mismatch");
  if (ctx->w_dev) cudaFree(ctx->w_dev);
  if (ctx->blob_dev) cudaFree(ctx->blob_dev);
  ctx->w_dev = nullptr;
  ctx->blob_dev = nullptr;
  if (dmalloc(ctx, &ctx->w_dev, dev.size(), "weights") != ETX_OK) return ETX_ERR_CUDA;
  if (dmalloc(ctx, &ctx->blob_dev, (size_t)n_floats, "weight blob") != ETX_OK) return ETX_ERR_CUDA;
  cudaError_t e = cudaMemcpy(ctx->w_dev, dev.data(), dev.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->blob_dev, blob, (size_t)n_floats * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "weight upload");
  ctx->w_dev_floats = dev.size();
  ctx->w_host = dev;
  // --- BF16 tensor-core operand images (hidden == 128) ------------------------
  if (ctx->w_tc) cudaFree(ctx->w_tc);
  ctx->w_tc = nullptr;
  std::vector<size_t> tc_off, f8_off;
  std::vector<float> f8_scale;
  if (H == 128) {
    std::vector<uint8_t> img, img8;
    auto push_img = [&](const Pending& q) {
      tc_off.push_back(img.size());
      append_bf16_image(q.w, q.n, q.k_in, img);
      const float sc = e4m3_scale(q.w, (size_t)q.n * q.k_in);
      f8_off.push_back(img8.size());
      f8_scale.push_back(sc);
      append_e4m3_image(q.w, q.n, q.k_in, sc, img8);
    };
    push_img(edge_enc.l1);
    push_img(edge_enc.l2);
    for (int k = 0; k < c.n_iters; ++k) {
      push_img(node[k].l1);
      push_img(node[k].l2);
      push_img(edge[k].l1);
      push_img(edge[k].l2);
    }
    push_img(cl1);
    const size_t b16 = img.size();
    img.insert(img.end(), img8.begin(), img8.end());  // FP8 images after the BF16 ones
    for (auto& o : f8_off) o += b16;
    if (dmalloc(ctx, &ctx->w_tc, img.size(), "tensor-core weights") != ETX_OK) return ETX_ERR_CUDA;
    e = cudaMemcpy(ctx->w_tc, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core weight upload");
  }
  float* base = ctx->w_dev;
  auto lin = [&](const Pending& q) {
    LinF32 l;
    l.wt = base + q.wt;
    l.b = base + q.b;
    l.k_in = q.k_in;
    l.k_pad = q.k_pad;
    l.n = q.n;
    return l;
  };
  auto blk = [&](const PB& b) {
    BlockF32 o;
    o.l1 = lin(b.l1);
    o.l2 = lin(b.l2);
    o.g1 = base + b.g1;
    o.be1 = base + b.be1;
    o.g2 = base + b.g2;
    o.be2 = base + b.be2;
    return o;
  };
  ctx->w = Weights();
  ctx->w.norm = base + norm_at;
  for (auto& q : emb) ctx->w.emb.push_back(lin(q));
  ctx->w.node_enc = blk(node_enc);
  ctx->w.edge_enc = blk(edge_enc);
  for (auto& b : node) ctx->w.node.push_back(blk(b));
  for (auto& b : edge) ctx->w.edge.push_back(blk(b));
  ctx->w.cls.l1 = lin(cl1);
  ctx->w.cls.g1 = base + cg1;
  ctx->w.cls.be1 = base + cbe1;
  ctx->w.cls.w2 = base + cw2;
  ctx->w.cls.b2 = base + cb2;
  if (H == 128) {
    size_t i = 0;
    // fills (w, w8, scale) of the next Linear in image order
    auto next = [&](const uint8_t** w, const uint8_t** w8, float* sc) {
      *w = ctx->w_tc + tc_off[i];
      *w8 = ctx->w_tc + f8_off[i];
      *sc = f8_scale[i];
      ++i;
    };
    auto block = [&](BlockTC& t) {
      next(&t.w1, &t.w1f8, &t.s1);
      next(&t.w2, &t.w2f8, &t.s2);
    };
    block(ctx->w.edge_enc_tc);
    for (int k = 0; k < c.n_iters; ++k) {
      BlockTC nb, eb;
      block(nb);
      block(eb);
      ctx->w.node_tc.push_back(nb);
      ctx->w.edge_tc.push_back(eb);
    }
    next(&ctx->w.cls_tc.w1, &ctx->w.cls_tc.w1f8, &ctx->w.cls_tc.s1);
    ctx->w.has_tc = true;
  }
  // repack plan of the interaction network for etx_set_gnn_params: every Linear
  // (W to W^T, its BF16 operand image when there is one) and bias, every vector
  {
    std::vector<RepackJob> jobs;
    auto lin_job = [&](const Pending& q, int64_t img) {
      const int64_t src = (int64_t)(q.w - blob) - gnn_offset;
      jobs.push_back(RepackJob{src, (int64_t)q.wt, img, q.k_in, q.n});
      jobs.push_back(RepackJob{src + (int64_t)q.n * q.k_in, (int64_t)q.b, -1, 0, q.n});
    };
    size_t ti = 0;  // next BF16 image (push_img order)
    auto img = [&]() { return H == 128 ? (int64_t)tc_off[ti++] : (int64_t)-1; };
    lin_job(node_enc.l1, -1);
    lin_job(node_enc.l2, -1);
    lin_job(edge_enc.l1, img());
    lin_job(edge_enc.l2, img());
    for (int k = 0; k < c.n_iters; ++k) {
      lin_job(node[k].l1, img());
      lin_job(node[k].l2, img());
      lin_job(edge[k].l1, img());
      lin_job(edge[k].l2, img());
    }
    lin_job(cl1, img());
    jobs.insert(jobs.end(), vec_jobs.begin(), vec_jobs.end());
    if (ctx->repack_dev) cudaFree(ctx->repack_dev);
    ctx->repack_dev = nullptr;
    if (dmalloc(ctx, &ctx->repack_dev, jobs.size(), "repack plan") != ETX_OK) return ETX_ERR_CUDA;
    e = cudaMemcpy(ctx->repack_dev, jobs.data(), jobs.size() * sizeof(RepackJob), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "repack plan upload");
    ctx->n_repack = (int)jobs.size();
    ctx->n_theta = n_floats - gnn_offset;
    // and of the embedding, for etx_set_embed_params (FP32 layers only)
    std::vector<RepackJob> ejobs;
    for (auto& q : emb) {
      const int64_t src = (int64_t)(q.w - blob) - 12;  // the embedding follows the 12 normalisation values
      ejobs.push_back(RepackJob{src, (int64_t)q.wt, -1, q.k_in, q.n});
      ejobs.push_back(RepackJob{src + (int64_t)q.n * q.k_in, (int64_t)q.b, -1, 0, q.n});
    }
    if (ctx->embed_repack_dev) cudaFree(ctx->embed_repack_dev);
    ctx->embed_repack_dev = nullptr;
    if (dmalloc(ctx, &ctx->embed_repack_dev, ejobs.size(), "embedding repack plan") != ETX_OK)
      return ETX_ERR_CUDA;
    e = cudaMemcpy(ctx->embed_repack_dev, ejobs.data(), ejobs.size() * sizeof(RepackJob),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "embedding repack plan upload");
    ctx->n_embed_repack = (int)ejobs.size();
  }
  ctx->w_host_pending = false;
  ctx->f8_stale = false;
  ctx->gnn_blob_offset = gnn_offset;
  ctx->fwd_saved = false;
  ctx->weights_loaded = true;
  return ETX_OK;
}

}  // extern "C"

namespace etx {
namespace {

// One repack job per block row of the grid: a Linear's W [n][k_in] (row-major,
// from the parameter vector) to W^T [k][n] in the FP32 weights, plus, when
// img >= 0, its BF16 K-major 128-byte-swizzle operand image (64-column chunks,
// 16-byte unit u of row o at position u ^ (o % 8)); or a plain vector copy.
__global__ void k_repack(const float* __restrict__ theta, const RepackJob* __restrict__ jobs,
                         float* __restrict__ w_dev, uint8_t* __restrict__ w_tc) {
  const RepackJob j = jobs[blockIdx.y];
  const int64_t total = j.k_in > 0 ? (int64_t)j.k_in * j.n : j.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = theta[j.src + i];
    if (j.k_in > 0) {
      const int o = (int)(i / j.k_in), kk = (int)(i % j.k_in);
      w_dev[j.dst + (int64_t)kk * j.n + o] = v;
      if (j.img >= 0) {
        const int cch = kk >> 6, u = (kk & 63) >> 3, jj = kk & 7;
        const int64_t off = j.img + (int64_t)cch * j.n * 128 + (int64_t)o * 128 + ((u ^ (o & 7)) << 4) + 2 * jj;
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16*>(w_tc + off) = b;
      }
    } else {
      w_dev[j.dst + i] = v;
    }
  }
}

}  // namespace
}  // namespace etx

extern "C" {

etx_status etx_set_gnn_params(etx_ctx* ctx, const float* theta, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->weights_loaded) return fail(ctx, ETX_ERR_STATE, "weights not loaded");
  if (!theta) return fail(ctx, ETX_ERR_ARG, "parameter vector is NULL");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->w_host_pinned) {
    cudaError_t e = cudaMallocHost((void**)&ctx->w_host_pinned, ctx->w_dev_floats * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pinned weight copy");
    e = cudaEventCreateWithFlags(&ctx->w_host_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weight copy event");
  }
  // a host copy still being filled must land before the buffer is reused
  if (ctx->w_host_pending) {
    cudaError_t e = cudaEventSynchronize(ctx->w_host_ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weight copy wait");
  }
  launch(ctx, "weights_repack", k_repack, dim3(32, ctx->n_repack), 256, 0, s, theta,
         (const RepackJob*)ctx->repack_dev, ctx->w_dev, ctx->w_tc);
  cudaError_t e = cudaMemcpyAsync(ctx->blob_dev + ctx->gnn_blob_offset, theta,
                                  (size_t)ctx->n_theta * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->w_host_pinned, ctx->w_dev, ctx->w_dev_floats * sizeof(float),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->w_host_ev, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_set_gnn_params");
  ctx->w_host_pending = true;
  ctx->f8_stale = ctx->w.has_tc;  // the e4m3 images keep the loaded weights
  ctx->fwd_saved = false;
  return ETX_OK;
}

etx_status etx_set_embed_params(etx_ctx* ctx, const float* theta, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->weights_loaded || !ctx->embed_repack_dev) return fail(ctx, ETX_ERR_STATE, "weights not loaded");
  if (!theta) return fail(ctx, ETX_ERR_ARG, "parameter vector is NULL");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "weights_repack", k_repack, dim3(32, ctx->n_embed_repack), 256, 0, s, theta,
         (const RepackJob*)ctx->embed_repack_dev, ctx->w_dev, (uint8_t*)nullptr);
  // the reverse pass reads the weights in blob order
  cudaError_t e = cudaMemcpyAsync(ctx->blob_dev + 12, theta,
                                  (size_t)embed_param_count(ctx->cfg) * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_set_embed_params");
  return ETX_OK;
}

etx_status etx_ctx_sync(etx_ctx* ctx, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  int word = 0;
  e = cudaMemcpy(&word, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "error word read");
  if (word) {
    e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word reset");
  }
  if (word & DERR_TIMEOUT) return fail(ctx, ETX_ERR_TIMEOUT, "a device loop reached its iteration cap");
  if (word & DERR_CAPACITY) return fail(ctx, ETX_ERR_CAPACITY, "an edge buffer was too small");
  if (word & DERR_UNSORTED) return fail(ctx, ETX_ERR_UNSORTED, "hits not plane-sorted / edges not sorted by source / bad offsets");
  if (word & DERR_RANGE) return fail(ctx, ETX_ERR_UNSORTED, "an index was out of range");
  return ETX_OK;
}

etx_status etx_embed(etx_ctx* ctx, const float* x, const float* y, const float* z, int64_t n_hits,
                     float* emb, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->weights_loaded) return fail(ctx, ETX_ERR_STATE, "weights not loaded");
  if (n_hits < 0 || n_hits >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "n_hits out of range");
  if (n_hits > 0 && (!x || !y || !z || !emb)) return fail(ctx, ETX_ERR_ARG, "NULL array");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_embed(ctx, x, y, z, n_hits, emb, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_embed launch");
  return ETX_OK;
}

etx_status etx_build_graph(etx_ctx* ctx, const float* emb, const int8_t* plane,
                           const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                           float radius, int32_t k_max, int32_t* src, int32_t* dst,
                           int64_t edge_capacity, int32_t* edge_offsets, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (n_hits < 0 || n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (!(radius >= 0.f) || radius > 1e18f) return fail(ctx, ETX_ERR_ARG, "radius must be finite and >= 0");
  if (k_max < 1) return fail(ctx, ETX_ERR_ARG, "k_max must be >= 1");
  if (edge_capacity < 0 || edge_capacity >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "edge_capacity out of range");
  if (!hit_offsets || !edge_offsets) return fail(ctx, ETX_ERR_ARG, "NULL offsets");
  if (n_hits > 0 && (!emb || !plane)) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (edge_capacity > 0 && (!src || !dst)) return fail(ctx, ETX_ERR_ARG, "NULL edge arrays");
  if (n_hits * (int64_t)k_max >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "n_hits * k_max must stay below 2^31");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_build_graph(ctx, emb, plane, hit_offsets, n_events, n_hits, radius, k_max,
                                     src, dst, edge_capacity, edge_offsets, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_build_graph launch");
  return ETX_OK;
}

etx_status etx_gnn_forward(etx_ctx* ctx, const float* x, const float* y, const float* z,
                           int64_t n_hits, const int32_t* src, const int32_t* dst,
                           const int32_t* edge_offsets, int32_t n_events, etx_dtype dtype,
                           float* logits, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->weights_loaded) return fail(ctx, ETX_ERR_STATE, "weights not loaded");
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (n_hits < 0 || n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (!edge_offsets || !src || !dst || !logits) return fail(ctx, ETX_ERR_ARG, "NULL edge array");
  if (n_hits > 0 && (!x || !y || !z)) return fail(ctx, ETX_ERR_ARG, "NULL hit array");
  if (dtype != ETX_F32 && dtype != ETX_BF16 && dtype != ETX_FP8E4M3 && dtype != ETX_BF16_EDGE_STORE)
    return fail(ctx, ETX_ERR_ARG, "unknown dtype");
  if (dtype == ETX_BF16_EDGE_STORE && ctx->cfg.train)
    return fail(ctx, ETX_ERR_UNSUPPORTED, "BF16 edge storage is for inference (train context)");
  if (dtype != ETX_F32 && !ctx->w.has_tc)
    return fail(ctx, ETX_ERR_UNSUPPORTED, "the tensor-core path needs hidden == 128");
  if (dtype == ETX_FP8E4M3 && ctx->f8_stale)
    return fail(ctx, ETX_ERR_STATE, "e4m3 weights predate etx_set_gnn_params: reload the weights");
  if (ctx->w_host_pending) {  // the kernels take some parameters by value from the host copy
    cudaError_t e = cudaEventSynchronize(ctx->w_host_ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weight copy wait");
    std::memcpy(ctx->w_host.data(), ctx->w_host_pinned, ctx->w_dev_floats * sizeof(float));
    ctx->w_host_pending = false;
  }
  if (n_hits == 0) return ETX_OK;  // no hits, hence no edges: nothing to compute
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "clamp_edges", k_clamp_edges, 1, 1, 0, s, edge_offsets, n_events, ctx->cfg.max_edges,
         ctx->n_edges, ctx->d_err);
  cudaError_t e = launch_edge_index(ctx, n_hits, src, dst, ctx->n_edges, s);
  if (e == cudaSuccess)
    e = launch_gnn_forward(ctx, x, y, z, n_hits, src, dst, ctx->n_edges, logits, dtype, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_gnn_forward launch");
  if (ctx->cfg.train) {
    ctx->fwd_x = x;
    ctx->fwd_y = y;
    ctx->fwd_z = z;
    ctx->fwd_src = src;
    ctx->fwd_dst = dst;
    ctx->fwd_n_hits = n_hits;
    ctx->fwd_saved = true;
  }
  return ETX_OK;
}

etx_status etx_gnn_checkpoints(etx_ctx* ctx, int32_t k, float* h_out, float* e_out, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->cfg.train || !ctx->fwd_saved) return fail(ctx, ETX_ERR_STATE, "no training forward kept");
  if (k < 0 || k > ctx->cfg.n_iters) return fail(ctx, ETX_ERR_ARG, "checkpoint index out of range");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t H = ctx->cfg.hidden, N = ctx->fwd_n_hits, Ecap = ctx->cfg.max_edges;
  cudaError_t e = cudaSuccess;
  if (h_out)
    e = cudaMemcpyAsync(h_out, ctx->h_ck + (size_t)k * N * H, (size_t)N * H * sizeof(float),
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && e_out)
    e = launch_checkpoint(ctx, e_out, ctx->e_ck + (size_t)k * Ecap * H, 0, ctx->n_edges, Ecap, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_gnn_checkpoints");
  return ETX_OK;
}

int64_t etx_fp8_scale_count(const etx_config* cfg) {
  if (config_problem(cfg)) return -1;
  return 4 * (int64_t)cfg->n_iters + 3;
}

etx_status etx_set_fp8_scales(etx_ctx* ctx, const float* host_scales, int64_t n) {
  if (!ctx) return ETX_ERR_ARG;
  if (n == 0 && !host_scales) {
    ctx->fp8_act.clear();
    return ETX_OK;
  }
  if (!host_scales) return fail(ctx, ETX_ERR_ARG, "fp8 scales are NULL");
  if (n != etx_fp8_scale_count(&ctx->cfg))
    return fail(ctx, ETX_ERR_ARG, "fp8 scale count must be 4 * n_iters + 3");
  for (int64_t i = 0; i < n; ++i) {
    const float v = host_scales[i];
    int ex = 0;
    if (!(v > 0.f) || !std::isfinite(v) || std::frexp(v, &ex) != 0.5f || ex < -99 || ex > 101)
      return fail(ctx, ETX_ERR_ARG, "fp8 scales must be powers of two in [2^-100, 2^100]");
  }
  ctx->fp8_act.assign(host_scales, host_scales + n);
  return ETX_OK;
}

etx_status etx_gnn_backward(etx_ctx* ctx, const float* dlogits, float* dparams, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->cfg.train) return fail(ctx, ETX_ERR_STATE, "context was not created for training");
  if (!ctx->fwd_saved) return fail(ctx, ETX_ERR_STATE, "no training forward since the weights were loaded");
  if (!dlogits || !dparams) return fail(ctx, ETX_ERR_ARG, "NULL array");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_gnn_backward(ctx, dlogits, dparams, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_gnn_backward launch");
  return ETX_OK;
}

etx_status etx_weighted_bce(etx_ctx* ctx, const float* logits, const float* targets,
                            const int32_t* edge_offsets, int32_t n_events, float pos_weight,
                            float* loss, float* dlogits, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!logits || !targets || !edge_offsets || !loss || !dlogits) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (!(pos_weight >= 0.f)) return fail(ctx, ETX_ERR_ARG, "pos_weight must be >= 0");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "clamp_edges", k_clamp_edges, 1, 1, 0, s, edge_offsets, n_events, ctx->cfg.max_edges,
         ctx->n_edges, ctx->d_err);
  cudaError_t e = launch_weighted_bce(ctx, logits, targets, ctx->n_edges, pos_weight, loss, dlogits, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_weighted_bce launch");
  return ETX_OK;
}

etx_status etx_focal_loss(etx_ctx* ctx, const float* logits, const float* targets,
                          const int32_t* edge_offsets, int32_t n_events, float alpha, float gamma,
                          float* loss, float* dlogits, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!logits || !targets || !edge_offsets || !loss || !dlogits) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (!(alpha >= 0.f && alpha <= 1.f) || !(gamma >= 0.f) || gamma > 1e6f)
    return fail(ctx, ETX_ERR_ARG, "alpha must lie in [0, 1] and gamma be >= 0");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "clamp_edges", k_clamp_edges, 1, 1, 0, s, edge_offsets, n_events, ctx->cfg.max_edges,
         ctx->n_edges, ctx->d_err);
  cudaError_t e = launch_focal_loss(ctx, logits, targets, ctx->n_edges, alpha, gamma, loss, dlogits, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_focal_loss launch");
  return ETX_OK;
}

etx_status etx_adam_step(etx_ctx* ctx, float* params, const float* grads, float* m, float* v,
                         int64_t n, float lr, float beta1, float beta2, float eps, int64_t step,
                         void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n < 0 || (n > 0 && (!params || !grads || !m || !v))) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (step < 1) return fail(ctx, ETX_ERR_ARG, "step counts from 1");
  if (n == 0) return ETX_OK;
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_adam(ctx, params, grads, m, v, n, lr, beta1, beta2, eps, step,
                              (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_adam_step launch");
  return ETX_OK;
}

etx_status etx_edges_to_tracks(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                               const float* logits, float threshold_logit,
                               const int32_t* edge_offsets, const int32_t* hit_offsets,
                               int32_t n_events, int64_t n_hits, int32_t min_hits,
                               int32_t* labels, int32_t* n_tracks, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (n_hits < 0 || n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (!edge_offsets || !hit_offsets || !src || !dst || !logits) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (n_hits > 0 && !labels) return fail(ctx, ETX_ERR_ARG, "NULL labels");
  if (threshold_logit != threshold_logit) return fail(ctx, ETX_ERR_ARG, "threshold is NaN");
  if (n_events == 0 && n_hits > 0) return fail(ctx, ETX_ERR_ARG, "hits without events");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "clamp_edges", k_clamp_edges, 1, 1, 0, s, edge_offsets, n_events, (int64_t)INT32_MAX,
         ctx->n_edges, ctx->d_err);
  cudaError_t e = launch_edges_to_tracks(ctx, src, dst, logits, threshold_logit, ctx->n_edges,
                                         hit_offsets, n_events, n_hits, min_hits, labels, n_tracks, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_edges_to_tracks launch");
  return ETX_OK;
}

etx_status etx_edges_to_tracks_sweep(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                     const float* logits, float threshold_logit,
                                     const int32_t* edge_offsets, const int8_t* plane,
                                     const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                                     int32_t* labels, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (n_hits < 0 || n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (!edge_offsets || !hit_offsets || !src || !dst || !logits) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (n_hits > 0 && (!labels || !plane)) return fail(ctx, ETX_ERR_ARG, "NULL labels or plane");
  if (threshold_logit != threshold_logit) return fail(ctx, ETX_ERR_ARG, "threshold is NaN");
  if (n_events == 0 && n_hits > 0) return fail(ctx, ETX_ERR_ARG, "hits without events");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "clamp_edges", k_clamp_edges, 1, 1, 0, s, edge_offsets, n_events, ctx->cfg.max_edges,
         ctx->n_edges, ctx->d_err);
  ctx->fwd_saved = false;  // the out-offsets of the last training forward are rebuilt
  cudaError_t e = launch_plane_bins(ctx, plane, hit_offsets, n_events, n_hits, s);
  if (e == cudaSuccess) e = launch_out_offsets(ctx, n_hits, src, dst, ctx->n_edges, s);
  if (e == cudaSuccess)
    e = launch_plane_sweep(ctx, src, dst, logits, threshold_logit, hit_offsets, n_events, n_hits,
                           labels, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_edges_to_tracks_sweep launch");
  return ETX_OK;
}

// ---- triplets (Sec. 5.3) -------------------------------------------------------

int64_t etx_triplet_weights_size(const etx_config* cfg) {
  if (!cfg || cfg->hidden < 1) return -1;
  return triplet_weights_size(cfg->hidden);
}

etx_status etx_load_triplet_weights(etx_ctx* ctx, const float* blob, int64_t n_floats) {
  if (!ctx) return ETX_ERR_ARG;
  if (!blob) return fail(ctx, ETX_ERR_ARG, "weight blob is NULL");
  if (n_floats != triplet_weights_size(ctx->cfg.hidden))
    return fail(ctx, ETX_ERR_ARG, "triplet blob size does not match the config");
  cudaSetDevice(ctx->device);
  cudaError_t e = load_triplet_weights(ctx, blob);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "triplet weight upload");
  return ETX_OK;
}

size_t etx_triplets_workspace(int64_t n_hits) {
  return n_hits < 0 ? 0 : triplets_workspace(n_hits);
}

etx_status etx_build_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                              const float* logits, float threshold_logit,
                              const int32_t* edge_offsets, int32_t n_events, int64_t n_hits,
                              void* workspace, size_t workspace_bytes, int32_t* first,
                              int32_t* second, int8_t* kind, int64_t capacity, int32_t* counts,
                              void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (n_hits < 0 || n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (!edge_offsets || !src || !dst || !logits || !counts || !workspace) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (capacity < 0 || capacity >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "capacity out of range");
  if (capacity > 0 && (!first || !second || !kind)) return fail(ctx, ETX_ERR_ARG, "NULL triplet arrays");
  if (threshold_logit != threshold_logit) return fail(ctx, ETX_ERR_ARG, "threshold is NaN");
  if (workspace_bytes < triplets_workspace(n_hits))
    return fail(ctx, ETX_ERR_CAPACITY, "workspace smaller than etx_triplets_workspace()");
  if (reinterpret_cast<uintptr_t>(workspace) & 3) return fail(ctx, ETX_ERR_ARG, "workspace not 4-byte aligned");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "clamp_edges", k_clamp_edges, 1, 1, 0, s, edge_offsets, n_events, ctx->cfg.max_edges,
         ctx->n_edges, ctx->d_err);
  ctx->fwd_saved = false;  // the edge index of the last training forward is rebuilt
  cudaError_t e = launch_build_triplets(ctx, src, dst, logits, threshold_logit, n_hits, workspace,
                                        capacity, first, second, kind, counts, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_build_triplets launch");
  return ETX_OK;
}

size_t etx_tracks_workspace(int64_t n_hits, int64_t max_edges, int64_t triplet_capacity) {
  if (n_hits < 0 || max_edges < 0 || triplet_capacity < 0) return 0;
  return tracks_workspace(n_hits, max_edges, triplet_capacity);
}

etx_status etx_tracks_from_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                    const float* logits, float threshold_logit,
                                    const int32_t* edge_offsets, int32_t n_events,
                                    int64_t n_hits, const int32_t* first, const int32_t* second,
                                    const float* triplet_logits, float triplet_threshold,
                                    const int32_t* counts, int64_t triplet_capacity,
                                    int32_t min_hits, void* workspace, size_t workspace_bytes,
                                    int32_t* track_offsets, int32_t* track_hits,
                                    int64_t track_capacity, int64_t hit_capacity,
                                    int32_t* n_out, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (n_hits < 0 || n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (!edge_offsets || !src || !dst || !logits || !counts || !workspace || !n_out || !track_offsets)
    return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (triplet_capacity < 0 || triplet_capacity >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "triplet capacity out of range");
  if (triplet_capacity > 0 && (!first || !second || !triplet_logits)) return fail(ctx, ETX_ERR_ARG, "NULL triplet arrays");
  if (track_capacity < 0 || hit_capacity < 0 || track_capacity >= ((int64_t)1 << 31) ||
      hit_capacity >= ((int64_t)1 << 31))
    return fail(ctx, ETX_ERR_ARG, "track or hit capacity out of range");
  if (hit_capacity > 0 && !track_hits) return fail(ctx, ETX_ERR_ARG, "NULL track hits");
  if (min_hits < 1) return fail(ctx, ETX_ERR_ARG, "min_hits must be >= 1");
  if (threshold_logit != threshold_logit || triplet_threshold != triplet_threshold)
    return fail(ctx, ETX_ERR_ARG, "threshold is NaN");
  if (ctx->cfg.max_edges + triplet_capacity >= ((int64_t)1 << 31))
    return fail(ctx, ETX_ERR_CAPACITY, "max_edges + triplet capacity must stay below 2^31");
  if (workspace_bytes < tracks_workspace(n_hits, ctx->cfg.max_edges, triplet_capacity))
    return fail(ctx, ETX_ERR_CAPACITY, "workspace smaller than etx_tracks_workspace()");
  if (reinterpret_cast<uintptr_t>(workspace) & 3) return fail(ctx, ETX_ERR_ARG, "workspace not 4-byte aligned");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  launch(ctx, "clamp_edges", k_clamp_edges, 1, 1, 0, s, edge_offsets, n_events, ctx->cfg.max_edges,
         ctx->n_edges, ctx->d_err);
  ctx->fwd_saved = false;  // the edge index of the last training forward is rebuilt
  cudaError_t e = launch_tracks_from_triplets(
      ctx, src, dst, logits, threshold_logit, n_hits, first, second, triplet_logits,
      triplet_threshold, counts, triplet_capacity, min_hits, workspace, track_offsets, track_hits,
      track_capacity, hit_capacity, n_out, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_tracks_from_triplets launch");
  return ETX_OK;
}

etx_status etx_classify_triplets(etx_ctx* ctx, const int32_t* first, const int32_t* second,
                                 const int32_t* counts, int64_t capacity, float* logits,
                                 void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->trip_loaded) return fail(ctx, ETX_ERR_STATE, "triplet weights not loaded");
  if (ctx->e_bf16)
    return fail(ctx, ETX_ERR_STATE, "the last forward stored the edge encodings in BF16; classify "
                                    "triplets after an FP32-storage forward");
  if (!counts || (capacity > 0 && (!first || !second || !logits))) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (capacity < 0 || capacity >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "capacity out of range");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_triplet_classifier(ctx, first, second, nullptr, counts + 1, capacity,
                                            ctx->trip_art, logits, s);
  if (e == cudaSuccess)
    e = launch_triplet_classifier(ctx, first, second, counts + 1, counts, capacity, ctx->trip_elb,
                                  logits, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_classify_triplets launch");
  return ETX_OK;
}

// ---- embedding training (Sec. 5.1, Eq. 2-3) ----------------------------------

int64_t etx_embed_param_count(const etx_config* cfg) {
  if (!cfg || cfg->emb_depth < 1 || cfg->emb_depth > ETX_MAX_EMB_LAYERS) return -1;
  return embed_param_count(*cfg);
}

size_t etx_embed_train_workspace(const etx_config* cfg, int64_t n_hits) {
  if (!cfg || n_hits < 0 || cfg->emb_depth < 1 || cfg->emb_depth > ETX_MAX_EMB_LAYERS) return 0;
  return embed_backward_workspace(*cfg, n_hits);
}

etx_status etx_embed_forward_train(etx_ctx* ctx, const float* x, const float* y, const float* z,
                                   int64_t n_hits, float* emb, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->weights_loaded) return fail(ctx, ETX_ERR_STATE, "weights not loaded");
  if (n_hits < 0 || n_hits >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "n_hits out of range");
  if (n_hits > 0 && (!x || !y || !z || !emb || !workspace)) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (workspace_bytes < embed_backward_workspace(ctx->cfg, n_hits))
    return fail(ctx, ETX_ERR_CAPACITY, "workspace smaller than etx_embed_train_workspace()");
  if (reinterpret_cast<uintptr_t>(workspace) & 15) return fail(ctx, ETX_ERR_ARG, "workspace not 16-byte aligned");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_embed_save(ctx, x, y, z, n_hits, emb, static_cast<float*>(workspace),
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_embed_forward_train launch");
  return ETX_OK;
}

etx_status etx_embed_backward(etx_ctx* ctx, int64_t n_hits, const float* d_emb, float* d_params,
                              void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (!ctx->weights_loaded || !ctx->blob_dev) return fail(ctx, ETX_ERR_STATE, "weights not loaded");
  if (n_hits < 0 || n_hits >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "n_hits out of range");
  if (!d_params || (n_hits > 0 && (!d_emb || !workspace))) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (workspace_bytes < embed_backward_workspace(ctx->cfg, n_hits))
    return fail(ctx, ETX_ERR_CAPACITY, "workspace smaller than etx_embed_train_workspace()");
  const int64_t EW = ctx->cfg.emb_widths[1];
  float* saved = static_cast<float*>(workspace);
  float* dz_a = saved + n_hits * 4 + (int64_t)(ctx->cfg.emb_depth - 1) * n_hits * EW;
  float* dz_b = dz_a + n_hits * EW;
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_embed_backward(ctx, n_hits, saved, d_emb, dz_a, dz_b, d_params,
                                        (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_embed_backward launch");
  return ETX_OK;
}

size_t etx_embedding_pairs_workspace(int32_t n_events, int64_t n_hits, int32_t k_max) {
  if (n_events < 0 || n_hits < 0 || k_max < 1) return 0;
  return embedding_pairs_workspace(n_events, n_hits, k_max);
}

etx_status etx_embedding_pairs(etx_ctx* ctx, const float* emb, const int8_t* plane,
                               const int32_t* particle_id, const int32_t* hit_offsets,
                               int32_t n_events, int64_t n_hits, float radius, int32_t k_max,
                               const uint32_t* rand, int32_t min_hits, void* workspace,
                               size_t workspace_bytes, int32_t* pair_q, int32_t* pair_a,
                               uint8_t* pair_genuine, int64_t capacity, int32_t* n_pairs,
                               void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_events < 0 || n_events > ctx->cfg.max_events) return fail(ctx, ETX_ERR_CAPACITY, "n_events exceeds the context capacity");
  if (n_hits < 0 || n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (n_events == 0 && n_hits > 0) return fail(ctx, ETX_ERR_ARG, "hits without events");
  if (!(radius >= 0.f) || radius > 1e18f) return fail(ctx, ETX_ERR_ARG, "radius must be finite and >= 0");
  if (k_max < 1 || n_hits * (int64_t)k_max >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "k_max out of range");
  if (min_hits < 1) return fail(ctx, ETX_ERR_ARG, "min_hits must be at least 1");
  if (capacity < 0 || capacity >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "capacity out of range");
  if (!hit_offsets || !n_pairs || !workspace) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (n_hits > 0 && (!emb || !plane || !particle_id || !rand)) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (capacity > 0 && (!pair_q || !pair_a || !pair_genuine)) return fail(ctx, ETX_ERR_ARG, "NULL pair arrays");
  if (workspace_bytes < embedding_pairs_workspace(n_events, n_hits, k_max))
    return fail(ctx, ETX_ERR_CAPACITY, "workspace smaller than etx_embedding_pairs_workspace()");
  if (reinterpret_cast<uintptr_t>(workspace) & 3) return fail(ctx, ETX_ERR_ARG, "workspace not 4-byte aligned");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_embedding_pairs(ctx, emb, plane, particle_id, hit_offsets, n_events, n_hits,
                                         radius, k_max, rand, min_hits, workspace, pair_q, pair_a,
                                         pair_genuine, capacity, n_pairs, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_embedding_pairs launch");
  return ETX_OK;
}

size_t etx_hinge_loss_workspace(int64_t n_hits, int64_t pair_capacity) {
  if (n_hits < 0 || pair_capacity < 0) return 0;
  return hinge_loss_workspace(n_hits, pair_capacity);
}

etx_status etx_hinge_loss(etx_ctx* ctx, const float* emb, int64_t n_hits, const int32_t* pair_q,
                          const int32_t* pair_a, const uint8_t* pair_genuine,
                          const int32_t* n_pairs, int64_t pair_capacity, float margin,
                          float w_genuine, float* loss, float* d_emb, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_hits < 0 || n_hits >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "n_hits out of range");
  if (n_hits > ctx->cfg.max_hits) return fail(ctx, ETX_ERR_CAPACITY, "n_hits exceeds the context capacity");
  if (pair_capacity < 0 || pair_capacity >= ((int64_t)1 << 31)) return fail(ctx, ETX_ERR_ARG, "pair_capacity out of range");
  if (!workspace) return fail(ctx, ETX_ERR_ARG, "NULL workspace");
  if (reinterpret_cast<uintptr_t>(workspace) & 15) return fail(ctx, ETX_ERR_ARG, "workspace not 16-byte aligned");
  if (workspace_bytes < hinge_loss_workspace(n_hits, pair_capacity))
    return fail(ctx, ETX_ERR_CAPACITY, "workspace smaller than etx_hinge_loss_workspace()");
  if (!n_pairs || !loss || (n_hits > 0 && (!emb || !d_emb))) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (pair_capacity > 0 && (!pair_q || !pair_a || !pair_genuine)) return fail(ctx, ETX_ERR_ARG, "NULL pair arrays");
  if (!(margin == margin) || !(w_genuine >= 0.f) || w_genuine > 1e30f) return fail(ctx, ETX_ERR_ARG, "bad margin or w_genuine");
  if (ctx->cfg.emb_widths[ctx->cfg.emb_depth] > 16) return fail(ctx, ETX_ERR_UNSUPPORTED, "embedding dimension above 16");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_hinge_loss(ctx, emb, n_hits, pair_q, pair_a, pair_genuine, n_pairs,
                                    pair_capacity, margin, w_genuine, loss, d_emb, workspace,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_hinge_loss launch");
  return ETX_OK;
}

size_t etx_track_metrics_workspace(int32_t n_events, int64_t n_hits) {
  if (n_events < 0 || n_hits < 0) return 0;
  return track_metrics_workspace(n_events, n_hits);
}

etx_status etx_track_metrics(etx_ctx* ctx, const int32_t* labels, const int32_t* particle_id,
                             const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                             int32_t min_hits, int32_t match_num, int32_t match_den,
                             void* workspace, size_t workspace_bytes, int64_t* counts,
                             double* values, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  if (n_events < 0 || n_hits < 0 || n_hits > INT32_MAX) return fail(ctx, ETX_ERR_ARG, "bad n_events or n_hits");
  if (n_events == 0 && n_hits > 0) return fail(ctx, ETX_ERR_ARG, "hits without events");
  if (!counts || !values || (n_events > 0 && !hit_offsets)) return fail(ctx, ETX_ERR_ARG, "NULL array");
  if (n_hits > 0 && (!labels || !particle_id)) return fail(ctx, ETX_ERR_ARG, "NULL labels or particle_id");
  if (min_hits < 1) return fail(ctx, ETX_ERR_ARG, "min_hits must be at least 1");
  if (match_num <= 0 || match_num > match_den || 2 * (int64_t)match_num <= match_den)
    return fail(ctx, ETX_ERR_ARG, "match fraction must lie in (1/2, 1]");
  if (workspace_bytes < track_metrics_workspace(n_events, n_hits))
    return fail(ctx, ETX_ERR_CAPACITY, "workspace smaller than etx_track_metrics_workspace()");
  if (n_events > 0 && (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 7)))
    return fail(ctx, ETX_ERR_ARG, "workspace NULL or not 8-byte aligned");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_track_metrics(ctx, labels, particle_id, hit_offsets, n_events, n_hits,
                                       min_hits, match_num, match_den, workspace, counts, values,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etx_track_metrics launch");
  return ETX_OK;
}

}  // extern "C"

// ---- autotuner ---------------------------------------------------------------

namespace {

const char* const kTcBlock[4] = {"edge_encoder", "node_update", "edge_update", "classifier"};
// k-NN launch candidates: blocks per (event, plane), candidate floats staged per block
constexpr int kKnnSplits[3] = {1, 2, 4};
constexpr int kKnnStages[5] = {1024, 2048, 4096, 8192, 16384};

// Milliseconds of the recorded launches whose name starts with `prefix`
// (waits for them); clears the record.
double prof_take(etx_ctx* ctx, const char* prefix) {
  double ms = 0.0;
  const size_t n = std::strlen(prefix);
  for (size_t i = 0; i < ctx->prof_used; ++i) {
    const ProfRec& r = ctx->prof[i];
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
      return -1.0;
    if (std::strncmp(r.name, prefix, n) == 0) ms += t;
  }
  ctx->prof_used = 0;
  return ms;
}

}  // namespace

extern "C" {

etx_status etx_autotune(etx_ctx* ctx, const float* x, const float* y, const float* z,
                        const int8_t* plane, const int32_t* hit_offsets, int32_t n_events,
                        int64_t n_hits, float radius, int32_t k_max, etx_dtype dtype, float* emb,
                        int32_t* src, int32_t* dst, int64_t edge_capacity, int32_t* edge_offsets,
                        float* logits, void* stream) {
  if (!ctx) return ETX_ERR_ARG;
  etx_status st = etx_embed(ctx, x, y, z, n_hits, emb, stream);
  if (st != ETX_OK) return st;
  const bool prof_was = ctx->prof_on;
  ctx->prof_on = true;
  ctx->prof_used = 0;
  constexpr int kReps = 2;
  // k-NN: blocks per (event, plane) x candidate stage per block
  double best = 1e300;
  int best_split = ctx->knn_split, best_stage = ctx->knn_stage;
  for (int stage : kKnnStages) {
    for (int split : kKnnSplits) {
      ctx->knn_split = split;
      ctx->knn_stage = stage;
      double ms = 0.0;
      for (int r = 0; r <= kReps && st == ETX_OK; ++r) {
        st = etx_build_graph(ctx, emb, plane, hit_offsets, n_events, n_hits, radius, k_max, src,
                             dst, edge_capacity, edge_offsets, stream);
        const double t = prof_take(ctx, "graph_knn");
        if (t < 0) st = fail(ctx, ETX_ERR_CUDA, "autotune timing");
        if (r > 0) ms += t;  // the first run warms up
      }
      if (st != ETX_OK) break;
      if (ms < best) {
        best = ms;
        best_split = split;
        best_stage = stage;
      }
    }
    if (st != ETX_OK) break;
  }
  ctx->knn_split = best_split;
  ctx->knn_stage = best_stage;
  if (st == ETX_OK)
    st = etx_build_graph(ctx, emb, plane, hit_offsets, n_events, n_hits, radius, k_max, src, dst,
                         edge_capacity, edge_offsets, stream);
  // tensor-core MLP kernels: ring slots per block
  if (st == ETX_OK && dtype != ETX_F32) {
    const int f8 = dtype == ETX_FP8E4M3 ? 1 : 0;
    const char* suffix = f8 ? "_fp8" : "_bf16";
    constexpr int NV = 4;  // ring slots 2 .. 5
    double ms[NV][4] = {};
    for (int v = 0; v < NV && st == ETX_OK; ++v) {
      for (int m = 0; m < 4; ++m) ctx->tc_stages[m][f8] = 2 + v;
      for (int r = 0; r <= kReps && st == ETX_OK; ++r) {
        st = etx_gnn_forward(ctx, x, y, z, n_hits, src, dst, edge_offsets, n_events, dtype, logits,
                             stream);
        for (int m = 0; m < 4 && st == ETX_OK; ++m) {
          const std::string name = std::string("gnn_") + kTcBlock[m] + suffix;
          double t = 0.0;
          for (size_t i = 0; i < ctx->prof_used; ++i) {
            const ProfRec& rec = ctx->prof[i];
            float e = 0.f;
            if (cudaEventSynchronize(rec.b) != cudaSuccess ||
                cudaEventElapsedTime(&e, rec.a, rec.b) != cudaSuccess) {
              st = fail(ctx, ETX_ERR_CUDA, "autotune timing");
              break;
            }
            if (name == rec.name) t += e;
          }
          if (r > 0) ms[v][m] += t;
        }
        ctx->prof_used = 0;
      }
    }
    for (int m = 0; m < 4; ++m) {
      int best_v = 0;
      for (int v = 1; v < NV; ++v)
        if (ms[v][m] < ms[best_v][m]) best_v = v;
      ctx->tc_stages[m][f8] = 2 + best_v;
    }
    if (st == ETX_OK)
      st = etx_gnn_forward(ctx, x, y, z, n_hits, src, dst, edge_offsets, n_events, dtype, logits,
                           stream);
  }
  ctx->prof_on = prof_was;
  ctx->prof_used = 0;
  if (st == ETX_OK) {
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "autotune");
  }
  return st;
}

int32_t etx_tuned(const etx_ctx* ctx, const char* knob) {
  if (!ctx || !knob) return -1;
  const std::string k(knob);
  if (k == "knn_split") return ctx->knn_split;
  if (k == "knn_stage") return ctx->knn_stage;
  for (int m = 0; m < 4; ++m)
    for (int f8 = 0; f8 < 2; ++f8)
      if (k == std::string("tc_stages/") + kTcBlock[m] + (f8 ? "/fp8" : "/bf16"))
        return ctx->tc_stages[m][f8];
  return -1;
}

etx_status etx_set_tuned(etx_ctx* ctx, const char* knob, int32_t value) {
  if (!ctx) return ETX_ERR_ARG;
  if (!knob) return fail(ctx, ETX_ERR_ARG, "knob name is NULL");
  const std::string k(knob);
  if (k == "knn_split") {
    if (value != 1 && value != 2 && value != 4) return fail(ctx, ETX_ERR_ARG, "knn_split must be 1, 2 or 4");
    ctx->knn_split = value;
    return ETX_OK;
  }
  if (k == "knn_stage") {
    if (std::find(std::begin(kKnnStages), std::end(kKnnStages), value) == std::end(kKnnStages))
      return fail(ctx, ETX_ERR_ARG, "knn_stage must be 1024, 2048, 4096, 8192 or 16384");
    ctx->knn_stage = value;
    return ETX_OK;
  }
  for (int m = 0; m < 4; ++m)
    for (int f8 = 0; f8 < 2; ++f8)
      if (k == std::string("tc_stages/") + kTcBlock[m] + (f8 ? "/fp8" : "/bf16")) {
        if (value < 2 || value > 5) return fail(ctx, ETX_ERR_ARG, "tc_stages must be 2 to 5");
        ctx->tc_stages[m][f8] = value;
        return ETX_OK;
      }
  return fail(ctx, ETX_ERR_ARG, "unknown knob");
}

}  // extern "C"
