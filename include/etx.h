/*
 * etx.h -- C ABI of the GB300 (sm_103a) ETX4VELO track-finding hot path.
 *
 * One batch = B events of uneven size, concatenated.  Hits are given as
 * structure-of-arrays float32 x, y, z plus an int8 plane index, and
 * hit_offsets[B+1] (event b owns hits [hit_offsets[b], hit_offsets[b+1])).
 * Inside an event, hits must be sorted by plane (non-decreasing).
 *
 * Pipeline (paper Sec. 5 and Sec. 7; the triplet stage is not on it, as in
 * the paper's own C++/CUDA port):
 *   etx_embed            hit embedding MLP                     (Sec. 5.1)
 *   etx_build_graph      radius-capped k-NN graph p -> p+1, p+2 (Eq. 1, Sec. 5.1, Sec. 7.2)
 *   etx_gnn_forward      interaction network edge logits       (Sec. 5.2, Eq. 4)
 *   etx_gnn_backward     gradient of the network parameters    (Sec. 5.2, Eq. 5)
 *   etx_edges_to_tracks  threshold + connected components      (Sec. 5, Sec. 7.3)
 *
 * Around it: training (etx_weighted_bce, etx_adam_step; the embedding's
 * training set, hinge loss and reverse pass, Sec. 5.1, Eq. 2-3), the paper's
 * plane-sweep labelling for comparison (etx_edges_to_tracks_sweep, Sec. 7.3),
 * the Table 1 metrics on truth (etx_track_metrics, Sec. 6), triplets and
 * their classifiers (etx_build_triplets, etx_classify_triplets, Sec. 5.3),
 * and the launch-configuration autotuner (etx_autotune).
 *
 * Conventions shared by every entry point
 *  - All array arguments are DEVICE pointers owned by the caller unless a
 *    comment says "host".  The library never frees caller memory.
 *  - Every call is asynchronous on the given stream (NULL = legacy default
 *    stream) and performs no host synchronisation, except etx_ctx_sync.
 *  - Host-detectable argument errors return a non-zero etx_status before
 *    anything is launched; the message is in etx_last_error().
 *  - Data-dependent errors found on the device (unsorted planes, edges out of
 *    order, capacity overflow, an iteration cap hit) are recorded in a device
 *    error word owned by the context; the kernels that detect them skip the
 *    offending work (never trap), and etx_ctx_sync() returns the status.
 *  - Indices (src, dst) are batch-global int32 hit indices.  Track labels
 *    are event-local.
 *  - A context is bound to one device and is not thread-safe; calls that
 *    share a context must be issued on one stream (they share scratch).
 */
#ifndef ETX_H
#define ETX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum etx_status {
  ETX_OK = 0,
  ETX_ERR_ARG = 1,          /* bad pointer, size, shape or configuration          */
  ETX_ERR_UNSORTED = 2,     /* hits not plane-sorted, plane out of range, or edges
                               not sorted by source / out of range                */
  ETX_ERR_CAPACITY = 3,     /* an output or context buffer is too small           */
  ETX_ERR_CUDA = 4,         /* a CUDA runtime call failed                          */
  ETX_ERR_TIMEOUT = 5,      /* a bounded device loop reached its iteration cap     */
  ETX_ERR_UNSUPPORTED = 6,  /* shape or dtype not supported by this build          */
  ETX_ERR_STATE = 7         /* weights not loaded, or saved activations missing    */
} etx_status;

/* Arithmetic type of the interaction-network GEMMs.  Accumulation, LayerNorm,
 * message sums and logits are FP32 in every mode; so are the residual streams
 * h and e, except in ETX_BF16_EDGE_STORE, which runs the BF16 GEMMs and stores
 * the edge stream e in BF16 (each residual edge update is added in FP32 and
 * the sum rounded to BF16 where it is written): half the bytes of the
 * dominant edge traffic, at the cost of that extra rounding.  Inference only
 * (train contexts reject it); after such a forward the final edge encodings
 * are BF16, so etx_classify_triplets refuses them (ETX_ERR_STATE). */
typedef enum etx_dtype {
  ETX_F32 = 0,
  ETX_BF16 = 1,
  ETX_FP8E4M3 = 2,
  ETX_BF16_EDGE_STORE = 3
} etx_dtype;

#define ETX_MAX_EMB_LAYERS 8

/* Model shapes and context capacities. */
typedef struct etx_config {
  int32_t emb_depth;                           /* Linear layers of the embedding MLP      */
  int32_t emb_widths[ETX_MAX_EMB_LAYERS + 1];  /* widths[0] = 3 ... widths[depth] = D     */
  int32_t hidden;                              /* n_h = n_e = H: 16, 32, 64 or 128         */
  int32_t n_iters;                             /* message-passing steps L >= 0             */
  int32_t n_planes;                            /* detector planes (26)                    */
  int32_t max_events;                          /* capacity: events per call               */
  int64_t max_hits;                            /* capacity: hits per call (< 2^31)        */
  int64_t max_edges;                           /* capacity: edges per call (< 2^31)       */
  int32_t train;                               /* nonzero: keep per-step activations for
                                                  etx_gnn_backward                        */
  int32_t uf_iter_cap;                         /* iteration cap of every union-find loop in
                                                  etx_edges_to_tracks (each find, and each
                                                  hook attempt of an edge); 0 = the
                                                  default (2^22 find steps, 2^20 hook
                                                  attempts).  Reaching it leaves the
                                                  labels unspecified and makes
                                                  etx_ctx_sync return ETX_ERR_TIMEOUT  */
} etx_config;

typedef struct etx_ctx etx_ctx;

/* Create a context on `device`: validates `cfg`, allocates every scratch
 * buffer for the given capacities (cudaMalloc; nothing is allocated later),
 * and records the SM count for persistent-grid sizing.  On failure *out is
 * NULL and the status says why. */
etx_status etx_ctx_create(const etx_config* cfg, int32_t device, etx_ctx** out);

/* Free the context and its device memory.  NULL is accepted. */
etx_status etx_ctx_destroy(etx_ctx* ctx);

/* Last error message of this context (static string when ctx is NULL). */
const char* etx_last_error(const etx_ctx* ctx);

/* Number of float32 values of the weight blob for `cfg` (or -1 if invalid).
 * Blob order: normalisation (emb mu[3], sigma[3], gnn mu[3], sigma[3]),
 * embedding layers (W[out][in], b[out]) ..., then the interaction network:
 * node encoder, edge encoder, L x (node net, edge net), each block as
 * W1[H][K] b1 g1 be1 W2[H][H] b2 g2 be2, and the classifier W1[H][H] b1 g1
 * be1 W2[1][H] b2[1]. */
int64_t etx_weights_size(const etx_config* cfg);

/* Copy a HOST weight blob of `n_floats` values into the context (device
 * repacking for every arithmetic type).  Synchronous. */
etx_status etx_load_weights(etx_ctx* ctx, const float* host_blob, int64_t n_floats);

/* Replace the interaction-network parameters with a DEVICE vector theta
 * (float32, etx_gnn_param_count(cfg) values in the blob's order from the node
 * encoder on; the layout etx_gnn_backward writes its gradient in), e.g. after
 * an etx_adam_step on the device: the context's FP32 weights and BF16
 * tensor-core images are rebuilt by a kernel on `stream` (no host round trip
 * of the weights; the few values the tensor-core kernels take by value come
 * back through an asynchronous copy that the next etx_gnn_forward waits for).
 * The e4m3 images are not rebuilt: ETX_FP8E4M3 returns ETX_ERR_STATE until
 * the next etx_load_weights.  A pending etx_gnn_backward is invalidated.  No
 * counterpart in the paper beyond "trained". */
etx_status etx_set_gnn_params(etx_ctx* ctx, const float* theta, void* stream);

/* Wait for `stream`, then return and clear the context's device error word
 * (ETX_OK if no kernel recorded an error). */
etx_status etx_ctx_sync(etx_ctx* ctx, void* stream);

/*
 * Hit embedding (Sec. 5.1): e_h = MLP((r, phi, z) normalised), r = sqrt(x^2 +
 * y^2), phi = atan2(y, x); hidden layers Linear -> ReLU, bare last Linear.
 *   x, y, z   float32 [n_hits]
 *   emb       float32 [n_hits][D] row-major, written
 * FP32 throughout.
 */
etx_status etx_embed(etx_ctx* ctx, const float* x, const float* y, const float* z,
                     int64_t n_hits, float* emb, void* stream);

/*
 * Rough graph (Eq. 1, Sec. 5.1, Sec. 7.2): for each hit i on plane p, the
 * hits j of the same event on planes p+1 and p+2 with
 *     d2(i, j) = sum_d (e_i,d - e_j,d)^2 < radius^2
 * (evaluated in FP32, one rounding per operation, dimensions in index order,
 * r^2 = radius * radius rounded to FP32); if more than k_max qualify, the
 * k_max smallest by (d2, j) are kept.  Edges i -> j are written sorted by
 * (i, j), so events are contiguous.
 *   emb          float32 [n_hits][D]
 *   plane        int8 [n_hits], 0 <= plane < n_planes, sorted within each event
 *   hit_offsets  int32 [n_events + 1] (device)
 *   src, dst     int32 [edge_capacity], written ([0, n_edges) valid)
 *   edge_offsets int32 [n_events + 1], written: edges of event b are
 *                [edge_offsets[b], edge_offsets[b+1]); n_edges = edge_offsets[n_events]
 * If the edges do not fit, ETX_ERR_CAPACITY is recorded on the device, src/dst
 * are left unwritten and edge_offsets still holds the required counts.
 * edge_capacity >= n_hits * k_max can never overflow.  When n_hits * k_max
 * fits the context's max_edges, one distance pass writes each source's kept
 * edges to fixed slots in context scratch and a compaction forms the list;
 * otherwise a counting pass precedes the emitting pass.  Same result.
 */
etx_status etx_build_graph(etx_ctx* ctx, const float* emb, const int8_t* plane,
                           const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                           float radius, int32_t k_max, int32_t* src, int32_t* dst,
                           int64_t edge_capacity, int32_t* edge_offsets, void* stream);

/*
 * Interaction network (Sec. 5.2, Eq. 4): node encoder on (x, y, z)
 * normalised, edge encoder on [h_i, h_j], then L steps of
 *     m_l = [sum_{l->j} e_lj, sum_{i->l} e_il]
 *     h  <- h + node_net_k([h, m])          (distinct weights per step)
 *     e  <- e + edge_net_k([e, h_i, h_j])   (with the updated h)
 * and the edge classifier; writes one FP32 logit per edge.
 *   src, dst     int32 [>= n_edges]: src non-decreasing (as etx_build_graph writes)
 *   edge_offsets int32 [n_events + 1]: only edge_offsets[n_events] (= n_edges)
 *                is read, on the device, so the call needs no host sync
 *   logits       float32 [>= n_edges], written
 * With cfg.train set, the per-step encodings are kept in the context for
 * etx_gnn_backward.
 */
etx_status etx_gnn_forward(etx_ctx* ctx, const float* x, const float* y, const float* z,
                           int64_t n_hits, const int32_t* src, const int32_t* dst,
                           const int32_t* edge_offsets, int32_t n_events, etx_dtype dtype,
                           float* logits, void* stream);

/*
 * Static per-tensor activation scales of the e4m3 path (ETX_FP8E4M3; the
 * paper calibrates its INT8 quantisation on simulated events, Sec. 7.4).
 * Each matrix-product operand x of the interaction network enters the
 * tensor cores as e4m3(x / s) and the accumulator is multiplied back by s
 * (and by the weight's own amax / 448 scale); s is a power of two, so the
 * scaling itself is exact and only moves e4m3's range (saturation at 448 s,
 * subnormals below 2^-6 s).  One scale covers a whole concatenated block
 * input ([e, h_i, h_j] or [h, m_out, m_in]).  Order, n = 4 L + 3 values:
 *   edge encoder input, edge encoder second-layer input,
 *   for k = 0 .. L-1: node net k input, its second-layer input,
 *                     edge net k input, its second-layer input,
 *   classifier input.
 * host_scales is a HOST array, copied; (NULL, 0) restores the default (all
 * 1).  ETX_ERR_ARG for a wrong count or a value that is not a power of two
 * in [2^-100, 2^100].  BF16 and FP32 ignore the scales.  Takes effect for
 * the next etx_gnn_forward.
 */
int64_t etx_fp8_scale_count(const etx_config* cfg);
etx_status etx_set_fp8_scales(etx_ctx* ctx, const float* host_scales, int64_t n);

/*
 * Reverse pass of the last etx_gnn_forward of this context (train contexts
 * only): given dlogits = dLoss/dlogit [n_edges], writes dparams, float32 in
 * the blob's interaction-network order, starting at the node encoder (the
 * normalisation and embedding entries are not part of it); its length is
 * etx_gnn_param_count(cfg).  Message-passing steps are recomputed from the
 * kept per-step encodings (checkpointing).  Arithmetic: for hidden width 128
 * the edge encoder, node and edge updates run on the tensor cores in TF32 (the
 * recomputed forward products split into high and low TF32 parts, within FP32
 * rounding of the exact products; the input-gradient products single TF32)
 * and every weight gradient in TF32 with FP32 accumulation; the node encoder,
 * the classifier and other widths use FP32 SIMT.  Every sum is formed in a
 * fixed order: the same inputs give the same bits.  The pass reads the edge index
 * that the forward built; etx_build_graph (single-pass k-NN),
 * etx_build_triplets and etx_edges_to_tracks_sweep reuse that scratch, so
 * after one of them on this context the backward returns ETX_ERR_STATE until
 * the next training forward.  The forward's input arrays (x, y, z, src, dst)
 * are read again by the backward: they must stay allocated and unchanged until
 * it has run (the caller owns them; the context keeps only their addresses).
 */
int64_t etx_gnn_param_count(const etx_config* cfg);
etx_status etx_gnn_backward(etx_ctx* ctx, const float* dlogits, float* dparams, void* stream);

/* The residual streams that the last training forward kept (train contexts):
 * h^k float32 [n_hits][H] and e^k float32 [n_edges][H] of step k (0 = after
 * the encoders, n_iters = final), copied to caller-owned device buffers (either
 * may be NULL).  These are the checkpoints etx_gnn_backward recomputes from;
 * exposed to check the reverse pass against an independent one on the same
 * inputs.  ETX_ERR_STATE without a training forward, ETX_ERR_ARG for k out of
 * range.  Asynchronous on `stream`. */
etx_status etx_gnn_checkpoints(etx_ctx* ctx, int32_t k, float* h_out, float* e_out, void* stream);

/*
 * Training loss: the edge term of Eq. 5 read as class-weighted binary cross
 * entropy on the logits (the paper uses a sigmoid focal loss; this build's
 * training workload asks for BCE with a positive-class weight):
 *     loss = mean_e [ w y_e softplus(-z_e) + (1 - y_e) softplus(z_e) ]
 * over the n_edges = edge_offsets[n_events] edges (read on the device).
 *   targets  float32 [n_edges], 1 for genuine edges, 0 otherwise
 *   loss     float32 [1], written
 *   dlogits  float32 [n_edges], written: d loss / d z_e
 */
etx_status etx_weighted_bce(etx_ctx* ctx, const float* logits, const float* targets,
                            const int32_t* edge_offsets, int32_t n_events, float pos_weight,
                            float* loss, float* dlogits, void* stream);

/*
 * The paper's own edge loss (Sec. 5.2, Eq. 5): the sigmoid focal loss of its
 * reference (Lin et al. 2017), p = sigmoid(z),
 *     loss = mean_e [ y alpha (1 - p)^gamma (-log p)
 *                     + (1 - y) (1 - alpha) p^gamma (-log(1 - p)) ]
 * (the paper gives no alpha or gamma; 0.25 and 2 are the reference's
 * defaults).  Arguments, layouts and errors as etx_weighted_bce; alpha in
 * [0, 1], gamma >= 0, else ETX_ERR_ARG.  The loss is summed per block and the
 * block sums added in a fixed order.
 */
etx_status etx_focal_loss(etx_ctx* ctx, const float* logits, const float* targets,
                          const int32_t* edge_offsets, int32_t n_events, float alpha, float gamma,
                          float* loss, float* dlogits, void* stream);

/*
 * One Adam update (Kingma & Ba) of n float32 parameters in place, with
 * bias-corrected moments; m and v are caller-owned state (zero before step 1),
 * step counts from 1.  No counterpart in the paper's text beyond "trained".
 */
etx_status etx_adam_step(etx_ctx* ctx, float* params, const float* grads, float* m, float* v,
                         int64_t n, float lr, float beta1, float beta2, float eps, int64_t step,
                         void* stream);

/*
 * Purified hit graph and tracks (Sec. 5, Sec. 7.3): keep edge e iff
 * logits[e] > threshold_logit (score > sigmoid(threshold_logit); 0.0f is the
 * paper's 0.5), then weakly connected components by lock-free union-find.
 *   labels      int32 [n_hits], written: smallest event-local hit index of the
 *               hit's component (a hit with no kept edge labels itself)
 *   n_tracks    int32 [n_events] or NULL: number of components per event with
 *               at least `min_hits` hits
 */
etx_status etx_edges_to_tracks(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                               const float* logits, float threshold_logit,
                               const int32_t* edge_offsets, const int32_t* hit_offsets,
                               int32_t n_events, int64_t n_hits, int32_t min_hits,
                               int32_t* labels, int32_t* n_tracks, void* stream);

/*
 * Allocation-free components (the paper has no counterpart to this call).
 *
 * Same result as etx_edges_to_tracks, but the call needs no context and
 * never allocates device memory: no cudaMalloc, no cudaFree, no allocating
 * library routine.  It is meant for callers that cannot allocate, such as a
 * host framework that reserves the whole device-memory budget at start-up
 * and hands out slices itself, or a real-time event loop where an
 * allocation (which can synchronise the device) is not allowed.  The caller
 * still passes every input and output array, as for etx_edges_to_tracks.
 *
 * Scratch: a file-scope device array of the library holding 2^21 hit slots
 * (8 MiB plus an error word), present on every GPU that loads the library
 * until the process exits.  n_hits above 2^21 returns ETX_ERR_CAPACITY
 * before anything is launched.  The first call on a device looks the
 * array's device address up (cudaGetSymbolAddress, on the current device)
 * and caches it, so make that first call before any stream capture.  Every
 * call re-initialises the part of the array it uses, but all calls share
 * it: calls that overlap on the GPU (different streams or devices sharing a
 * context's memory) race and give wrong labels.  Runs on the current device
 * and the given stream; asynchronous.  The union-find loops carry the
 * default iteration caps of etx_edges_to_tracks, and there is no context to
 * report to, so device-side problems come back through `status`.
 *   status   int32 [1] (device) or NULL: once the call's kernels have run it
 *            holds ETX_OK, ETX_ERR_TIMEOUT (a union-find iteration cap was
 *            reached: labels unspecified) or ETX_ERR_UNSORTED (an edge index
 *            outside [0, n_hits) was skipped).  The array's error word is
 *            cleared at the start of every call, so `status` describes this
 *            call alone.
 * The return value covers host-side checks and launch failures of this
 * call's own kernels.
 */
etx_status etx_edges_to_tracks_noalloc(const int32_t* src, const int32_t* dst,
                                       const float* logits, float threshold_logit,
                                       const int32_t* edge_offsets, const int32_t* hit_offsets,
                                       int32_t n_events, int64_t n_hits, int32_t min_hits,
                                       int32_t* labels, int32_t* n_tracks, int32_t* status,
                                       void* stream);

/*
 * The paper's own track-building kernel (Sec. 7.3), for comparison with
 * etx_edges_to_tracks: a plane-ordered propagation of minimum labels.  Every
 * hit starts with its own index; forward, for planes 1 .. n_planes-1 in turn,
 * each hit of the plane takes the smallest label among itself and the hits
 * that its kept incoming edges (logit > threshold_logit) come from; backward,
 * for planes n_planes-2 .. 0 in turn, each hit takes the smallest label among
 * itself and the hits its kept outgoing edges go to.  This is not an exact
 * connected-components algorithm (one component can end with several
 * labels); labels[i] is the event-local index of a hit of the same component.
 * Needs plane (int8 [n_hits], ascending within each event) and edges sorted by
 * (src, dst) as etx_build_graph writes them; edge_offsets[n_events] is the
 * edge count.  Errors as etx_edges_to_tracks; unsorted planes or edges are
 * reported by etx_ctx_sync.  Asynchronous on `stream`.
 */
etx_status etx_edges_to_tracks_sweep(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                     const float* logits, float threshold_logit,
                                     const int32_t* edge_offsets, const int8_t* plane,
                                     const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                                     int32_t* labels, void* stream);

/*
 * Triplets (Sec. 5.3) of the kept edges (logit > threshold_logit) and their
 * two classifiers; etx_tracks_from_triplets (below) builds the tracks of
 * Sec. 5.4 from them.
 *
 * etx_build_triplets: every pair of kept edges sharing a hit C, as
 *   articulation  A->C, C->B   (kind 0; first = the edge into C)
 *   left elbow    C->A, C->B   (kind 1; first < second)
 *   right elbow   A->C, B->C   (kind 2; first < second)
 * written type-major (all articulations, then left, then right elbows), by
 * C, then first, then second: first, second int32 [capacity] edge indices,
 * kind int8 [capacity]; counts int32 [4] (device) = {total, articulations,
 * left elbows, right elbows}.  Edges sorted by (src, dst) as etx_build_graph
 * writes them, edge_offsets[n_events] = edge count.  workspace: at least
 * etx_triplets_workspace() bytes, 4-byte aligned, caller-owned scratch.
 * Rebuilds the context's edge index structures for these edges (the final
 * edge encodings of the last etx_gnn_forward are kept).  More triplets than
 * `capacity`: ETX_ERR_CAPACITY at etx_ctx_sync and counts all 0.
 *
 * etx_load_triplet_weights: HOST blob of etx_triplet_weights_size() floats:
 * articulation classifier then elbow classifier, each W1[H][2H] b1[H]
 * g1[H] be1[H] W2[1][H] b2[1] (Lin -> LN -> ReLU -> Lin).  Synchronous.
 *
 * etx_classify_triplets: logits float32 [capacity] (rows [0, counts[0])
 * written) of the triplets from etx_build_triplets, on [e_first, e_second]
 * of the final edge encodings of the last etx_gnn_forward of this context
 * (FP32 SIMT, any dtype of that forward).  Articulations use the first
 * classifier, elbows the second.
 */
int64_t etx_triplet_weights_size(const etx_config* cfg);
etx_status etx_load_triplet_weights(etx_ctx* ctx, const float* host_blob, int64_t n_floats);
size_t etx_triplets_workspace(int64_t n_hits);
etx_status etx_build_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                              const float* logits, float threshold_logit,
                              const int32_t* edge_offsets, int32_t n_events, int64_t n_hits,
                              void* workspace, size_t workspace_bytes, int32_t* first,
                              int32_t* second, int8_t* kind, int64_t capacity, int32_t* counts,
                              void* stream);
etx_status etx_classify_triplets(etx_ctx* ctx, const int32_t* first, const int32_t* second,
                                 const int32_t* counts, int64_t capacity, float* logits,
                                 void* stream);

/*
 * Track building on the purified edge graph (Sec. 5.4): tracks that may
 * share hits (e+e- pairs share their first hits).  The graph's nodes are the
 * kept edges (logits > threshold_logit), its links the kept triplets
 * (triplet_logits > triplet_threshold) of the list etx_build_triplets wrote
 * for the same edges and threshold_logit.  Four steps, as read here (the
 * paper gives them in prose and a figure):
 *   1. at each hit C, kept edges into C joined by kept right elbows form a
 *      group, and so do kept edges out of C joined by kept left elbows; an
 *      articulation (i, o) at C is present when a kept articulation links
 *      i's group to o's group (an elbow's two edges share their
 *      continuations through C; an articulation implied twice counts once);
 *   2. a present articulation (i, o) is shared when i has two or more
 *      present articulations at C, or o has (a fork or a merge); weakly
 *      connected components are formed over the kept edges linked by the
 *      present, unshared articulations;
 *   3. every component that no shared articulation touches is a track, and
 *      every shared articulation (i, o) is a track of its own: the union of
 *      i's and o's components (the shared part is duplicated);
 *   4. a track's hits are the end points of its edges; tracks with fewer
 *      than min_hits hits are dropped.
 * Output: track_offsets int32 [track_capacity + 1] and track_hits int32
 * [hit_capacity] (batch-global hit indices, ascending within a track) as a
 * CSR of n_out[0] tracks and n_out[1] hits (n_out: int32 [2], device): first
 * the components in order of their smallest edge index, then the shared
 * articulations in list order.  Tracks never span events.
 *   first, second  int32 [triplet_capacity], counts int32 [4]: the output of
 *                  etx_build_triplets (its capacity as triplet_capacity)
 *   triplet_logits float32 [triplet_capacity]: etx_classify_triplets' output
 *   workspace      >= etx_tracks_workspace(n_hits, max_edges of the context,
 *                  triplet_capacity) bytes, 4-byte aligned, caller-owned
 * More than 64 kept edges into or out of one hit: that hit's articulations
 * are dropped and etx_ctx_sync reports ETX_ERR_CAPACITY, as it does for a
 * component of more than 8,192 hits (whose hits are then left unsorted;
 * a component never spans events); a triplet list that
 * does not belong to these edges is reported as ETX_ERR_UNSORTED; more
 * tracks or hits than the capacities: ETX_ERR_CAPACITY and n_out = {0, 0}.
 * Rebuilds the context's edge index (as etx_build_triplets does).
 * Asynchronous on `stream`.
 */
size_t etx_tracks_workspace(int64_t n_hits, int64_t max_edges, int64_t triplet_capacity);
etx_status etx_tracks_from_triplets(etx_ctx* ctx, const int32_t* src, const int32_t* dst,
                                    const float* logits, float threshold_logit,
                                    const int32_t* edge_offsets, int32_t n_events,
                                    int64_t n_hits, const int32_t* first, const int32_t* second,
                                    const float* triplet_logits, float triplet_threshold,
                                    const int32_t* counts, int64_t triplet_capacity,
                                    int32_t min_hits, void* workspace, size_t workspace_bytes,
                                    int32_t* track_offsets, int32_t* track_hits,
                                    int64_t track_capacity, int64_t hit_capacity,
                                    int32_t* n_out, void* stream);

/*
 * Training of the hit embedding (Sec. 5.1, Eq. 2-3).  A step is
 *   etx_embed_forward_train -> etx_embedding_pairs -> etx_hinge_loss ->
 *   etx_embed_backward -> etx_adam_step on the embedding parameters ->
 *   etx_set_embed_params (on the device; etx_load_weights with a host blob
 *   does the same through the host).
 * The batch has its noise hits removed (Sec. 5.1), hits plane-sorted per
 * event as everywhere.
 *
 * etx_embed_param_count: number of embedding parameters, in blob order
 * (W[out][in], b[out] per layer; they follow the 12 normalisation values of
 * the blob), or -1 for an invalid config.
 *
 * etx_embed_forward_train: etx_embed that also keeps, in `workspace` (at
 * least etx_embed_train_workspace() bytes, 16-byte aligned, owned by the
 * caller), the normalised inputs and every hidden layer's activations for
 * etx_embed_backward.  emb float32 [n_hits][D] is written.
 *
 * etx_embed_backward: d_params float32 [etx_embed_param_count] receives
 * dL/dtheta for the upstream gradient d_emb float32 [n_hits][D], through the
 * activations that the last etx_embed_forward_train of the same n_hits and
 * weights left in `workspace` (the rest of the workspace is scratch).  The
 * weights are read from the context's copy of the blob.  FP32 SIMT; the
 * weight gradients and bias sums are formed as per-split partials in the
 * workspace's tail and added in a fixed order (the same d_emb gives the same
 * bits).
 *
 * etx_embedding_pairs: the training set T (Sec. 5.1).  For each query q (a
 * hit whose particle has at least min_hits hits in its event) on plane p,
 * partners on planes p+1 and p+2 of the event: the pairs of the graph rule
 * (etx_build_graph with `radius` and `k_max`: hard negatives), one random
 * partner (the (rand[q] mod c)-th of the c hits on p+1 and p+2, in index
 * order; rand uint32 [n_hits] is an input), and the genuine edge q -> next
 * hit of q's particle when it lies on p+1 or p+2.  The union is written
 * sorted by (q, a): pair_q, pair_a int32 [capacity] batch-global hit
 * indices, pair_genuine uint8 [capacity] (1 iff a is the next hit of q's
 * particle); n_pairs int32 (device) receives the count.
 *   particle_id  int32 [n_hits], event-local in [0, hits of the event), no
 *                noise (-1 is reported by etx_ctx_sync as out of range)
 *   workspace    at least etx_embedding_pairs_workspace() bytes, 4-byte
 *                aligned, caller-owned scratch
 * Uses the context's graph scratch (so n_events and n_hits within its
 * capacity).  More pairs than `capacity`: ETX_ERR_CAPACITY at etx_ctx_sync and
 * n_pairs = 0.  Asynchronous on `stream`.
 *
 * etx_hinge_loss: Eq. 2-3 over the n_pairs (device) pairs: loss float32 [3]
 * (device) = {L_fake + w_genuine * L_genuine, L_genuine, L_fake}, L_genuine
 * = mean d2 over genuine pairs, L_fake = mean max(0, margin - d2) over fake
 * pairs (an empty set contributes 0; the hinge is inactive at d2 = margin);
 * d_emb float32 [n_hits][D] = dL/d emb (every row overwritten).  No atomics
 * on floating point: each hit's gradient is summed over its pairs as query,
 * then as partner, each in ascending pair index, and the loss from per-block
 * FP64 sums added in block order, so the same inputs on the same context
 * give the same bits.  pair_capacity bounds n_pairs and sizes the grid and
 * the workspace (at least etx_hinge_loss_workspace(n_hits, pair_capacity)
 * bytes of device scratch, 16-byte aligned, owned by the caller); n_pairs
 * outside [0, pair_capacity] is reported as ETX_ERR_CAPACITY by etx_ctx_sync
 * and no pair is used.  n_hits <= the context's max_hits.  D <= 16.
 * Indices outside [0, n_hits) are skipped and reported by etx_ctx_sync.
 */
int64_t etx_embed_param_count(const etx_config* cfg);
size_t etx_embed_train_workspace(const etx_config* cfg, int64_t n_hits);
etx_status etx_embed_forward_train(etx_ctx* ctx, const float* x, const float* y, const float* z,
                                   int64_t n_hits, float* emb, void* workspace,
                                   size_t workspace_bytes, void* stream);
etx_status etx_embed_backward(etx_ctx* ctx, int64_t n_hits, const float* d_emb, float* d_params,
                              void* workspace, size_t workspace_bytes, void* stream);

/* The embedding's parameters (Sec. 5.1) replaced from a device vector theta
 * float32 [etx_embed_param_count] in blob order (W[out][in], b[out] per layer),
 * e.g. after an optimiser step: the context's transposed FP32 copies are
 * rebuilt from it by one kernel and its copy of the blob updated, all on
 * `stream` (asynchronous; no host round trip).  Later etx_embed,
 * etx_embed_forward_train and etx_embed_backward see the new weights.
 * ETX_ERR_STATE before etx_load_weights, ETX_ERR_ARG for a NULL vector. */
etx_status etx_set_embed_params(etx_ctx* ctx, const float* theta, void* stream);
size_t etx_embedding_pairs_workspace(int32_t n_events, int64_t n_hits, int32_t k_max);
etx_status etx_embedding_pairs(etx_ctx* ctx, const float* emb, const int8_t* plane,
                               const int32_t* particle_id, const int32_t* hit_offsets,
                               int32_t n_events, int64_t n_hits, float radius, int32_t k_max,
                               const uint32_t* rand, int32_t min_hits, void* workspace,
                               size_t workspace_bytes, int32_t* pair_q, int32_t* pair_a,
                               uint8_t* pair_genuine, int64_t capacity, int32_t* n_pairs,
                               void* stream);
size_t etx_hinge_loss_workspace(int64_t n_hits, int64_t pair_capacity);
etx_status etx_hinge_loss(etx_ctx* ctx, const float* emb, int64_t n_hits, const int32_t* pair_q,
                          const int32_t* pair_a, const uint8_t* pair_genuine,
                          const int32_t* n_pairs, int64_t pair_capacity, float margin,
                          float w_genuine, float* loss, float* d_emb, void* workspace,
                          size_t workspace_bytes, void* stream);

/*
 * Track-finding performance against truth (Sec. 6, Table 1), for evaluating
 * labels on synthetic or simulated events.  A track is a set of hits of one
 * event that share a label; it counts when it has at least min_hits hits.  A
 * particle counts (is reconstructible, Sec. 3) when it has at least min_hits
 * hits.  A track and a particle form a matching candidate when at least
 * match_num / match_den of the track's hits belong to the particle (the
 * paper: 3 hits, 7/10).
 *
 * labels       int32 [n_hits], event-local, each in [0, hits of its event)
 *              (the output of etx_edges_to_tracks or _sweep)
 * particle_id  int32 [n_hits], event-local particle index in [0, hits of its
 *              event), -1 for noise
 * hit_offsets  int32 [n_events + 1], as everywhere
 * workspace    device scratch of at least etx_track_metrics_workspace()
 *              bytes, 8-byte aligned, owned by the caller
 * counts       int64 [6] (device) receives: reconstructible particles,
 *              those with a candidate, candidates, distinct particles among
 *              the candidates, tracks, tracks without a candidate
 * values       double [7] (device) receives: sum over candidates of matched /
 *              particle hits, sum over candidates of matched / track hits,
 *              efficiency, clone rate, fake rate, hit efficiency, hit purity
 *              (the last five are NaN where their denominator is zero)
 *
 * Counts are exact; the FP64 sums are formed in a fixed order (the same
 * inputs give the same bits).  ETX_ERR_ARG for NULL arrays, min_hits < 1, a
 * match fraction outside (1/2, 1] (at most one particle per track) or an
 * unaligned workspace; ETX_ERR_CAPACITY for a small workspace.  Labels or
 * particle ids out of range are skipped and reported by etx_ctx_sync
 * (ETX_ERR_UNSORTED, "an index was out of range").  Asynchronous on `stream`; writes nothing but the workspace
 * and the two outputs.
 */
size_t etx_track_metrics_workspace(int32_t n_events, int64_t n_hits);
etx_status etx_track_metrics(etx_ctx* ctx, const int32_t* labels, const int32_t* particle_id,
                             const int32_t* hit_offsets, int32_t n_events, int64_t n_hits,
                             int32_t min_hits, int32_t match_num, int32_t match_den,
                             void* workspace, size_t workspace_bytes, int64_t* counts,
                             double* values, void* stream);

/*
 * Autotuner (no counterpart in the paper: it picks launch configurations, not
 * results).  Runs the embedding, the graph and (for ETX_BF16 / ETX_FP8E4M3)
 * the interaction network on the given batch, timing with CUDA events each
 * candidate of
 *   "knn_split"                 blocks that share the sources of one
 *                               (event, plane) in the k-NN: 1, 2 or 4
 *                               (per-event work partitioning);
 *   "knn_stage"                 floats of candidate embeddings a k-NN block
 *                               stages in shared memory: 1024, 2048, 4096
 *                               (the default), 8192 or 16384 (an (event,
 *                               plane) whose two candidate planes hold more
 *                               reads them from global memory; a smaller
 *                               stage keeps more blocks resident per SM);
 *   "tc_stages/<block>/<dtype>" A-operand ring slots of the tensor-core MLP
 *                               kernel, 2 to 5 (capped by shared memory),
 *                               for block edge_encoder, node_update,
 *                               edge_update or classifier and dtype bf16 or
 *                               fp8,
 * and keeps the fastest in the context for all later calls.  Outputs do not
 * depend on these choices.  On return emb, src, dst, edge_offsets (and logits
 * for the tensor-core dtypes) hold the results of the chosen configuration,
 * as the regular calls would write them; arguments, layouts and errors are
 * those of etx_embed, etx_build_graph and etx_gnn_forward.  Synchronises the
 * stream (the host waits) and clears any pending profile record.
 * etx_tuned returns the current value of a knob by the names above, or -1;
 * etx_set_tuned sets one (a value outside the candidates above, or an unknown
 * knob, is ETX_ERR_ARG), e.g. to restore a configuration tuned earlier.
 */
etx_status etx_autotune(etx_ctx* ctx, const float* x, const float* y, const float* z,
                        const int8_t* plane, const int32_t* hit_offsets, int32_t n_events,
                        int64_t n_hits, float radius, int32_t k_max, etx_dtype dtype, float* emb,
                        int32_t* src, int32_t* dst, int64_t edge_capacity, int32_t* edge_offsets,
                        float* logits, void* stream);
int32_t etx_tuned(const etx_ctx* ctx, const char* knob);
etx_status etx_set_tuned(etx_ctx* ctx, const char* knob, int32_t value);

/*
 * Instrumentation (no counterpart in the paper; used by the benchmark).
 *   etx_launch_count    number of kernels this context has launched so far.
 *   etx_profile_enable  when on, every kernel launch is bracketed by a CUDA
 *                       event pair recorded on its own stream.
 *   etx_profile_read    synchronises on the recorded events and aggregates
 *                       them by kernel name: names[i] (static strings owned
 *                       by the library), total_ms[i], counts[i]; returns the
 *                       number of entries written (<= max_entries) or -1,
 *                       and clears the record.
 */
int64_t etx_launch_count(const etx_ctx* ctx);
etx_status etx_profile_enable(etx_ctx* ctx, int32_t on);
int32_t etx_profile_read(etx_ctx* ctx, const char** names, double* total_ms, int64_t* counts,
                         int32_t max_entries);

#ifdef __cplusplus
}
#endif

#endif /* ETX_H */
