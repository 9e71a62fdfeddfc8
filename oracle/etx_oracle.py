"""FP64 CPU oracle of the ETX4VELO hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module.  The product path (the CUDA library and its Python
binding) never imports, links or runs it, and this module shares no code
with that path: it depends on numpy and on the seeded input generator
(``velo_synth``) alone.

Every function writes out the definition the paper gives, in FP64, with no
blocking, fusion or reordering beyond what the definition states:

  normalise / embed     Sec. 5.1 (normalised cylindrical inputs, footnote) and
                        the embedding MLP of Sec. 5.1
  d2                    Eq. 1
  build_graph           Sec. 5.1: hits on plane p connect to hits on p+1 and
                        p+2 with d2 below the cut, at most k_max per node
                        (Sec. 7.2 keeps the nearest ones)
  gnn_forward           Sec. 5.2: node and edge encoders, Eq. 4 messages,
                        residual node then edge updates with distinct weights
                        per step, edge classifier
  weighted_bce          the training loss used here for the edge term of Eq. 5
  gnn_backward          reverse-mode derivative of gnn_forward + loss, by hand
  connected_components  weakly connected components of the purified hit graph
                        (Sec. 5 overview, Sec. 7.3), by breadth-first search
  plane_sweep_components  the paper's plane-ordered two-sweep labelling
                        (Sec. 7.3), which is not exact
  track_metrics         the counts behind the Table 1 metrics (Sec. 6):
                        70% matching, efficiency, clone and fake rates, hit
                        efficiency and purity
  embedding_pairs       the embedding's training set (Sec. 5.1): hard
                        negatives from the graph rule, one random pair per
                        query, the genuine edges
  hinge_embedding_loss  Eq. 2-3 and its gradient with respect to the embedding
  embed_backward        reverse pass of the embedding MLP
  build_triplets        articulations and left / right elbows of the purified
                        graph (Sec. 5.3)
  triplet_logits        the articulation and elbow classifiers (Sec. 5.3)

Readings where the paper is silent (also listed in the design notes):
  * radius r is Euclidean: keep d2 < r*r (strict); the k_max cap is joint over
    planes p+1 and p+2 and keeps the smallest (d2, j) pairs;
  * edges point from the lower to the higher plane and are listed by (i, j);
  * every MLP layer of the interaction network is Linear -> LayerNorm(eps
    1e-5, biased variance, affine) -> ReLU, except the classifier's last
    Linear; the embedding MLP is Linear -> ReLU with a bare last Linear;
  * node network input [h, m_out, m_in], edge network input [e, h_i, h_j]
    with the updated h, edge encoder input [h_i, h_j];
  * an edge is kept iff its logit > 0 (score > 0.5);
  * a track label is the smallest event-local hit index of the component;
  * a reconstructed track needs at least three hits, like a reconstructible
    particle (Sec. 3).

Parity of every function is pinned by the non-GPU tests (brute force,
closed forms, invariants, torch float64 cross-checks and finite differences).
"""
from __future__ import annotations

import numpy as np

LN_EPS = 1e-5


# ----------------------------------------------------------------------------
# input features and embedding (Sec. 5.1)
# ----------------------------------------------------------------------------
def cylindrical(x, y, z):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    return np.stack([np.sqrt(x * x + y * y), np.arctan2(y, x), z], axis=1)


def normalise(feat, mu, sigma):
    return (feat - np.asarray(mu, np.float64)) / np.asarray(sigma, np.float64)


def embed(weights, n_layers, x, y, z):
    """Embedding MLP on normalised (r, phi, z): ReLU between layers, bare
    output.  Returns [N, D] float64."""
    a = normalise(cylindrical(x, y, z), weights["emb_mu"], weights["emb_sigma"])
    for i in range(n_layers):
        W = weights[f"emb{i}.W"].astype(np.float64)
        b = weights[f"emb{i}.b"].astype(np.float64)
        a = a @ W.T + b
        if i < n_layers - 1:
            a = np.maximum(a, 0.0)
    return a


# ----------------------------------------------------------------------------
# rough graph (Eq. 1, Sec. 5.1, Sec. 7.2)
# ----------------------------------------------------------------------------
def d2_fp64(ea, eb):
    """Eq. 1 for all pairs: ea [n, D], eb [m, D] -> [n, m]."""
    diff = ea[:, None, :].astype(np.float64) - eb[None, :, :].astype(np.float64)
    return (diff * diff).sum(-1)


def d2_fp32(ea, eb):
    """Eq. 1 evaluated in FP32, one IEEE rounding per operation, summed over
    the embedding dimensions in index order (no fused multiply-add).  This is
    the precision in which the cut and the nearest-k choice are decided when
    both sides start from the same FP32 embedding."""
    ea = np.asarray(ea, np.float32)
    eb = np.asarray(eb, np.float32)
    s = np.zeros((ea.shape[0], eb.shape[0]), np.float32)
    for i in range(ea.shape[1]):
        d = ea[:, None, i] - eb[None, :, i]
        s = s + d * d
    return s


def build_graph(emb, plane, hit_offsets, radius, k_max, precision="fp64"):
    """Per event: for hit i on plane p, candidates j on planes p+1, p+2 with
    d2(i, j) < r^2; keep the k_max smallest by (d2, j); emit edges (i, j)
    sorted by (i, j).  Indices are batch-global.

    precision "fp64": d2 and r^2 in float64 (the definition);
    precision "fp32": d2 by ``d2_fp32`` and r^2 = fl32(fl32(r) * fl32(r)).
    Returns (src int64 [E], dst int64 [E], edge_offsets int64 [B+1])."""
    plane = np.asarray(plane, np.int64)
    hit_offsets = np.asarray(hit_offsets, np.int64)
    if precision == "fp64":
        r2 = float(radius) * float(radius)
        dist = d2_fp64
    elif precision == "fp32":
        rf = np.float32(radius)
        r2 = rf * rf
        dist = d2_fp32
    else:
        raise ValueError(precision)
    src_all, dst_all, counts = [], [], []
    for b in range(hit_offsets.shape[0] - 1):
        lo, hi = int(hit_offsets[b]), int(hit_offsets[b + 1])
        ne = 0
        pl = plane[lo:hi]
        for p in np.unique(pl):
            src_idx = lo + np.nonzero(pl == p)[0]
            cand = lo + np.nonzero((pl == p + 1) | (pl == p + 2))[0]
            if cand.size == 0:
                continue
            d2 = dist(emb[src_idx], emb[cand])
            for row, i in enumerate(src_idx):
                ok = d2[row] < r2
                js, ds = cand[ok], d2[row][ok]
                order = np.lexsort((js, ds))          # by d2, then j
                keep = np.sort(js[order[:k_max]])
                src_all.append(np.full(keep.size, i, np.int64))
                dst_all.append(keep.astype(np.int64))
                ne += keep.size
        counts.append(ne)
    src = np.concatenate(src_all) if src_all else np.zeros(0, np.int64)
    dst = np.concatenate(dst_all) if dst_all else np.zeros(0, np.int64)
    order = np.lexsort((dst, src))
    eo = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=eo[1:])
    return src[order], dst[order], eo


# ----------------------------------------------------------------------------
# interaction network (Sec. 5.2, Eq. 4)
# ----------------------------------------------------------------------------
def layer_norm(a, g, be):
    mu = a.mean(-1, keepdims=True)
    var = ((a - mu) ** 2).mean(-1, keepdims=True)
    rstd = 1.0 / np.sqrt(var + LN_EPS)
    n = (a - mu) * rstd
    return n * g + be, n, rstd


def round_bf16(a):
    """Round to BF16 as a tensor core operand is formed from an FP32 value:
    first to FP32, then to the nearest BF16 (8 significand bits), ties to
    even.  Returned as float64."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def round_e4m3(a):
    """Round to the FP8 e4m3 format (1 sign, 4 exponent bits with bias 7, 3
    mantissa bits, no infinities, largest finite 448): first to FP32, then to
    the nearest e4m3 value, ties to even; magnitudes above 448 saturate."""
    x = np.asarray(a, np.float32).astype(np.float64)
    ax = np.abs(x)
    _, e = np.frexp(ax)                        # ax in [2^(e-1), 2^e)
    ex = np.maximum(e - 1, -6)                 # subnormal spacing 2^-9 below 2^-6
    step = np.ldexp(1.0, ex - 3)
    r = np.minimum(np.round(ax / step) * step, 448.0)   # np.round: half to even
    return np.copysign(r, x)


def quant_weight_e4m3(W):
    """Per-tensor scaled e4m3 weights: s = amax|W| / 448 (FP32), W ~ e4m3(W / s) * s."""
    W32 = np.asarray(W, np.float32)
    amax = np.float32(np.abs(W32).max()) if W32.size else np.float32(0)
    s = np.float32(amax / np.float32(448.0)) if amax > 0 else np.float32(1.0)
    return round_e4m3(W32 / s) * float(s)


def quant_act_e4m3(a, scale):
    """e4m3 operand of an activation tensor with a per-tensor scale s that is a
    power of two: e4m3(a / s) * s (a rounded to FP32 first).  Dividing by a
    power of two is exact, so the scale only moves the e4m3 range: values
    above 448 s saturate, spacing below 2^-6 s is subnormal."""
    s = float(scale)
    if s <= 0 or np.frexp(s)[0] != 0.5:
        raise ValueError("activation scale must be a positive power of two")
    return round_e4m3(np.asarray(a, np.float32).astype(np.float64) / s) * s


def fp8_act_scale(amax):
    """Static per-tensor activation scale of the e4m3 reading: the smallest
    power of two s with amax / s <= 448 (1 for an all-zero tensor)."""
    amax = float(amax)
    if not amax > 0:
        return 1.0
    s = 2.0 ** int(np.ceil(np.log2(amax / 448.0)))
    while amax / s > 448.0:     # guard the logarithm's rounding at exact powers
        s *= 2.0
    while s > 2.0 ** -126 and amax / (s / 2.0) <= 448.0:
        s /= 2.0
    return s


def _identity(a):
    return a


GEMM_READINGS = {
    "fp64": (_identity, _identity),
    "bf16": (round_bf16, round_bf16),
    "fp8": (round_e4m3, quant_weight_e4m3),
}


def n_act_scales(n_iters):
    """Number of e4m3 activation scales of a network with n_iters steps: the
    two matrix products of the edge encoder and of every node and edge
    network, and the classifier's first one."""
    return 2 * (1 + 2 * n_iters) + 1


def act_scale_names(n_iters):
    """Order of the activation scales (and of ``activation_amax``):
    edge_enc in/mid, then per step node{k} in/mid, edge{k} in/mid, then cls in.
    "in" is the block input (first product), "mid" the ReLU output of its
    first layer (second product)."""
    names = ["edge_enc.in", "edge_enc.mid"]
    for k in range(n_iters):
        names += [f"node{k}.in", f"node{k}.mid", f"edge{k}.in", f"edge{k}.mid"]
    return names + ["cls.in"]


def mlp_block(X, w, prefix, cache=None, op=_identity, op_w=None, op2=None):
    """Lin -> LN -> ReLU -> Lin -> LN -> ReLU on rows of X.  ``op`` is applied
    to the activation operand of the first matrix product, ``op2`` (default
    ``op``) to that of the second, and ``op_w`` (default ``op``) to the weight
    operand of both (identity: exact FP64)."""
    op_w = op if op_w is None else op_w
    op2 = op if op2 is None else op2
    f = lambda k: w[f"{prefix}.{k}"].astype(np.float64)
    a1 = op(X) @ op_w(w[f"{prefix}.W1"]).T + f("b1")
    y1, n1, s1 = layer_norm(a1, f("g1"), f("be1"))
    r1 = np.maximum(y1, 0.0)
    a2 = op2(r1) @ op_w(w[f"{prefix}.W2"]).T + f("b2")
    y2, n2, s2 = layer_norm(a2, f("g2"), f("be2"))
    out = np.maximum(y2, 0.0)
    if cache is not None:
        cache[prefix] = dict(X=X, y1=y1, n1=n1, s1=s1, r1=r1, y2=y2, n2=n2, s2=s2)
    return out


def messages(e, src, dst, n_nodes):
    """Eq. 4: m_l = [sum over edges l->j of e_lj, sum over edges i->l of e_il]."""
    H = e.shape[1]
    m_out = np.zeros((n_nodes, H))
    m_in = np.zeros((n_nodes, H))
    np.add.at(m_out, src, e)
    np.add.at(m_in, dst, e)
    return np.concatenate([m_out, m_in], axis=1)


def gnn_forward(weights, n_iters, x, y, z, src, dst, cache=None, gemm="fp64", act_scales=None,
                edge_store="fp32"):
    """Edge logits [E] (float64) of the interaction network.

    gemm="bf16" reads the mixed-precision configuration: the operands of every
    matrix product with a hidden-width input (edge encoder, node and edge
    networks, first classifier layer) are rounded to BF16 and the products
    accumulate exactly; the node encoder (3 inputs), LayerNorm, residual adds,
    message sums and the last classifier dot product stay exact.
    gemm="fp8" rounds the weights to per-tensor scaled e4m3
    (``quant_weight_e4m3``) and each of those activation operands to e4m3
    with its static per-tensor scale (``quant_act_e4m3``): ``act_scales``
    lists them in ``act_scale_names`` order (powers of two; None = all 1).
    One scale covers a whole concatenated block input ([e, h_i, h_j] or
    [h, m_out, m_in]).

    edge_store="bf16" (with gemm="bf16") reads the variant that stores the
    edge stream in BF16: e is rounded to BF16 where it is written (after the
    edge encoder and after every residual edge update, the addition itself
    exact), so the messages sum and the next blocks read the rounded values;
    h stays exact."""
    op, op_w = GEMM_READINGS[gemm]
    if edge_store not in ("fp32", "bf16") or (edge_store == "bf16" and gemm != "bf16"):
        raise ValueError("edge_store='bf16' is read with gemm='bf16' only")
    store = round_bf16 if edge_store == "bf16" else _identity
    n_sc = n_act_scales(n_iters)
    if act_scales is not None and gemm != "fp8":
        raise ValueError("activation scales belong to the e4m3 reading")
    sc = [1.0] * n_sc if act_scales is None else [float(v) for v in act_scales]
    if len(sc) != n_sc:
        raise ValueError(f"expected {n_sc} activation scales")
    if gemm == "fp8":
        q = lambda i: (lambda a, s=sc[i]: quant_act_e4m3(a, s))
    else:
        q = lambda i: op
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    N = np.asarray(x).shape[0]
    xin = normalise(np.stack([np.asarray(x, np.float64), np.asarray(y, np.float64),
                              np.asarray(z, np.float64)], axis=1),
                    weights["gnn_mu"], weights["gnn_sigma"])
    h = mlp_block(xin, weights, "node_enc", cache)
    e = store(mlp_block(np.concatenate([h[src], h[dst]], axis=1), weights, "edge_enc", cache, q(0),
                        op_w, q(1)))
    for k in range(n_iters):
        m = messages(e, src, dst, N)
        h = h + mlp_block(np.concatenate([h, m], axis=1), weights, f"node{k}", cache, q(2 + 4 * k),
                          op_w, q(3 + 4 * k))
        e = store(e + mlp_block(np.concatenate([e, h[src], h[dst]], axis=1), weights, f"edge{k}",
                                cache, q(4 + 4 * k), op_w, q(5 + 4 * k)))
    a1 = q(n_sc - 1)(e) @ op_w(weights["cls.W1"]).T + weights["cls.b1"].astype(np.float64)
    y1, n1, s1 = layer_norm(a1, weights["cls.g1"].astype(np.float64),
                            weights["cls.be1"].astype(np.float64))
    r1 = np.maximum(y1, 0.0)
    logits = r1 @ weights["cls.W2"].astype(np.float64)[0] + float(weights["cls.b2"][0])
    if cache is not None:
        cache["cls"] = dict(X=e, y1=y1, n1=n1, s1=s1, r1=r1)
        cache["meta"] = dict(N=N, src=src, dst=dst, n_iters=n_iters)
    return logits


def activation_amax(weights, n_iters, x, y, z, src, dst):
    """Largest magnitude of every e4m3 activation operand of the exact
    (FP64) forward, in ``act_scale_names`` order: the calibration that
    ``fp8_act_scale`` turns into static per-tensor scales."""
    cache = {}
    gnn_forward(weights, n_iters, x, y, z, src, dst, cache=cache)
    amax = lambda a: float(np.abs(a).max()) if np.size(a) else 0.0
    out = [amax(cache["edge_enc"]["X"]), amax(cache["edge_enc"]["r1"])]
    for k in range(n_iters):
        for p in (f"node{k}", f"edge{k}"):
            out += [amax(cache[p]["X"]), amax(cache[p]["r1"])]
    return out + [amax(cache["cls"]["X"])]


# ----------------------------------------------------------------------------
# loss and reverse pass
# ----------------------------------------------------------------------------
def softplus(t):
    return np.logaddexp(0.0, t)


def sigmoid(t):
    return 0.5 * (1.0 + np.tanh(0.5 * t))


def weighted_bce(logits, target, pos_weight=10.0):
    """mean_e [ w y softplus(-z) + (1 - y) softplus(z) ] and d loss / d z."""
    z = np.asarray(logits, np.float64)
    yv = np.asarray(target, np.float64)
    E = max(z.shape[0], 1)
    loss = float(np.sum(pos_weight * yv * softplus(-z) + (1.0 - yv) * softplus(z)) / E)
    dz = (-pos_weight * yv * sigmoid(-z) + (1.0 - yv) * sigmoid(z)) / E
    return loss, dz


def focal_loss(logits, target, alpha=0.25, gamma=2.0):
    """Sigmoid focal loss, the edge loss the paper trains with (Sec. 5.2, Eq. 5;
    the form of its reference, Lin et al. 2017): mean over edges of
    y alpha (1 - p)^gamma (-log p) + (1 - y) (1 - alpha) p^gamma (-log(1 - p)),
    p = sigmoid(z); and d loss / d z, differentiated by hand:
    y alpha (1 - p)^gamma (gamma p log p - (1 - p))
    + (1 - y) (1 - alpha) p^gamma (p - gamma (1 - p) log(1 - p)), over E.
    Reading: the paper gives neither alpha nor gamma; the reference's values
    alpha = 0.25, gamma = 2 are the defaults."""
    z = np.asarray(logits, np.float64)
    yv = np.asarray(target, np.float64)
    E = max(z.shape[0], 1)
    p, q = sigmoid(z), sigmoid(-z)   # p and 1 - p, each without cancellation
    lp, lq = -softplus(-z), -softplus(z)   # log p, log(1 - p)
    l1 = -alpha * q ** gamma * lp
    l0 = -(1.0 - alpha) * p ** gamma * lq
    loss = float(np.sum(yv * l1 + (1.0 - yv) * l0) / E)
    d1 = alpha * q ** gamma * (gamma * p * lp - q)
    d0 = (1.0 - alpha) * p ** gamma * (p - gamma * q * lq)
    dz = (yv * d1 + (1.0 - yv) * d0) / E
    return loss, dz


def _ln_backward(dy, n, rstd, g):
    """LayerNorm backward: returns (d input, d gamma, d beta)."""
    dn = dy * g
    H = n.shape[-1]
    da = rstd * (dn - dn.sum(-1, keepdims=True) / H - n * (dn * n).sum(-1, keepdims=True) / H)
    return da, (dy * n).sum(0), dy.sum(0)


def _mlp_block_backward(dout, w, prefix, c, grads):
    f = lambda k: w[f"{prefix}.{k}"].astype(np.float64)
    dy2 = dout * (c["y2"] > 0)
    da2, grads[f"{prefix}.g2"], grads[f"{prefix}.be2"] = _ln_backward(dy2, c["n2"], c["s2"], f("g2"))
    grads[f"{prefix}.W2"] = da2.T @ c["r1"]
    grads[f"{prefix}.b2"] = da2.sum(0)
    dr1 = da2 @ f("W2")
    dy1 = dr1 * (c["y1"] > 0)
    da1, grads[f"{prefix}.g1"], grads[f"{prefix}.be1"] = _ln_backward(dy1, c["n1"], c["s1"], f("g1"))
    grads[f"{prefix}.W1"] = da1.T @ c["X"]
    grads[f"{prefix}.b1"] = da1.sum(0)
    return da1 @ f("W1")


def _recompute_exact(weights, cache):
    """A copy of a forward cache whose block internals are recomputed exactly
    (FP64) from each block's cached input: the checkpointed residual streams
    of a forward taken in any reading, with exact blocks around them."""
    out = {"meta": cache["meta"]}
    for prefix, c in cache.items():
        if prefix in ("meta", "cls"):
            continue
        tmp = {}
        mlp_block(c["X"], weights, prefix, tmp)
        out[prefix] = tmp[prefix]
    X = cache["cls"]["X"]
    a1 = X @ weights["cls.W1"].astype(np.float64).T + weights["cls.b1"].astype(np.float64)
    y1, n1, s1 = layer_norm(a1, weights["cls.g1"].astype(np.float64),
                            weights["cls.be1"].astype(np.float64))
    out["cls"] = dict(X=X, y1=y1, n1=n1, s1=s1, r1=np.maximum(y1, 0.0))
    return out


def forward_cache_from_streams(weights, n_iters, x, y, z, src, dst, hs, es):
    """A forward cache (the inputs of every block) built from given residual
    streams h^0..h^L, e^0..e^L instead of from this module's own forward: to
    take the reverse pass of ``gnn_backward(recompute=True)`` at another
    implementation's checkpoints (stage-isolated parity of a backward).
    Only the block inputs are filled; recompute=True rebuilds the rest."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    N = np.asarray(x).shape[0]
    hs = [np.asarray(h, np.float64) for h in hs]
    es = [np.asarray(e, np.float64) for e in es]
    xin = normalise(np.stack([np.asarray(x, np.float64), np.asarray(y, np.float64),
                              np.asarray(z, np.float64)], axis=1),
                    weights["gnn_mu"], weights["gnn_sigma"])
    cache = {"node_enc": {"X": xin},
             "edge_enc": {"X": np.concatenate([hs[0][src], hs[0][dst]], axis=1)}}
    for k in range(n_iters):
        cache[f"node{k}"] = {"X": np.concatenate([hs[k], messages(es[k], src, dst, N)], axis=1)}
        cache[f"edge{k}"] = {"X": np.concatenate([es[k], hs[k + 1][src], hs[k + 1][dst]], axis=1)}
    cache["cls"] = {"X": es[n_iters]}
    cache["meta"] = dict(N=N, src=src, dst=dst, n_iters=n_iters)
    return cache


def gnn_backward(weights, cache, dlogits, recompute=False):
    """Gradients (float64) of sum_e dlogits[e] * logit[e] w.r.t. every
    interaction-network parameter, by the chain rule through gnn_forward.

    recompute=True reads the training path of a mixed-precision forward: the
    forward (gemm="bf16") keeps its residual streams h^k, e^k (the inputs of
    every block), and the reverse pass recomputes each block's internals from
    them in exact arithmetic before differentiating it (checkpointing with an
    exact backward)."""
    if recompute:
        cache = _recompute_exact(weights, cache)
    meta = cache["meta"]
    src, dst, N, L = meta["src"], meta["dst"], meta["N"], meta["n_iters"]
    grads = {}
    c = cache["cls"]
    dz = np.asarray(dlogits, np.float64)
    W2c = weights["cls.W2"].astype(np.float64)
    grads["cls.W2"] = (dz @ c["r1"])[None, :]
    grads["cls.b2"] = np.array([dz.sum()])
    dr1 = dz[:, None] * W2c
    dy1 = dr1 * (c["y1"] > 0)
    da1, grads["cls.g1"], grads["cls.be1"] = _ln_backward(dy1, c["n1"], c["s1"],
                                                          weights["cls.g1"].astype(np.float64))
    grads["cls.W1"] = da1.T @ c["X"]
    grads["cls.b1"] = da1.sum(0)
    de = da1 @ weights["cls.W1"].astype(np.float64)
    H = de.shape[1]
    dh = np.zeros((N, H))
    for k in reversed(range(L)):
        # e_{k+1} = e_k + f_edge([e_k, h_{k+1}[src], h_{k+1}[dst]])
        dX = _mlp_block_backward(de, weights, f"edge{k}", cache[f"edge{k}"], grads)
        de = de + dX[:, :H]
        np.add.at(dh, src, dX[:, H:2 * H])
        np.add.at(dh, dst, dX[:, 2 * H:])
        # h_{k+1} = h_k + f_node([h_k, m_out(e_k), m_in(e_k)])
        dX = _mlp_block_backward(dh, weights, f"node{k}", cache[f"node{k}"], grads)
        dh = dh + dX[:, :H]
        de = de + dX[:, H:2 * H][src] + dX[:, 2 * H:][dst]
    dX = _mlp_block_backward(de, weights, "edge_enc", cache["edge_enc"], grads)
    np.add.at(dh, src, dX[:, :H])
    np.add.at(dh, dst, dX[:, H:])
    _mlp_block_backward(dh, weights, "node_enc", cache["node_enc"], grads)
    return grads


# ----------------------------------------------------------------------------
# purified graph and tracks (Sec. 5 overview, Sec. 7.3)
# ----------------------------------------------------------------------------
def edge_mask(logits):
    """Keep an edge iff its score exceeds 0.5, i.e. its logit is > 0."""
    return np.asarray(logits) > 0


def connected_components(src, dst, mask, hit_offsets):
    """Weakly connected components of the kept edges, by breadth-first
    search per event.  Returns int32 labels: for each hit, the smallest
    event-local index in its component."""
    hit_offsets = np.asarray(hit_offsets, np.int64)
    N = int(hit_offsets[-1])
    src = np.asarray(src, np.int64)[np.asarray(mask, bool)]
    dst = np.asarray(dst, np.int64)[np.asarray(mask, bool)]
    adj = [[] for _ in range(N)]
    for a, b in zip(src.tolist(), dst.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    labels = np.full(N, -1, np.int64)
    event_of = np.searchsorted(hit_offsets, np.arange(N), side="right") - 1
    for s in range(N):  # ascending: the first node reached is the component minimum
        if labels[s] >= 0:
            continue
        lab = s - hit_offsets[event_of[s]]
        labels[s] = lab
        frontier = [s]
        while frontier:
            nxt = []
            for u in frontier:
                for v in adj[u]:
                    if labels[v] < 0:
                        labels[v] = lab
                        nxt.append(v)
            frontier = nxt
    return labels.astype(np.int32)


def plane_sweep_components(src, dst, mask, plane, hit_offsets, n_planes=26):
    """The paper's plane-ordered label propagation (Sec. 7.3), a variant of the
    components step that is not exact.  Every hit starts with its own index.
    Forward: for planes 1 .. n_planes-1 in turn, every hit of the plane takes,
    all at once, the smallest label among itself and the hits its kept
    incoming edges come from (lower planes, final by then).  Backward: for
    planes n_planes-2 .. 0 in turn, every hit of the plane takes the smallest
    label among itself and the hits its kept outgoing edges go to.  Returns
    event-local labels (int32)."""
    hit_offsets = np.asarray(hit_offsets, np.int64)
    N = int(hit_offsets[-1])
    keep = np.asarray(mask, bool)
    s = np.asarray(src, np.int64)[keep]
    d = np.asarray(dst, np.int64)[keep]
    plane = np.asarray(plane, np.int64)
    lab = np.arange(N, dtype=np.int64)
    for p in range(1, n_planes):
        sel = plane[d] == p
        new = lab.copy()
        np.minimum.at(new, d[sel], lab[s[sel]])
        lab = new
    for p in range(n_planes - 2, -1, -1):
        sel = plane[s] == p
        new = lab.copy()
        np.minimum.at(new, s[sel], lab[d[sel]])
        lab = new
    event_of = np.searchsorted(hit_offsets, np.arange(N), side="right") - 1
    return (lab - hit_offsets[event_of]).astype(np.int32)


# ----------------------------------------------------------------------------
# track-finding performance on truth (Sec. 6, Table 1)
# ----------------------------------------------------------------------------
TRACK_METRIC_COUNTS = ("particles", "matched_particles", "candidates", "candidate_particles",
                       "tracks", "unmatched_tracks")


def track_metrics(labels, particle_id, hit_offsets, min_hits=3, match_num=7, match_den=10):
    """Counts and sums behind the Table 1 metrics, event by event.

    A track is a set of hits of one event sharing a label, kept if it has at
    least ``min_hits`` hits; a particle counts (is reconstructible, Sec. 3) if
    it has at least ``min_hits`` hits; noise hits have particle id -1.  A track
    and a particle form a matching candidate when at least match_num/match_den
    (70%) of the track's hits belong to the particle (Sec. 6), so a track has
    at most one candidate particle.  Returns a dict of integer counts
    (TRACK_METRIC_COUNTS: reconstructible particles, those with a candidate,
    candidates, distinct particles among the candidates, tracks, tracks with
    no candidate) and the FP64 sums over candidates of matched/particle hits
    ("hit_eff_sum") and matched/track hits ("hit_purity_sum").  With the
    paper's 3 hits and 70%, a matched track has at least 3 hits of its
    particle, so every candidate particle is reconstructible."""
    hit_offsets = np.asarray(hit_offsets, np.int64)
    labels = np.asarray(labels, np.int64)
    particle_id = np.asarray(particle_id, np.int64)
    out = dict.fromkeys(TRACK_METRIC_COUNTS, 0)
    out["hit_eff_sum"] = 0.0
    out["hit_purity_sum"] = 0.0
    for b in range(hit_offsets.shape[0] - 1):
        lab = labels[hit_offsets[b]:hit_offsets[b + 1]].tolist()
        pid = particle_id[hit_offsets[b]:hit_offsets[b + 1]].tolist()
        particle_hits = {}
        for p in pid:
            if p >= 0:
                particle_hits[p] = particle_hits.get(p, 0) + 1
        reconstructible = {p for p, n in particle_hits.items() if n >= min_hits}
        tracks = {}
        for lb, p in zip(lab, pid):
            tracks.setdefault(lb, []).append(p)
        matched = set()
        for members in tracks.values():
            size = len(members)
            if size < min_hits:
                continue
            out["tracks"] += 1
            owner = None
            for p in set(members):
                n = members.count(p)
                if p >= 0 and n * match_den >= match_num * size:
                    owner, n_owned = p, n
            if owner is None:
                out["unmatched_tracks"] += 1
                continue
            out["candidates"] += 1
            matched.add(owner)
            out["hit_eff_sum"] += n_owned / particle_hits[owner]
            out["hit_purity_sum"] += n_owned / size
        out["particles"] += len(reconstructible)
        out["matched_particles"] += len(matched & reconstructible)
        out["candidate_particles"] += len(matched)
    return out


def track_metric_rates(m):
    """The Table 1 ratios from ``track_metrics`` totals (NaN where a
    denominator is zero)."""
    div = lambda a, b: a / b if b else float("nan")
    return {"efficiency": div(m["matched_particles"], m["particles"]),
            "clone_rate": div(m["candidates"] - m["candidate_particles"], m["candidates"]),
            "fake_rate": div(m["unmatched_tracks"], m["tracks"]),
            "hit_efficiency": div(m["hit_eff_sum"], m["candidates"]),
            "hit_purity": div(m["hit_purity_sum"], m["candidates"])}


# ----------------------------------------------------------------------------
# embedding training (Sec. 5.1, Eq. 2-3)
# ----------------------------------------------------------------------------
def embedding_queries(particle_id, hit_offsets, min_hits=3):
    """Query nodes (Sec. 5.1): hits of particles with at least ``min_hits``
    hits in their event (reconstructible, Sec. 3).  Noise (-1) never."""
    particle_id = np.asarray(particle_id, np.int64)
    hit_offsets = np.asarray(hit_offsets, np.int64)
    q = np.zeros(particle_id.shape[0], bool)
    for b in range(hit_offsets.shape[0] - 1):
        lo, hi = int(hit_offsets[b]), int(hit_offsets[b + 1])
        pid = particle_id[lo:hi]
        for p in set(pid.tolist()) - {-1}:
            members = np.nonzero(pid == p)[0]
            if members.size >= min_hits:
                q[lo + members] = True
    return q


def next_hit_of_particle(particle_id, hit_offsets):
    """For every hit, the hit of the same particle that follows it in plane
    order (hits are plane-sorted within an event, at most one hit per
    particle and plane), or -1."""
    particle_id = np.asarray(particle_id, np.int64)
    hit_offsets = np.asarray(hit_offsets, np.int64)
    nxt = np.full(particle_id.shape[0], -1, np.int64)
    for b in range(hit_offsets.shape[0] - 1):
        lo, hi = int(hit_offsets[b]), int(hit_offsets[b + 1])
        last = {}
        for i in range(hi - 1, lo - 1, -1):
            p = int(particle_id[i])
            if p >= 0:
                nxt[i] = last.get(p, -1)
                last[p] = i
    return nxt


def embedding_pairs(emb, plane, particle_id, hit_offsets, radius, k_max, rand, min_hits=3,
                    precision="fp32"):
    """Training set T of Sec. 5.1 for a batch whose noise hits were removed.

    From every query q (``embedding_queries``) on plane p, to hits a on planes
    p+1 and p+2 of its event:
      * hard negatives: the pairs the graph rule itself produces
        (``build_graph`` with the training radius and k_max);
      * one random pair: the (rand[q] mod c)-th hit, in index order, of the c
        hits on planes p+1 and p+2 (none when c = 0); the random numbers are
        inputs;
      * the genuine edge: q -> the next hit of q's particle, when it lies on
        p+1 or p+2.
    T is the union as a set.  A pair is genuine iff a is the next hit of q's
    particle (a genuine edge: successive hits of one particle).  Returns
    (q int64 [T], a int64 [T], genuine bool [T]) sorted by (q, a)."""
    plane = np.asarray(plane, np.int64)
    rand = np.asarray(rand, np.uint64)
    hit_offsets = np.asarray(hit_offsets, np.int64)
    is_q = embedding_queries(particle_id, hit_offsets, min_hits)
    nxt = next_hit_of_particle(particle_id, hit_offsets)
    s, d, _ = build_graph(emb, plane, hit_offsets, radius, k_max, precision=precision)
    pairs = {(int(i), int(j)) for i, j in zip(s.tolist(), d.tolist()) if is_q[i]}
    for b in range(hit_offsets.shape[0] - 1):
        lo, hi = int(hit_offsets[b]), int(hit_offsets[b + 1])
        for q in range(lo, hi):
            if not is_q[q]:
                continue
            p = plane[q]
            cand = [j for j in range(lo, hi) if plane[j] in (p + 1, p + 2)]
            if cand:
                pairs.add((q, cand[int(rand[q] % np.uint64(len(cand)))]))
            if nxt[q] >= 0 and plane[nxt[q]] - p <= 2:
                pairs.add((q, int(nxt[q])))
    out = sorted(pairs)
    q = np.array([x for x, _ in out], np.int64)
    a = np.array([y for _, y in out], np.int64)
    return q, a, (nxt[q] == a) if out else np.zeros(0, bool)


def hinge_embedding_loss(emb, q, a, genuine, margin=1.0, w_genuine=2.0):
    """Eq. 2-3: L = L_fake + w_genuine * L_genuine with L_genuine the mean of
    d2(q, a) over genuine pairs and L_fake the mean of max(0, margin - d2)
    over fake pairs (an empty set contributes 0; at d2 = margin the hinge
    is inactive).  Returns (L, L_genuine, L_fake, dL/d emb [N, D])."""
    emb = np.asarray(emb, np.float64)
    q = np.asarray(q, np.int64)
    a = np.asarray(a, np.int64)
    g = np.asarray(genuine, bool)
    diff = emb[q] - emb[a]
    d2 = (diff * diff).sum(1)
    n_g, n_f = int(g.sum()), int((~g).sum())
    L_g = d2[g].mean() if n_g else 0.0
    hinge = np.maximum(0.0, margin - d2[~g])
    L_f = hinge.mean() if n_f else 0.0
    # dL/d d2 per pair
    coef = np.zeros(q.shape[0])
    if n_g:
        coef[g] = w_genuine / n_g
    if n_f:
        coef[~g] = np.where(d2[~g] < margin, -1.0 / n_f, 0.0)
    grad = np.zeros_like(emb)
    contrib = 2.0 * coef[:, None] * diff
    np.add.at(grad, q, contrib)
    np.add.at(grad, a, -contrib)
    return L_f + w_genuine * L_g, L_g, L_f, grad


def embed_backward(weights, n_layers, x, y, z, d_emb):
    """Reverse pass of ``embed`` for dL/d emb = d_emb: returns
    {"emb{i}.W": [out, in], "emb{i}.b": [out]} in float64."""
    acts = [normalise(cylindrical(x, y, z), weights["emb_mu"], weights["emb_sigma"])]
    for i in range(n_layers):
        W = weights[f"emb{i}.W"].astype(np.float64)
        b = weights[f"emb{i}.b"].astype(np.float64)
        out = acts[-1] @ W.T + b
        acts.append(np.maximum(out, 0.0) if i < n_layers - 1 else out)
    grads = {}
    dz = np.asarray(d_emb, np.float64)               # d L / d (pre-activation of the last layer)
    for i in range(n_layers - 1, -1, -1):
        grads[f"emb{i}.W"] = dz.T @ acts[i]
        grads[f"emb{i}.b"] = dz.sum(0)
        if i > 0:
            W = weights[f"emb{i}.W"].astype(np.float64)
            dz = (dz @ W) * (acts[i] > 0)               # through Linear, then ReLU of layer i-1
    return grads


# ----------------------------------------------------------------------------
# triplets of the purified graph (Sec. 5.3) and their classifiers
# ----------------------------------------------------------------------------
TRIPLET_ARTICULATION, TRIPLET_LEFT_ELBOW, TRIPLET_RIGHT_ELBOW = 0, 1, 2


def build_triplets(src, dst, mask, n_hits):
    """Triplets of the kept edges (Sec. 5.3), each a pair of edges sharing a
    common hit C: articulations A->C, C->B (first = the edge into C), left
    elbows C->A, C->B and right elbows A->C, B->C (first < second by edge
    index).  Returned as (first, second, kind) int64 arrays: all
    articulations, then all left elbows, then all right elbows; within a kind
    by C, then first, then second."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    keep = np.nonzero(np.asarray(mask, bool))[0]
    out_e = [[] for _ in range(n_hits)]
    in_e = [[] for _ in range(n_hits)]
    for k in keep.tolist():
        out_e[src[k]].append(k)
        in_e[dst[k]].append(k)
    lists = ([], [], [])
    for c in range(n_hits):
        for i in in_e[c]:
            for o in out_e[c]:
                lists[TRIPLET_ARTICULATION].append((i, o))
        for x in range(len(out_e[c])):
            for y in range(x + 1, len(out_e[c])):
                lists[TRIPLET_LEFT_ELBOW].append((out_e[c][x], out_e[c][y]))
        for x in range(len(in_e[c])):
            for y in range(x + 1, len(in_e[c])):
                lists[TRIPLET_RIGHT_ELBOW].append((in_e[c][x], in_e[c][y]))
    first = np.array([p[0] for l in lists for p in l], np.int64)
    second = np.array([p[1] for l in lists for p in l], np.int64)
    kind = np.concatenate([np.full(len(l), t, np.int64) for t, l in enumerate(lists)])
    return first, second, kind


def triplet_logits(tw, e, first, second, kind):
    """The two triplet classifiers (Sec. 5.3; articulations "art", elbows
    "elb"): Lin(2H, H) -> LN -> ReLU -> Lin(H, 1) on [e_first, e_second],
    the final edge encodings.  Returns float64 logits."""
    e = np.asarray(e, np.float64)
    first = np.asarray(first, np.int64)
    second = np.asarray(second, np.int64)
    kind = np.asarray(kind, np.int64)
    x = np.concatenate([e[first], e[second]], axis=1) if first.size else np.zeros((0, 2 * e.shape[1]))
    out = np.zeros(first.shape[0])
    for name, sel in (("art", kind == TRIPLET_ARTICULATION), ("elb", kind != TRIPLET_ARTICULATION)):
        if not sel.any():
            continue
        a = x[sel] @ np.asarray(tw[f"{name}.W1"], np.float64).T + np.asarray(tw[f"{name}.b1"], np.float64)
        a = np.maximum(layer_norm(a, np.asarray(tw[f"{name}.g1"], np.float64),
                                  np.asarray(tw[f"{name}.be1"], np.float64))[0], 0.0)
        out[sel] = a @ np.asarray(tw[f"{name}.W2"], np.float64)[0] + float(np.asarray(tw[f"{name}.b2"])[0])
    return out


# ----------------------------------------------------------------------------
# track building on the purified edge graph (Sec. 5.4)
# ----------------------------------------------------------------------------
def _find(parent, x):
    while parent[x] != x:
        x = parent[x]
    return x


def _union(parent, a, b):
    ra, rb = _find(parent, a), _find(parent, b)
    if ra != rb:
        parent[max(ra, rb)] = min(ra, rb)


def tracks_from_triplets(src, dst, edge_mask, first, second, kind, triplet_mask, min_hits=3):
    """Tracks that may share hits, built from the purified edge graph: the
    kept edges (``edge_mask``) linked by the kept triplets (``triplet_mask``
    over ``build_triplets``'s list), in the four steps of Sec. 5.4 as read
    here (the paper gives them in prose and a figure):

    1. Elbows join continuations.  At each hit C, the kept edges entering C
       that a chain of kept right elbows joins form one group, and so do the
       kept edges leaving C joined by kept left elbows.  An articulation
       (i, o) at C is taken as present when a kept articulation links some
       edge of i's group to some edge of o's group: two edges of one elbow
       share their continuations through C.  An articulation that the
       classifier kept is present once, however many elbows also imply it
       (the duplicates are dropped).
    2. An articulation (i, o) at C is shared when i continues into two or
       more present articulations at C (a fork after i) or o into two or more
       (a merge before o).  Weakly connected components are taken over the
       kept edges linked by the present, unshared articulations.
    3. Every component touched by no shared articulation is a track; every
       shared articulation (i, o) is a track of its own, the union of i's and
       o's components (so a shared part is duplicated into each track).
    4. A track's hits are the end points of its edges.

    Tracks with fewer than ``min_hits`` hits are dropped.  Returns the list of
    tracks, each a sorted tuple of batch-global hit indices, in lexicographic
    order (the order is not part of the result)."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    emask = np.asarray(edge_mask, bool)
    first = np.asarray(first, np.int64)
    second = np.asarray(second, np.int64)
    kind = np.asarray(kind, np.int64)
    tmask = np.asarray(triplet_mask, bool)
    E = src.shape[0]
    # kept edges entering and leaving each hit, ascending edge index
    ins, outs = {}, {}
    for k in range(E):
        if emask[k]:
            outs.setdefault(int(src[k]), []).append(k)
            ins.setdefault(int(dst[k]), []).append(k)
    kept = {(int(f), int(s), int(t)) for f, s, t, m in zip(first, second, kind, tmask) if m}
    parent = list(range(E))          # union-find over edge indices
    shared = []
    for c in sorted(set(ins) & set(outs)):
        I, O = ins[c], outs[c]
        # step 1: elbow groups of the in-edges (right elbows) and out-edges (left elbows)
        gi, go = {i: i for i in I}, {o: o for o in O}
        for x in range(len(I)):
            for y in range(x + 1, len(I)):
                if (I[x], I[y], TRIPLET_RIGHT_ELBOW) in kept:
                    _union(gi, I[x], I[y])
        for x in range(len(O)):
            for y in range(x + 1, len(O)):
                if (O[x], O[y], TRIPLET_LEFT_ELBOW) in kept:
                    _union(go, O[x], O[y])
        linked = {(_find(gi, i), _find(go, o)) for i in I for o in O
                  if (i, o, TRIPLET_ARTICULATION) in kept}
        present = [(i, o) for i in I for o in O if (_find(gi, i), _find(go, o)) in linked]
        # step 2: shared articulations; the others link edges
        n_out = {i: sum(1 for a, _ in present if a == i) for i in I}
        n_in = {o: sum(1 for _, b in present if b == o) for o in O}
        for i, o in present:
            if n_out[i] >= 2 or n_in[o] >= 2:
                shared.append((i, o))
            else:
                _union(parent, i, o)
    # step 3: tracks as sets of edges (by component root)
    comp_edges = {}
    for k in range(E):
        if emask[k]:
            comp_edges.setdefault(_find(parent, k), []).append(k)
    touched = {_find(parent, i) for i, _ in shared} | {_find(parent, o) for _, o in shared}
    track_edges = [comp_edges[r] for r in sorted(comp_edges) if r not in touched]
    for i, o in shared:
        ri, ro = _find(parent, i), _find(parent, o)
        track_edges.append(comp_edges[ri] + (comp_edges[ro] if ro != ri else []))
    # step 4: edges -> hits
    tracks = []
    for es in track_edges:
        hits = sorted({int(src[k]) for k in es} | {int(dst[k]) for k in es})
        if len(hits) >= min_hits:
            tracks.append(tuple(hits))
    return sorted(tracks)
