"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer outputs (edge lists, offsets, labels) must match exactly when both
sides start from the same inputs; FP32 logits within max-abs 1e-4; the only
allowed graph differences end to end are pairs within 1e-5 of the radius (or
of the k-th kept distance), which are counted and reported.
"""
import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import (WORKLOADS, ModelConfig, concat_events, make_batch, make_event,
                        make_weights, pack_blob)

pytestmark = pytest.mark.gpu

LOGIT_TOL = 1e-4      # FP32 logits vs FP64 oracle (max-abs)
NEAR_CUT = 1e-5       # distance band around the radius / k-th distance


@pytest.fixture(scope="module")
def etx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import etx as m
    return m


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def events(recipe, seeds, extra=()):
    parts = [make_event(recipe, s) for s in seeds]
    for pos, part in extra:
        parts.insert(pos, part)
    return concat_events(parts)


def empty_event():
    z = np.zeros(0, np.float32)
    return (z, z, z, np.zeros(0, np.int8), np.zeros(0, np.int32))


class Setup:
    def __init__(self, etx, model, batch, weights, max_edges=None):
        self.model, self.b, self.W = model, batch, weights
        N = max(batch.n_hits, 1)
        self.ctx = etx.Context(model, max(batch.n_events, 1), N,
                               max_edges or max(N * model.k_max, 1))
        self.ctx.load_weights(pack_blob(model, weights))
        self.x, self.y, self.z = (cuda(batch.x), cuda(batch.y), cuda(batch.z))
        self.plane = cuda(batch.plane)
        self.hoff = cuda(batch.hit_offsets)
        self.depth = len(model.emb_widths) - 1

    def oracle_emb(self):
        return O.embed(self.W, self.depth, self.b.x, self.b.y, self.b.z)


def setup_for(etx, name, n_events=None, perturb=0.2, extra=(), model=None, seeds=None):
    wl = WORKLOADS[name]
    model = model or wl.model
    if seeds is None:
        seeds = [wl.base_seed + i for i in range(n_events or wl.n_events)]
    b = events(wl.recipe, seeds, extra)
    W = make_weights(model, wl.calibration(), perturb=perturb)
    return Setup(etx, model, b, W)


def oracle_graph32(st, emb64, radius=None, k=None):
    emb32 = emb64.astype(np.float32)
    s, d, eo = O.build_graph(emb32, st.b.plane, st.b.hit_offsets,
                             st.model.radius if radius is None else radius,
                             st.model.k_max if k is None else k, precision="fp32")
    return emb32, s, d, eo


def gpu_graph(st, emb32, radius=None, k=None, cap=None):
    src, dst, eo = st.ctx.build_graph(cuda(emb32), st.plane, st.hoff,
                                      st.model.radius if radius is None else radius,
                                      st.model.k_max if k is None else k, edge_capacity=cap)
    st.ctx.sync()
    eo = eo.cpu().numpy()
    E = int(eo[-1])
    return src[:E].cpu().numpy(), dst[:E].cpu().numpy(), eo


# ---------------------------------------------------------------------------
# embedding
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,n", [("plain", 1), ("batch500", 4)])
def test_embed_parity(etx, name, n):
    st = setup_for(etx, name, n)
    ref = st.oracle_emb()
    out = st.ctx.embed(st.x, st.y, st.z)
    st.ctx.sync()
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    # FP32 MLP: the error scales with the magnitude of the outputs
    bound = 2e-6 * (1.0 + np.abs(ref).max())
    print(f"embed {name}: max |err| {err.max():.3e}, bound {bound:.3e}")
    assert err.max() <= bound


# ---------------------------------------------------------------------------
# graph, stage-isolated: both sides start from the same FP32 embedding
# ---------------------------------------------------------------------------
def _check_graph_exact(st, emb64, radius=None, k=None):
    emb32, s, d, eo = oracle_graph32(st, emb64, radius, k)
    gs, gd, geo = gpu_graph(st, emb32, radius, k)
    np.testing.assert_array_equal(geo, eo)
    np.testing.assert_array_equal(gs, s)
    np.testing.assert_array_equal(gd, d)
    return s.size


def test_graph_exact_plain(etx):
    st = setup_for(etx, "plain", 1)
    assert _check_graph_exact(st, st.oracle_emb()) > 0


def test_graph_exact_ragged_batch_with_empty_events(etx):
    wl = WORKLOADS["batch500"]
    st = setup_for(etx, "batch500", seeds=[1000, 1001, 1002, 1003, 1004],
                   extra=[(0, empty_event()), (3, empty_event())])
    assert st.b.n_events == 7
    assert _check_graph_exact(st, st.oracle_emb()) > 0


def test_graph_exact_k_cap_binding(etx):
    st = setup_for(etx, "batch500", 3)
    emb = st.oracle_emb()
    n = _check_graph_exact(st, emb, radius=3.0, k=4)
    assert n > 0
    # the cap binds for most sources here
    _, s, _, _ = oracle_graph32(st, emb, radius=3.0, k=4)
    assert np.bincount(s).max() == 4


def test_graph_exact_ties_between_duplicate_hits(etx):
    wl = WORKLOADS["plain"]
    x, y, z, p, pid = make_event(wl.recipe, 7)
    # every hit twice: identical embeddings, so distances tie exactly
    order = np.argsort(np.concatenate([p, p]), kind="stable")
    dup = tuple(np.concatenate([a, a])[order] for a in (x, y, z, p, pid))
    b = concat_events([dup])
    W = make_weights(wl.model, wl.calibration(), perturb=0.2)
    st = Setup(etx, wl.model, b, W)
    assert _check_graph_exact(st, st.oracle_emb(), k=3) > 0


@pytest.mark.parametrize("counts", [[12, 500, 500, 5], [12, 1100, 1100, 5]])
def test_graph_exact_large_candidate_sets(etx, counts):
    # 1,000 candidates: the 64-key register path; 2,200: more than the
    # shared-memory stage holds, so the generic path reads global memory
    rng = np.random.default_rng(3)
    plane = np.concatenate([np.full(c, i, np.int8) for i, c in enumerate(counts)])
    r = np.sqrt(rng.uniform(5.1 ** 2, 40 ** 2, plane.size))
    ph = rng.uniform(0, 2 * np.pi, plane.size)
    ev = ((r * np.cos(ph)).astype(np.float32), (r * np.sin(ph)).astype(np.float32),
          np.linspace(-287, 750, 26)[plane].astype(np.float32), plane, np.full(plane.size, -1, np.int32))
    b = concat_events([ev])
    model = WORKLOADS["batch500"].model
    W = make_weights(model, WORKLOADS["batch500"].calibration(), perturb=0.2)
    st = Setup(etx, model, b, W)
    assert _check_graph_exact(st, st.oracle_emb(), radius=2.0, k=8) > 0


def test_graph_literal_radius_gives_no_edges(etx):
    st = setup_for(etx, "batch500", 2)
    emb = st.oracle_emb()
    assert _check_graph_exact(st, emb, radius=1e-3) == 0


def test_graph_capacity_overflow_is_reported(etx):
    st = setup_for(etx, "plain", 1)
    emb32, s, d, eo = oracle_graph32(st, st.oracle_emb())
    src, dst, geo = st.ctx.build_graph(cuda(emb32), st.plane, st.hoff, st.model.radius,
                                       st.model.k_max, edge_capacity=max(1, s.size // 2))
    with pytest.raises(etx.EtxError) as ei:
        st.ctx.sync()
    assert ei.value.status == etx.ETX_ERR_CAPACITY
    np.testing.assert_array_equal(geo.cpu().numpy(), eo)  # counts are still reported


# ---------------------------------------------------------------------------
# graph, end to end: GPU embedding + GPU graph vs FP64 oracle
# ---------------------------------------------------------------------------
def test_graph_end_to_end_only_near_cut_pairs_differ(etx):
    st = setup_for(etx, "batch500", 4)
    emb64 = st.oracle_emb()
    s, d, _ = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    emb = st.ctx.embed(st.x, st.y, st.z)
    src, dst, eo = st.ctx.build_graph(emb, st.plane, st.hoff, st.model.radius, st.model.k_max)
    st.ctx.sync()
    E = int(eo[-1].item())
    gset = set(zip(src[:E].cpu().tolist(), dst[:E].cpu().tolist()))
    oset = set(zip(s.tolist(), d.tolist()))
    diff = gset ^ oset
    r, k = st.model.radius, st.model.k_max
    unexplained = 0
    for i, j in diff:
        dist = np.sqrt(((emb64[i] - emb64[j]) ** 2).sum())
        if abs(dist - r) <= NEAR_CUT:
            continue
        # rank near-tie: the cap binds and j sits at the k-th kept distance
        cand = np.nonzero(np.isin(st.b.plane.astype(int) - int(st.b.plane[i]), [1, 2]))[0]
        ev = np.searchsorted(st.b.hit_offsets, i, side="right") - 1
        cand = cand[(cand >= st.b.hit_offsets[ev]) & (cand < st.b.hit_offsets[ev + 1])]
        dd = np.sort(np.sqrt(((emb64[cand] - emb64[i]) ** 2).sum(1)))
        dd = dd[dd < r]
        if dd.size > k and abs(dist - dd[k - 1]) <= NEAR_CUT:
            continue
        unexplained += 1
    print(f"end-to-end graph: {len(oset)} oracle edges, {len(diff)} differ, all near the cut")
    assert unexplained == 0
    assert len(diff) <= 1e-3 * max(len(oset), 1)


# ---------------------------------------------------------------------------
# interaction network
# ---------------------------------------------------------------------------
GNN_CASES = [
    ("plain", 1, None),
    ("batch500", 2, None),
    ("batch500", 2, ModelConfig(emb_widths=(3, 128, 128, 128, 8), hidden=64, n_iters=3,
                                radius=1.14, k_max=32)),
    ("plain", 2, ModelConfig(emb_widths=(3, 32, 32, 4), hidden=16, n_iters=4, radius=1.5,
                             k_max=16)),
]


@pytest.mark.parametrize("name,n,model", GNN_CASES)
def test_gnn_forward_parity(etx, name, n, model):
    st = setup_for(etx, name, n, model=model)
    emb64 = st.oracle_emb()
    s, d, eo = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    ref = O.gnn_forward(st.W, st.model.n_iters, st.b.x, st.b.y, st.b.z, s, d)
    logits = st.ctx.gnn_forward(st.x, st.y, st.z, cuda(s, torch.int32), cuda(d, torch.int32),
                                cuda(eo, torch.int32))
    st.ctx.sync()
    err = np.abs(logits.cpu().numpy().astype(np.float64) - ref)
    print(f"gnn {name} H={st.model.hidden} L={st.model.n_iters}: E={s.size} max |err| {err.max():.3e}")
    assert err.max() <= LOGIT_TOL


def test_gnn_forward_without_edges(etx):
    st = setup_for(etx, "plain", 1)
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    eo = torch.zeros(2, dtype=torch.int32, device="cuda")
    logits = st.ctx.gnn_forward(st.x, st.y, st.z, z, z, eo)
    st.ctx.sync()
    assert logits.shape[0] == 1


def test_gnn_rejects_unsorted_edges(etx):
    st = setup_for(etx, "plain", 1)
    s = cuda(np.array([5, 2], np.int32))
    d = cuda(np.array([40, 41], np.int32))
    eo = cuda(np.array([0, 2], np.int32))
    st.ctx.gnn_forward(st.x, st.y, st.z, s, d, eo)
    with pytest.raises(etx.EtxError) as ei:
        st.ctx.sync()
    assert ei.value.status == etx.ETX_ERR_UNSORTED


# ---------------------------------------------------------------------------
# components: same mask on both sides -> identical labels
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("quantile", [0.0, 0.5, 0.9, 0.99, 1.0])
def test_cc_labels_exact(etx, quantile):
    st = setup_for(etx, "batch500", 3)
    emb64 = st.oracle_emb()
    s, d, eo = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    rng = np.random.default_rng(int(quantile * 100))
    logits = rng.normal(size=s.size).astype(np.float32)
    thr = np.float32(np.quantile(logits, quantile)) if quantile < 1.0 else np.float32(10.0)
    ref = O.connected_components(s, d, logits > thr, st.b.hit_offsets)
    labels, nt = st.ctx.edges_to_tracks(cuda(s, torch.int32), cuda(d, torch.int32), cuda(logits),
                                        float(thr), cuda(eo, torch.int32), st.hoff, min_hits=3)
    st.ctx.sync()
    np.testing.assert_array_equal(labels.cpu().numpy(), ref)
    # tracks with >= 3 hits per event
    for b in range(st.b.n_events):
        lo, hi = st.b.hit_offsets[b], st.b.hit_offsets[b + 1]
        sizes = np.bincount(ref[lo:hi], minlength=hi - lo)
        assert int(nt[b].item()) == int((sizes >= 3).sum())


def test_cc_golden_graphs_on_gpu(etx):
    import json
    from pathlib import Path
    cases = json.loads((Path(__file__).parent / "golden" / "wcc_graphs.json").read_text())["cases"]
    model = WORKLOADS["plain"].model
    ctx = etx.Context(model, 8, 64, 64)
    for c in cases:
        logits = np.where(np.array(c["mask"]) > 0, 1.0, -1.0).astype(np.float32)
        hoff = np.array(c["hit_offsets"], np.int32)
        eo = np.array([0] * (len(hoff) - 1) + [len(c["src"])], np.int32)
        labels, _ = ctx.edges_to_tracks(cuda(np.array(c["src"], np.int32)),
                                        cuda(np.array(c["dst"], np.int32)), cuda(logits), 0.0,
                                        cuda(eo), cuda(hoff))
        ctx.sync()
        assert labels.cpu().tolist() == c["labels"], c["name"]


# ---------------------------------------------------------------------------
# whole pipeline and host-side errors
# ---------------------------------------------------------------------------
def test_pipeline_end_to_end_labels(etx):
    st = setup_for(etx, "batch500", 3, perturb=0.0)
    thr = st.model.threshold_logit
    emb64 = st.oracle_emb()
    s, d, _ = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    z = O.gnn_forward(st.W, st.model.n_iters, st.b.x, st.b.y, st.b.z, s, d)
    ref = O.connected_components(s, d, z > thr, st.b.hit_offsets)
    emb = st.ctx.embed(st.x, st.y, st.z)
    src, dst, eo = st.ctx.build_graph(emb, st.plane, st.hoff, st.model.radius, st.model.k_max)
    logits = st.ctx.gnn_forward(st.x, st.y, st.z, src, dst, eo)
    labels, _ = st.ctx.edges_to_tracks(src, dst, logits, thr, eo, st.hoff)
    st.ctx.sync()
    agree = float((labels.cpu().numpy() == ref).mean())
    print(f"pipeline label agreement {agree:.6f}")
    assert agree >= 0.99


def test_host_argument_errors(etx):
    st = setup_for(etx, "plain", 1)
    emb = st.ctx.embed(st.x, st.y, st.z)
    with pytest.raises(etx.EtxError) as ei:
        st.ctx.build_graph(emb, st.plane, st.hoff, 1.0, 0)
    assert ei.value.status == etx.ETX_ERR_ARG
    big = cuda(np.array([0, 0, 0, st.b.n_hits], np.int32))
    with pytest.raises(etx.EtxError) as ei:
        st.ctx.build_graph(emb, st.plane, big, 1.0, 4)
    assert ei.value.status == etx.ETX_ERR_CAPACITY
    ctx2 = etx.Context(st.model, 1, 1000, 1000)
    with pytest.raises(etx.EtxError) as ei:
        ctx2.embed(st.x, st.y, st.z)
    assert ei.value.status == etx.ETX_ERR_STATE
    st.ctx.sync()


def test_unsorted_planes_are_reported(etx):
    st = setup_for(etx, "plain", 1)
    emb = st.ctx.embed(st.x, st.y, st.z)
    bad = st.b.plane.copy()[::-1].copy()
    st.ctx.build_graph(emb, cuda(bad), st.hoff, st.model.radius, st.model.k_max)
    with pytest.raises(etx.EtxError) as ei:
        st.ctx.sync()
    assert ei.value.status == etx.ETX_ERR_UNSORTED
    st.ctx.sync()  # the error word was cleared


# ---------------------------------------------------------------------------
# tensor-core (BF16 operand) interaction network
# ---------------------------------------------------------------------------
BF16_TOL = 2e-2   # vs the oracle's BF16-operand reading (max-abs)


@pytest.mark.parametrize("n_events", [1, 3])
def test_gnn_forward_bf16_tensor_cores(etx, n_events):
    st = setup_for(etx, "batch500", n_events)
    emb64 = st.oracle_emb()
    s, d, eo = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    args = (st.W, st.model.n_iters, st.b.x, st.b.y, st.b.z, s, d)
    ref64 = O.gnn_forward(*args)
    ref16 = O.gnn_forward(*args, gemm="bf16")
    logits = st.ctx.gnn_forward(st.x, st.y, st.z, cuda(s, torch.int32), cuda(d, torch.int32),
                                cuda(eo, torch.int32), dtype="bf16")
    st.ctx.sync()
    got = logits.cpu().numpy().astype(np.float64)
    e16, e64 = np.abs(got - ref16), np.abs(got - ref64)
    print(f"bf16 E={s.size}: max|err| vs bf16 reading {e16.max():.3e} (mean {e16.mean():.2e}), "
          f"vs fp64 {e64.max():.3e} (mean {e64.mean():.2e}), oracle bf16-vs-fp64 "
          f"{np.abs(ref16 - ref64).max():.3e}")
    assert e16.max() <= BF16_TOL


@pytest.mark.parametrize("n_events", [1, 3])
def test_gnn_forward_bf16_edge_store(etx, n_events):
    """BF16 GEMMs with the edge stream stored in BF16 against the oracle's
    matching reading (edge_store="bf16")."""
    st = setup_for(etx, "batch500", n_events)
    emb64 = st.oracle_emb()
    s, d, eo = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    args = (st.W, st.model.n_iters, st.b.x, st.b.y, st.b.z, s, d)
    ref = O.gnn_forward(*args, gemm="bf16", edge_store="bf16")
    ref16 = O.gnn_forward(*args, gemm="bf16")
    logits = st.ctx.gnn_forward(st.x, st.y, st.z, cuda(s, torch.int32), cuda(d, torch.int32),
                                cuda(eo, torch.int32), dtype="bf16s")
    st.ctx.sync()
    got = logits.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    print(f"bf16s E={s.size}: max|err| vs its reading {err.max():.3e} (mean {err.mean():.2e}); "
          f"the reading vs the FP32-storage BF16 reading {np.abs(ref - ref16).max():.3e}")
    assert err.max() <= BF16_TOL
    # the triplet classifier reads FP32 edge encodings: refused after a BF16-storage forward
    from velo_synth import make_triplet_weights, pack_triplet_blob
    st.ctx.load_triplet_weights(pack_triplet_blob(st.model, make_triplet_weights(st.model)))
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(etx.EtxError) as ei:
        st.ctx.classify_triplets(z, z, z)
    assert ei.value.status == etx.ETX_ERR_STATE


# vs the oracle's e4m3 reading (max-abs).  e4m3 keeps 3 mantissa bits: where an FP32
# operand and its FP64 counterpart fall on either side of a rounding boundary the two
# roundings differ by a whole e4m3 step, and the network carries such flips on, so the
# largest difference from the reading is of the order of the format's own error (the
# reading differs from FP64 by up to 0.2 here); the mean check below is the sharp one
FP8_TOL = 0.25


@pytest.mark.parametrize("n_events,scales", [(1, "unit"), (3, "unit"), (3, "calibrated")])
def test_gnn_forward_fp8_tensor_cores(etx, n_events, scales):
    st = setup_for(etx, "batch500", n_events)
    sc = st.model.fp8_act_scales if scales == "calibrated" else None
    assert scales == "unit" or sc is not None
    st.ctx.set_fp8_scales(sc)
    emb64 = st.oracle_emb()
    s, d, eo = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    args = (st.W, st.model.n_iters, st.b.x, st.b.y, st.b.z, s, d)
    ref64 = O.gnn_forward(*args)
    ref8 = O.gnn_forward(*args, gemm="fp8", act_scales=sc)
    logits = st.ctx.gnn_forward(st.x, st.y, st.z, cuda(s, torch.int32), cuda(d, torch.int32),
                                cuda(eo, torch.int32), dtype="fp8")
    st.ctx.sync()
    got = logits.cpu().numpy().astype(np.float64)
    e8, e64 = np.abs(got - ref8), np.abs(got - ref64)
    print(f"fp8 ({scales} scales) E={s.size}: max|err| vs e4m3 reading {e8.max():.3e} "
          f"(mean {e8.mean():.2e}), vs fp64 {e64.max():.3e} (mean {e64.mean():.2e}), oracle "
          f"fp8-vs-fp64 {np.abs(ref8 - ref64).max():.3e} (mean {np.abs(ref8 - ref64).mean():.2e})")
    assert e8.max() <= FP8_TOL
    # a layout or scale error would be far larger than the e4m3 rounding itself
    assert e8.mean() <= 0.5 * max(np.abs(ref8 - ref64).mean(), 1e-6) + 1e-2


# Per-dtype bounds against the FP64 oracle on the batch500 sample (random weights: logits
# 2.44 +- 0.23 around the cut 2.848).  An edge mask can only differ where the FP64 logit
# lies closer to the cut than the dtype's logit error, so the band |z64 - cut| <= NEAR_LOGIT
# is "near the cut" (counted); outside it the masks must agree exactly.
NEAR_LOGIT = {"f32": 1e-4, "bf16": 2e-2, "bf16s": 2e-2, "fp8": 0.25}
MAX_ABS_VS_FP64 = {"f32": 1e-4, "bf16": 2e-2, "bf16s": 2e-2, "fp8": 0.25}
# bf16s (edge stream stored in BF16) is a speed variant: its extra rounding puts it a
# little above the 1e-3 target (1.1e-3 in the oracle's own reading on these events)
MASK_DIS_MAX = {"f32": 1e-4, "bf16": 1e-3, "bf16s": 2e-3}
LABEL_AGREE_MIN = {"f32": 0.999, "bf16": 0.99, "bf16s": 0.99, "fp8": 0.8}


def test_dtype_report_vs_fp64_oracle(etx):
    """Per arithmetic type: max-abs logit error against the FP64 oracle, edge-mask
    disagreement at the workload's cut (split into near-cut and the rest) and
    track-label agreement, all on the oracle's graph of 5 events.  FP32 and BF16
    must keep the mask disagreement within the bound; e4m3's is set by its
    3-bit mantissa, which the oracle's own e4m3 reading shows independently of
    the GPU: the GPU may not exceed that reading's disagreement by more than
    one part in four, plus 1e-3."""
    st = setup_for(etx, "batch500", 5, perturb=0.0)
    st.ctx.set_fp8_scales(st.model.fp8_act_scales)
    emb64 = st.oracle_emb()
    s, d, eo = O.build_graph(emb64, st.b.plane, st.b.hit_offsets, st.model.radius, st.model.k_max)
    args = (st.W, st.model.n_iters, st.b.x, st.b.y, st.b.z, s, d)
    z64 = O.gnn_forward(*args)
    thr = st.model.threshold_logit
    z8 = O.gnn_forward(*args, gemm="fp8", act_scales=st.model.fp8_act_scales)
    reading8_dis = float(((z8 > thr) != (z64 > thr)).mean())
    lab64 = O.connected_components(s, d, z64 > thr, st.b.hit_offsets)
    s_t, d_t, eo_t = cuda(s, torch.int32), cuda(d, torch.int32), cuda(eo, torch.int32)
    report = {}
    for dt in ("f32", "bf16", "bf16s", "fp8"):
        z = st.ctx.gnn_forward(st.x, st.y, st.z, s_t, d_t, eo_t, dtype=dt)
        lab, _ = st.ctx.edges_to_tracks(s_t, d_t, z, thr, eo_t, st.hoff)
        st.ctx.sync()
        zg = z.cpu().numpy().astype(np.float64)
        flip = (zg > thr) != (z64 > thr)
        near = np.abs(z64 - thr) <= NEAR_LOGIT[dt]
        report[dt] = dict(max_abs=float(np.abs(zg - z64).max()), mask_dis=float(flip.mean()),
                          flips_far=int((flip & ~near).sum()), near=int(near.sum()),
                          label_agree=float((lab.cpu().numpy() == lab64).mean()))
    for dt, r in report.items():
        print(f"{dt}: E={s.size} max|logit err| {r['max_abs']:.3e}, mask disagreement "
              f"{r['mask_dis']:.2e} ({r['near']} edges near the cut, {r['flips_far']} flips "
              f"outside), label agreement {r['label_agree']:.5f}")
    print(f"oracle e4m3 reading vs fp64: mask disagreement {reading8_dis:.2e}")
    for dt, r in report.items():
        assert r["max_abs"] <= MAX_ABS_VS_FP64[dt], dt
        assert r["flips_far"] == 0, dt
        assert r["label_agree"] >= LABEL_AGREE_MIN[dt], dt
        if dt in MASK_DIS_MAX:
            assert r["mask_dis"] <= MASK_DIS_MAX[dt], dt
    assert report["fp8"]["mask_dis"] <= 1.25 * reading8_dis + 1e-3
