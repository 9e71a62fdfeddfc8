"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, brute force, library routines (scipy, torch float64),
invariants and finite differences.  CPU only."""
import json
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import etx_oracle as O
from velo_synth import (WORKLOADS, ModelConfig, Z_PLANES, concat_events, global_particle_ids,
                        make_batch, make_weights, truth_edge_labels)

GOLDEN = Path(__file__).parent / "golden"
TINY = ModelConfig(emb_widths=(3, 16, 16, 4), hidden=16, n_iters=2, radius=1.0, k_max=4)


def tiny_batch(n_events=3, seed=0):
    return make_batch(WORKLOADS["plain"].recipe, n_events, 100 + seed)


def random_event_arrays(rng, n, n_planes=5, D=3):
    plane = np.sort(rng.integers(0, n_planes, size=n)).astype(np.int8)
    emb = rng.normal(size=(n, D))
    return emb, plane


# ---------------------------------------------------------------------------
# embedding (Sec. 5.1)
# ---------------------------------------------------------------------------
def test_embed_closed_form_golden():
    g = json.loads((GOLDEN / "embed_closed_form.json").read_text())
    w = {"emb_mu": np.zeros(3), "emb_sigma": np.ones(3),
         "emb0.W": np.eye(3), "emb0.b": np.zeros(3),
         "emb1.W": np.array(g["W1"], float), "emb1.b": np.array(g["b1"], float)}
    for case in g["cases"]:
        out = O.embed(w, 2, [case["x"]], [case["y"]], [case["z"]])[0]
        np.testing.assert_allclose(out, case["expected"], rtol=0, atol=1e-12)


def test_embed_normalisation_is_affine():
    # doubling sigma and shifting mu must equal transforming the raw features
    rng = np.random.default_rng(3)
    x, y, z = rng.normal(size=(3, 7)) * 10
    W = {"emb_mu": np.array([1.0, -0.5, 2.0]), "emb_sigma": np.array([2.0, 0.5, 4.0]),
         "emb0.W": np.eye(3), "emb0.b": np.full(3, 100.0),   # +100 keeps ReLU linear
         "emb1.W": np.eye(3), "emb1.b": np.full(3, -100.0)}
    out = O.embed(W, 2, x, y, z)
    r = np.hypot(x, y)
    phi = np.arctan2(y, x)
    ref = np.stack([(r - 1.0) / 2.0, (phi + 0.5) / 0.5, (z - 2.0) / 4.0], 1)
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_embed_matches_torch_float64():
    torch = pytest.importorskip("torch")
    wl = WORKLOADS["plain"]
    b = tiny_batch(1)
    W = make_weights(wl.model, b, perturb=0.2)
    depth = len(wl.model.emb_widths) - 1
    feats = np.stack([np.hypot(b.x.astype(float), b.y.astype(float)),
                      np.arctan2(b.y.astype(float), b.x.astype(float)), b.z.astype(float)], 1)
    t = (torch.tensor(feats) - torch.tensor(W["emb_mu"], dtype=torch.float64)) / \
        torch.tensor(W["emb_sigma"], dtype=torch.float64)
    layers = []
    for i in range(depth):
        lin = torch.nn.Linear(wl.model.emb_widths[i], wl.model.emb_widths[i + 1]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.tensor(W[f"emb{i}.W"], dtype=torch.float64))
            lin.bias.copy_(torch.tensor(W[f"emb{i}.b"], dtype=torch.float64))
        layers.append(lin)
        if i < depth - 1:
            layers.append(torch.nn.ReLU())
    with torch.no_grad():
        ref = torch.nn.Sequential(*layers)(t).numpy()
    np.testing.assert_allclose(O.embed(W, depth, b.x, b.y, b.z), ref, atol=1e-12)


# ---------------------------------------------------------------------------
# Eq. 1 and the rough graph (Sec. 5.1, Sec. 7.2)
# ---------------------------------------------------------------------------
def test_d2_matches_scipy_cdist():
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=(9, 8)), rng.normal(size=(11, 8))
    np.testing.assert_allclose(O.d2_fp64(a, b), cdist(a, b, "sqeuclidean"), rtol=1e-12)


def test_d2_fp32_properties():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(20, 8)).astype(np.float32)
    b = rng.normal(size=(30, 8)).astype(np.float32)
    s = O.d2_fp32(a, b)
    assert s.dtype == np.float32
    # exact symmetry: (a-b)^2 == (b-a)^2 in IEEE arithmetic
    np.testing.assert_array_equal(s, O.d2_fp32(b, a).T)
    np.testing.assert_array_equal(np.diag(O.d2_fp32(a, a)), np.zeros(20, np.float32))
    # within the FP32 rounding bound of the exact value (2D+1 roundings)
    ref = O.d2_fp64(a.astype(np.float64), b.astype(np.float64))
    assert np.all(np.abs(s - ref) <= (2 * 8 + 1) * 2.0 ** -24 * ref + 1e-30)


def brute_force_graph(emb, plane, hit_offsets, radius, k_max, fp32=False):
    """All-pairs reference written with plain Python loops."""
    edges = []
    for b in range(len(hit_offsets) - 1):
        lo, hi = int(hit_offsets[b]), int(hit_offsets[b + 1])
        for i in range(lo, hi):
            cands = []
            for j in range(lo, hi):
                if int(plane[j]) - int(plane[i]) not in (1, 2):
                    continue
                if fp32:
                    s = np.float32(0)
                    for d in range(emb.shape[1]):
                        t = np.float32(emb[i, d]) - np.float32(emb[j, d])
                        s = np.float32(s + np.float32(t * t))
                    r2 = np.float32(radius) * np.float32(radius)
                    d2 = float(s)
                    ok = s < r2
                else:
                    d2 = sum((float(emb[i, d]) - float(emb[j, d])) ** 2 for d in range(emb.shape[1]))
                    ok = d2 < radius * radius
                if ok:
                    cands.append((d2, j))
            cands.sort()
            for _, j in sorted(cands[:k_max], key=lambda t: t[1]):
                edges.append((i, j))
    return edges


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("fp32", [False, True])
def test_graph_brute_force(seed, fp32):
    rng = np.random.default_rng(seed)
    parts_emb, parts_plane, offs = [], [], [0]
    for n in (0, 37, 1, 52, 20):  # includes an empty and a single-hit event
        e, p = random_event_arrays(rng, n, n_planes=6, D=3)
        parts_emb.append(e)
        parts_plane.append(p)
        offs.append(offs[-1] + n)
    emb = np.concatenate(parts_emb) if offs[-1] else np.zeros((0, 3))
    plane = np.concatenate(parts_plane)
    if fp32:
        emb = emb.astype(np.float32)
    radius, k = 1.3, 3
    s, d, eo = O.build_graph(emb, plane, np.array(offs), radius, k,
                             precision="fp32" if fp32 else "fp64")
    ref = brute_force_graph(emb, plane, offs, radius, k, fp32=fp32)
    assert list(zip(s.tolist(), d.tolist())) == ref
    for b in range(len(offs) - 1):
        es = slice(int(eo[b]), int(eo[b + 1]))
        assert np.all((s[es] >= offs[b]) & (s[es] < offs[b + 1]))
        assert np.all((d[es] >= offs[b]) & (d[es] < offs[b + 1]))


def test_graph_special_cases():
    rng = np.random.default_rng(5)
    emb, _ = random_event_arrays(rng, 30, D=4)
    one_plane = np.full(30, 3, np.int8)
    s, d, eo = O.build_graph(emb, one_plane, np.array([0, 30]), 1e9, 10 ** 6)
    assert s.size == 0 and eo.tolist() == [0, 0]
    # r = inf, k = inf: complete p -> p+1, p+2 bipartite graph
    plane = np.sort(rng.integers(0, 6, size=30)).astype(np.int8)
    s, d, eo = O.build_graph(emb, plane, np.array([0, 30]), np.inf, 10 ** 6)
    n_p = np.bincount(plane, minlength=8)
    expected = sum(int(n_p[p]) * (int(n_p[p + 1]) + int(n_p[p + 2])) for p in range(6))
    assert s.size == expected
    assert np.all(np.isin(plane[d] - plane[s], [1, 2]))
    # k = 1 keeps the nearest candidate of every hit
    s1, d1, _ = O.build_graph(emb, plane, np.array([0, 30]), np.inf, 1)
    for i, j in zip(s1, d1):
        cand = np.nonzero(np.isin(plane - plane[i], [1, 2]))[0]
        dist = ((emb[cand] - emb[i]) ** 2).sum(1)
        assert j == cand[np.lexsort((cand, dist))[0]]
    # empty batch
    s, d, eo = O.build_graph(np.zeros((0, 4)), np.zeros(0, np.int8), np.array([0, 0, 0]), 1.0, 5)
    assert s.size == 0 and eo.tolist() == [0, 0, 0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_cut_is_strict(precision):
    # d2 exactly equal to r^2 (0.25 = 0.5^2, exact in binary) is outside the cut
    emb = np.array([[0.0, 0.0], [0.5, 0.0], [0.0, -0.25], [0.0, -0.5]])
    plane = np.array([0, 1, 1, 2], np.int8)
    s, d, _ = O.build_graph(emb, plane, np.array([0, 4]), 0.5, 8, precision=precision)
    assert list(zip(s.tolist(), d.tolist())) == [(0, 2), (2, 3)]


def test_graph_ties_broken_by_index():
    # three candidates at exactly the same distance: the lowest indices win
    emb = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])
    plane = np.array([0, 1, 1, 2], np.int8)
    s, d, _ = O.build_graph(emb, plane, np.array([0, 4]), 2.0, 2)
    assert list(zip(s.tolist(), d.tolist()))[:2] == [(0, 1), (0, 2)]


# ---------------------------------------------------------------------------
# messages (Eq. 4)
# ---------------------------------------------------------------------------
def test_messages_are_incidence_products():
    import scipy.sparse as sp
    rng = np.random.default_rng(7)
    N, E, H = 13, 40, 5
    src, dst = rng.integers(0, N, E), rng.integers(0, N, E)
    e = rng.normal(size=(E, H))
    m = O.messages(e, src, dst, N)
    S_out = sp.csr_matrix((np.ones(E), (src, np.arange(E))), shape=(N, E))
    S_in = sp.csr_matrix((np.ones(E), (dst, np.arange(E))), shape=(N, E))
    np.testing.assert_allclose(m[:, :H], S_out @ e, atol=1e-12)
    np.testing.assert_allclose(m[:, H:], S_in @ e, atol=1e-12)


# ---------------------------------------------------------------------------
# interaction network (Sec. 5.2)
# ---------------------------------------------------------------------------
def small_problem(H=16, L=2, n_events=2, seed=0, perturb=0.3):
    cfg = ModelConfig(emb_widths=(3, 16, 16, 4), hidden=H, n_iters=L, radius=1.5, k_max=6)
    b = tiny_batch(n_events, seed)
    W = make_weights(cfg, b, seed=seed, perturb=perturb)
    emb = O.embed(W, 3, b.x, b.y, b.z)
    s, d, eo = O.build_graph(emb, b.plane, b.hit_offsets, cfg.radius, cfg.k_max)
    return cfg, b, W, s, d, eo


def test_gnn_permutation_equivariance():
    cfg, b, W, s, d, _ = small_problem()
    z = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d)
    rng = np.random.default_rng(11)
    N, E = b.n_hits, s.size
    hp = rng.permutation(N)            # new index of hit i is inv[i]
    inv = np.empty(N, np.int64)
    inv[hp] = np.arange(N)
    ep = rng.permutation(E)
    z2 = O.gnn_forward(W, cfg.n_iters, b.x[hp], b.y[hp], b.z[hp], inv[s][ep], inv[d][ep])
    np.testing.assert_allclose(z2, z[ep], rtol=0, atol=1e-12)


def test_gnn_zero_step_networks_are_identity():
    # blocks whose last Linear and LN shift are zero add exactly 0 (ReLU(LN(0)*g + 0) = 0),
    # so L such steps must equal L = 0 (residual structure of the node/edge updates)
    cfg, b, W, s, d, _ = small_problem(L=3)
    W0 = dict(W)
    for k in range(3):
        for net in ("node", "edge"):
            W0[f"{net}{k}.W2"] = np.zeros_like(W[f"{net}{k}.W2"])
            W0[f"{net}{k}.b2"] = np.zeros_like(W[f"{net}{k}.b2"])
            W0[f"{net}{k}.be2"] = np.zeros_like(W[f"{net}{k}.be2"])
    z3 = O.gnn_forward(W0, 3, b.x, b.y, b.z, s, d)
    z0 = O.gnn_forward(W0, 0, b.x, b.y, b.z, s, d)
    np.testing.assert_array_equal(z3, z0)


def test_gnn_hidden1_closed_form():
    # H = 1: LayerNorm of one value is 0, so every block outputs ReLU(beta2); the
    # residual streams just add those constants and logit = W2 * ReLU(be1) + b2
    cfg = ModelConfig(emb_widths=(3, 16, 16, 4), hidden=1, n_iters=3)
    b = tiny_batch(1)
    W = make_weights(cfg, b, perturb=1.0)
    s = np.array([0, 0, 5]); d = np.array([3, 4, 9])
    z = O.gnn_forward(W, 3, b.x, b.y, b.z, s, d)
    e = max(W["edge_enc.be2"][0], 0.0) + sum(max(W[f"edge{k}.be2"][0], 0.0) for k in range(3))
    assert e >= 0  # e only enters through LN, which discards it for H = 1
    expected = float(W["cls.W2"][0, 0]) * max(float(W["cls.be1"][0]), 0.0) + float(W["cls.b2"][0])
    np.testing.assert_allclose(z, expected, atol=1e-12)


def test_gnn_event_batching_invariance():
    cfg, b, W, s, d, eo = small_problem(n_events=3)
    z = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d)
    for ev in range(3):
        lo, hi = int(b.hit_offsets[ev]), int(b.hit_offsets[ev + 1])
        es = slice(int(eo[ev]), int(eo[ev + 1]))
        zi = O.gnn_forward(W, cfg.n_iters, b.x[lo:hi], b.y[lo:hi], b.z[lo:hi], s[es] - lo, d[es] - lo)
        np.testing.assert_allclose(zi, z[es], atol=1e-12)


def torch_reference_forward(torch, W, L, x, y, z, src, dst):
    """Independent float64 restatement with torch.nn modules and index_add_."""
    t = lambda a: torch.tensor(np.asarray(a, np.float64))
    H = W["node_enc.W1"].shape[0]

    def block(X, p):
        seq = torch.nn.Sequential(torch.nn.Linear(X.shape[1], H), torch.nn.LayerNorm(H, eps=1e-5),
                                  torch.nn.ReLU(), torch.nn.Linear(H, H),
                                  torch.nn.LayerNorm(H, eps=1e-5), torch.nn.ReLU()).double()
        seq[0].weight = torch.nn.Parameter(t(W[p + ".W1"]))
        seq[0].bias = torch.nn.Parameter(t(W[p + ".b1"]))
        seq[1].weight = torch.nn.Parameter(t(W[p + ".g1"]))
        seq[1].bias = torch.nn.Parameter(t(W[p + ".be1"]))
        seq[3].weight = torch.nn.Parameter(t(W[p + ".W2"]))
        seq[3].bias = torch.nn.Parameter(t(W[p + ".b2"]))
        seq[4].weight = torch.nn.Parameter(t(W[p + ".g2"]))
        seq[4].bias = torch.nn.Parameter(t(W[p + ".be2"]))
        return seq(X), list(seq.parameters())

    params = {}
    si, di = torch.tensor(src), torch.tensor(dst)
    xin = (torch.stack([t(x), t(y), t(z)], 1) - t(W["gnn_mu"])) / t(W["gnn_sigma"])
    h, params["node_enc"] = block(xin, "node_enc")
    e, params["edge_enc"] = block(torch.cat([h[si], h[di]], 1), "edge_enc")
    N = h.shape[0]
    for k in range(L):
        mo = torch.zeros(N, H, dtype=torch.float64).index_add_(0, si, e)
        mi = torch.zeros(N, H, dtype=torch.float64).index_add_(0, di, e)
        dh, params[f"node{k}"] = block(torch.cat([h, mo, mi], 1), f"node{k}")
        h = h + dh
        de, params[f"edge{k}"] = block(torch.cat([e, h[si], h[di]], 1), f"edge{k}")
        e = e + de
    c1 = torch.nn.Linear(H, H).double()
    c1.weight = torch.nn.Parameter(t(W["cls.W1"]))
    c1.bias = torch.nn.Parameter(t(W["cls.b1"]))
    ln = torch.nn.LayerNorm(H, eps=1e-5).double()
    ln.weight = torch.nn.Parameter(t(W["cls.g1"]))
    ln.bias = torch.nn.Parameter(t(W["cls.be1"]))
    c2 = torch.nn.Linear(H, 1).double()
    c2.weight = torch.nn.Parameter(t(W["cls.W2"]))
    c2.bias = torch.nn.Parameter(t(W["cls.b2"]))
    logits = c2(torch.relu(ln(c1(e))))[:, 0]
    params["cls"] = [c1.weight, c1.bias, ln.weight, ln.bias, c2.weight, c2.bias]
    return logits, params


def test_gnn_forward_and_backward_match_torch_autograd():
    torch = pytest.importorskip("torch")
    cfg, b, W, s, d, _ = small_problem(H=16, L=2, n_events=2)
    cache = {}
    z = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d, cache)
    zt, params = torch_reference_forward(torch, W, cfg.n_iters, b.x, b.y, b.z, s, d)
    np.testing.assert_allclose(z, zt.detach().numpy(), atol=1e-10)
    y = truth_edge_labels(global_particle_ids(b), b.plane, s, d)
    loss, dz = O.weighted_bce(z, y, 10.0)
    lt = torch.nn.functional.binary_cross_entropy_with_logits(
        zt, torch.tensor(y, dtype=torch.float64), pos_weight=torch.tensor(10.0, dtype=torch.float64))
    np.testing.assert_allclose(loss, float(lt), rtol=1e-12)
    lt.backward()
    grads = O.gnn_backward(W, cache, dz)
    names = ["W1", "b1", "g1", "be1", "W2", "b2", "g2", "be2"]
    for blk, plist in params.items():
        nm = ["W1", "b1", "g1", "be1", "W2", "b2"] if blk == "cls" else names
        for n, p in zip(nm, plist):
            np.testing.assert_allclose(grads[f"{blk}.{n}"], p.grad.numpy(), rtol=1e-8, atol=1e-12,
                                       err_msg=f"{blk}.{n}")


def test_backward_central_finite_differences():
    cfg, b, W, s, d, _ = small_problem(H=16, L=2, n_events=1, perturb=0.3)
    y = truth_edge_labels(global_particle_ids(b), b.plane, s, d)
    Wd = {k: np.asarray(v, np.float64) for k, v in W.items()}
    cache = {}
    z = O.gnn_forward(Wd, cfg.n_iters, b.x, b.y, b.z, s, d, cache)
    _, dz = O.weighted_bce(z, y)
    grads = O.gnn_backward(Wd, cache, dz)
    rng = np.random.default_rng(0)
    h = 1e-6
    for name in ["node_enc.W1", "edge_enc.g2", "node0.W1", "node1.b1", "edge0.W2", "edge1.be1",
                 "cls.W1", "cls.W2", "cls.b2"]:
        flat = Wd[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        fd, an = [], []
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp, _ = O.weighted_bce(O.gnn_forward(Wd, cfg.n_iters, b.x, b.y, b.z, s, d), y)
            flat[i] = old - h
            lm, _ = O.weighted_bce(O.gnn_forward(Wd, cfg.n_iters, b.x, b.y, b.z, s, d), y)
            flat[i] = old
            fd.append((lp - lm) / (2 * h))
            an.append(grads[name].reshape(-1)[i])
        fd, an = np.array(fd), np.array(an)
        assert np.linalg.norm(fd - an) <= 1e-6 * max(np.linalg.norm(fd), 1e-8) + 1e-9, name


def test_weighted_bce_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    z = rng.normal(size=50) * 3
    y = (rng.uniform(size=50) < 0.3).astype(float)
    zt = torch.tensor(z, requires_grad=True)
    lt = torch.nn.functional.binary_cross_entropy_with_logits(
        zt, torch.tensor(y), pos_weight=torch.tensor(10.0, dtype=torch.float64))
    lt.backward()
    loss, dz = O.weighted_bce(z, y, 10.0)
    np.testing.assert_allclose(loss, float(lt), rtol=1e-13)
    np.testing.assert_allclose(dz, zt.grad.numpy(), rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------
# components (Sec. 5 overview, Sec. 7.3)
# ---------------------------------------------------------------------------
def scipy_labels(src, dst, mask, hit_offsets):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    N = int(hit_offsets[-1])
    m = np.asarray(mask, bool)
    A = sp.coo_matrix((np.ones(int(m.sum())), (np.asarray(src)[m], np.asarray(dst)[m])), shape=(N, N))
    _, comp = connected_components(A, directed=True, connection="weak")
    first = {}
    for i in range(N):
        first.setdefault(comp[i], i)
    ev = np.searchsorted(hit_offsets, np.arange(N), side="right") - 1
    return np.array([first[comp[i]] - hit_offsets[ev[i]] for i in range(N)], np.int64)


def test_cc_matches_scipy_random_graphs():
    rng = np.random.default_rng(9)
    offs = np.array([0, 0, 40, 41, 90, 150])
    src, dst = [], []
    for b in range(5):
        lo, hi = offs[b], offs[b + 1]
        if hi - lo < 2:
            continue
        ne = rng.integers(0, 2 * (hi - lo))
        src.append(rng.integers(lo, hi, ne))
        dst.append(rng.integers(lo, hi, ne))
    src, dst = np.concatenate(src), np.concatenate(dst)
    mask = rng.uniform(size=src.size) < 0.4
    lab = O.connected_components(src, dst, mask, offs)
    np.testing.assert_array_equal(lab, scipy_labels(src, dst, mask, offs))


def test_cc_golden_graphs():
    for case in json.loads((GOLDEN / "wcc_graphs.json").read_text())["cases"]:
        lab = O.connected_components(case["src"], case["dst"], case["mask"], case["hit_offsets"])
        assert lab.tolist() == case["labels"], case["name"]


def test_cc_truth_edges_reproduce_particles():
    b = make_batch(WORKLOADS["batch500"].recipe, 3, 1000)
    pid = global_particle_ids(b)
    src, dst = [], []
    for p in np.unique(pid[pid >= 0]):
        hits = np.nonzero(pid == p)[0]
        hits = hits[np.argsort(b.plane[hits], kind="stable")]
        src.append(hits[:-1])
        dst.append(hits[1:])
    src, dst = np.concatenate(src), np.concatenate(dst)
    y = truth_edge_labels(pid, b.plane, src, dst)
    assert y.min() == 1.0  # the generator's truth agrees: every such edge is genuine
    lab = O.connected_components(src, dst, np.ones(src.size, bool), b.hit_offsets)
    ev = np.searchsorted(b.hit_offsets, np.arange(b.n_hits), side="right") - 1
    glab = lab + b.hit_offsets[ev]
    for p in np.unique(pid[pid >= 0]):
        hits = np.nonzero(pid == p)[0]
        assert np.all(glab[hits] == hits.min())
    noise = np.nonzero(pid < 0)[0]
    assert np.all(glab[noise] == noise)


def test_plane_sweep_counterexample_worked_by_hand():
    # Sec. 7.3 sweep on the golden counter-example (hits e=0, a=1, c=2 on plane 0,
    # b=3, d=4 on plane 1): forward b <- min(3, a, c) = 1, d <- min(4, c, e) = 0;
    # backward a <- min(1, b) = 1, c <- min(2, b, d) = 0, e <- min(0, d) = 0.
    case = next(c for c in json.loads((GOLDEN / "wcc_graphs.json").read_text())["cases"]
                if c["name"] == "plane_sweep_counterexample")
    plane = np.array([0, 0, 0, 1, 1])
    lab = O.plane_sweep_components(case["src"], case["dst"], case["mask"], plane,
                                   case["hit_offsets"])
    assert lab.tolist() == [0, 1, 0, 1, 0]
    assert case["labels"] == [0, 0, 0, 0, 0]  # the exact components differ


def random_plane_graph(rng, sizes, n_planes=26, p_edge=0.15):
    """Plane-sorted events of random sizes with random edges p -> p+1, p+2."""
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    plane = np.concatenate([np.sort(rng.integers(0, n_planes, n)) for n in sizes]).astype(np.int8)
    src, dst = [], []
    for b in range(len(sizes)):
        lo, hi = offs[b], offs[b + 1]
        for i in range(lo, hi):
            for j in range(lo, hi):
                if 1 <= plane[j] - plane[i] <= 2 and rng.uniform() < p_edge:
                    src.append(i)
                    dst.append(j)
    return np.array(src, np.int64), np.array(dst, np.int64), plane, offs


def test_plane_sweep_refines_exact_components():
    inexact = 0
    for seed in range(12):
        rng = np.random.default_rng(seed)
        src, dst, plane, offs = random_plane_graph(rng, [0, 60, 1, 45, 80], p_edge=0.25)
        mask = rng.uniform(size=src.size) < 0.5
        sweep = O.plane_sweep_components(src, dst, mask, plane, offs)
        exact = O.connected_components(src, dst, mask, offs)
        ev = np.searchsorted(offs, np.arange(offs[-1]), side="right") - 1
        g_sweep = sweep + offs[ev]
        g_exact = exact + offs[ev]
        # every sweep label names a hit of the same exact component (so of the same
        # event), no lower than the component minimum; equal sweep labels imply
        # equal exact labels
        assert np.all(g_exact[g_sweep] == g_exact)
        assert np.all(sweep >= exact)
        for lab in np.unique(g_sweep):
            assert len(np.unique(g_exact[g_sweep == lab])) == 1
        inexact += int(np.any(sweep != exact))
    assert inexact > 0  # the random graphs exercise the inexactness


def test_plane_sweep_special_cases():
    rng = np.random.default_rng(5)
    src, dst, plane, offs = random_plane_graph(rng, [30, 30])
    none = O.plane_sweep_components(src, dst, np.zeros(src.size, bool), plane, offs)
    ev = np.searchsorted(offs, np.arange(offs[-1]), side="right") - 1
    np.testing.assert_array_equal(none, np.arange(offs[-1]) - offs[ev])
    # tracks (one hit per plane, consecutive): the sweep is exact
    b = make_batch(WORKLOADS["batch500"].recipe, 2, 1000)
    pid = global_particle_ids(b)
    s, d = [], []
    for p in np.unique(pid[pid >= 0]):
        hits = np.nonzero(pid == p)[0]
        hits = hits[np.argsort(b.plane[hits], kind="stable")]
        s.append(hits[:-1])
        d.append(hits[1:])
    s, d = np.concatenate(s), np.concatenate(d)
    keep = np.ones(s.size, bool)
    np.testing.assert_array_equal(O.plane_sweep_components(s, d, keep, b.plane, b.hit_offsets),
                                  O.connected_components(s, d, keep, b.hit_offsets))


def test_generator_geometry():
    b = make_batch(WORKLOADS["batch500"].recipe, 4, 1000)
    r = np.hypot(b.x.astype(float), b.y.astype(float))
    assert np.all((r > 5.0) & (r < 40.1))
    np.testing.assert_array_equal(b.z, Z_PLANES[b.plane].astype(np.float32))
    for e in range(b.n_events):
        p = b.plane[b.hit_offsets[e]:b.hit_offsets[e + 1]]
        assert np.all(np.diff(p.astype(int)) >= 0)
    # an event is identical alone and inside a batch
    one = make_batch(WORKLOADS["batch500"].recipe, 1, 1002)
    lo, hi = b.hit_offsets[2], b.hit_offsets[3]
    np.testing.assert_array_equal(one.x, b.x[lo:hi])
    # straight tracks from the vertex: hits of one particle share phi
    pid = b.particle_id[b.hit_offsets[0]:b.hit_offsets[1]]
    x, y = b.x[:b.hit_offsets[1]], b.y[:b.hit_offsets[1]]
    for p in np.unique(pid[pid >= 0])[:10]:
        ph = np.arctan2(y[pid == p], x[pid == p])
        assert np.ptp(np.unwrap(ph)) < 0.01
    assert concat_events([]).n_hits == 0
    assert math.isclose(float(np.diff(b.hit_offsets).mean()), 1700, rel_tol=0.5)


# ---------------------------------------------------------------------------
# BF16 operand reading of the mixed-precision configuration
# ---------------------------------------------------------------------------
def test_round_bf16_closed_forms():
    one = 1.0
    cases = [(one, one), (one + 2 ** -8, one),                 # tie -> even (down)
             (one + 3 * 2 ** -8, one + 2 ** -6),               # tie -> even (up)
             (one + 2 ** -8 + 2 ** -20, one + 2 ** -7),        # above the tie
             (-(one + 2 ** -9), -one), (0.0, 0.0), (2.0 ** -130, 2.0 ** -130)]
    for x, want in cases:
        assert O.round_bf16(np.array([x]))[0] == want, x


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    a = (rng.normal(size=4000) * np.exp(rng.uniform(-20, 20, 4000))).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_bf16(a), ref)


def test_gnn_bf16_reading_is_close_to_exact():
    cfg, b, W, s, d, _ = small_problem(H=16, L=2, n_events=1)
    z64 = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d)
    z16 = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d, gemm="bf16")
    err = np.abs(z16 - z64).max()
    assert 0 < err < 0.1   # rounding operands to 8 significand bits moves the logits a little


def test_round_e4m3_closed_forms():
    cases = [(1.0, 1.0), (1.0625, 1.0),                 # tie between 1 and 1.125 -> even (1)
             (1.1875, 1.25),                            # tie between 1.125 and 1.25 -> even (1.25)
             (448.0, 448.0), (500.0, 448.0), (-1e9, -448.0),   # saturation
             (2.0 ** -9, 2.0 ** -9), (2.0 ** -10, 0.0),        # smallest subnormal / tie to zero
             (3 * 2.0 ** -10, 2.0 ** -8),               # tie between 1 and 2 subnormal steps -> 2
             (0.0, 0.0), (240.0, 240.0), (232.0, 224.0)]      # 232: tie between 224 and 240 -> 224
    for x, want in cases:
        assert O.round_e4m3(np.array([x]))[0] == want, x


def test_round_e4m3_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    rng = np.random.default_rng(6)
    a = (rng.normal(size=4000) * np.exp(rng.uniform(-12, 5, 4000))).astype(np.float32)
    a = np.clip(a, -448, 448)
    ref = torch.from_numpy(a).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_e4m3(a), ref)


def test_quant_weight_e4m3_scale():
    W = np.array([[0.5, -2.0], [0.25, 0.0]], np.float32)
    q = O.quant_weight_e4m3(W)
    # the largest magnitude maps to 448 s, i.e. back to itself up to the rounding of s
    np.testing.assert_allclose(q[0, 1], -2.0, rtol=1e-6)
    assert np.all(np.abs(q - W) <= 2.0 ** -4 * np.abs(W) + 1e-12)


# ---------------------------------------------------------------------------
# track-finding metrics (Sec. 6, Table 1)
# ---------------------------------------------------------------------------
def test_track_metrics_worked_by_hand():
    case = json.loads((GOLDEN / "track_metrics.json").read_text())["cases"][0]
    m = O.track_metrics(case["labels"], case["particle_id"], case["hit_offsets"])
    exp = case["expected"]
    for k in O.TRACK_METRIC_COUNTS:
        assert m[k] == exp[k], k
    assert m["hit_eff_sum"] == pytest.approx(exp["hit_eff_sum"], abs=1e-15)
    assert m["hit_purity_sum"] == pytest.approx(exp["hit_purity_sum"], abs=1e-15)
    r = O.track_metric_rates(m)
    assert r["efficiency"] == exp["efficiency"]
    assert r["clone_rate"] == exp["clone_rate"]
    assert r["fake_rate"] == exp["fake_rate"][0] / exp["fake_rate"][1]
    assert r["hit_efficiency"] == exp["hit_efficiency"]
    assert r["hit_purity"] == exp["hit_purity"]


def truth_labels(batch):
    """Every particle's hits form one track (label = its first hit), noise alone."""
    lab = np.empty(batch.n_hits, np.int64)
    for b in range(batch.n_events):
        lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
        first = {}
        for i in range(lo, hi):
            p = int(batch.particle_id[i])
            lab[i] = i - lo if p < 0 else first.setdefault(p, i - lo)
    return lab


def test_track_metrics_of_the_truth_partition_are_perfect():
    batch = tiny_batch(4)
    m = O.track_metrics(truth_labels(batch), batch.particle_id, batch.hit_offsets)
    n_rec = sum(int((np.bincount(batch.event(b).particle_id[batch.event(b).particle_id >= 0]) >= 3).sum())
                for b in range(batch.n_events))
    assert n_rec > 50
    assert m["particles"] == m["matched_particles"] == m["candidates"] == m["tracks"] == n_rec
    assert m["candidate_particles"] == n_rec and m["unmatched_tracks"] == 0
    assert m["hit_eff_sum"] == m["hit_purity_sum"] == n_rec
    r = O.track_metric_rates(m)
    assert (r["efficiency"], r["clone_rate"], r["fake_rate"]) == (1.0, 0.0, 0.0)


def test_track_metrics_special_cases():
    # one event, every hit one label: one track, matched only if a particle holds 70%
    pid = np.array([0] * 7 + [1] * 3)
    m = O.track_metrics(np.zeros(10), pid, [0, 10])
    assert (m["tracks"], m["candidates"], m["particles"], m["matched_particles"]) == (1, 1, 2, 1)
    assert m["hit_eff_sum"] == 1.0 and m["hit_purity_sum"] == 0.7
    m = O.track_metrics(np.zeros(10), np.array([0] * 6 + [1] * 4), [0, 10])
    assert (m["tracks"], m["unmatched_tracks"], m["candidates"]) == (1, 1, 0)
    # every hit alone: no track, nothing matched
    m = O.track_metrics(np.arange(10), pid, [0, 10])
    assert (m["tracks"], m["candidates"], m["particles"], m["matched_particles"]) == (0, 0, 2, 0)
    # all noise: no particle; empty batch
    m = O.track_metrics(np.zeros(5), -np.ones(5), [0, 5])
    assert (m["particles"], m["tracks"], m["unmatched_tracks"]) == (0, 1, 1)
    m = O.track_metrics(np.zeros(0), np.zeros(0), [0, 0, 0])
    assert all(m[k] == 0 for k in O.TRACK_METRIC_COUNTS)
    assert math.isnan(O.track_metric_rates(m)["efficiency"])


def test_track_metrics_invariant_under_relabelling():
    rng = np.random.default_rng(11)
    batch = tiny_batch(3, seed=5)
    lab = truth_labels(batch)
    # split some particles in two and move hits between tracks, so that
    # clones and unmatched tracks occur
    for b in range(batch.n_events):
        lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
        n, seg, pid = hi - lo, lab[lo:hi], batch.particle_id[lo:hi]
        for p in np.unique(pid[pid >= 0])[::3]:
            hits = np.nonzero(pid == p)[0]
            seg[hits[len(hits) // 2:]] = hits[len(hits) // 2]
        pick = np.nonzero(rng.uniform(size=n) < 0.2)[0]
        seg[pick] = seg[rng.integers(0, n, size=pick.size)]
    m = O.track_metrics(lab, batch.particle_id, batch.hit_offsets)
    assert m["unmatched_tracks"] > 0 and m["candidates"] > m["candidate_particles"] > 0
    lab2, pid2 = lab.copy(), batch.particle_id.astype(np.int64).copy()
    for b in range(batch.n_events):
        lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
        perm = rng.permutation(hi - lo)
        lab2[lo:hi] = perm[lab[lo:hi]]                     # bijection of label values
        sig = pid2[lo:hi] >= 0
        pperm = rng.permutation(int(pid2[lo:hi][sig].max()) + 1)
        pid2[lo:hi][sig] = pperm[pid2[lo:hi][sig]]         # bijection of particle ids
        order = rng.permutation(hi - lo) + lo              # hit order inside the event
        lab2[lo:hi], pid2[lo:hi] = lab2[order].copy(), pid2[order].copy()
    m2 = O.track_metrics(lab2, pid2, batch.hit_offsets)
    for k in O.TRACK_METRIC_COUNTS:
        assert m2[k] == m[k], k
    assert m2["hit_eff_sum"] == pytest.approx(m["hit_eff_sum"], rel=1e-14)
    assert m2["hit_purity_sum"] == pytest.approx(m["hit_purity_sum"], rel=1e-14)


def test_track_metrics_against_a_contingency_table():
    """The same quantities from a (track, particle) count matrix built with
    scipy.sparse, on random labellings of a synthetic batch."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(2)
    batch = tiny_batch(3, seed=9)
    for trial in range(4):
        lab = truth_labels(batch)
        pick = rng.uniform(size=lab.size) < 0.1 * (trial + 1)
        for b in range(batch.n_events):
            lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
            sel = pick[lo:hi]
            lab[lo:hi][sel] = rng.integers(0, max(hi - lo, 1), size=int(sel.sum()))
        tot = dict.fromkeys(O.TRACK_METRIC_COUNTS, 0)
        tot["hit_eff_sum"] = tot["hit_purity_sum"] = 0.0
        for b in range(batch.n_events):
            lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
            n, l, p = hi - lo, lab[lo:hi], batch.particle_id[lo:hi].astype(np.int64)
            C = sp.coo_matrix((np.ones(n), (l, p + 1)), shape=(n, n + 1)).toarray()  # col 0 = noise
            size, phits = C.sum(1), C.sum(0)
            is_track = size >= 3
            cand = is_track[:, None] & (10 * C >= 7 * size[:, None])
            cand[:, 0] = False
            tr, pa = np.nonzero(cand)
            tot["particles"] += int((phits[1:] >= 3).sum())
            tot["matched_particles"] += int(np.unique(pa[phits[pa] >= 3]).size)
            tot["candidates"] += tr.size
            tot["candidate_particles"] += int(np.unique(pa).size)
            tot["tracks"] += int(is_track.sum())
            tot["unmatched_tracks"] += int(is_track.sum()) - tr.size
            tot["hit_eff_sum"] += float((C[tr, pa] / phits[pa]).sum())
            tot["hit_purity_sum"] += float((C[tr, pa] / size[tr]).sum())
        m = O.track_metrics(lab, batch.particle_id, batch.hit_offsets)
        for k in O.TRACK_METRIC_COUNTS:
            assert m[k] == tot[k], (trial, k)
        assert m["hit_eff_sum"] == pytest.approx(tot["hit_eff_sum"], rel=1e-13)
        assert m["hit_purity_sum"] == pytest.approx(tot["hit_purity_sum"], rel=1e-13)


# ---------------------------------------------------------------------------
# embedding training (Sec. 5.1, Eq. 2-3)
# ---------------------------------------------------------------------------
def training_batch(n_events=2, seed=3):
    from velo_synth import drop_noise
    return drop_noise(tiny_batch(n_events, seed))


def test_embedding_pairs_against_brute_force():
    b = training_batch()
    rng = np.random.default_rng(4)
    emb = rng.normal(size=(b.n_hits, 3)).astype(np.float32)
    rand = rng.integers(0, 2 ** 32, size=b.n_hits, dtype=np.uint64)
    radius, k_max = 1.2, 5
    q, a, g = O.embedding_pairs(emb, b.plane, b.particle_id, b.hit_offsets, radius, k_max, rand)
    r2 = np.float32(radius) * np.float32(radius)
    want = {}
    for ev in range(b.n_events):
        lo, hi = int(b.hit_offsets[ev]), int(b.hit_offsets[ev + 1])
        pid, pl = b.particle_id[lo:hi], b.plane[lo:hi].astype(int)
        sizes = {p: int((pid == p).sum()) for p in set(pid.tolist())}
        for i in range(hi - lo):
            if sizes[int(pid[i])] < 3:
                continue
            cand = [j for j in range(hi - lo) if pl[j] - pl[i] in (1, 2)]
            scored = sorted((float(O.d2_fp32(emb[lo + i][None], emb[lo + j][None])[0, 0]), j)
                            for j in cand)
            chosen = {j for _, j in [(d, j) for d, j in scored if d < r2][:k_max]}
            if cand:
                chosen.add(cand[int(rand[lo + i]) % len(cand)])
            later = [j for j in range(i + 1, hi - lo) if pid[j] == pid[i]]
            if later and pl[later[0]] - pl[i] <= 2:
                chosen.add(later[0])
            for j in chosen:
                want[(lo + i, lo + j)] = bool(later and later[0] == j)
    got = {(int(x), int(y)): bool(f) for x, y, f in zip(q, a, g)}
    assert got == want
    assert list(zip(q.tolist(), a.tolist())) == sorted(got)
    assert 0 < g.sum() < g.size


def test_embedding_pairs_truth_and_structure():
    b = training_batch(3, seed=8)
    rng = np.random.default_rng(1)
    emb = rng.normal(size=(b.n_hits, 4)).astype(np.float32)
    rand = rng.integers(0, 2 ** 32, size=b.n_hits, dtype=np.uint64)
    q, a, g = O.embedding_pairs(emb, b.plane, b.particle_id, b.hit_offsets, 1.5, 8, rand)
    # the genuine flag is the generator's own genuine-edge definition
    y = truth_edge_labels(global_particle_ids(b), b.plane, q, a)
    assert np.array_equal(g, y > 0)
    gap = b.plane[a].astype(int) - b.plane[q].astype(int)
    assert set(gap.tolist()) <= {1, 2}
    is_q = O.embedding_queries(b.particle_id, b.hit_offsets)
    assert is_q[q].all()
    # every query with a successor within two planes has its genuine pair
    nxt = O.next_hit_of_particle(b.particle_id, b.hit_offsets)
    need = {(i, int(nxt[i])) for i in np.nonzero(is_q)[0]
            if nxt[i] >= 0 and b.plane[nxt[i]] - b.plane[i] <= 2}
    assert need <= set(zip(q.tolist(), a.tolist()))
    # radius 0: only the random and the genuine pair of each query remain
    q0, a0, g0 = O.embedding_pairs(emb, b.plane, b.particle_id, b.hit_offsets, 0.0, 8, rand)
    per_q = np.bincount(q0, minlength=b.n_hits)
    assert per_q.max() <= 2 and set(zip(q0[g0].tolist(), a0[g0].tolist())) == need
    # query definition: particles with at least three hits
    counts = {}
    for ev in range(b.n_events):
        lo, hi = int(b.hit_offsets[ev]), int(b.hit_offsets[ev + 1])
        for i in range(lo, hi):
            counts[(ev, int(b.particle_id[i]))] = counts.get((ev, int(b.particle_id[i])), 0) + 1
    ev_of = np.searchsorted(b.hit_offsets, np.arange(b.n_hits), side="right") - 1
    assert all(is_q[i] == (counts[(int(ev_of[i]), int(b.particle_id[i]))] >= 3)
               for i in range(b.n_hits))


def test_hinge_loss_closed_forms():
    emb = np.array([[0.0, 0.0], [0.3, 0.4], [3.0, 4.0]])
    L, Lg, Lf, d = O.hinge_embedding_loss(emb, [0], [1], [True], w_genuine=2.0)
    assert (L, Lg, Lf) == pytest.approx((0.5, 0.25, 0.0), abs=1e-15)
    np.testing.assert_allclose(d[0], [-1.2, -1.6], atol=1e-15)
    np.testing.assert_allclose(d[1], [1.2, 1.6], atol=1e-15)
    L, Lg, Lf, d = O.hinge_embedding_loss(emb, [0, 0], [1, 2], [False, False])
    assert (L, Lg, Lf) == pytest.approx((0.375, 0.0, 0.375), abs=1e-15)   # (0.75 + 0) / 2
    np.testing.assert_allclose(d[0], [0.3, 0.4], atol=1e-15)               # -2 (e0 - e1) / 2
    assert not d[2].any()                                                   # d2 = 25 > margin
    L, *_ = O.hinge_embedding_loss(emb, [0], [2], [False], margin=25.0)    # d2 = margin: inactive
    assert L == 0.0
    L, Lg, Lf, d = O.hinge_embedding_loss(emb, [], [], [])
    assert (L, Lg, Lf) == (0.0, 0.0, 0.0) and not d.any()


def test_hinge_loss_against_torch_autograd_and_differences():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    emb = rng.normal(scale=0.6, size=(12, 3))
    q = rng.integers(0, 12, 40)
    a = (q + 1 + rng.integers(0, 11, 40)) % 12
    g = rng.uniform(size=40) < 0.3
    L, Lg, Lf, d = O.hinge_embedding_loss(emb, q, a, g, margin=1.0, w_genuine=3.0)
    t = torch.tensor(emb, dtype=torch.float64, requires_grad=True)
    d2 = ((t[torch.tensor(q)] - t[torch.tensor(a)]) ** 2).sum(1)
    gt = torch.tensor(g)
    lt = torch.relu(1.0 - d2[~gt]).mean() + 3.0 * d2[gt].mean()
    lt.backward()
    assert L == pytest.approx(lt.item(), rel=1e-14)
    np.testing.assert_allclose(d, t.grad.numpy(), rtol=1e-12, atol=1e-14)
    h = 1e-6
    for (i, k) in [(0, 0), (5, 2), (11, 1)]:
        e2 = emb.copy(); e2[i, k] += h
        e1 = emb.copy(); e1[i, k] -= h
        fd = (O.hinge_embedding_loss(e2, q, a, g, 1.0, 3.0)[0]
              - O.hinge_embedding_loss(e1, q, a, g, 1.0, 3.0)[0]) / (2 * h)
        assert d[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_embed_backward_against_torch_autograd_and_differences():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    widths = (3, 16, 16, 4)
    W = {"emb_mu": rng.normal(size=3), "emb_sigma": rng.uniform(0.5, 2.0, 3)}
    for i in range(3):
        W[f"emb{i}.W"] = rng.normal(scale=0.5, size=(widths[i + 1], widths[i]))
        W[f"emb{i}.b"] = rng.normal(scale=0.3, size=widths[i + 1])
    x, y, z = rng.normal(size=(3, 30)) * np.array([[10.0], [10.0], [100.0]])
    up = rng.normal(size=(30, 4))
    grads = O.embed_backward(W, 3, x, y, z, up)
    feat = torch.tensor(O.normalise(O.cylindrical(x, y, z), W["emb_mu"], W["emb_sigma"]))
    lins = [torch.nn.Linear(widths[i], widths[i + 1]).double() for i in range(3)]
    with torch.no_grad():
        for i, lin in enumerate(lins):
            lin.weight.copy_(torch.tensor(W[f"emb{i}.W"]))
            lin.bias.copy_(torch.tensor(W[f"emb{i}.b"]))
    h = feat
    for i, lin in enumerate(lins):
        h = lin(h)
        if i < 2:
            h = torch.relu(h)
    (h * torch.tensor(up)).sum().backward()
    for i, lin in enumerate(lins):
        np.testing.assert_allclose(grads[f"emb{i}.W"], lin.weight.grad.numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(grads[f"emb{i}.b"], lin.bias.grad.numpy(), rtol=1e-12, atol=1e-12)
    f = lambda WW: float((O.embed(WW, 3, x, y, z) * up).sum())
    for name, idx in [("emb0.W", (3, 1)), ("emb1.b", (7,)), ("emb2.W", (2, 9))]:
        Wp = {k: v.copy() for k, v in W.items()}; Wp[name][idx] += 1e-6
        Wm = {k: v.copy() for k, v in W.items()}; Wm[name][idx] -= 1e-6
        assert grads[name][idx] == pytest.approx((f(Wp) - f(Wm)) / 2e-6, rel=1e-5, abs=1e-7)


def test_embedding_pairs_worked_by_hand():
    g = json.loads((GOLDEN / "embedding_pairs.json").read_text())
    ev = g["event"]
    emb = np.zeros((8, 2), np.float32)
    for case in g["cases"]:
        q, a, gen = O.embedding_pairs(emb, ev["plane"], ev["particle_id"], [0, 8], 0.0, 5,
                                      np.array(case["rand"], np.uint64))
        assert [[int(x), int(y), bool(f)] for x, y, f in zip(q, a, gen)] == case["pairs"]


def test_hinge_gradient_vanishes_at_the_margin():
    emb = np.array([[0.0, 0.0], [3.0, 4.0]])
    L, _, _, d = O.hinge_embedding_loss(emb, [0], [1], [False], margin=25.0)
    assert L == 0.0 and not d.any()


# ---------------------------------------------------------------------------
# triplets (Sec. 5.3)
# ---------------------------------------------------------------------------
def random_edges(rng, n_hits=30, n_planes=6, p=0.3):
    plane = np.sort(rng.integers(0, n_planes, n_hits))
    e = [(i, j) for i in range(n_hits) for j in range(n_hits)
         if 1 <= plane[j] - plane[i] <= 2 and rng.uniform() < p]
    src = np.array([a for a, _ in e], np.int64)
    dst = np.array([b for _, b in e], np.int64)
    return src, dst


def test_triplets_against_brute_force_pairs():
    rng = np.random.default_rng(12)
    for trial in range(5):
        src, dst = random_edges(rng)
        mask = rng.uniform(size=src.size) < 0.6
        f, s, k = O.build_triplets(src, dst, mask, 30)
        want = []
        kept = np.nonzero(mask)[0].tolist()
        for a in kept:
            for b in kept:
                if a == b:
                    continue
                if dst[a] == src[b]:
                    want.append((O.TRIPLET_ARTICULATION, int(dst[a]), a, b))
                if a < b and src[a] == src[b]:
                    want.append((O.TRIPLET_LEFT_ELBOW, int(src[a]), a, b))
                if a < b and dst[a] == dst[b]:
                    want.append((O.TRIPLET_RIGHT_ELBOW, int(dst[a]), a, b))
        want.sort()
        assert [(int(t), int(f_), int(s_)) for t, f_, s_ in zip(k, f, s)] == [(t, a, b) for t, _, a, b in want]
        # closed-form counts from the kept in- and out-degrees
        indeg = np.bincount(dst[mask], minlength=30)
        outdeg = np.bincount(src[mask], minlength=30)
        assert (k == 0).sum() == int((indeg * outdeg).sum())
        assert (k == 1).sum() == int((outdeg * (outdeg - 1) // 2).sum())
        assert (k == 2).sum() == int((indeg * (indeg - 1) // 2).sum())


def test_triplets_of_a_track_chain_are_articulations():
    # hits 0..5 on planes 0..5, edges i -> i+1: n-2 articulations, no elbows
    src, dst = np.arange(5), np.arange(1, 6)
    f, s, k = O.build_triplets(src, dst, np.ones(5, bool), 6)
    assert k.tolist() == [0] * 4 and f.tolist() == [0, 1, 2, 3] and s.tolist() == [1, 2, 3, 4]
    # a fork at hit 1 (1 -> 2 and 1 -> 3) and a merge at hit 4 (2 -> 4, 3 -> 4)
    src, dst = np.array([0, 1, 1, 2, 3]), np.array([1, 2, 3, 4, 4])
    f, s, k = O.build_triplets(src, dst, np.ones(5, bool), 5)
    assert list(zip(k.tolist(), f.tolist(), s.tolist())) == [
        (0, 0, 1), (0, 0, 2), (0, 1, 3), (0, 2, 4), (1, 1, 2), (2, 3, 4)]
    f, s, k = O.build_triplets(src, dst, np.zeros(5, bool), 5)
    assert f.size == 0


def test_triplet_classifiers_against_torch():
    torch = pytest.importorskip("torch")
    from velo_synth import make_triplet_weights
    cfg = ModelConfig(emb_widths=(3, 8, 4), hidden=16, n_iters=1, radius=1.0, k_max=4)
    tw = make_triplet_weights(cfg, perturb=0.3)
    rng = np.random.default_rng(2)
    e = rng.normal(size=(20, 16))
    f, s = rng.integers(0, 20, 30), rng.integers(0, 20, 30)
    k = rng.integers(0, 3, 30)
    z = O.triplet_logits(tw, e, f, s, k)
    for name, sel in (("art", k == 0), ("elb", k != 0)):
        l1 = torch.nn.Linear(32, 16).double()
        ln = torch.nn.LayerNorm(16, eps=1e-5).double()
        l2 = torch.nn.Linear(16, 1).double()
        with torch.no_grad():
            l1.weight.copy_(torch.tensor(tw[f"{name}.W1"])); l1.bias.copy_(torch.tensor(tw[f"{name}.b1"]))
            ln.weight.copy_(torch.tensor(tw[f"{name}.g1"])); ln.bias.copy_(torch.tensor(tw[f"{name}.be1"]))
            l2.weight.copy_(torch.tensor(tw[f"{name}.W2"])); l2.bias.copy_(torch.tensor(tw[f"{name}.b2"]))
            x = torch.cat([torch.tensor(e[f[sel]]), torch.tensor(e[s[sel]])], 1)
            want = l2(torch.relu(ln(l1(x))))[:, 0].numpy()
        np.testing.assert_allclose(z[sel], want, rtol=1e-12, atol=1e-12)


def test_backward_recompute_reading():
    """gnn_backward(recompute=True): on an exact forward it is the plain
    backward (to rounding); on a BF16-reading forward it differs from the exact
    gradient by about the BF16 forward error, and recomputing changes the
    result against differentiating the rounded internals."""
    from velo_synth import ModelConfig, WORKLOADS, make_batch, make_weights
    cfg = ModelConfig(emb_widths=(3, 32, 32, 4), hidden=16, n_iters=2, radius=1.5, k_max=16)
    wl = WORKLOADS["plain"]
    b = make_batch(wl.recipe, 1, 5001)
    W = make_weights(cfg, wl.calibration(), perturb=0.3)
    emb = O.embed(W, 3, b.x, b.y, b.z)
    s, d, _ = O.build_graph(emb, b.plane, b.hit_offsets, cfg.radius, cfg.k_max)
    rng = np.random.default_rng(0)
    dz = rng.normal(size=s.size)
    c64 = {}
    O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d, cache=c64)
    g64 = O.gnn_backward(W, c64, dz)
    g64r = O.gnn_backward(W, c64, dz, recompute=True)
    for k in g64:
        np.testing.assert_allclose(g64r[k], g64[k], rtol=1e-12, atol=1e-14)
    c16 = {}
    O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d, cache=c16, gemm="bf16")
    g16r = O.gnn_backward(W, c16, dz, recompute=True)
    g16 = O.gnn_backward(W, c16, dz)
    rel = lambda a, b_: np.linalg.norm(a - b_) / max(np.linalg.norm(b_), 1e-30)
    # the BF16 forward moves the gradients by a few per cent (activations one BF16
    # step off, ReLU masks and LayerNorm of small spreads are sensitive)
    devs = [rel(g16r[k], g64[k]) for k in g64]
    assert 1e-3 < np.median(devs) < 0.15 and max(devs) < 0.5
    assert max(rel(g16r[k], g16[k]) for k in g64) > 1e-6


def test_forward_cache_from_streams_matches_the_forward():
    """forward_cache_from_streams, given the residual streams of the oracle's own
    forward, rebuilds that forward's block inputs exactly, so the reverse pass
    taken at given checkpoints is the one taken along the forward (a block fed
    h^k where it needs h^(k+1), or e^(k+1) where it needs e^k, fails here)."""
    from velo_synth import ModelConfig, WORKLOADS, make_batch, make_weights
    cfg = ModelConfig(emb_widths=(3, 32, 32, 4), hidden=16, n_iters=3, radius=1.5, k_max=16)
    wl = WORKLOADS["plain"]
    b = make_batch(wl.recipe, 1, 5002)
    W = make_weights(cfg, wl.calibration(), perturb=0.3)
    emb = O.embed(W, 3, b.x, b.y, b.z)
    s, d, _ = O.build_graph(emb, b.plane, b.hit_offsets, cfg.radius, cfg.k_max)
    H, L = cfg.hidden, cfg.n_iters
    for gemm in ("fp64", "bf16"):
        c = {}
        O.gnn_forward(W, L, b.x, b.y, b.z, s, d, cache=c, gemm=gemm)
        hs = [c[f"node{k}"]["X"][:, :H] for k in range(L)]
        hL = np.zeros_like(hs[0])
        hL[s] = c[f"edge{L - 1}"]["X"][:, H:2 * H]
        hL[d] = c[f"edge{L - 1}"]["X"][:, 2 * H:]
        es = [c[f"edge{k}"]["X"][:, :H] for k in range(L)] + [c["cls"]["X"]]
        r = O.forward_cache_from_streams(W, L, b.x, b.y, b.z, s, d, hs + [hL], es)
        for name in ["node_enc", "edge_enc", "cls"] + [f"{p}{k}" for k in range(L) for p in ("node", "edge")]:
            np.testing.assert_array_equal(r[name]["X"], c[name]["X"])
        dz = np.random.default_rng(1).normal(size=s.size)
        g0 = O.gnn_backward(W, c, dz, recompute=True)
        g1 = O.gnn_backward(W, r, dz, recompute=True)
        for k in g0:
            np.testing.assert_array_equal(g1[k], g0[k])


def test_focal_loss_pins():
    """The sigmoid focal loss (Sec. 5.2, Eq. 5): gamma = 0 with alpha = 1/2 is
    half the plain binary cross-entropy (pinned separately against torch);
    hand values at z = 0 (p = 1/2: alpha / 4 ln 2 and (1 - alpha) / 4 ln 2);
    its gradient against central differences; an edge classified with a large
    margin costs next to nothing."""
    rng = np.random.default_rng(3)
    z = rng.normal(scale=3.0, size=200)
    y = (rng.random(200) < 0.3).astype(np.float64)
    lb, db = O.weighted_bce(z, y, 1.0)
    lf, df = O.focal_loss(z, y, alpha=0.5, gamma=0.0)
    assert abs(lf - 0.5 * lb) <= 1e-12 * abs(lb)
    np.testing.assert_allclose(df, 0.5 * db, rtol=1e-12, atol=1e-15)
    l, d = O.focal_loss(np.zeros(2), np.array([1.0, 0.0]))
    ln2 = np.log(2.0)
    assert abs(l - 0.5 * (0.25 * 0.25 * ln2 + 0.75 * 0.25 * ln2)) <= 1e-15
    # at z = 0 (p = 1/2, gamma = 2): d/dz for y = 1 is 0.25 * 0.25 * (2 * 0.5 * -ln2 - 0.5) / 2
    assert abs(d[0] - 0.25 * 0.25 * (-ln2 - 0.5) / 2) <= 1e-15
    h = 1e-6
    for i in rng.choice(200, size=12, replace=False):
        zp, zm = z.copy(), z.copy()
        zp[i] += h
        zm[i] -= h
        fd = (O.focal_loss(zp, y)[0] - O.focal_loss(zm, y)[0]) / (2 * h)
        # central differences carry ~eps * loss / h = 2e-11 of rounding
        assert abs(O.focal_loss(z, y)[1][i] - fd) <= 1e-5 * abs(fd) + 1e-10
    big, _ = O.focal_loss(np.array([20.0, -20.0]), np.array([1.0, 0.0]))
    assert 0.0 < big < 1e-20
