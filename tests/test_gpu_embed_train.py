"""Embedding training (Sec. 5.1, Eq. 2-3) on the GPU against the oracle:
the training pairs bit-exact (integers and flags; the graph rule's cut and
nearest-k decided in FP32 on both sides), the hinge loss and its embedding
gradient, and the embedding MLP's reverse pass within FP32 tolerances."""
import json
from pathlib import Path

import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import WORKLOADS, compact_particle_ids, drop_noise, pack_blob

pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).parent / "golden"


@pytest.fixture(scope="module")
def etx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import etx as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rand_bits(rng, n):
    u = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    return u, cuda(u.view(np.int32))


def gpu_pairs(ctx, emb, plane, pid, hoff, radius, k_max, rand_t, capacity=None):
    n = plane.shape[0]
    cap = n * (k_max + 2) if capacity is None else capacity
    pq, pa, pg, npairs = ctx.embedding_pairs(cuda(emb), cuda(plane), cuda(pid), cuda(hoff), radius,
                                             k_max, rand_t, cap)
    ctx.sync()
    k = int(npairs.item())
    return pq[:k].cpu().numpy(), pa[:k].cpu().numpy(), pg[:k].cpu().numpy().astype(bool)


def test_pairs_worked_by_hand(etx):
    g = json.loads((GOLDEN / "embedding_pairs.json").read_text())
    ev = g["event"]
    m = WORKLOADS["plain"].model
    ctx = etx.Context(m, 4, 64, 64)
    D = m.emb_widths[-1]
    for case in g["cases"]:
        r = np.array(case["rand"], np.uint32)
        q, a, f = gpu_pairs(ctx, np.zeros((8, D), np.float32), np.array(ev["plane"], np.int8),
                            np.array(ev["particle_id"], np.int32), np.array([0, 8], np.int32), 0.0, 5,
                            cuda(r.view(np.int32)))
        assert [[int(x), int(y), bool(z)] for x, y, z in zip(q, a, f)] == case["pairs"]


@pytest.mark.parametrize("k_max,radius,seed", [(50, float(np.sqrt(1.5)), 0), (4, 1.0, 1), (1, 2.0, 2)])
def test_pairs_match_oracle(etx, k_max, radius, seed):
    rng = np.random.default_rng(seed)
    wl = WORKLOADS["plain"]
    b = drop_noise(wl.batch(6))
    pid = compact_particle_ids(b)
    D = wl.model.emb_widths[-1]
    emb = (rng.normal(size=(b.n_hits, D)) * 0.8).astype(np.float32)
    r, rt = rand_bits(rng, b.n_hits)
    ctx = etx.Context(wl.model, b.n_events, b.n_hits, 1)
    q, a, f = gpu_pairs(ctx, emb, b.plane, pid, b.hit_offsets, radius, k_max, rt)
    qo, ao, fo = O.embedding_pairs(emb, b.plane, pid, b.hit_offsets, radius, k_max, r,
                                   precision="fp32")
    assert np.array_equal(q, qo) and np.array_equal(a, ao) and np.array_equal(f, fo)
    assert 0 < f.sum() < f.size


def test_pairs_capacity_and_noise_are_reported(etx):
    wl = WORKLOADS["plain"]
    b = drop_noise(wl.batch(2))
    pid = compact_particle_ids(b)
    emb = np.zeros((b.n_hits, wl.model.emb_widths[-1]), np.float32)
    _, rt = rand_bits(np.random.default_rng(0), b.n_hits)
    ctx = etx.Context(wl.model, b.n_events, b.n_hits, 1)
    out = ctx.embedding_pairs(cuda(emb), cuda(b.plane), cuda(pid), cuda(b.hit_offsets), 1.0, 8, rt, 5)
    with pytest.raises(etx.EtxError) as e:
        ctx.sync()
    assert e.value.status == etx.ETX_ERR_CAPACITY
    assert int(out[3].item()) == 0                        # nothing exposed on overflow
    bad = pid.copy()
    bad[3] = -1                                           # a noise hit left in
    ctx.embedding_pairs(cuda(emb), cuda(b.plane), cuda(bad), cuda(b.hit_offsets), 1.0, 8, rt, 10 ** 5)
    with pytest.raises(etx.EtxError):
        ctx.sync()


def test_hinge_loss_matches_oracle(etx):
    rng = np.random.default_rng(5)
    wl = WORKLOADS["plain"]
    b = drop_noise(wl.batch(4))
    pid = compact_particle_ids(b)
    D = wl.model.emb_widths[-1]
    emb = (rng.normal(size=(b.n_hits, D)) * 0.4).astype(np.float32)
    r, _ = rand_bits(rng, b.n_hits)
    q, a, g = O.embedding_pairs(emb, b.plane, pid, b.hit_offsets, 1.0, 20, r, precision="fp32")
    ctx = etx.Context(wl.model, b.n_events, b.n_hits, 1)
    cap = q.size + 7                                     # grid sized by the capacity
    pad = lambda v, dt: np.concatenate([v.astype(dt), np.zeros(7, dt)])
    loss, d = ctx.hinge_loss(cuda(emb), cuda(pad(q, np.int32)), cuda(pad(a, np.int32)),
                             cuda(pad(g, np.uint8)), cuda(np.array([q.size], np.int32)), 1.0, 2.5)
    ctx.sync()
    L, Lg, Lf, dref = O.hinge_embedding_loss(emb, q, a, g, 1.0, 2.5)
    np.testing.assert_allclose(loss.cpu().numpy(), [L, Lg, Lf], rtol=2e-6)
    # FP32 terms summed per hit: error far below 1e-5 of the largest entry
    dg = d.cpu().numpy()
    assert np.abs(dg - dref).max() <= 1e-5 * np.abs(dref).max()
    assert cap > q.size


def test_hinge_loss_fixed_order_and_any_pair_order(etx):
    """The hinge loss and its gradient come out bit for bit the same on a
    repeat; pairs in any order (here shuffled) give the oracle's values; a
    pair with an index out of range is skipped and reported; a pair count
    above the capacity is reported and uses no pair."""
    rng = np.random.default_rng(11)
    wl = WORKLOADS["batch500"]
    b = drop_noise(wl.batch(6))
    pid = compact_particle_ids(b)
    D = wl.model.emb_widths[-1]
    emb = (rng.normal(size=(b.n_hits, D)) * 0.3).astype(np.float32)
    r, _ = rand_bits(rng, b.n_hits)
    q, a, g = O.embedding_pairs(emb, b.plane, pid, b.hit_offsets, 1.2, 30, r, precision="fp32")
    ctx = etx.Context(wl.model, b.n_events, b.n_hits, 1)
    args = (cuda(emb), cuda(q.astype(np.int32)), cuda(a.astype(np.int32)), cuda(g.astype(np.uint8)),
            cuda(np.array([q.size], np.int32)), 1.0, 2.0)
    l1, d1 = (t.clone() for t in ctx.hinge_loss(*args))
    l2, d2 = ctx.hinge_loss(*args)
    ctx.sync()
    assert torch.equal(l1, l2) and torch.equal(d1, d2)
    L, Lg, Lf, dref = O.hinge_embedding_loss(emb, q, a, g, 1.0, 2.0)
    np.testing.assert_allclose(l1.cpu().numpy(), [L, Lg, Lf], rtol=2e-6)
    assert np.abs(d1.cpu().numpy() - dref).max() <= 1e-5 * np.abs(dref).max()
    perm = rng.permutation(q.size)
    ls, ds = ctx.hinge_loss(cuda(emb), cuda(q[perm].astype(np.int32)), cuda(a[perm].astype(np.int32)),
                            cuda(g[perm].astype(np.uint8)), cuda(np.array([q.size], np.int32)), 1.0, 2.0)
    ctx.sync()
    np.testing.assert_allclose(ls.cpu().numpy(), [L, Lg, Lf], rtol=2e-6)
    assert np.abs(ds.cpu().numpy() - dref).max() <= 1e-5 * np.abs(dref).max()
    # an index out of range: that pair is left out of the loss and the gradient
    qb = q.astype(np.int32).copy()
    qb[0] = b.n_hits
    ctx.hinge_loss(cuda(emb), cuda(qb), cuda(a.astype(np.int32)), cuda(g.astype(np.uint8)),
                   cuda(np.array([q.size], np.int32)), 1.0, 2.0)
    with pytest.raises(etx.EtxError):
        ctx.sync()
    # more pairs than the capacity: reported, nothing used (loss 0, gradient 0)
    lc, dc = ctx.hinge_loss(*args[:4], cuda(np.array([q.size + 1], np.int32)), 1.0, 2.0)
    with pytest.raises(etx.EtxError) as e:
        ctx.sync()
    assert e.value.status == etx.ETX_ERR_CAPACITY
    assert not lc.any() and not dc.any()


def test_embed_backward_matches_oracle(etx):
    rng = np.random.default_rng(7)
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = drop_noise(wl.batch(3))
    W = wl.weights(perturb=0.2)
    blob = pack_blob(m, W)
    ctx = etx.Context(m, b.n_events, b.n_hits, 1)
    ctx.load_weights(blob)
    ws = ctx.embed_train_workspace(b.n_hits)
    x, y, z = cuda(b.x), cuda(b.y), cuda(b.z)
    emb = ctx.embed_forward_train(x, y, z, ws)
    plain = ctx.embed(x, y, z)
    assert torch.equal(emb, plain)                       # the saving forward computes the same
    up = rng.normal(size=(b.n_hits, m.emb_widths[-1])).astype(np.float32)
    grads = ctx.embed_backward(cuda(up), ws).cpu().numpy()
    ref = O.embed_backward(W, len(m.emb_widths) - 1, b.x, b.y, b.z, up)
    off = 0
    for i in range(len(m.emb_widths) - 1):
        for name in (f"emb{i}.W", f"emb{i}.b"):
            r = ref[name].ravel()
            g = grads[off:off + r.size]
            off += r.size
            # FP32 sums over ~5k rows (partials added in a fixed order): within 1e-4 of
            # the largest entry
            assert np.abs(g - r).max() <= 1e-4 * np.abs(r).max(), name
    assert off == grads.size == ctx.embed_param_count
    # the same upstream gradient gives the same bits (no atomics in the reverse pass)
    again = ctx.embed_backward(cuda(up), ws).cpu().numpy()
    assert np.array_equal(again, grads)


def test_embed_backward_many_splits(etx):
    """64 noise-free events (~100k hits): the weight gradients take one row split
    per SM and the bias sums several hundred partials, all added in a fixed
    order; sampled against the oracle and reproducible bit for bit."""
    rng = np.random.default_rng(8)
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = drop_noise(wl.batch(64))
    W = wl.weights(perturb=0.2)
    ctx = etx.Context(m, b.n_events, b.n_hits, 1)
    ctx.load_weights(pack_blob(m, W))
    ws = ctx.embed_train_workspace(b.n_hits)
    x, y, z = cuda(b.x), cuda(b.y), cuda(b.z)
    ctx.embed_forward_train(x, y, z, ws)
    up = rng.normal(size=(b.n_hits, m.emb_widths[-1])).astype(np.float32)
    g1 = ctx.embed_backward(cuda(up), ws).cpu().numpy()
    g2 = ctx.embed_backward(cuda(up), ws).cpu().numpy()
    assert np.array_equal(g1, g2)
    ref = O.embed_backward(W, len(m.emb_widths) - 1, b.x, b.y, b.z, up)
    off = 0
    for i in range(len(m.emb_widths) - 1):
        for name in (f"emb{i}.W", f"emb{i}.b"):
            r = ref[name].ravel()
            g = g1[off:off + r.size]
            off += r.size
            # per-tensor relative L2 (as the network's gradient tests): over ~100k
            # random-sign rows a hidden unit's ReLU decided differently by the FP32
            # and FP64 recomputation (pre-activation within rounding of zero) moves
            # an entry by one term, ~1/sqrt(rows) of it
            assert np.linalg.norm(g - r) <= 1e-3 * np.linalg.norm(r), name


def test_embedding_training_reduces_the_loss(etx):
    from paper_2407_12119_gb300.train import EmbeddingTrainer
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = drop_noise(wl.batch(8))
    pid = compact_particle_ids(b)
    tr = EmbeddingTrainer(m, pack_blob(m, wl.weights()), b.n_events, b.n_hits, lr=1e-3)
    args = [cuda(v) for v in (b.x, b.y, b.z, b.plane, pid, b.hit_offsets)]
    first = tr.step(*args).cpu().numpy().copy()
    for _ in range(40):
        last = tr.step(*args).cpu().numpy().copy()
    tr.ctx.sync()
    print("embedding training: loss", first, "->", last)
    assert last[0] < 0.8 * first[0]


def test_embedding_training_steps_are_reproducible(etx):
    """Two trainers with the same seed give the same parameters bit for bit
    after several steps (pairs, hinge gradient, reverse pass and Adam all in a
    fixed order)."""
    from paper_2407_12119_gb300.train import EmbeddingTrainer
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = drop_noise(wl.batch(4))
    pid = compact_particle_ids(b)
    args = [cuda(v) for v in (b.x, b.y, b.z, b.plane, pid, b.hit_offsets)]
    thetas, losses = [], []
    for _ in range(2):
        tr = EmbeddingTrainer(m, pack_blob(m, wl.weights()), b.n_events, b.n_hits, lr=1e-3, seed=3)
        for _ in range(4):
            loss = tr.step(*args)
        tr.ctx.sync()
        thetas.append(tr.theta.clone())
        losses.append(loss.clone())
    assert torch.equal(thetas[0], thetas[1])
    assert torch.equal(losses[0], losses[1])


def test_device_embed_update_equals_a_reload(etx):
    """etx_set_embed_params with a device vector gives the same embedding and the
    same reverse pass as loading a blob that holds the same parameters."""
    rng = np.random.default_rng(9)
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = drop_noise(wl.batch(3))
    blob = pack_blob(m, wl.weights(perturb=0.2))
    ctx = etx.Context(m, b.n_events, b.n_hits, 1)
    ctx.load_weights(blob)
    n_theta = ctx.embed_param_count
    theta = blob[12:12 + n_theta] + rng.normal(scale=0.05, size=n_theta).astype(np.float32)
    ctx.set_embed_params(cuda(theta.astype(np.float32)))
    blob2 = blob.copy()
    blob2[12:12 + n_theta] = theta
    ref = etx.Context(m, b.n_events, b.n_hits, 1)
    ref.load_weights(blob2)
    x, y, z = cuda(b.x), cuda(b.y), cuda(b.z)
    assert torch.equal(ctx.embed(x, y, z), ref.embed(x, y, z))
    up = cuda(rng.normal(size=(b.n_hits, m.emb_widths[-1])).astype(np.float32))
    ws1, ws2 = ctx.embed_train_workspace(b.n_hits), ref.embed_train_workspace(b.n_hits)
    e1, e2 = ctx.embed_forward_train(x, y, z, ws1), ref.embed_forward_train(x, y, z, ws2)
    assert torch.equal(e1, e2)
    assert torch.equal(ctx.embed_backward(up, ws1), ref.embed_backward(up, ws2))
