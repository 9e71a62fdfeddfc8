"""Triplets (Sec. 5.3) on the GPU against the oracle: the lists bit-exact
(integers), the articulation / elbow classifier logits within the FP32 logit
tolerance.  Graphs, logits and edge encodings of the oracle side come from
the oracle itself; the GPU gets the same edges and logits as inputs."""
import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import (WORKLOADS, make_batch, make_triplet_weights, make_weights, pack_blob,
                        pack_triplet_blob)

pytestmark = pytest.mark.gpu
LOGIT_TOL = 1e-4


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
    return (t.to(dtype) if dtype is not None else t).cuda()


def gpu_triplets(ctx, src, dst, logits, thr, eoff, n_hits, cap=None):
    cap = 4 * max(len(src), 1) if cap is None else cap
    f, s, k, c = ctx.build_triplets(cuda(src, torch.int32), cuda(dst, torch.int32),
                                    cuda(np.asarray(logits, np.float32)), thr,
                                    cuda(eoff, torch.int32), n_hits, cap)
    ctx.sync()
    n = int(c[0].item())
    return f[:n].cpu().numpy(), s[:n].cpu().numpy(), k[:n].cpu().numpy(), c.cpu().numpy(), (f, s, c)


def test_triplets_chain_and_fork(etx):
    m = WORKLOADS["plain"].model
    ctx = etx.Context(m, 1, 8, 16)
    src, dst = np.array([0, 1, 1, 2, 3]), np.array([1, 2, 3, 4, 4])
    f, s, k, c, _ = gpu_triplets(ctx, src, dst, np.ones(5), 0.0, [0, 5], 5)
    assert list(zip(k.tolist(), f.tolist(), s.tolist())) == [
        (0, 0, 1), (0, 0, 2), (0, 1, 3), (0, 2, 4), (1, 1, 2), (2, 3, 4)]
    assert c.tolist() == [6, 4, 1, 1]
    f, s, k, c, _ = gpu_triplets(ctx, src, dst, -np.ones(5), 0.0, [0, 5], 5)
    assert c.tolist() == [0, 0, 0, 0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_triplets_random_graphs_match_oracle(etx, seed):
    rng = np.random.default_rng(seed)
    sizes = [40, 0, 25, 60]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    plane = np.concatenate([np.sort(rng.integers(0, 8, n)) for n in sizes])
    src, dst = [], []
    for b in range(len(sizes)):
        for i in range(offs[b], offs[b + 1]):
            for j in range(offs[b], offs[b + 1]):
                if 1 <= plane[j] - plane[i] <= 2 and rng.uniform() < 0.3:
                    src.append(i)
                    dst.append(j)
    src, dst = np.array(src), np.array(dst)
    eoff = np.searchsorted(src, offs)
    logits = rng.normal(size=src.size).astype(np.float32)
    thr = float(np.quantile(logits, 0.3))
    ctx = etx.Context(WORKLOADS["plain"].model, len(sizes), int(offs[-1]), src.size)
    f, s, k, c, _ = gpu_triplets(ctx, src, dst, logits, thr, eoff, int(offs[-1]))
    fo, so, ko = O.build_triplets(src, dst, logits > np.float32(thr), int(offs[-1]))
    assert np.array_equal(f, fo) and np.array_equal(s, so) and np.array_equal(k, ko)
    assert c.tolist() == [fo.size, int((ko == 0).sum()), int((ko == 1).sum()), int((ko == 2).sum())]


def test_triplet_capacity_overflow_is_reported(etx):
    ctx = etx.Context(WORKLOADS["plain"].model, 1, 8, 16)
    src, dst = np.array([0, 1, 1, 2, 3]), np.array([1, 2, 3, 4, 4])
    out = ctx.build_triplets(cuda(src, torch.int32), cuda(dst, torch.int32), cuda(np.ones(5, np.float32)),
                             0.0, cuda(np.array([0, 5]), torch.int32), 5, 5)
    with pytest.raises(etx.EtxError) as e:
        ctx.sync()
    assert e.value.status == etx.ETX_ERR_CAPACITY
    assert out[3].cpu().tolist() == [0, 0, 0, 0]


def test_triplets_and_classifiers_on_an_oracle_graph(etx):
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = make_batch(wl.recipe, 2, wl.base_seed)
    W = make_weights(m, wl.calibration(), perturb=0.2)
    emb = O.embed(W, len(m.emb_widths) - 1, b.x, b.y, b.z)
    src, dst, eoff = O.build_graph(emb, b.plane, b.hit_offsets, m.radius, m.k_max)
    cache = {}
    z = O.gnn_forward(W, m.n_iters, b.x, b.y, b.z, src, dst, cache=cache)
    thr = float(np.quantile(z, 0.9))                  # keep the top 10% of the edges
    keep = z.astype(np.float32) > np.float32(thr)
    tw = make_triplet_weights(m, perturb=0.2)
    ctx = etx.Context(m, b.n_events, b.n_hits, src.size)
    ctx.load_weights(pack_blob(m, W))
    ctx.load_triplet_weights(pack_triplet_blob(m, tw))
    # GPU forward (FP32) on the oracle's edges: leaves the final edge encodings in the context
    ctx.gnn_forward(cuda(b.x), cuda(b.y), cuda(b.z), cuda(src, torch.int32), cuda(dst, torch.int32),
                    cuda(eoff, torch.int32), dtype="f32")
    f, s, k, c, (ft, st, ct) = gpu_triplets(ctx, src, dst, z, thr, eoff, b.n_hits)
    fo, so, ko = O.build_triplets(src, dst, keep, b.n_hits)
    assert np.array_equal(f, fo) and np.array_equal(s, so) and np.array_equal(k, ko)
    assert c[1] > 0 and c[2] + c[3] > 0
    logits = ctx.classify_triplets(ft, st, ct)
    ctx.sync()
    ref = O.triplet_logits(tw, cache["cls"]["X"], fo, so, ko)
    got = logits[:fo.size].cpu().numpy()
    err = np.abs(got - ref).max()
    print(f"triplets: {fo.size} ({c[1]} articulations), max |logit err| {err:.2e}")
    assert err <= LOGIT_TOL
