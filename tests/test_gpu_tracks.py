"""GPU track building on the purified edge graph (Sec. 5.4) against the
oracle's ``tracks_from_triplets``: the same kept edges and kept triplets on
both sides give exactly the same tracks (compared as sets of hit tuples: the
order of the tracks is not part of the result)."""
import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import WORKLOADS, make_batch, make_weights

pytestmark = pytest.mark.gpu


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


def gpu_tracks(etx, model, src, dst, hoff, edge_logits, edge_thr, trip_decide, min_hits=3):
    """Triplets built on the GPU; their logits set by ``trip_decide(first,
    second, kind) -> float array``; tracks built on the GPU.  Returns
    (tracks as sorted hit tuples, the triplet list and its logits)."""
    n_hits = int(hoff[-1])
    E = src.size
    ctx = etx.Context(model, len(hoff) - 1, max(n_hits, 1), max(E, 1))
    eo = np.array([0] * (len(hoff) - 1) + [E], np.int32)
    s_t, d_t, l_t, eo_t = cuda(src, torch.int32), cuda(dst, torch.int32), cuda(edge_logits), cuda(eo)
    cap = max(4 * E, 16)
    f, s2, k, counts = ctx.build_triplets(s_t, d_t, l_t, edge_thr, eo_t, n_hits, cap)
    ctx.sync()
    n = int(counts[0].item())
    fh, sh, kh = f[:n].cpu().numpy(), s2[:n].cpu().numpy(), k[:n].cpu().numpy().astype(np.int64)
    tl = np.full(cap, -1.0, np.float32)
    tl[:n] = trip_decide(fh, sh, kh)
    offs, hits, n_out = ctx.tracks_from_triplets(s_t, d_t, l_t, edge_thr, eo_t, n_hits, f, s2,
                                                 cuda(tl), 0.0, counts, min_hits=min_hits)
    ctx.sync()
    nt, nh = n_out.cpu().tolist()
    offs, hits = offs[:nt + 1].cpu().numpy(), hits[:nh].cpu().numpy()
    tracks = sorted(tuple(hits[offs[t]:offs[t + 1]].tolist()) for t in range(nt))
    for tr in tracks:                           # ascending, no repeats within a track
        assert list(tr) == sorted(set(tr))
    return tracks, (fh, sh, kh), tl[:n] > 0


CASES = {
    "fork": ([0, 1, 1, 2, 4], [1, 2, 4, 3, 5], []),
    "fork_elbow_restores": ([0, 1, 1, 2, 4], [1, 2, 4, 3, 5], [(0, 2, 0)]),
    "fork_no_elbow": ([0, 1, 1, 2, 4], [1, 2, 4, 3, 5], [(0, 2, 0), (1, 2, 1)]),
    "first_hit": ([0, 1, 2, 0, 4, 5], [1, 2, 3, 4, 5, 6], []),
    "merge": ([0, 1, 2, 3, 4], [1, 4, 3, 4, 5], []),
    "merge_no_elbow": ([0, 1, 2, 3, 4], [1, 4, 3, 4, 5], [(3, 4, 0), (1, 3, 2)]),
    "crossing": ([0, 1, 2, 3, 5, 6, 2, 7], [1, 2, 3, 4, 6, 2, 7, 8], []),
    "crossing_resolved": ([0, 1, 2, 3, 5, 6, 2, 7], [1, 2, 3, 4, 6, 2, 7, 8],
                          [(1, 6, 0), (5, 2, 0), (2, 6, 1), (1, 5, 2)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_hand_worked_cases(etx, name):
    src, dst, drop = CASES[name]
    src, dst = np.array(src), np.array(dst)
    # the oracle's edge order is (src, dst)-sorted like the library's
    order = np.lexsort((dst, src))
    assert np.array_equal(order, np.arange(src.size)), "cases are listed sorted"
    n = int(max(src.max(), dst.max())) + 1
    model = WORKLOADS["plain"].model
    drop = set(drop)
    decide = lambda f, s, k: np.array([-1.0 if (int(a), int(b), int(c)) in drop else 1.0
                                       for a, b, c in zip(f, s, k)], np.float32)
    got, (f, s, k), tm = gpu_tracks(etx, model, src, dst, np.array([0, n], np.int32),
                                    np.ones(src.size, np.float32), 0.0, decide)
    ref = O.tracks_from_triplets(src, dst, np.ones(src.size, bool), f, s, k, tm)
    assert got == ref, (name, got, ref)


@pytest.mark.parametrize("seed,edge_keep,trip_keep", [(1, 0.3, 0.9), (2, 0.5, 0.6), (3, 0.4, 0.3)])
def test_random_masks_on_event_graphs(etx, seed, edge_keep, trip_keep):
    """batch500 events: the oracle's graph, random edge logits (keeping about
    edge_keep of the edges) and random triplet logits (about trip_keep)."""
    wl = WORKLOADS["batch500"]
    b = make_batch(wl.recipe, 3, wl.base_seed + 20 + seed)
    W = make_weights(wl.model, b)
    emb = O.embed(W, len(wl.model.emb_widths) - 1, b.x, b.y, b.z)
    src, dst, _ = O.build_graph(emb, b.plane, b.hit_offsets, wl.model.radius, wl.model.k_max)
    rng = np.random.default_rng(seed)
    el = rng.normal(size=src.size).astype(np.float32)
    thr = float(np.quantile(el, 1.0 - edge_keep))
    tr_rng = np.random.default_rng(100 + seed)
    decide = lambda f, s, k: np.where(tr_rng.random(f.size) < trip_keep, 1.0, -1.0).astype(np.float32)
    got, (f, s, k), tm = gpu_tracks(etx, wl.model, src, dst, b.hit_offsets, el, thr, decide)
    # the GPU's triplet list is the oracle's (bit-exact elsewhere); the oracle builds
    # its tracks from the same kept edges and kept triplets
    rf, rs, rk = O.build_triplets(src, dst, el > np.float32(thr), b.n_hits)
    assert np.array_equal(rf, f) and np.array_equal(rs, s) and np.array_equal(rk, k)
    ref = O.tracks_from_triplets(src, dst, el > np.float32(thr), f, s, k, tm)
    shared = sum(1 for t in ref for u in ref if t < u and set(t) & set(u))
    print(f"seed {seed}: {src.size} edges, {int((el > thr).sum())} kept, {f.size} triplets, "
          f"{int(tm.sum())} kept; {len(ref)} tracks, {shared} pairs of tracks sharing hits")
    assert got == ref
    assert len(ref) > 0


def test_capacity_and_mismatched_list_are_reported(etx):
    src, dst = np.array([0, 1, 1, 2, 4]), np.array([1, 2, 4, 3, 5])
    model = WORKLOADS["plain"].model
    ctx = etx.Context(model, 1, 6, 5)
    s_t, d_t = cuda(src, torch.int32), cuda(dst, torch.int32)
    l_t, eo_t = cuda(np.ones(5, np.float32)), cuda(np.array([0, 5], np.int32))
    f, s2, k, counts = ctx.build_triplets(s_t, d_t, l_t, 0.0, eo_t, 6, 32)
    tl = cuda(np.ones(32, np.float32))
    # too small a hit capacity: reported, no tracks
    offs, hits, n_out = ctx.tracks_from_triplets(s_t, d_t, l_t, 0.0, eo_t, 6, f, s2, tl, 0.0,
                                                 counts, track_capacity=4, hit_capacity=3)
    with pytest.raises(etx.EtxError) as ei:
        ctx.sync()
    assert ei.value.status == etx.ETX_ERR_CAPACITY
    assert n_out.cpu().tolist() == [0, 0]
    # a triplet list built for another edge cut does not match these edges
    f2, s3, k2, c2 = ctx.build_triplets(s_t, d_t, l_t, 2.0, eo_t, 6, 32)   # keeps nothing
    ctx.tracks_from_triplets(s_t, d_t, l_t, 0.0, eo_t, 6, f2, s3, tl, 0.0, c2)
    with pytest.raises(etx.EtxError) as ei:
        ctx.sync()
    assert ei.value.status == etx.ETX_ERR_UNSORTED
