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


def gpu_tracks(etx, model, src, dst, hoff, edge_logits, edge_thr, trip_decide, min_hits=3,
               n_tracks=None, n_track_hits=None):
    """Triplets built on the GPU; their logits set by ``trip_decide(first,
    second, kind) -> float array``; tracks built on the GPU (capacities from
    the expected counts when given).  Returns (tracks as sorted hit tuples,
    the triplet list and its kept mask)."""
    n_hits = int(hoff[-1])
    E = src.size
    ctx = etx.Context(model, len(hoff) - 1, max(n_hits, 1), max(E, 1))
    eo = np.array([0] * (len(hoff) - 1) + [E], np.int32)
    s_t, d_t, l_t, eo_t = cuda(src, torch.int32), cuda(dst, torch.int32), cuda(edge_logits), cuda(eo)
    cap = max(4 * E, 16)
    f, s2, k, counts = ctx.build_triplets(s_t, d_t, l_t, edge_thr, eo_t, n_hits, cap)
    ctx.sync()
    n = int(counts[0].item())
    assert n <= cap
    fh, sh, kh = f[:n].cpu().numpy(), s2[:n].cpu().numpy(), k[:n].cpu().numpy().astype(np.int64)
    tl = np.full(cap, -1.0, np.float32)
    tl[:n] = trip_decide(fh, sh, kh)
    kw = {}
    if n_tracks is not None:
        kw = dict(track_capacity=n_tracks + 8, hit_capacity=n_track_hits + 64)
    offs, hits, n_out = ctx.tracks_from_triplets(s_t, d_t, l_t, edge_thr, eo_t, n_hits, f, s2,
                                                 cuda(tl), 0.0, counts, min_hits=min_hits, **kw)
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
    # the library takes edges sorted by (src, dst): renumber them, and the
    # dropped triplets' edge indices with them (elbows keep first < second)
    order = np.lexsort((dst, src))
    new = np.argsort(order)                     # new index of old edge e
    src, dst = src[order], dst[order]
    drop = {(int(new[a]), int(new[b]), c) if c == 0 else
            (int(min(new[a], new[b])), int(max(new[a], new[b])), c) for a, b, c in drop}
    n = int(max(src.max(), dst.max())) + 1
    model = WORKLOADS["plain"].model
    decide = lambda f, s, k: np.array([-1.0 if (int(a), int(b), int(c)) in drop else 1.0
                                       for a, b, c in zip(f, s, k)], np.float32)
    got, (f, s, k), tm = gpu_tracks(etx, model, src, dst, np.array([0, n], np.int32),
                                    np.ones(src.size, np.float32), 0.0, decide)
    ref = O.tracks_from_triplets(src, dst, np.ones(src.size, bool), f, s, k, tm)
    assert got == ref, (name, got, ref)


@pytest.mark.parametrize("seed,edge_keep,trip_keep", [(1, 0.3, 0.9), (2, 0.15, 0.6), (3, 0.2, 0.3)])
def test_random_masks_on_event_graphs(etx, seed, edge_keep, trip_keep):
    """batch500 events: the oracle's graph, random edge logits (keeping about
    edge_keep of the edges) and random triplet logits (about trip_keep); the
    output capacities come from the oracle's counts."""
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
    # the oracle on the same kept edges, with the same triplet decisions
    rf, rs, rk = O.build_triplets(src, dst, el > np.float32(thr), b.n_hits)
    tm = decide(rf, rs, rk) > 0
    ref = O.tracks_from_triplets(src, dst, el > np.float32(thr), rf, rs, rk, tm)
    tr_rng = np.random.default_rng(100 + seed)   # same draws for the GPU's list
    got, (f, s, k), tm_gpu = gpu_tracks(etx, wl.model, src, dst, b.hit_offsets, el, thr, decide,
                                        n_tracks=len(ref), n_track_hits=sum(len(t) for t in ref))
    # the GPU's triplet list is the oracle's (bit-exact elsewhere), so are the decisions
    assert np.array_equal(rf, f) and np.array_equal(rs, s) and np.array_equal(rk, k)
    assert np.array_equal(tm, tm_gpu)
    hits_in = {}
    for t in ref:
        for h in t:
            hits_in[h] = hits_in.get(h, 0) + 1
    print(f"seed {seed}: {src.size} edges, {int((el > thr).sum())} kept, {f.size} triplets, "
          f"{int(tm.sum())} kept; {len(ref)} tracks, {sum(c > 1 for c in hits_in.values())} "
          f"hits in more than one track")
    assert got == ref
    assert len(ref) > 0


def test_genuine_tracks_with_noise_edges(etx):
    """The genuine edges of batch500 events (long tracks) plus 3% of the other
    graph edges kept as noise; every articulation kept, elbows kept at
    random: forks and merges on long tracks."""
    from velo_synth import global_particle_ids, truth_edge_labels
    wl = WORKLOADS["batch500"]
    b = make_batch(wl.recipe, 2, wl.base_seed + 31)
    W = make_weights(wl.model, b)
    emb = O.embed(W, len(wl.model.emb_widths) - 1, b.x, b.y, b.z)
    src, dst, _ = O.build_graph(emb, b.plane, b.hit_offsets, wl.model.radius, wl.model.k_max)
    gen = truth_edge_labels(global_particle_ids(b), b.plane, src, dst) > 0
    rng = np.random.default_rng(7)
    keep = gen | (rng.random(src.size) < 0.03)
    el = np.where(keep, 1.0, -1.0).astype(np.float32)
    el_rng = np.random.default_rng(8)
    decide = lambda f, s, k: np.where((k == 0) | (el_rng.random(f.size) < 0.5), 1.0, -1.0).astype(np.float32)
    rf, rs, rk = O.build_triplets(src, dst, keep, b.n_hits)
    ref = O.tracks_from_triplets(src, dst, keep, rf, rs, rk, decide(rf, rs, rk) > 0)
    el_rng = np.random.default_rng(8)
    got, _, _ = gpu_tracks(etx, wl.model, src, dst, b.hit_offsets, el, 0.0, decide,
                           n_tracks=len(ref), n_track_hits=sum(len(t) for t in ref))
    print(f"{int(gen.sum())} genuine + {int((keep & ~gen).sum())} noise edges: {len(ref)} tracks, "
          f"longest {max(len(t) for t in ref)} hits")
    assert got == ref


def test_long_component_is_sorted(etx):
    """One chain through 5,000 hits numbered in random order: a component
    longer than the per-thread sort takes (the block-wide sort handles it)."""
    n = 5000
    rng = np.random.default_rng(3)
    perm = rng.permutation(n)
    src, dst = perm[:-1].astype(np.int64), perm[1:].astype(np.int64)
    o = np.lexsort((dst, src))
    src, dst = src[o], dst[o]
    model = WORKLOADS["plain"].model
    got, _, _ = gpu_tracks(etx, model, src, dst, np.array([0, n], np.int32),
                           np.ones(src.size, np.float32), 0.0,
                           lambda f, s, k: np.ones(f.size, np.float32), n_tracks=1, n_track_hits=n)
    assert got == [tuple(range(n))]


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
