"""Pins of the oracle's track building on the purified edge graph (Sec. 5.4,
``tracks_from_triplets``): hand-worked forks, merges and elbow cases with
their tracks written out, the reduction to connected components when no hit
is shared, and invariance under relabelling of the edges."""
import numpy as np
import pytest

from oracle import etx_oracle as O

ART, LEFT, RIGHT = O.TRIPLET_ARTICULATION, O.TRIPLET_LEFT_ELBOW, O.TRIPLET_RIGHT_ELBOW


def run(src, dst, drop=(), edge_mask=None, min_hits=3):
    """Tracks with every triplet kept except the (first, second, kind) in ``drop``."""
    src, dst = np.asarray(src), np.asarray(dst)
    em = np.ones(src.size, bool) if edge_mask is None else np.asarray(edge_mask, bool)
    n = int(max(src.max(), dst.max())) + 1
    f, s, k = O.build_triplets(src, dst, em, n)
    tm = np.array([(int(a), int(b), int(c)) not in set(drop) for a, b, c in zip(f, s, k)], bool)
    return O.tracks_from_triplets(src, dst, em, f, s, k, tm, min_hits=min_hits)


# e+e- pair sharing its first two hits 0, 1: P1 = 0 1 2 3, P2 = 0 1 4 5
# edges: 0: 0->1, 1: 1->2, 2: 1->4, 3: 2->3, 4: 4->5
FORK = ([0, 1, 1, 2, 4], [1, 2, 4, 3, 5])


def test_fork_sharing_two_hits_duplicates_the_shared_part():
    # articulations (0,1) and (0,2) share edge 0: both shared; edge 0 is
    # duplicated into each track
    assert run(*FORK) == [(0, 1, 2, 3), (0, 1, 4, 5)]


def test_plain_components_would_merge_the_pair():
    labels = O.connected_components(*FORK, np.ones(5, bool), np.array([0, 6]))
    assert len(set(labels.tolist())) == 1          # one component: the pair is lost


def test_elbow_restores_a_missing_articulation():
    # the classifier drops articulation (0, 2); the kept left elbow (1, 2) at hit 1
    # joins edges 1 and 2, so edge 2 shares edge 1's continuation (0, 1): same tracks
    assert run(*FORK, drop=[(0, 2, ART)]) == [(0, 1, 2, 3), (0, 1, 4, 5)]
    # without the elbow, edge 0 continues only into edge 1; edges 2, 4 form their own track
    assert run(*FORK, drop=[(0, 2, ART), (1, 2, LEFT)]) == [(0, 1, 2, 3), (1, 4, 5)]


def test_fork_at_the_first_hit():
    # tracks sharing only hit 0: 0->1->2->3 and 0->4->5->6; no edge is shared,
    # the left elbow (0, 3) links nothing to join; two tracks, both with hit 0
    src, dst = [0, 1, 2, 0, 4, 5], [1, 2, 3, 4, 5, 6]
    assert run(src, dst) == [(0, 1, 2, 3), (0, 4, 5, 6)]


def test_merge_sharing_the_last_hits():
    # P1 = 0 1 4 5, P2 = 2 3 4 5: edges 0: 0->1, 1: 1->4, 2: 2->3, 3: 3->4, 4: 4->5;
    # articulations (1, 4) and (3, 4) share edge 4 (two articulations into it)
    src, dst = [0, 1, 2, 3, 4], [1, 4, 3, 4, 5]
    assert run(src, dst) == [(0, 1, 4, 5), (2, 3, 4, 5)]
    # a right elbow (1, 3) restores a dropped articulation (3, 4)
    assert run(src, dst, drop=[(3, 4, ART)]) == [(0, 1, 4, 5), (2, 3, 4, 5)]
    assert run(src, dst, drop=[(3, 4, ART), (1, 3, RIGHT)]) == [(0, 1, 4, 5), (2, 3, 4)]


def test_dropped_articulation_splits_a_track():
    src, dst = [0, 1, 2, 3, 4], [1, 2, 3, 4, 5]       # one chain of six hits
    assert run(src, dst) == [(0, 1, 2, 3, 4, 5)]
    assert run(src, dst, drop=[(1, 2, ART)]) == [(0, 1, 2), (2, 3, 4, 5)]


def test_min_hits_and_removed_edges():
    src, dst = [0, 1, 3], [1, 2, 4]                      # a 3-hit chain and a lone edge
    assert run(src, dst) == [(0, 1, 2)]
    assert run(src, dst, min_hits=2) == [(0, 1, 2), (3, 4)]
    assert run(src, dst, edge_mask=[True, False, True], min_hits=2) == [(0, 1), (3, 4)]


def test_skip_plane_edges_and_a_shared_middle():
    # two tracks crossing at hit 2: 0->1->2->3->4 and 5->6->2->7->8; at hit 2 both
    # in-edges continue into both out-edges (4 articulations): all shared, so each
    # articulation is a track: 4 tracks, the two genuine and the two crossed ones
    src, dst = [0, 1, 2, 3, 5, 6, 2, 7], [1, 2, 3, 4, 6, 2, 7, 8]
    t = run(src, dst)
    assert t == sorted([(0, 1, 2, 3, 4), (0, 1, 2, 7, 8), (2, 3, 4, 5, 6), (2, 5, 6, 7, 8)])
    # a classifier that keeps only the two genuine articulations at hit 2 (and no
    # elbows there) separates them
    drop = [(1, 6, ART), (5, 2, ART), (2, 6, LEFT), (1, 5, RIGHT)]
    assert run(src, dst, drop=drop) == [(0, 1, 2, 3, 4), (2, 5, 6, 7, 8)]


def _random_graph(rng, n_hits, n_planes, p_edge, p_drop):
    plane = np.sort(rng.integers(0, n_planes, n_hits))
    src, dst = [], []
    for i in range(n_hits):
        for j in range(n_hits):
            if plane[j] in (plane[i] + 1, plane[i] + 2) and rng.random() < p_edge:
                src.append(i)
                dst.append(j)
    return np.array(src, np.int64), np.array(dst, np.int64)


def test_without_shared_hits_tracks_are_the_components():
    """A graph where every hit has at most one kept edge in and one out, and
    every articulation is kept: the tracks are the connected components of the
    kept hit graph with at least 3 hits (the exact-components path, Sec. 7.3)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(10, 60))
        perm = rng.permutation(n)
        cuts = np.sort(rng.choice(np.arange(1, n), size=int(rng.integers(1, n // 3)), replace=False))
        src, dst = [], []
        for chain in np.split(perm, cuts):
            for a, b in zip(chain[:-1], chain[1:]):
                src.append(int(a))
                dst.append(int(b))
        src, dst = np.array(src), np.array(dst)
        labels = O.connected_components(src, dst, np.ones(src.size, bool), np.array([0, n]))
        comps = {}
        for h, lab in enumerate(labels.tolist()):
            comps.setdefault(lab, []).append(h)
        expect = sorted(tuple(sorted(c)) for c in comps.values() if len(c) >= 3)
        assert run(src, dst) == expect


def test_invariant_under_edge_relabelling():
    rng = np.random.default_rng(11)
    for _ in range(10):
        src, dst = _random_graph(rng, 25, 6, 0.2, 0.0)
        if src.size == 0:
            continue
        n = 25
        em = rng.random(src.size) < 0.8
        f, s, k = O.build_triplets(src, dst, em, n)
        tm = rng.random(f.size) < 0.7
        ref = O.tracks_from_triplets(src, dst, em, f, s, k, tm)
        # relabel edges by a permutation, carrying the triplet decisions along
        p = rng.permutation(src.size)
        inv = np.argsort(p)                       # new index of old edge e: inv[e]
        src2, dst2, em2 = src[p], dst[p], em[p]
        f2, s2, k2 = O.build_triplets(src2, dst2, em2, n)
        decide = {(int(a), int(b), int(c)): bool(m) for a, b, c, m in zip(f, s, k, tm)}
        tm2 = []
        for a, b, c in zip(f2, s2, k2):
            oa, ob = int(p[a]), int(p[b])
            if c != ART and (oa, ob, int(c)) not in decide:
                oa, ob = ob, oa                   # elbows are listed with first < second
            tm2.append(decide[(oa, ob, int(c))])
        got = O.tracks_from_triplets(src2, dst2, em2, f2, s2, k2, np.array(tm2, bool))
        assert got == ref
        assert inv.size == p.size
