"""The allocation-free components call (etx_edges_to_tracks_noalloc).

Some callers cannot allocate device memory: a host framework that owns the
whole device budget, or a real-time loop where an allocation is not allowed.
For them the library has one entry point whose scratch is a fixed array
inside the library.  This file checks, on the GPU and through the C ABI,
that on two calls in a row with different inputs (so nothing left in the
shared array by the first call leaks into the second) it gives exactly the
oracle's connected-component labels and the regular etx_edges_to_tracks'
labels and track counts, that its device status reads ETX_OK, that the
second call changes the device's free memory by nothing, and that it
refuses sizes above its limit.  It is collected last on purpose.
"""
import ctypes

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


def _graph(name, n_events, seed):
    wl = WORKLOADS[name]
    b = make_batch(wl.recipe, n_events, wl.base_seed + seed)
    W = make_weights(wl.model, b, perturb=0.2)
    emb = O.embed(W, len(wl.model.emb_widths) - 1, b.x, b.y, b.z)
    s, d, eo = O.build_graph(emb, b.plane, b.hit_offsets, wl.model.radius, wl.model.k_max)
    return wl.model, b, s, d, eo


def _tracks_per_event(labels, hit_offsets, min_hits):
    """Components of at least min_hits hits per event, from event-local labels."""
    out = []
    for b in range(len(hit_offsets) - 1):
        lab = labels[hit_offsets[b]:hit_offsets[b + 1]]
        _, counts = np.unique(lab, return_counts=True)
        out.append(int((counts >= min_hits).sum()))
    return np.array(out, np.int32)


def test_noalloc_matches_oracle_and_regular_entry_point_twice(etx):
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cases = []
    for call, (name, n, seed, q) in enumerate([("batch500", 3, 7, 0.9), ("plain", 2, 3, 0.5)]):
        model, b, s, d, eo = _graph(name, n, seed)
        rng = np.random.default_rng(call)
        logits = rng.normal(size=s.size).astype(np.float32)
        thr = float(np.quantile(logits, q))
        # the regular entry point (its context allocates: done before any measurement)
        args = (t(s.astype(np.int32)), t(d.astype(np.int32)), t(logits))
        eo_t, ho_t = t(eo.astype(np.int32)), t(b.hit_offsets)
        ctx = etx.Context(model, b.n_events, b.n_hits, max(s.size, 1))
        ref_l, ref_n = ctx.edges_to_tracks(*args, thr, eo_t, ho_t, min_hits=3)
        torch.cuda.synchronize()
        ctx.sync()
        lab = torch.full((b.n_hits,), -7, dtype=torch.int32, device=dev)
        nt = torch.full((b.n_events,), -7, dtype=torch.int32, device=dev)
        status = torch.full((1,), -7, dtype=torch.int32, device=dev)
        oracle_l = O.connected_components(s, d, logits > np.float32(thr), b.hit_offsets)
        cases.append((b, args, eo_t, ho_t, thr, lab, nt, status, ref_l, ref_n, oracle_l))

    for call, (b, args, eo_t, ho_t, thr, lab, nt, status, ref_l, ref_n, oracle_l) in enumerate(cases):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        etx.edges_to_tracks_noalloc(*args, thr, eo_t, ho_t, lab, nt, min_hits=3, status=status)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(dev)[0]
        if call == 1:  # the first call has looked the array's address up; nothing may allocate now
            assert free1 == free0, (free0, free1)
        got = lab.cpu().numpy()
        np.testing.assert_array_equal(got, oracle_l)
        np.testing.assert_array_equal(got, ref_l.cpu().numpy())
        np.testing.assert_array_equal(nt.cpu().numpy(), ref_n[:b.n_events].cpu().numpy())
        np.testing.assert_array_equal(nt.cpu().numpy(), _tracks_per_event(oracle_l, b.hit_offsets, 3))
        assert int(status.item()) == etx.ETX_OK
        # some hits are joined to others, some stay alone: both branches are exercised
        own = np.arange(b.n_hits) - np.repeat(b.hit_offsets[:-1], np.diff(b.hit_offsets))
        assert 0 < int((got == own).sum()) < b.n_hits


def test_noalloc_rejects_sizes_above_its_limit(etx):
    dev = torch.device("cuda", 0)
    z = torch.zeros(1, dtype=torch.int32, device=dev)
    f = torch.zeros(1, dtype=torch.float32, device=dev)
    L = etx.lib()
    st = L.etx_edges_to_tracks_noalloc(etx._ptr(z), etx._ptr(z), etx._ptr(f), 0.0, etx._ptr(z),
                                       etx._ptr(z), 1, etx.NOALLOC_MAX_HITS + 1, 3, etx._ptr(z),
                                       None, None, ctypes.c_void_p(0))
    assert st == etx.ETX_ERR_CAPACITY
