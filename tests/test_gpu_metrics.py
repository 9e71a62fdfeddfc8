"""Table 1 track-finding counts (Sec. 6) on the GPU against the oracle:
integer counts exact, FP64 sums and ratios to 1e-12 relative (the kernel
adds the same fractions in another order)."""
import json
import math
from pathlib import Path

import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import WORKLOADS, compact_particle_ids, pack_blob

pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).parent / "golden"
RTOL = 1e-12


@pytest.fixture(scope="module")
def etx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import etx as m
    return m


@pytest.fixture(scope="module")
def ctx(etx):
    return etx.Context(WORKLOADS["plain"].model, 64, 1 << 16, 1 << 16)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_metrics(ctx, labels, pid, hoff, **kw):
    c, v = ctx.track_metrics(cuda(np.asarray(labels, np.int32)), cuda(np.asarray(pid, np.int32)),
                             cuda(np.asarray(hoff, np.int32)), **kw)
    ctx.sync()
    return c.cpu().numpy(), v.cpu().numpy()


def check_against_oracle(etx, counts, values, labels, pid, hoff):
    ref = O.track_metrics(labels, pid, hoff)
    rates = O.track_metric_rates(ref)
    assert dict(zip(etx.TRACK_COUNTS, counts.tolist())) == {k: ref[k] for k in O.TRACK_METRIC_COUNTS}
    exp = [ref["hit_eff_sum"], ref["hit_purity_sum"]] + [rates[k] for k in etx.TRACK_VALUES[2:]]
    for name, got, want in zip(etx.TRACK_VALUES, values.tolist(), exp):
        if math.isnan(want):
            assert math.isnan(got), name
        else:
            assert got == pytest.approx(want, rel=RTOL, abs=0), name


def test_metrics_worked_by_hand(etx, ctx):
    case = json.loads((GOLDEN / "track_metrics.json").read_text())["cases"][0]
    counts, values = gpu_metrics(ctx, case["labels"], case["particle_id"], case["hit_offsets"])
    exp = case["expected"]
    assert counts.tolist() == [exp[k] for k in etx.TRACK_COUNTS]
    assert values[0] == pytest.approx(2.5, rel=RTOL) and values[1] == pytest.approx(3.5, rel=RTOL)
    assert values[2:].tolist() == pytest.approx([0.75, 0.25, 2 / 6, 0.625, 0.875], rel=RTOL)


def scrambled_labels(batch, pid, rng, split_every=3, move=0.2):
    """Truth tracks, some particles split in two, a fraction of hits moved to
    another hit's track: clones and unmatched tracks occur."""
    lab = np.empty(batch.n_hits, np.int32)
    for b in range(batch.n_events):
        lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
        n, seg, p = hi - lo, lab[lo:hi], pid[lo:hi]
        seg[:] = np.arange(n)
        for q in np.unique(p[p >= 0]):
            hits = np.nonzero(p == q)[0]
            seg[hits] = hits[0]
            if q % split_every == 0:
                seg[hits[len(hits) // 2:]] = hits[len(hits) // 2]
        if n:
            pick = np.nonzero(rng.uniform(size=n) < move)[0]
            seg[pick] = seg[rng.integers(0, n, size=pick.size)]
    return lab


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_metrics_random_labellings_match_oracle(etx, ctx, seed):
    rng = np.random.default_rng(seed)
    wl = WORKLOADS["plain"]
    from velo_synth import concat_events, make_event
    parts = [make_event(wl.recipe, 500 + seed * 50 + b) for b in range(9)]
    # an empty event and a noise-only event among them
    empty = tuple(np.zeros(0, dt) for dt in (np.float32, np.float32, np.float32, np.int8, np.int32))
    noise = (np.zeros(5, np.float32),) * 3 + (np.arange(5, dtype=np.int8), -np.ones(5, np.int32))
    batch = concat_events(parts[:3] + [empty] + parts[3:6] + [noise] + parts[6:])
    pid = compact_particle_ids(batch)
    lab = scrambled_labels(batch, pid, rng, move=0.1 * (seed + 1))
    counts, values = gpu_metrics(ctx, lab, pid, batch.hit_offsets)
    check_against_oracle(etx, counts, values, lab, pid, batch.hit_offsets)
    assert counts[2] > counts[3] > 0 and counts[5] > 0     # clones and fakes occur
    counts2, values2 = gpu_metrics(ctx, lab, pid, batch.hit_offsets)
    assert np.array_equal(counts, counts2) and values.tobytes() == values2.tobytes()


def test_metrics_other_thresholds(etx, ctx):
    rng = np.random.default_rng(5)
    batch = WORKLOADS["plain"].batch(4)
    pid = compact_particle_ids(batch)
    lab = scrambled_labels(batch, pid, rng)
    for min_hits, match in ((4, (3, 4)), (1, (1, 1)), (3, (51, 100))):
        c, v = gpu_metrics(ctx, lab, pid, batch.hit_offsets, min_hits=min_hits, match=match)
        ref = O.track_metrics(lab, pid, batch.hit_offsets, min_hits=min_hits,
                              match_num=match[0], match_den=match[1])
        assert c.tolist() == [ref[k] for k in O.TRACK_METRIC_COUNTS], (min_hits, match)
        assert v[0] == pytest.approx(ref["hit_eff_sum"], rel=RTOL)
        assert v[1] == pytest.approx(ref["hit_purity_sum"], rel=RTOL)


def test_metrics_degenerate_inputs(etx, ctx):
    c, v = gpu_metrics(ctx, np.zeros(0), np.zeros(0), [0])           # one empty event
    assert c.tolist() == [0] * 6 and all(math.isnan(x) for x in v[2:])
    c, v = gpu_metrics(ctx, np.zeros(0), np.zeros(0), [0, 0, 0])
    assert c.tolist() == [0] * 6
    c, v = gpu_metrics(ctx, np.zeros(6), [0, 0, 0, 0, 0, -1], [0, 6])  # one track, 5/6 one particle
    assert c.tolist() == [1, 1, 1, 1, 1, 0] and v[1] == pytest.approx(5 / 6, rel=RTOL)


def test_metrics_argument_errors(etx, ctx):
    lab, pid, hoff = cuda(np.zeros(4, np.int32)), cuda(np.zeros(4, np.int32)), cuda(np.array([0, 4], np.int32))
    with pytest.raises(etx.EtxError) as e:
        ctx.track_metrics(lab, pid, hoff, match=(1, 2))   # a track could match two particles
    assert e.value.status == etx.ETX_ERR_ARG
    with pytest.raises(etx.EtxError) as e:
        ctx.track_metrics(lab, pid, hoff, min_hits=0)
    assert e.value.status == etx.ETX_ERR_ARG
    with pytest.raises(etx.EtxError) as e:
        ctx.track_metrics(lab, pid, hoff, workspace=torch.empty(8, dtype=torch.uint8, device="cuda"))
    assert e.value.status == etx.ETX_ERR_CAPACITY


def test_metrics_out_of_range_ids_are_reported(etx):
    """A label or particle id outside the event is skipped by the kernel's own
    bounds check and reported at the next sync."""
    c = etx.Context(WORKLOADS["plain"].model, 4, 64, 64)
    lab = cuda(np.array([0, 0, 7, 0], np.int32))              # 7 >= 4 hits
    pid = cuda(np.array([0, 0, 0, 9], np.int32))              # 9 >= 4 hits
    c.track_metrics(lab, pid, cuda(np.array([0, 4], np.int32)))
    with pytest.raises(etx.EtxError):
        c.sync()


def test_metrics_of_oracle_tracks(etx, ctx):
    """Tracks of the oracle's own pipeline on two events of the 500-event
    recipe (exact components and the plane sweep of its graph and FP64 logits):
    GPU metrics equal the oracle's on the same labels."""
    from velo_synth import make_batch, make_weights
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = make_batch(wl.recipe, 2, wl.base_seed)
    W = make_weights(m, wl.calibration(), perturb=0.2)
    emb = O.embed(W, len(m.emb_widths) - 1, b.x, b.y, b.z)
    src, dst, _ = O.build_graph(emb, b.plane, b.hit_offsets, m.radius, m.k_max)
    z = O.gnn_forward(W, m.n_iters, b.x, b.y, b.z, src, dst)
    keep = z > np.quantile(z, 0.9)
    pid = compact_particle_ids(b)
    big = etx.Context(m, b.n_events, b.n_hits, 1)
    for name, lab in (("components", O.connected_components(src, dst, keep, b.hit_offsets)),
                      ("plane sweep", O.plane_sweep_components(src, dst, keep, b.plane, b.hit_offsets))):
        counts, values = gpu_metrics(big, lab, pid, b.hit_offsets)
        check_against_oracle(etx, counts, values, lab, pid, b.hit_offsets)
        print(name, dict(zip(etx.TRACK_VALUES[2:], np.round(values[2:], 4))))
