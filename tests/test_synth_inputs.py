"""The input-preparation helpers of the synthetic generator (CPU): removing
noise hits and renumbering particle ids keep the event structure that the
kernels rely on."""
import numpy as np

from velo_synth import WORKLOADS, compact_particle_ids, drop_noise, make_batch


def test_drop_noise_keeps_order_and_offsets():
    b = make_batch(WORKLOADS["batch500"].recipe, 5, 1000)
    c = drop_noise(b)
    assert c.n_events == b.n_events
    assert (c.particle_id >= 0).all()
    assert c.n_hits == int((b.particle_id >= 0).sum())
    for ev in range(b.n_events):
        orig, kept = b.event(ev), c.event(ev)
        sig = orig.particle_id >= 0
        np.testing.assert_array_equal(kept.x, orig.x[sig])
        np.testing.assert_array_equal(kept.plane, orig.plane[sig])
        assert np.all(np.diff(kept.plane.astype(int)) >= 0)       # still plane-sorted


def test_compact_particle_ids_partition_and_range():
    b = make_batch(WORKLOADS["batch500"].recipe, 5, 1000)
    pid = compact_particle_ids(b)
    for ev in range(b.n_events):
        lo, hi = int(b.hit_offsets[ev]), int(b.hit_offsets[ev + 1])
        old, new = b.particle_id[lo:hi], pid[lo:hi]
        assert np.array_equal(old < 0, new < 0)                   # noise stays noise
        sig = old >= 0
        if sig.any():
            assert new[sig].max() < hi - lo                       # below the event's hit count
            assert np.array_equal(np.unique(new[sig]), np.arange(np.unique(old[sig]).size))
            # same partition of the hits: equal old ids <=> equal new ids
            o, n = old[sig], new[sig]
            assert np.array_equal(o[:, None] == o[None, :], n[:, None] == n[None, :])


def test_fp8_scales_of_the_presets_are_the_calibrated_ones():
    """The e4m3 activation scales in the presets are those that
    ``python -m oracle.calibrate --fp8`` wrote to oracle/calibration.json,
    one per tensor-core operand (4 L + 3), and each is a power of two."""
    import json
    from pathlib import Path

    from velo_synth import WORKLOADS
    cal = json.loads((Path(__file__).resolve().parents[1] / "oracle" / "calibration.json").read_text())
    for name in ("batch500", "pileup4x"):
        m = WORKLOADS[name].model
        assert list(m.fp8_act_log2) == cal[name]["fp8_act_log2"]
        assert len(m.fp8_act_scales) == 4 * m.n_iters + 3
        for s, amax in zip(m.fp8_act_scales, cal[name]["fp8_act_amax"]):
            assert amax / s <= 448.0 < amax / (s / 2)
