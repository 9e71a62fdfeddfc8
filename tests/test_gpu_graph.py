"""The whole inference step captured in one CUDA graph (TrackFinder.capture /
replay) gives bit-identical results to the eager launches, also after new
hits of the same sizes are copied into the captured input tensors."""
import numpy as np
import pytest
import torch

from velo_synth import WORKLOADS, pack_blob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pipeline():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import pipeline as p
    return p


def inputs(batch):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return [t(batch.x), t(batch.y), t(batch.z), t(batch.plane), t(batch.hit_offsets)]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_graph_replay_matches_eager(pipeline, dtype):
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = wl.batch(6)
    tf = pipeline.TrackFinder(m, pack_blob(m, wl.weights()), b.n_events, b.n_hits,
                              b.n_hits * m.k_max, dtype=dtype)
    x, y, z, plane, hoff = inputs(b)
    labels_g, nt_g = tf.capture(x, y, z, plane, hoff, b.n_hits, b.n_events)
    logits_g = tf.logits.clone()
    labels_g, nt_g = labels_g.clone(), nt_g.clone()
    # eager run on copies of the same hits (other addresses, outside the graph)
    x2, y2, z2, p2, h2 = inputs(b)
    labels_e, nt_e = tf.run_device(x2, y2, z2, p2, h2, b.n_hits, b.n_events)
    torch.cuda.synchronize()
    assert torch.equal(labels_e, labels_g)
    assert torch.equal(nt_e, nt_g)
    assert torch.equal(tf.logits, logits_g)
    tf.ctx.sync()

    # new hits, same sizes: shift every hit by a small random offset in x, y
    rng = np.random.default_rng(7)
    xs = (b.x + rng.normal(0, 0.02, b.n_hits)).astype(np.float32)
    ys = (b.y + rng.normal(0, 0.02, b.n_hits)).astype(np.float32)
    x.copy_(torch.from_numpy(xs))
    y.copy_(torch.from_numpy(ys))
    launches = tf.ctx.launch_count
    labels_r, nt_r = tf.replay()
    labels_r, nt_r = labels_r.clone(), nt_r.clone()
    logits_r = tf.logits.clone()
    torch.cuda.synchronize()
    assert tf.ctx.launch_count == launches  # the replay issues no eager launches
    x3, y3 = torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda()
    labels_e2, nt_e2 = tf.run_device(x3, y3, z2, p2, h2, b.n_hits, b.n_events)
    torch.cuda.synchronize()
    assert torch.equal(labels_e2, labels_r)
    assert torch.equal(nt_e2, nt_r)
    assert torch.equal(tf.logits, logits_r)
    assert not torch.equal(logits_r, logits_g)  # the replay saw the new hits
    tf.ctx.sync()


def test_replay_without_capture_is_an_error(pipeline):
    wl = WORKLOADS["plain"]
    m = wl.model
    b = wl.batch(1)
    tf = pipeline.TrackFinder(m, pack_blob(m, wl.weights()), b.n_events, b.n_hits)
    with pytest.raises(RuntimeError):
        tf.replay()
