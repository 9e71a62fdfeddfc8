"""Launch configurations (k-NN work partitioning and candidate stage,
tensor-core ring depth) do not change any output, and the autotuner picks one
of its candidates."""
import numpy as np
import pytest
import torch

from velo_synth import WORKLOADS, pack_blob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def finder():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300.pipeline import TrackFinder
    wl = WORKLOADS["batch500"]
    m = wl.model
    b = wl.batch(12)
    tf = TrackFinder(m, pack_blob(m, wl.weights()), b.n_events, b.n_hits, b.n_hits * m.k_max)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (t(b.x), t(b.y), t(b.z), t(b.plane), t(b.hit_offsets), b.n_hits, b.n_events)
    return tf, args


def outputs(tf, args):
    labels, nt = tf.run_device(*args)
    E = int(tf.eoff[args[-1]].item())
    out = (tf.src[:E].clone(), tf.dst[:E].clone(), tf.eoff.clone(), tf.logits[:E].clone(),
           labels.clone(), nt.clone())
    tf.ctx.sync()
    return out


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_every_configuration_gives_the_same_results(finder, dtype):
    tf, args = finder
    tf.dtype = dtype
    tf.ctx.set_tuned(knn_split=1, knn_stage=16384)
    for blk in ("edge_encoder", "node_update", "edge_update", "classifier"):
        tf.ctx.set_tuned(**{f"tc_stages__{blk}__{dtype}": 3})
    ref = outputs(tf, args)
    # stage 1024 (128 candidates of dimension 8) leaves most (event, plane)
    # blocks reading their candidates from global memory
    for split, stage, stages in ((2, 1024, 2), (4, 2048, 3), (4, 4096, 2), (1, 8192, 4),
                                 (2, 1024, 5)):
        tf.ctx.set_tuned(knn_split=split, knn_stage=stage)
        for blk in ("edge_encoder", "node_update", "edge_update", "classifier"):
            tf.ctx.set_tuned(**{f"tc_stages__{blk}__{dtype}": stages})
        got = outputs(tf, args)
        for a, b in zip(ref, got):
            assert torch.equal(a, b)


def test_autotune_picks_candidates_and_keeps_results(finder):
    tf, args = finder
    tf.dtype = "bf16"
    ref = outputs(tf, args)
    choice = tf.autotune(*args)
    assert choice["knn_split"] in (1, 2, 4)
    assert choice["knn_stage"] in (1024, 2048, 4096, 8192, 16384)
    for blk in ("edge_encoder", "node_update", "edge_update", "classifier"):
        assert choice[f"tc_stages/{blk}/bf16"] in (2, 3, 4, 5)
    E = int(tf.eoff[args[-1]].item())
    assert torch.equal(tf.logits[:E], ref[3])  # the tuner's own last forward
    got = outputs(tf, args)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_set_tuned_rejects_bad_values(finder):
    tf, _ = finder
    from paper_2407_12119_gb300.etx import EtxError
    with pytest.raises(EtxError):
        tf.ctx.set_tuned(knn_split=3)
    with pytest.raises(EtxError):
        tf.ctx.set_tuned(knn_stage=3000)
    with pytest.raises(EtxError):
        tf.ctx.set_tuned(tc_stages__edge_update__bf16=6)
    with pytest.raises(EtxError):
        tf.ctx.set_tuned(no_such_knob=1)
