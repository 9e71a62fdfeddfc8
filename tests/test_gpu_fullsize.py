"""Parity at the full sizes, in the launch configuration the benchmark times:
the whole 500-event batch (and the 1,000-event pile-up batch) goes through the
autotuned step replayed from its CUDA graph; sampled events, which are
independent of the rest of the batch, are then recomputed one by one by the
FP64 oracle from its own inputs and compared: embeddings within the FP32
bound, edge lists exactly apart from pairs within 1e-5 of the radius or of
the k-th kept distance (counted), logits within the dtype's tolerance on
events whose graphs agree, labels exactly where the edge masks agree."""
import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import WORKLOADS, pack_blob

pytestmark = pytest.mark.gpu
NEAR_CUT = 1e-5
LOGIT_TOL = {"f32": 1e-4, "bf16": 2e-2}   # bf16: vs the oracle's BF16 reading, as the stage tests


@pytest.fixture(scope="module")
def pipeline():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import pipeline as p
    return p


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def near_cut(emb64, i, j, plane, lo, hi, r, k):
    dist = np.sqrt(((emb64[i] - emb64[j]) ** 2).sum())
    if abs(dist - r) <= NEAR_CUT:
        return True
    cand = np.arange(lo, hi)[np.isin(plane[lo:hi].astype(int) - int(plane[i]), [1, 2])]
    dd = np.sort(np.sqrt(((emb64[cand] - emb64[i]) ** 2).sum(1)))
    dd = dd[dd < r]
    return dd.size > k and abs(dist - dd[k - 1]) <= NEAR_CUT


def run_full(pipeline, name, dtype):
    wl = WORKLOADS[name]
    m = wl.model
    b = wl.batch()
    W = wl.weights()
    tf = pipeline.TrackFinder(m, pack_blob(m, W), b.n_events, b.n_hits, b.n_hits * m.k_max,
                              dtype=dtype)
    x, y, z, p, h = cuda(b.x), cuda(b.y), cuda(b.z), cuda(b.plane), cuda(b.hit_offsets)
    tf.autotune(x, y, z, p, h, b.n_hits, b.n_events)
    tf.capture(x, y, z, p, h, b.n_hits, b.n_events)
    labels, _ = tf.replay()
    torch.cuda.synchronize()
    E = int(tf.eoff[b.n_events].item())
    out = dict(emb=tf.emb[:b.n_hits].cpu().numpy().astype(np.float64),
               src=tf.src[:E].cpu().numpy(), dst=tf.dst[:E].cpu().numpy(),
               eoff=tf.eoff[:b.n_events + 1].cpu().numpy(), logits=tf.logits[:E].cpu().numpy(),
               labels=labels.cpu().numpy())
    tf.ctx.sync()
    return wl, b, W, out


def check_event(wl, b, W, g, ev, dtype):
    m = wl.model
    lo, hi = int(b.hit_offsets[ev]), int(b.hit_offsets[ev + 1])
    e = b.event(ev)
    emb64 = O.embed(W, len(m.emb_widths) - 1, e.x, e.y, e.z)
    bound = 2e-6 * (1.0 + np.abs(emb64).max())
    assert np.abs(g["emb"][lo:hi] - emb64).max() <= bound
    s, d, _ = O.build_graph(emb64, e.plane, e.hit_offsets, m.radius, m.k_max)
    e0, e1 = int(g["eoff"][ev]), int(g["eoff"][ev + 1])
    gs, gd = g["src"][e0:e1] - lo, g["dst"][e0:e1] - lo
    diff = set(zip(gs.tolist(), gd.tolist())) ^ set(zip(s.tolist(), d.tolist()))
    assert all(near_cut(emb64, i, j, e.plane, 0, hi - lo, m.radius, m.k_max) for i, j in diff)
    if diff:
        return f"event {ev}: {len(diff)} near-cut pairs differ", False
    ref = O.gnn_forward(W, m.n_iters, e.x, e.y, e.z, s, d,
                        gemm="bf16" if dtype == "bf16" else "fp64")
    err = np.abs(g["logits"][e0:e1] - ref).max() if s.size else 0.0
    assert err <= LOGIT_TOL[dtype], (ev, err)
    mask_gpu = g["logits"][e0:e1] > m.threshold_logit
    mask_ref = ref > m.threshold_logit
    flips = int((mask_gpu != mask_ref).sum())
    if flips == 0:
        ref_lab = O.connected_components(s, d, mask_ref, e.hit_offsets)
        np.testing.assert_array_equal(g["labels"][lo:hi], ref_lab)
    return f"event {ev}: {hi - lo} hits, {s.size} edges, max |logit err| {err:.2e}, mask flips {flips}", True


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_full_batch500_sampled_events(pipeline, dtype):
    wl, b, W, g = run_full(pipeline, "batch500", dtype)
    sizes = np.diff(b.hit_offsets)
    sample = sorted({0, b.n_events // 2, b.n_events - 1, int(np.argmax(sizes))})
    agreed = 0
    for ev in sample:
        msg, ok = check_event(wl, b, W, g, ev, dtype)
        agreed += ok
        print(dtype, msg)
    assert agreed >= 2


def test_full_pileup_sampled_events(pipeline):
    wl, b, W, g = run_full(pipeline, "pileup4x", "bf16")
    sample = [0, b.n_events - 1]
    agreed = 0
    for ev in sample:
        msg, ok = check_event(wl, b, W, g, ev, "bf16")
        agreed += ok
        print("pileup", msg)
    assert agreed >= 1
