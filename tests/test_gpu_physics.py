"""End to end with training: the embedding (Sec. 5.1) and the interaction
network trained on synthetic events by the library's own kernels give tracks
that the Table 1 metrics rate as physical on held-out events (the random
weights give almost no matched particles)."""
import dataclasses

import numpy as np
import pytest
import torch

from velo_synth import (WORKLOADS, compact_particle_ids, drop_noise, global_particle_ids,
                        make_batch, pack_blob, truth_edge_labels)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import pipeline, train
    return pipeline, train


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_trained_pipeline_finds_the_tracks(lib):
    pipeline, train = lib
    wl = WORKLOADS["batch500"]
    m = dataclasses.replace(wl.model, radius=float(np.sqrt(0.9)), k_max=50, threshold_logit=0.0)
    blob = pack_blob(m, wl.weights())
    batches = [make_batch(wl.recipe, 16, 90000 + 16 * i) for i in range(2)]
    max_hits = max(b.n_hits for b in batches)
    et = train.EmbeddingTrainer(m, blob, 16, max_hits)
    nf = [drop_noise(b) for b in batches]
    args = [[cuda(v) for v in (c.x, c.y, c.z, c.plane, compact_particle_ids(c), c.hit_offsets)] for c in nf]
    for k in range(250):
        et.step(*args[k % 2])
    blob = et.blob.copy()
    probe = pipeline.TrackFinder(m, blob, 16, max_hits)
    graphs = []
    for b in batches:
        x, y, z, p, h = cuda(b.x), cuda(b.y), cuda(b.z), cuda(b.plane), cuda(b.hit_offsets)
        src, dst, eo = probe.ctx.build_graph(probe.ctx.embed(x, y, z), p, h, m.radius, m.k_max)
        probe.ctx.sync()
        E = int(eo[-1].item())
        yb = truth_edge_labels(global_particle_ids(b), b.plane, src[:E].cpu().numpy(), dst[:E].cpu().numpy())
        graphs.append((x, y, z, src[:E].contiguous(), dst[:E].contiguous(), eo, cuda(yb)))
    gt = train.Trainer(m, blob, 16, max_hits, max(g[3].shape[0] for g in graphs), dtype="bf16",
                       pos_weight=1.0)
    for k in range(250):
        gt.step(*graphs[k % 2])
    ev = make_batch(wl.recipe, 32, wl.base_seed)
    pid = cuda(compact_particle_ids(ev))
    out = {}
    for name, weights in (("random", pack_blob(m, wl.weights())), ("trained", gt.blob)):
        tf = pipeline.TrackFinder(m, weights, ev.n_events, ev.n_hits, dtype="bf16")
        x, y, z, p, h = cuda(ev.x), cuda(ev.y), cuda(ev.z), cuda(ev.plane), cuda(ev.hit_offsets)
        labels, _ = tf.run_device(x, y, z, p, h, ev.n_hits, ev.n_events)
        _, vals = tf.ctx.track_metrics(labels, pid, h)
        tf.ctx.sync()
        out[name] = vals.cpu().numpy()[2:]
    print("efficiency, clone, fake, hit efficiency, hit purity:", out)
    # a short training on 32 events (150 + 150 steps gave 70% efficiency, 16% fakes)
    assert out["trained"][0] > 0.5 and out["trained"][2] < 0.3
    assert out["trained"][0] > 10 * max(out["random"][0], 1e-3)
