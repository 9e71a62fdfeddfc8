"""Calibrate the graph radius and the edge-score cut of a workload with the
oracle (test infrastructure; run by hand, results recorded in the presets).

The paper's networks are trained; here the weights are random, so the
literal radii of the workload descriptions (0.05, 0.1) give almost no edges.
This script picks, on the calibration events (seed 12345), the radius whose
mean edge count per hit is ``EDGES_PER_HIT`` (about 20k edges for a
1,740-hit event, the density the workloads ask for and close to the paper's
30k edges for 2,200 hits, Sec. 5), and the logit cut whose kept fraction
equals the genuine-edge fraction of that graph (the trained classifier keeps
roughly the genuine edges, Sec. 5.2).

    python -m oracle.calibrate batch500 plain

With ``--fp8`` it calibrates the static e4m3 activation scales instead
(Sec. 7.4 calibrates its INT8 quantisation on simulated events; here the
largest magnitude of every activation operand of the exact forward over the
first calibration events, per event so that memory stays small, turned into
the smallest power-of-two scale that keeps it within e4m3's 448):

    python -m oracle.calibrate --fp8 batch500 pileup4x
"""
from __future__ import annotations

import json
import sys

import numpy as np

from velo_synth import WORKLOADS, global_particle_ids, make_batch, truth_edge_labels
from velo_synth.presets import CALIB_SEED

from . import etx_oracle as O

EDGES_PER_HIT = 11.5


def calibrate(name: str, n_graph_events: int = 50, n_gnn_events: int = 3,
              keep_radius: bool = False) -> dict:
    """``keep_radius``: keep the workload's radius (a workload sharing another
    one's embedding) and calibrate the logit cut only."""
    wl = WORKLOADS[name]
    cfg = wl.model
    W = wl.weights()
    depth = len(cfg.emb_widths) - 1
    b = make_batch(wl.recipe, n_graph_events, CALIB_SEED)
    emb = O.embed(W, depth, b.x, b.y, b.z)
    lo, hi = 0.05, 8.0
    for _ in range(0 if keep_radius else 30):
        r = 0.5 * (lo + hi)
        _, _, eo = O.build_graph(emb, b.plane, b.hit_offsets, r, cfg.k_max)
        if eo[-1] / b.n_hits < EDGES_PER_HIT:
            lo = r
        else:
            hi = r
    radius = cfg.radius if keep_radius else float(f"{0.5 * (lo + hi):.3g}")
    _, _, eo = O.build_graph(emb, b.plane, b.hit_offsets, radius, cfg.k_max)
    gb = make_batch(wl.recipe, n_gnn_events, CALIB_SEED)
    gemb = O.embed(W, depth, gb.x, gb.y, gb.z)
    s, d, _ = O.build_graph(gemb, gb.plane, gb.hit_offsets, radius, cfg.k_max)
    z = O.gnn_forward(W, cfg.n_iters, gb.x, gb.y, gb.z, s, d)
    y = truth_edge_labels(global_particle_ids(gb), gb.plane, s, d)
    frac = float(y.mean()) if y.size else 0.0
    thr = float(f"{np.quantile(z, 1.0 - frac):.6g}") if z.size else 0.0
    return {"radius": radius, "edges_per_hit": float(eo[-1] / b.n_hits),
            "edges_per_event": float(eo[-1] / b.n_events), "genuine_fraction": frac,
            "threshold_logit": thr, "kept_fraction": float((z > thr).mean()) if z.size else 0.0,
            "logit_mean": float(z.mean()) if z.size else 0.0,
            "logit_std": float(z.std()) if z.size else 0.0}


def calibrate_fp8(name: str, n_events: int) -> dict:
    """log2 of the e4m3 activation scales (``O.act_scale_names`` order) from
    the amax over the first ``n_events`` calibration events."""
    wl = WORKLOADS[name]
    cfg = wl.model
    W = wl.weights()
    depth = len(cfg.emb_widths) - 1
    b = make_batch(wl.recipe, n_events, CALIB_SEED)
    amax = np.zeros(O.n_act_scales(cfg.n_iters))
    for i in range(b.n_events):
        ev = b.event(i)
        emb = O.embed(W, depth, ev.x, ev.y, ev.z)
        s, d, _ = O.build_graph(emb, ev.plane, ev.hit_offsets, cfg.radius, cfg.k_max)
        if s.size:
            amax = np.maximum(amax, O.activation_amax(W, cfg.n_iters, ev.x, ev.y, ev.z, s, d))
    log2 = [int(np.log2(O.fp8_act_scale(a))) for a in amax]
    return {"fp8_events": n_events, "fp8_act_amax": [float(f"{a:.6g}") for a in amax],
            "fp8_act_log2": log2}


if __name__ == "__main__":
    args = sys.argv[1:]
    if "--fp8" in args:
        names = [a for a in args if not a.startswith("--")]
        n_ev = {"batch500": 40, "pileup4x": 8}
        print(json.dumps({n: calibrate_fp8(n, n_ev.get(n, 20)) for n in names}, indent=1))
        sys.exit(0)
    keep = "--keep-radius" in args
    names = [a for a in args if not a.startswith("--")] or ["plain", "batch500"]
    print(json.dumps({n: calibrate(n, n_graph_events=5 if keep else 50, keep_radius=keep)
                      for n in names}, indent=1))
