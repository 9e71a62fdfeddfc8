"""Whole hot path in one object: hits of a ragged event batch in, track labels
out (paper Sec. 5 without the triplet stage, as in its Sec. 7 port).

``TrackFinder.run_device`` works on device-resident tensors; ``find_tracks``
takes host arrays, copies them to the GPU, runs the four library calls and
copies the labels back; ``capture`` records one ``run_device`` call (every
launch of the four steps) into a CUDA graph that ``replay`` re-issues with a
single launch.  All of them only marshal arguments: every step runs in libetx.
"""
from __future__ import annotations

import numpy as np
import torch

from .etx import Context


class TrackFinder:
    """Context + reusable device buffers sized for a batch capacity."""

    def __init__(self, model, blob: np.ndarray, max_events: int, max_hits: int,
                 max_edges: int | None = None, device: int = 0, dtype: str = "f32"):
        self.model = model
        self.dtype = dtype
        self.max_edges = int(max_edges or max_hits * model.k_max)
        self.ctx = Context(model, max_events, max_hits, self.max_edges, device=device)
        self.ctx.load_weights(blob)
        # static e4m3 activation scales of the model (used by dtype "fp8" only)
        self.ctx.set_fp8_scales(getattr(model, "fp8_act_scales", None))
        dev = self.ctx.device
        self.dev = dev
        self.emb = torch.empty((max_hits, model.emb_widths[-1]), dtype=torch.float32, device=dev)
        self.src = torch.empty(self.max_edges, dtype=torch.int32, device=dev)
        self.dst = torch.empty(self.max_edges, dtype=torch.int32, device=dev)
        self.eoff = torch.empty(max_events + 1, dtype=torch.int32, device=dev)
        self.logits = torch.empty(self.max_edges, dtype=torch.float32, device=dev)
        self.labels = torch.empty(max_hits, dtype=torch.int32, device=dev)
        self.n_tracks = torch.empty(max(max_events, 1), dtype=torch.int32, device=dev)
        self.in_x = torch.empty(max_hits, dtype=torch.float32, device=dev)
        self.in_y = torch.empty_like(self.in_x)
        self.in_z = torch.empty_like(self.in_x)
        self.in_plane = torch.empty(max_hits, dtype=torch.int8, device=dev)
        self.in_hoff = torch.empty(max_events + 1, dtype=torch.int32, device=dev)

    def run_device(self, x, y, z, plane, hit_offsets, n_hits: int, n_events: int,
                   min_hits: int = 3):
        """All four steps on device tensors; returns (labels, n_tracks) views."""
        m, c = self.model, self.ctx
        emb = c.embed(x[:n_hits], y[:n_hits], z[:n_hits], out=self.emb[:n_hits])
        eoff = self.eoff[:n_events + 1]
        c.build_graph(emb, plane[:n_hits], hit_offsets[:n_events + 1], m.radius, m.k_max,
                      out=(self.src, self.dst, eoff))
        c.gnn_forward(x[:n_hits], y[:n_hits], z[:n_hits], self.src, self.dst, eoff,
                      dtype=self.dtype, logits=self.logits)
        labels, nt = c.edges_to_tracks(self.src, self.dst, self.logits, m.threshold_logit, eoff,
                                       hit_offsets[:n_events + 1], min_hits=min_hits,
                                       labels=self.labels[:n_hits],
                                       n_tracks=self.n_tracks[:max(n_events, 1)])
        return labels, nt

    def autotune(self, x, y, z, plane, hit_offsets, n_hits: int, n_events: int):
        """Let the library time its candidate launch configurations on this batch
        (k-NN work partitioning, tensor-core ring depth) and keep the fastest;
        returns the choices.  Capture after tuning: a graph keeps the
        configuration it was recorded with."""
        m = self.model
        eoff = self.eoff[:n_events + 1]
        return self.ctx.autotune(x[:n_hits], y[:n_hits], z[:n_hits], plane[:n_hits],
                                 hit_offsets[:n_events + 1], m.radius, m.k_max,
                                 self.emb[:n_hits], self.src, self.dst, eoff, self.logits,
                                 dtype=self.dtype)

    def capture(self, x, y, z, plane, hit_offsets, n_hits: int, n_events: int,
                min_hits: int = 3):
        """Record ``run_device`` on these device tensors into one CUDA graph.

        The graph is specialised to the tensors' addresses and to ``n_hits`` and
        ``n_events``: to process another batch of the same sizes, copy its hits
        into the same tensors and call ``replay``.  One eager call runs first, so
        one-time set-up (kernel attributes) happens outside the capture.
        Returns the (labels, n_tracks) views that each replay rewrites.
        """
        self.run_device(x, y, z, plane, hit_offsets, n_hits, n_events, min_hits)
        torch.cuda.synchronize(self.dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.graph_out = self.run_device(x, y, z, plane, hit_offsets, n_hits, n_events,
                                             min_hits)
        torch.cuda.synchronize(self.dev)
        return self.graph_out

    def replay(self):
        """Re-issue the captured step on the current stream; returns its outputs."""
        if getattr(self, "graph", None) is None:
            raise RuntimeError("TrackFinder.replay: nothing captured (call capture first)")
        self.graph.replay()
        return self.graph_out

    def find_tracks(self, x, y, z, plane, hit_offsets, labels_out=None, n_tracks_out=None,
                    min_hits: int = 3):
        """Host tensors in (pinned for asynchronous copies), host labels out."""
        n_hits, n_events = int(x.shape[0]), int(hit_offsets.shape[0] - 1)
        self.in_x[:n_hits].copy_(x, non_blocking=True)
        self.in_y[:n_hits].copy_(y, non_blocking=True)
        self.in_z[:n_hits].copy_(z, non_blocking=True)
        self.in_plane[:n_hits].copy_(plane, non_blocking=True)
        self.in_hoff[:n_events + 1].copy_(hit_offsets, non_blocking=True)
        labels, nt = self.run_device(self.in_x, self.in_y, self.in_z, self.in_plane, self.in_hoff,
                                     n_hits, n_events, min_hits)
        if labels_out is None:
            labels_out = torch.empty(n_hits, dtype=torch.int32, pin_memory=True)
        if n_tracks_out is None:
            n_tracks_out = torch.empty(max(n_events, 1), dtype=torch.int32, pin_memory=True)
        labels_out.copy_(labels, non_blocking=True)
        n_tracks_out.copy_(nt, non_blocking=True)
        return labels_out, n_tracks_out
