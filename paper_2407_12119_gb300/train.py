"""Training step of the interaction network on the library's kernels:
forward (FP32 or BF16 tensor cores, per-step checkpoints kept), weighted BCE,
hand-written backward with recomputation, Adam -- every step runs in libetx.

``InteractionNetworkFn`` is the torch.autograd.Function view of the same
forward / backward pair, for callers that build their own optimiser loop.
"""
from __future__ import annotations

import numpy as np
import torch

from .etx import Context


class InteractionNetworkFn(torch.autograd.Function):
    """logits = f(theta; graph).  ``theta`` is the flat interaction-network
    parameter vector (blob order from the node encoder on); the context must
    hold the same values (``Trainer.sync`` loads them)."""

    @staticmethod
    def forward(fctx, theta, etx_ctx: Context, x, y, z, src, dst, edge_offsets, dtype: str):
        logits = etx_ctx.gnn_forward(x, y, z, src, dst, edge_offsets, dtype=dtype)
        fctx.etx_ctx = etx_ctx
        return logits

    @staticmethod
    def backward(fctx, dlogits):
        dtheta = fctx.etx_ctx.gnn_backward(dlogits.contiguous())
        return (dtheta,) + (None,) * 8


class Trainer:
    """Owns a training context, the parameters and the Adam state."""

    def __init__(self, model, blob: np.ndarray, max_events: int, max_hits: int, max_edges: int,
                 device: int = 0, dtype: str = "bf16", lr: float = 1e-3, pos_weight: float = 10.0):
        self.ctx = Context(model, max_events, max_hits, max_edges, device=device, train=True)
        self.blob = np.array(blob, dtype=np.float32, copy=True)
        self.n_theta = self.ctx.gnn_param_count
        self.head = self.blob.size - self.n_theta        # normalisation + embedding
        dev = self.ctx.device
        self.theta = torch.from_numpy(self.blob[self.head:].copy()).to(dev)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.dtype, self.lr, self.pos_weight = dtype, lr, pos_weight
        self.t = 0
        self.sync()

    def sync(self):
        """Load the current parameters into the context."""
        self.blob[self.head:] = self.theta.detach().cpu().numpy()
        self.ctx.load_weights(self.blob)

    def step(self, x, y, z, src, dst, edge_offsets, targets):
        """One forward / loss / backward / Adam step; returns the loss tensor."""
        logits = self.ctx.gnn_forward(x, y, z, src, dst, edge_offsets, dtype=self.dtype)
        loss, dlogits = self.ctx.weighted_bce(logits, targets, edge_offsets, self.pos_weight)
        grads = self.ctx.gnn_backward(dlogits)
        self.t += 1
        self.ctx.adam_step(self.theta, grads, self.m, self.v, self.t, lr=self.lr)
        self.sync()
        return loss
