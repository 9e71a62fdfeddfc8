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
        # the library's backward reads these again: keep them alive until then
        fctx.inputs = (x, y, z, src, dst, edge_offsets)
        return logits

    @staticmethod
    def backward(fctx, dlogits):
        dtheta = fctx.etx_ctx.gnn_backward(dlogits.contiguous())
        return (dtheta,) + (None,) * 8


class Trainer:
    """Owns a training context, the parameters and the Adam state.  The edge
    loss is the class-weighted BCE (``loss="bce"``, ``pos_weight``) or the
    paper's sigmoid focal loss (``loss="focal"``, ``alpha``, ``gamma``)."""

    def __init__(self, model, blob: np.ndarray, max_events: int, max_hits: int, max_edges: int,
                 device: int = 0, dtype: str = "bf16", lr: float = 1e-3, pos_weight: float = 10.0,
                 loss: str = "bce", alpha: float = 0.25, gamma: float = 2.0):
        if loss not in ("bce", "focal"):
            raise ValueError("loss must be 'bce' or 'focal'")
        self.loss_kind, self.alpha, self.gamma = loss, alpha, gamma
        self.ctx = Context(model, max_events, max_hits, max_edges, device=device, train=True)
        self._blob = np.array(blob, dtype=np.float32, copy=True)
        self.n_theta = self.ctx.gnn_param_count
        self.head = self._blob.size - self.n_theta       # normalisation + embedding
        dev = self.ctx.device
        self.theta = torch.from_numpy(self._blob[self.head:].copy()).to(dev)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.dtype, self.lr, self.pos_weight = dtype, lr, pos_weight
        self.t = 0
        self.sync()

    @property
    def blob(self) -> np.ndarray:
        """The whole weight blob with the current parameters (a host copy)."""
        self._blob[self.head:] = self.theta.detach().cpu().numpy()
        return self._blob

    def sync(self):
        """Load the current parameters into the context from the host (the
        full reload, which also rebuilds the e4m3 images)."""
        self.ctx.load_weights(self.blob)

    def step(self, x, y, z, src, dst, edge_offsets, targets, reload: bool = True):
        """One forward / loss / backward / Adam step; returns the loss tensor.
        The updated parameters go into the context on the device
        (``set_gnn_params``); ``reload=False`` leaves the context's weights at
        their old values (for timing; call ``sync`` before the next step)."""
        logits = self.ctx.gnn_forward(x, y, z, src, dst, edge_offsets, dtype=self.dtype)
        if self.loss_kind == "focal":
            loss, dlogits = self.ctx.focal_loss(logits, targets, edge_offsets, self.alpha, self.gamma)
        else:
            loss, dlogits = self.ctx.weighted_bce(logits, targets, edge_offsets, self.pos_weight)
        grads = self.ctx.gnn_backward(dlogits)
        self.t += 1
        self.ctx.adam_step(self.theta, grads, self.m, self.v, self.t, lr=self.lr)
        if reload:  # on the device: no host round trip of the weights
            self.ctx.set_gnn_params(self.theta)
        return loss


class EmbeddingTrainer:
    """Training of the hit embedding (Sec. 5.1): the training pairs of the
    current embedding (hard negatives from the graph rule, one random pair
    per query, the genuine edges), the hinge loss of Eq. 2-3, the reverse pass
    and Adam -- every step runs in libetx.  Batches have their noise hits
    removed and event-local particle ids (velo_synth.drop_noise,
    compact_particle_ids).  Defaults follow the paper: k_max 50 and d2 below
    1.5 for the hard negatives, margin 1; w_genuine (> 1 in the paper, value
    not given) is 2."""

    EMB_OFFSET = 12  # the embedding parameters follow the 12 normalisation values

    def __init__(self, model, blob: np.ndarray, max_events: int, max_hits: int, device: int = 0,
                 lr: float = 1e-3, radius: float = float(np.sqrt(1.5)), k_max: int = 50,
                 margin: float = 1.0, w_genuine: float = 2.0, seed: int = 0):
        self.ctx = Context(model, max_events, max_hits, 1, device=device)
        dev = self.ctx.device
        self._blob = np.array(blob, dtype=np.float32, copy=True)
        self.n_theta = self.ctx.embed_param_count
        o = self.EMB_OFFSET
        self.theta = torch.from_numpy(self._blob[o:o + self.n_theta].copy()).to(dev)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.lr, self.radius, self.k_max = lr, radius, k_max
        self.margin, self.w_genuine = margin, w_genuine
        self.t = 0
        D = int(model.emb_widths[-1])
        self.emb = torch.empty(max_hits, D, dtype=torch.float32, device=dev)
        self.d_emb = torch.empty_like(self.emb)
        self.ws = self.ctx.embed_train_workspace(max_hits)
        self.capacity = max_hits * (k_max + 2)
        self.pairs = (torch.empty(self.capacity, dtype=torch.int32, device=dev),
                      torch.empty(self.capacity, dtype=torch.int32, device=dev),
                      torch.empty(self.capacity, dtype=torch.uint8, device=dev),
                      torch.empty(1, dtype=torch.int32, device=dev))
        self.hinge_ws = torch.empty(max(self.ctx.hinge_loss_workspace(max_hits, self.capacity), 16),
                                    dtype=torch.uint8, device=dev)
        self.gen = torch.Generator(device=dev)
        self.gen.manual_seed(seed)
        self.loss = torch.empty(3, dtype=torch.float32, device=dev)
        self.ctx.load_weights(self._blob)

    def sync(self):
        """Load the current embedding parameters into the context from the host
        (the steps update the context on the device: etx_set_embed_params)."""
        self.ctx.load_weights(self.current_blob())

    def current_blob(self) -> np.ndarray:
        """The weight blob with the current embedding parameters (host copy)."""
        o = self.EMB_OFFSET
        self._blob[o:o + self.n_theta] = self.theta.detach().cpu().numpy()
        return self._blob

    @property
    def blob(self) -> np.ndarray:
        """The weight blob with the current (trained) embedding parameters."""
        return self.current_blob()

    def step(self, x, y, z, plane, particle_id, hit_offsets):
        """One step; returns the loss tensor {L, L_genuine, L_fake} of the
        embedding before the update."""
        n = x.shape[0]
        emb = self.ctx.embed_forward_train(x, y, z, self.ws, emb=self.emb[:n])
        rand = torch.randint(-2 ** 31, 2 ** 31 - 1, (n,), dtype=torch.int32, device=x.device,
                             generator=self.gen)
        pq, pa, pg, npairs = self.ctx.embedding_pairs(emb, plane, particle_id, hit_offsets,
                                                      self.radius, self.k_max, rand,
                                                      self.capacity, out=self.pairs)
        self.ctx.hinge_loss(emb, pq, pa, pg, npairs, self.margin, self.w_genuine, loss=self.loss,
                            d_emb=self.d_emb[:n], workspace=self.hinge_ws)
        grads = self.ctx.embed_backward(self.d_emb[:n], self.ws)
        self.t += 1
        self.ctx.adam_step(self.theta, grads, self.m, self.v, self.t, lr=self.lr)
        self.ctx.set_embed_params(self.theta)  # on the device: no host round trip
        return self.loss
