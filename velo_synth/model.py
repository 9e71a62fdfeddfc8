"""Model shapes, seeded random weights and the flat weight-blob format.

Input generator only: nothing here evaluates a network.  The paper trains
its networks (Sec. 5.1, 5.2); no trained weights exist here, so weights are
Kaiming-normal draws (fan-in, gain sqrt 2) from ``numpy.default_rng(seed)``
in the fixed parameter order of ``blob_layout``.  Biases are zero and
LayerNorm affines are (1, 0) unless ``perturb > 0``, which adds
N(0, perturb) to all of them so tests can see every bias and affine term.

Input normalisation (Sec. 5.1 footnote): per-feature mean and population
standard deviation over a calibration batch, for the embedding features
(r, phi, z) and for the interaction-network features (x, y, z).  They are
model parameters stored at the head of the blob, and both the oracle and
the CUDA path read them from there.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class ModelConfig:
    emb_widths: tuple = (3, 32, 32, 4)  # embedding MLP 3 -> ... -> D
    hidden: int = 32                    # n_h = n_e
    n_iters: int = 2                    # message-passing steps
    radius: float = 0.05                # graph cut: d^2 < radius^2
    k_max: int = 16                     # max edges per source hit
    n_planes: int = 26
    threshold_logit: float = 0.0        # keep an edge iff logit > this (0 = score 0.5)
    # log2 of the static e4m3 activation scales (one per matrix-product operand
    # of the interaction network, 4 n_iters + 3 of them); empty = all 1
    fp8_act_log2: tuple = ()

    @property
    def emb_dim(self) -> int:
        return int(self.emb_widths[-1])

    @property
    def fp8_act_scales(self):
        """The e4m3 activation scales (powers of two), or None for all 1."""
        return tuple(2.0 ** int(k) for k in self.fp8_act_log2) if self.fp8_act_log2 else None


def blob_layout(cfg: ModelConfig):
    """Ordered (name, shape) list of the flat float32 weight blob.

    Linear weights are [out, in] row-major.  MLP blocks of the interaction
    network are Lin -> LN -> ReLU -> Lin -> LN -> ReLU; the classifier is
    Lin -> LN -> ReLU -> Lin(H, 1)."""
    H, L = cfg.hidden, cfg.n_iters
    out = [("emb_mu", (3,)), ("emb_sigma", (3,)), ("gnn_mu", (3,)), ("gnn_sigma", (3,))]
    w = cfg.emb_widths
    for i in range(len(w) - 1):
        out += [(f"emb{i}.W", (w[i + 1], w[i])), (f"emb{i}.b", (w[i + 1],))]

    def block(prefix, k_in):
        return [(f"{prefix}.W1", (H, k_in)), (f"{prefix}.b1", (H,)),
                (f"{prefix}.g1", (H,)), (f"{prefix}.be1", (H,)),
                (f"{prefix}.W2", (H, H)), (f"{prefix}.b2", (H,)),
                (f"{prefix}.g2", (H,)), (f"{prefix}.be2", (H,))]

    out += block("node_enc", 3)
    out += block("edge_enc", 2 * H)
    for k in range(L):
        out += block(f"node{k}", 3 * H)
        out += block(f"edge{k}", 3 * H)
    out += [("cls.W1", (H, H)), ("cls.b1", (H,)), ("cls.g1", (H,)), ("cls.be1", (H,)),
            ("cls.W2", (1, H)), ("cls.b2", (1,))]
    return out


def blob_size(cfg: ModelConfig) -> int:
    return int(sum(int(np.prod(s)) for _, s in blob_layout(cfg)))


def normalisation_from(x, y, z):
    """(mu, sigma) for (r, phi, z) and for (x, y, z) over calibration hits."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    cyl = np.stack([np.hypot(x, y), np.arctan2(y, x), z])
    car = np.stack([x, y, z])
    return cyl.mean(1), cyl.std(1), car.mean(1), car.std(1)


def make_weights(cfg: ModelConfig, calib, seed: int = 0, perturb: float = 0.0) -> dict:
    """Named float32 parameter arrays.  ``calib`` is a Batch (or x, y, z)."""
    if hasattr(calib, "x"):
        calib = (calib.x, calib.y, calib.z)
    emb_mu, emb_sigma, gnn_mu, gnn_sigma = normalisation_from(*calib)
    rng = np.random.default_rng(seed)
    prng = np.random.default_rng(seed + 7919)
    p = {"emb_mu": emb_mu, "emb_sigma": emb_sigma, "gnn_mu": gnn_mu, "gnn_sigma": gnn_sigma}
    for name, shape in blob_layout(cfg):
        if name in p:
            continue
        leaf = name.rsplit(".", 1)[1]
        if leaf.startswith("W"):
            fan_in = shape[1]
            v = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shape)
        elif leaf.startswith("g"):
            v = np.ones(shape)
            if perturb:
                v = v + prng.normal(0.0, perturb, size=shape)
        else:  # biases and LN shifts
            v = np.zeros(shape)
            if perturb:
                v = v + prng.normal(0.0, perturb, size=shape)
        p[name] = v
    return {k: np.asarray(v, np.float32) for k, v in p.items()}


def pack_blob(cfg: ModelConfig, weights: dict) -> np.ndarray:
    parts = []
    for name, shape in blob_layout(cfg):
        a = np.asarray(weights[name], np.float32)
        if a.shape != tuple(shape):
            raise ValueError(f"{name}: shape {a.shape} != {shape}")
        parts.append(a.reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def unpack_blob(cfg: ModelConfig, blob: np.ndarray) -> dict:
    blob = np.asarray(blob, np.float32).reshape(-1)
    if blob.shape[0] != blob_size(cfg):
        raise ValueError("blob size does not match the model config")
    out, o = {}, 0
    for name, shape in blob_layout(cfg):
        n = int(np.prod(shape))
        out[name] = blob[o:o + n].reshape(shape)
        o += n
    return out


def triplet_layout(cfg: ModelConfig):
    """Ordered (name, shape) list of the triplet-classifier blob: one MLP for
    articulations ("art") and one for elbows ("elb"), each Lin(2H, H) -> LN
    -> ReLU -> Lin(H, 1) on the two edges' final encodings."""
    H = cfg.hidden
    out = []
    for p in ("art", "elb"):
        out += [(f"{p}.W1", (H, 2 * H)), (f"{p}.b1", (H,)), (f"{p}.g1", (H,)), (f"{p}.be1", (H,)),
                (f"{p}.W2", (1, H)), (f"{p}.b2", (1,))]
    return out


def make_triplet_weights(cfg: ModelConfig, seed: int = 0, perturb: float = 0.0) -> dict:
    """Kaiming-normal weights (fan-in, gain sqrt 2); biases 0, LayerNorm (1, 0),
    optionally perturbed like ``make_weights``."""
    rng = np.random.default_rng(seed + 104729)
    prng = np.random.default_rng(seed + 130363)
    p = {}
    for name, shape in triplet_layout(cfg):
        leaf = name.rsplit(".", 1)[1]
        if leaf.startswith("W"):
            v = rng.normal(0.0, np.sqrt(2.0 / shape[1]), size=shape)
        else:
            v = np.ones(shape) if leaf.startswith("g") else np.zeros(shape)
            if perturb:
                v = v + prng.normal(0.0, perturb, size=shape)
        p[name] = v
    return {k: np.asarray(v, np.float32) for k, v in p.items()}


def pack_triplet_blob(cfg: ModelConfig, weights: dict) -> np.ndarray:
    parts = []
    for name, shape in triplet_layout(cfg):
        a = np.asarray(weights[name], np.float32)
        if a.shape != tuple(shape):
            raise ValueError(f"{name}: shape {a.shape} != {shape}")
        parts.append(a.reshape(-1))
    return np.concatenate(parts).astype(np.float32)
