"""Thin ctypes binding of libetx (include/etx.h).

Argument marshalling only: every step of the pipeline runs in the CUDA
library.  PyTorch provides device memory and the current stream.  If the
library has not been built the import of this module still works, but the
first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np
import torch

# ETX_LIBRARY may name another build of the same library (same ABI)
_LIB_PATH = Path(os.environ.get("ETX_LIBRARY") or Path(__file__).resolve().parent / "libetx.so")
_lib = None

ETX_OK, ETX_ERR_ARG, ETX_ERR_UNSORTED, ETX_ERR_CAPACITY = 0, 1, 2, 3
ETX_ERR_CUDA, ETX_ERR_TIMEOUT, ETX_ERR_UNSUPPORTED, ETX_ERR_STATE = 4, 5, 6, 7
_STATUS_NAMES = {0: "ETX_OK", 1: "ETX_ERR_ARG", 2: "ETX_ERR_UNSORTED", 3: "ETX_ERR_CAPACITY",
                 4: "ETX_ERR_CUDA", 5: "ETX_ERR_TIMEOUT", 6: "ETX_ERR_UNSUPPORTED",
                 7: "ETX_ERR_STATE"}
DTYPES = {"f32": 0, "bf16": 1, "fp8": 2, "bf16s": 3}  # bf16s: BF16 GEMMs, edge stream stored in BF16
MAX_EMB_LAYERS = 8

EXPORTED = ["etx_ctx_create", "etx_ctx_destroy", "etx_last_error", "etx_weights_size",
            "etx_load_weights", "etx_ctx_sync", "etx_embed", "etx_build_graph",
            "etx_gnn_forward", "etx_gnn_param_count", "etx_gnn_backward",
            "etx_edges_to_tracks", "etx_edges_to_tracks_noalloc", "etx_launch_count",
            "etx_profile_enable", "etx_profile_read", "etx_weighted_bce", "etx_adam_step",
            "etx_autotune", "etx_tuned", "etx_set_tuned", "etx_edges_to_tracks_sweep",
            "etx_track_metrics_workspace", "etx_track_metrics", "etx_embed_param_count",
            "etx_embed_train_workspace", "etx_embed_forward_train", "etx_embed_backward",
            "etx_embedding_pairs_workspace", "etx_embedding_pairs", "etx_hinge_loss_workspace",
            "etx_hinge_loss",
            "etx_triplet_weights_size", "etx_load_triplet_weights", "etx_triplets_workspace",
            "etx_build_triplets", "etx_classify_triplets", "etx_fp8_scale_count",
            "etx_set_fp8_scales", "etx_tracks_workspace", "etx_tracks_from_triplets",
            "etx_set_gnn_params", "etx_gnn_checkpoints", "etx_set_embed_params", "etx_focal_loss"]
# etx_track_metrics outputs
TRACK_COUNTS = ["particles", "matched_particles", "candidates", "candidate_particles", "tracks",
                "unmatched_tracks"]
TRACK_VALUES = ["hit_eff_sum", "hit_purity_sum", "efficiency", "clone_rate", "fake_rate",
                "hit_efficiency", "hit_purity"]
# knob names of the autotuner (etx_tuned)
TUNE_KNOBS = ["knn_split", "knn_stage"] + [f"tc_stages/{b}/{d}" for b in
                              ("edge_encoder", "node_update", "edge_update", "classifier")
                              for d in ("bf16", "fp8")]


class EtxConfig(ctypes.Structure):
    _fields_ = [("emb_depth", ctypes.c_int32),
                ("emb_widths", ctypes.c_int32 * (MAX_EMB_LAYERS + 1)),
                ("hidden", ctypes.c_int32),
                ("n_iters", ctypes.c_int32),
                ("n_planes", ctypes.c_int32),
                ("max_events", ctypes.c_int32),
                ("max_hits", ctypes.c_int64),
                ("max_edges", ctypes.c_int64),
                ("train", ctypes.c_int32),
                ("uf_iter_cap", ctypes.c_int32)]


class EtxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def library_path() -> Path:
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """Load libetx.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"{_LIB_PATH.name} is not built: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(str(_LIB_PATH))
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    cfgp = ctypes.POINTER(EtxConfig)
    sig = {
        "etx_ctx_create": (i32, [cfgp, i32, ctypes.POINTER(vp)]),
        "etx_ctx_destroy": (i32, [vp]),
        "etx_last_error": (ctypes.c_char_p, [vp]),
        "etx_weights_size": (i64, [cfgp]),
        "etx_gnn_param_count": (i64, [cfgp]),
        "etx_load_weights": (i32, [vp, vp, i64]),
        "etx_ctx_sync": (i32, [vp, vp]),
        "etx_embed": (i32, [vp, vp, vp, vp, i64, vp, vp]),
        "etx_build_graph": (i32, [vp, vp, vp, vp, i32, i64, f32, i32, vp, vp, i64, vp, vp]),
        "etx_gnn_forward": (i32, [vp, vp, vp, vp, i64, vp, vp, vp, i32, i32, vp, vp]),
        "etx_gnn_backward": (i32, [vp, vp, vp, vp]),
        "etx_edges_to_tracks": (i32, [vp, vp, vp, vp, f32, vp, vp, i32, i64, i32, vp, vp, vp]),
        "etx_edges_to_tracks_noalloc": (i32, [vp, vp, vp, f32, vp, vp, i32, i64, i32, vp, vp, vp,
                                              vp]),
        "etx_weighted_bce": (i32, [vp, vp, vp, vp, i32, f32, vp, vp, vp]),
        "etx_adam_step": (i32, [vp, vp, vp, vp, vp, i64, f32, f32, f32, f32, i64, vp]),
        "etx_autotune": (i32, [vp, vp, vp, vp, vp, vp, i32, i64, f32, i32, i32, vp, vp, vp, i64,
                               vp, vp, vp]),
        "etx_tuned": (i32, [vp, ctypes.c_char_p]),
        "etx_edges_to_tracks_sweep": (i32, [vp, vp, vp, vp, f32, vp, vp, vp, i32, i64, vp, vp]),
        "etx_set_tuned": (i32, [vp, ctypes.c_char_p, i32]),
        "etx_track_metrics_workspace": (ctypes.c_size_t, [i32, i64]),
        "etx_embed_param_count": (i64, [cfgp]),
        "etx_embed_train_workspace": (ctypes.c_size_t, [cfgp, i64]),
        "etx_embed_forward_train": (i32, [vp, vp, vp, vp, i64, vp, vp, ctypes.c_size_t, vp]),
        "etx_embed_backward": (i32, [vp, i64, vp, vp, vp, ctypes.c_size_t, vp]),
        "etx_embedding_pairs_workspace": (ctypes.c_size_t, [i32, i64, i32]),
        "etx_embedding_pairs": (i32, [vp, vp, vp, vp, vp, i32, i64, f32, i32, vp, i32, vp,
                                      ctypes.c_size_t, vp, vp, vp, i64, vp, vp]),
        "etx_hinge_loss_workspace": (ctypes.c_size_t, [i64, i64]),
        "etx_hinge_loss": (i32, [vp, vp, i64, vp, vp, vp, vp, i64, f32, f32, vp, vp, vp,
                                 ctypes.c_size_t, vp]),
        "etx_triplet_weights_size": (i64, [cfgp]),
        "etx_load_triplet_weights": (i32, [vp, vp, i64]),
        "etx_triplets_workspace": (ctypes.c_size_t, [i64]),
        "etx_build_triplets": (i32, [vp, vp, vp, vp, f32, vp, i32, i64, vp, ctypes.c_size_t, vp,
                                     vp, vp, i64, vp, vp]),
        "etx_classify_triplets": (i32, [vp, vp, vp, vp, i64, vp, vp]),
        "etx_track_metrics": (i32, [vp, vp, vp, vp, i32, i64, i32, i32, i32, vp, ctypes.c_size_t,
                                    vp, vp, vp]),
        "etx_tracks_workspace": (ctypes.c_size_t, [i64, i64, i64]),
        "etx_tracks_from_triplets": (i32, [vp, vp, vp, vp, f32, vp, i32, i64, vp, vp, vp, f32, vp,
                                           i64, i32, vp, ctypes.c_size_t, vp, vp, i64, i64, vp,
                                           vp]),
        "etx_fp8_scale_count": (i64, [cfgp]),
        "etx_set_gnn_params": (i32, [vp, vp, vp]),
        "etx_gnn_checkpoints": (i32, [vp, i32, vp, vp, vp]),
        "etx_set_embed_params": (i32, [vp, vp, vp]),
        "etx_focal_loss": (i32, [vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, vp, vp, vp]),
        "etx_set_fp8_scales": (i32, [vp, vp, i64]),
        "etx_launch_count": (i64, [vp]),
        "etx_profile_enable": (i32, [vp, i32]),
        "etx_profile_read": (i32, [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int64), i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def make_config(model, max_events: int, max_hits: int, max_edges: int, train: bool = False,
                uf_iter_cap: int = 0) -> EtxConfig:
    """``model`` needs emb_widths, hidden, n_iters and n_planes attributes;
    ``uf_iter_cap`` > 0 replaces the union-find loops' default iteration caps."""
    c = EtxConfig()
    w = list(model.emb_widths)
    if len(w) - 1 > MAX_EMB_LAYERS:
        raise ValueError("too many embedding layers")
    c.emb_depth = len(w) - 1
    for i, v in enumerate(w):
        c.emb_widths[i] = int(v)
    c.hidden = int(model.hidden)
    c.n_iters = int(model.n_iters)
    c.n_planes = int(getattr(model, "n_planes", 26))
    c.max_events = int(max_events)
    c.max_hits = int(max_hits)
    c.max_edges = int(max_edges)
    c.train = int(bool(train))
    c.uf_iter_cap = int(uf_iter_cap)
    return c


def weights_size(model) -> int:
    return int(lib().etx_weights_size(ctypes.byref(make_config(model, 1, 1, 1))))


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, dtype, name, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


NOALLOC_MAX_HITS = 1 << 21


def edges_to_tracks_noalloc(src, dst, logits, threshold_logit: float, edge_offsets, hit_offsets,
                            labels, n_tracks=None, min_hits: int = 3, status=None, stream=None):
    """etx_edges_to_tracks_noalloc: the components step without a context and
    without any device allocation (its scratch is a fixed array inside the
    library, at most NOALLOC_MAX_HITS hits).  Every array is caller-owned;
    ``status`` (int32 [1] on the device, optional) receives the call's
    device-side status (ETX_OK, ETX_ERR_TIMEOUT or ETX_ERR_UNSORTED)."""
    dev = labels.device
    _need(src, torch.int32, "src", dev)
    _need(dst, torch.int32, "dst", dev)
    _need(logits, torch.float32, "logits", dev)
    _need(edge_offsets, torch.int32, "edge_offsets", dev)
    _need(hit_offsets, torch.int32, "hit_offsets", dev)
    _need(labels, torch.int32, "labels", dev)
    if n_tracks is not None:
        _need(n_tracks, torch.int32, "n_tracks", dev)
    if status is not None:
        _need(status, torch.int32, "status", dev)
    st = lib().etx_edges_to_tracks_noalloc(_ptr(src), _ptr(dst), _ptr(logits), float(threshold_logit),
                                           _ptr(edge_offsets), _ptr(hit_offsets),
                                           hit_offsets.shape[0] - 1, labels.shape[0], int(min_hits),
                                           _ptr(labels), _ptr(n_tracks), _ptr(status),
                                           _stream(stream))
    if st != ETX_OK:
        raise EtxError(st, "etx_edges_to_tracks_noalloc failed")
    return labels, n_tracks


class Context:
    """An etx_ctx: model shapes, capacities, loaded weights and scratch."""

    def __init__(self, model, max_events: int, max_hits: int, max_edges: int, device: int = 0,
                 train: bool = False, uf_iter_cap: int = 0):
        L = lib()
        self.model = model
        self.cfg = make_config(model, max_events, max_hits, max_edges, train, uf_iter_cap)
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        st = L.etx_ctx_create(ctypes.byref(self.cfg), int(device), ctypes.byref(h))
        if st != ETX_OK:
            raise EtxError(st, "etx_ctx_create failed (bad config or out of device memory)")
        self._h = h
        self.emb_dim = int(model.emb_widths[-1])

    def close(self):
        if getattr(self, "_h", None):
            lib().etx_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != ETX_OK:
            msg = lib().etx_last_error(self._h)
            raise EtxError(st, msg.decode() if msg else "")

    # ---- entry points ------------------------------------------------------
    def load_weights(self, blob: np.ndarray):
        b = np.ascontiguousarray(blob, dtype=np.float32)
        self._check(lib().etx_load_weights(self._h, b.ctypes.data_as(ctypes.c_void_p), b.size))

    def set_gnn_params(self, theta, stream=None):
        """etx_set_gnn_params: the interaction-network parameters from a device
        float32 vector (blob order from the node encoder on), repacked on the
        device."""
        _need(theta, torch.float32, "theta", self.device)
        if theta.numel() != self.gnn_param_count:
            raise ValueError("theta must hold gnn_param_count values")
        self._check(lib().etx_set_gnn_params(self._h, _ptr(theta), _stream(stream)))

    def set_embed_params(self, theta, stream=None):
        """etx_set_embed_params: the embedding parameters from a device float32
        vector (blob order), repacked on the device."""
        _need(theta, torch.float32, "theta", self.device)
        if theta.numel() != self.embed_param_count:
            raise ValueError("theta must hold embed_param_count values")
        self._check(lib().etx_set_embed_params(self._h, _ptr(theta), _stream(stream)))

    def gnn_checkpoints(self, k: int, n_hits: int, n_edges: int, stream=None):
        """etx_gnn_checkpoints: (h^k [n_hits][H], e^k [n_edges][H]) that the last
        training forward kept."""
        H = int(self.model.hidden)
        h = torch.empty((n_hits, H), dtype=torch.float32, device=self.device)
        e = torch.empty((max(n_edges, 1), H), dtype=torch.float32, device=self.device)
        self._check(lib().etx_gnn_checkpoints(self._h, int(k), _ptr(h), _ptr(e), _stream(stream)))
        return h, e[:n_edges]

    def set_fp8_scales(self, scales=None):
        """Static e4m3 activation scales (powers of two, 4 L + 3 of them in the
        order of include/etx.h); None restores all 1."""
        if scales is None:
            self._check(lib().etx_set_fp8_scales(self._h, None, 0))
            return
        a = np.ascontiguousarray(scales, dtype=np.float32)
        self._check(lib().etx_set_fp8_scales(self._h, a.ctypes.data_as(ctypes.c_void_p), a.size))

    @property
    def launch_count(self) -> int:
        """Kernels launched by this context so far."""
        return int(lib().etx_launch_count(self._h))

    def profile(self, on: bool = True):
        self._check(lib().etx_profile_enable(self._h, int(bool(on))))

    def profile_read(self, max_entries: int = 64) -> dict:
        """{kernel name: (total ms, launches)} since the last read."""
        names = (ctypes.c_char_p * max_entries)()
        ms = (ctypes.c_double * max_entries)()
        cnt = (ctypes.c_int64 * max_entries)()
        n = lib().etx_profile_read(self._h, names, ms, cnt, max_entries)
        if n < 0:
            raise EtxError(ETX_ERR_CUDA, "etx_profile_read failed")
        return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}

    def sync(self, stream=None):
        self._check(lib().etx_ctx_sync(self._h, _stream(stream)))

    def embed(self, x, y, z, out=None, stream=None):
        dev = self.device
        for t, n in ((x, "x"), (y, "y"), (z, "z")):
            _need(t, torch.float32, n, dev)
        n = x.shape[0]
        if out is None:
            out = torch.empty((n, self.emb_dim), dtype=torch.float32, device=dev)
        _need(out, torch.float32, "emb", dev)
        self._check(lib().etx_embed(self._h, _ptr(x), _ptr(y), _ptr(z), n, _ptr(out), _stream(stream)))
        return out

    def build_graph(self, emb, plane, hit_offsets, radius: float, k_max: int,
                    edge_capacity: int | None = None, out=None, stream=None):
        dev = self.device
        _need(emb, torch.float32, "emb", dev)
        _need(plane, torch.int8, "plane", dev)
        _need(hit_offsets, torch.int32, "hit_offsets", dev)
        n_hits = emb.shape[0]
        n_events = hit_offsets.shape[0] - 1
        if edge_capacity is None:
            edge_capacity = max(1, n_hits * int(k_max))
        if out is None:
            src = torch.empty(edge_capacity, dtype=torch.int32, device=dev)
            dst = torch.empty(edge_capacity, dtype=torch.int32, device=dev)
            eoff = torch.empty(n_events + 1, dtype=torch.int32, device=dev)
        else:
            src, dst, eoff = out
        self._check(lib().etx_build_graph(self._h, _ptr(emb), _ptr(plane), _ptr(hit_offsets),
                                          n_events, n_hits, float(radius), int(k_max), _ptr(src),
                                          _ptr(dst), int(src.shape[0]), _ptr(eoff), _stream(stream)))
        return src, dst, eoff

    def gnn_forward(self, x, y, z, src, dst, edge_offsets, dtype: str = "f32", logits=None,
                    stream=None):
        dev = self.device
        for t, n in ((x, "x"), (y, "y"), (z, "z")):
            _need(t, torch.float32, n, dev)
        _need(src, torch.int32, "src", dev)
        _need(dst, torch.int32, "dst", dev)
        _need(edge_offsets, torch.int32, "edge_offsets", dev)
        if logits is None:
            logits = torch.empty(src.shape[0], dtype=torch.float32, device=dev)
        _need(logits, torch.float32, "logits", dev)
        n_events = edge_offsets.shape[0] - 1
        self._check(lib().etx_gnn_forward(self._h, _ptr(x), _ptr(y), _ptr(z), x.shape[0], _ptr(src),
                                          _ptr(dst), _ptr(edge_offsets), n_events, DTYPES[dtype],
                                          _ptr(logits), _stream(stream)))
        return logits

    def edges_to_tracks_sweep(self, src, dst, logits, threshold_logit: float, edge_offsets,
                              plane, hit_offsets, labels=None, stream=None):
        """The paper's plane-sweep labels (Sec. 7.3; not exact components)."""
        dev = self.device
        _need(src, torch.int32, "src", dev)
        _need(dst, torch.int32, "dst", dev)
        _need(logits, torch.float32, "logits", dev)
        _need(edge_offsets, torch.int32, "edge_offsets", dev)
        _need(plane, torch.int8, "plane", dev)
        _need(hit_offsets, torch.int32, "hit_offsets", dev)
        n_hits, n_events = plane.shape[0], hit_offsets.shape[0] - 1
        if labels is None:
            labels = torch.empty(n_hits, dtype=torch.int32, device=dev)
        _need(labels, torch.int32, "labels", dev)
        self._check(lib().etx_edges_to_tracks_sweep(self._h, _ptr(src), _ptr(dst), _ptr(logits),
                                                    float(threshold_logit), _ptr(edge_offsets),
                                                    _ptr(plane), _ptr(hit_offsets), n_events,
                                                    n_hits, _ptr(labels), _stream(stream)))
        return labels

    # ---- triplets (Sec. 5.3) -----------------------------------------------
    def load_triplet_weights(self, blob: np.ndarray):
        b = np.ascontiguousarray(blob, dtype=np.float32)
        self._check(lib().etx_load_triplet_weights(self._h, b.ctypes.data_as(ctypes.c_void_p), b.size))

    @staticmethod
    def triplets_workspace(n_hits: int) -> int:
        return int(lib().etx_triplets_workspace(int(n_hits)))

    def build_triplets(self, src, dst, logits, threshold_logit: float, edge_offsets, n_hits: int,
                       capacity: int, workspace=None, out=None, stream=None):
        """Returns (first, second, kind, counts) device tensors; counts =
        {total, articulations, left elbows, right elbows}."""
        dev = self.device
        _need(src, torch.int32, "src", dev)
        _need(dst, torch.int32, "dst", dev)
        _need(logits, torch.float32, "logits", dev)
        _need(edge_offsets, torch.int32, "edge_offsets", dev)
        n_events = edge_offsets.shape[0] - 1
        if workspace is None:
            need = lib().etx_triplets_workspace(int(n_hits))
            workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
        _need(workspace, torch.uint8, "workspace", dev)
        if out is None:
            cap = max(int(capacity), 1)
            out = (torch.empty(cap, dtype=torch.int32, device=dev),
                   torch.empty(cap, dtype=torch.int32, device=dev),
                   torch.empty(cap, dtype=torch.int8, device=dev),
                   torch.empty(4, dtype=torch.int32, device=dev))
        first, second, kind, counts = out
        self._check(lib().etx_build_triplets(self._h, _ptr(src), _ptr(dst), _ptr(logits),
                                             float(threshold_logit), _ptr(edge_offsets), n_events,
                                             int(n_hits), _ptr(workspace), workspace.numel(),
                                             _ptr(first), _ptr(second), _ptr(kind), int(capacity),
                                             _ptr(counts), _stream(stream)))
        return first, second, kind, counts

    def classify_triplets(self, first, second, counts, logits=None, stream=None):
        dev = self.device
        _need(first, torch.int32, "first", dev)
        _need(second, torch.int32, "second", dev)
        _need(counts, torch.int32, "counts", dev)
        if logits is None:
            logits = torch.empty(first.shape[0], dtype=torch.float32, device=dev)
        _need(logits, torch.float32, "logits", dev)
        self._check(lib().etx_classify_triplets(self._h, _ptr(first), _ptr(second), _ptr(counts),
                                                first.shape[0], _ptr(logits), _stream(stream)))
        return logits

    def tracks_workspace(self, n_hits: int, triplet_capacity: int) -> int:
        return int(lib().etx_tracks_workspace(int(n_hits), int(self.cfg.max_edges),
                                              int(triplet_capacity)))

    def tracks_from_triplets(self, src, dst, logits, threshold_logit: float, edge_offsets,
                             n_hits: int, first, second, triplet_logits, triplet_threshold: float,
                             counts, min_hits: int = 3, track_capacity: int | None = None,
                             hit_capacity: int | None = None, workspace=None, out=None,
                             stream=None):
        """etx_tracks_from_triplets (Sec. 5.4): tracks that may share hits, as a
        CSR (track_offsets, track_hits) plus n_out = [tracks, hits] on the
        device.  ``first``/``second``/``counts`` come from build_triplets,
        ``triplet_logits`` from classify_triplets."""
        dev = self.device
        for t, n in ((src, "src"), (dst, "dst"), (edge_offsets, "edge_offsets"), (first, "first"),
                     (second, "second"), (counts, "counts")):
            _need(t, torch.int32, n, dev)
        _need(logits, torch.float32, "logits", dev)
        _need(triplet_logits, torch.float32, "triplet_logits", dev)
        cap = first.shape[0]
        if track_capacity is None:
            track_capacity = int(self.cfg.max_edges) + cap
        if hit_capacity is None:
            hit_capacity = 2 * (int(self.cfg.max_edges) + cap)
        if workspace is None:
            workspace = torch.empty(max(self.tracks_workspace(n_hits, cap), 4), dtype=torch.uint8,
                                    device=dev)
        if out is None:
            out = (torch.empty(track_capacity + 1, dtype=torch.int32, device=dev),
                   torch.empty(max(hit_capacity, 1), dtype=torch.int32, device=dev),
                   torch.empty(2, dtype=torch.int32, device=dev))
        offs, hits, n_out = out
        self._check(lib().etx_tracks_from_triplets(
            self._h, _ptr(src), _ptr(dst), _ptr(logits), float(threshold_logit), _ptr(edge_offsets),
            edge_offsets.shape[0] - 1, int(n_hits), _ptr(first), _ptr(second), _ptr(triplet_logits),
            float(triplet_threshold), _ptr(counts), cap, int(min_hits), _ptr(workspace),
            workspace.numel(), _ptr(offs), _ptr(hits), int(track_capacity), int(hit_capacity),
            _ptr(n_out), _stream(stream)))
        return offs, hits, n_out

    # ---- embedding training (Sec. 5.1, Eq. 2-3) ----------------------------
    @property
    def embed_param_count(self) -> int:
        return int(lib().etx_embed_param_count(ctypes.byref(self.cfg)))

    def embed_train_workspace(self, n_hits: int):
        """Device scratch for embed_forward_train / embed_backward."""
        n = int(lib().etx_embed_train_workspace(ctypes.byref(self.cfg), int(n_hits)))
        return torch.empty(max(n, 16), dtype=torch.uint8, device=self.device)

    def embed_forward_train(self, x, y, z, workspace, emb=None, stream=None):
        dev = self.device
        for t, n in ((x, "x"), (y, "y"), (z, "z")):
            _need(t, torch.float32, n, dev)
        _need(workspace, torch.uint8, "workspace", dev)
        n_hits = x.shape[0]
        D = int(self.cfg.emb_widths[self.cfg.emb_depth])
        if emb is None:
            emb = torch.empty(n_hits, D, dtype=torch.float32, device=dev)
        _need(emb, torch.float32, "emb", dev)
        self._check(lib().etx_embed_forward_train(self._h, _ptr(x), _ptr(y), _ptr(z), n_hits,
                                                  _ptr(emb), _ptr(workspace), workspace.numel(),
                                                  _stream(stream)))
        return emb

    def embed_backward(self, d_emb, workspace, d_params=None, stream=None):
        dev = self.device
        _need(d_emb, torch.float32, "d_emb", dev)
        _need(workspace, torch.uint8, "workspace", dev)
        if d_params is None:
            d_params = torch.empty(self.embed_param_count, dtype=torch.float32, device=dev)
        _need(d_params, torch.float32, "d_params", dev)
        self._check(lib().etx_embed_backward(self._h, d_emb.shape[0], _ptr(d_emb), _ptr(d_params),
                                             _ptr(workspace), workspace.numel(), _stream(stream)))
        return d_params

    def embedding_pairs(self, emb, plane, particle_id, hit_offsets, radius: float, k_max: int,
                        rand, capacity: int, min_hits: int = 3, workspace=None, out=None,
                        stream=None):
        """Training set of Sec. 5.1; returns (pair_q, pair_a, pair_genuine, n_pairs) device
        tensors (the first n_pairs entries are valid)."""
        dev = self.device
        _need(emb, torch.float32, "emb", dev)
        _need(plane, torch.int8, "plane", dev)
        _need(particle_id, torch.int32, "particle_id", dev)
        _need(hit_offsets, torch.int32, "hit_offsets", dev)
        _need(rand, torch.int32, "rand (uint32 bits in an int32 tensor)", dev)
        n_hits, n_events = plane.shape[0], hit_offsets.shape[0] - 1
        if workspace is None:
            need = lib().etx_embedding_pairs_workspace(n_events, n_hits, int(k_max))
            workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
        _need(workspace, torch.uint8, "workspace", dev)
        if out is None:
            cap = max(int(capacity), 1)
            out = (torch.empty(cap, dtype=torch.int32, device=dev),
                   torch.empty(cap, dtype=torch.int32, device=dev),
                   torch.empty(cap, dtype=torch.uint8, device=dev),
                   torch.empty(1, dtype=torch.int32, device=dev))
        pq, pa, pg, npairs = out
        self._check(lib().etx_embedding_pairs(self._h, _ptr(emb), _ptr(plane), _ptr(particle_id),
                                              _ptr(hit_offsets), n_events, n_hits, float(radius),
                                              int(k_max), _ptr(rand), int(min_hits),
                                              _ptr(workspace), workspace.numel(), _ptr(pq),
                                              _ptr(pa), _ptr(pg), int(capacity), _ptr(npairs),
                                              _stream(stream)))
        return pq, pa, pg, npairs

    @staticmethod
    def hinge_loss_workspace(n_hits: int, pair_capacity: int) -> int:
        """Bytes of device scratch that hinge_loss needs."""
        return int(lib().etx_hinge_loss_workspace(int(n_hits), int(pair_capacity)))

    def hinge_loss(self, emb, pair_q, pair_a, pair_genuine, n_pairs, margin: float = 1.0,
                   w_genuine: float = 2.0, loss=None, d_emb=None, workspace=None, stream=None):
        """Eq. 2-3; returns (loss float32[3] = {L, L_genuine, L_fake}, d_emb) on the device."""
        dev = self.device
        _need(emb, torch.float32, "emb", dev)
        _need(pair_q, torch.int32, "pair_q", dev)
        _need(pair_a, torch.int32, "pair_a", dev)
        _need(pair_genuine, torch.uint8, "pair_genuine", dev)
        _need(n_pairs, torch.int32, "n_pairs", dev)
        if loss is None:
            loss = torch.empty(3, dtype=torch.float32, device=dev)
        if d_emb is None:
            d_emb = torch.empty_like(emb)
        _need(d_emb, torch.float32, "d_emb", dev)
        if workspace is None:
            need = self.hinge_loss_workspace(emb.shape[0], pair_q.shape[0])
            workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
        _need(workspace, torch.uint8, "workspace", dev)
        self._check(lib().etx_hinge_loss(self._h, _ptr(emb), emb.shape[0], _ptr(pair_q),
                                         _ptr(pair_a), _ptr(pair_genuine), _ptr(n_pairs),
                                         pair_q.shape[0], float(margin), float(w_genuine),
                                         _ptr(loss), _ptr(d_emb), _ptr(workspace),
                                         workspace.numel(), _stream(stream)))
        return loss, d_emb

    @staticmethod
    def track_metrics_workspace(n_events: int, n_hits: int) -> int:
        """Bytes of device scratch that track_metrics needs."""
        return int(lib().etx_track_metrics_workspace(int(n_events), int(n_hits)))

    def track_metrics(self, labels, particle_id, hit_offsets, min_hits: int = 3,
                      match=(7, 10), workspace=None, stream=None):
        """Table 1 counts and ratios (Sec. 6) computed on the device; returns
        (counts int64[6], values float64[7]) device tensors ordered as
        TRACK_COUNTS and TRACK_VALUES."""
        dev = self.device
        _need(labels, torch.int32, "labels", dev)
        _need(particle_id, torch.int32, "particle_id", dev)
        _need(hit_offsets, torch.int32, "hit_offsets", dev)
        n_hits, n_events = labels.shape[0], hit_offsets.shape[0] - 1
        if particle_id.shape[0] != n_hits:
            raise ValueError("labels and particle_id differ in length")
        need = lib().etx_track_metrics_workspace(n_events, n_hits)
        if workspace is None:
            workspace = torch.empty(max(need, 8), dtype=torch.uint8, device=dev)
        _need(workspace, torch.uint8, "workspace", dev)
        counts = torch.empty(6, dtype=torch.int64, device=dev)
        values = torch.empty(7, dtype=torch.float64, device=dev)
        self._check(lib().etx_track_metrics(self._h, _ptr(labels), _ptr(particle_id),
                                            _ptr(hit_offsets), n_events, n_hits, int(min_hits),
                                            int(match[0]), int(match[1]), _ptr(workspace),
                                            workspace.numel(), _ptr(counts), _ptr(values),
                                            _stream(stream)))
        return counts, values

    def autotune(self, x, y, z, plane, hit_offsets, radius: float, k_max: int, emb, src, dst,
                 edge_offsets, logits, dtype: str = "bf16", stream=None):
        """Time the candidate launch configurations on this batch and keep the
        fastest (see etx_autotune); returns {knob: value}.  The output tensors
        receive the results of the chosen configuration."""
        dev = self.device
        for t, n in ((x, "x"), (y, "y"), (z, "z"), (emb, "emb"), (logits, "logits")):
            _need(t, torch.float32, n, dev)
        _need(plane, torch.int8, "plane", dev)
        for t, n in ((hit_offsets, "hit_offsets"), (src, "src"), (dst, "dst"),
                     (edge_offsets, "edge_offsets")):
            _need(t, torch.int32, n, dev)
        n_hits, n_events = x.shape[0], hit_offsets.shape[0] - 1
        self._check(lib().etx_autotune(self._h, _ptr(x), _ptr(y), _ptr(z), _ptr(plane),
                                       _ptr(hit_offsets), n_events, n_hits, float(radius),
                                       int(k_max), DTYPES[dtype], _ptr(emb), _ptr(src), _ptr(dst),
                                       int(src.shape[0]), _ptr(edge_offsets), _ptr(logits),
                                       _stream(stream)))
        return self.tuned()

    def tuned(self) -> dict:
        """Current launch configuration chosen by the autotuner, by knob name."""
        return {k: int(lib().etx_tuned(self._h, k.encode())) for k in TUNE_KNOBS}

    def set_tuned(self, **knobs):
        """Set launch-configuration knobs (names as in ``tuned()``, with '/'
        written as '__'), e.g. ``set_tuned(knn_split=2)``."""
        for k, v in knobs.items():
            self._check(lib().etx_set_tuned(self._h, k.replace("__", "/").encode(), int(v)))

    @property
    def gnn_param_count(self) -> int:
        return int(lib().etx_gnn_param_count(ctypes.byref(self.cfg)))

    def gnn_backward(self, dlogits, dparams=None, stream=None):
        """Gradient of sum(dlogits * logits) w.r.t. the interaction-network
        parameters (blob order from the node encoder on) for the last training
        forward of this context."""
        _need(dlogits, torch.float32, "dlogits", self.device)
        if dparams is None:
            dparams = torch.empty(self.gnn_param_count, dtype=torch.float32, device=self.device)
        _need(dparams, torch.float32, "dparams", self.device)
        self._check(lib().etx_gnn_backward(self._h, _ptr(dlogits), _ptr(dparams), _stream(stream)))
        return dparams

    def weighted_bce(self, logits, targets, edge_offsets, pos_weight: float = 10.0, stream=None):
        """(loss [1], dlogits [len(logits)]) of the class-weighted BCE."""
        dev = self.device
        _need(logits, torch.float32, "logits", dev)
        _need(targets, torch.float32, "targets", dev)
        _need(edge_offsets, torch.int32, "edge_offsets", dev)
        loss = torch.empty(1, dtype=torch.float32, device=dev)
        dlogits = torch.zeros_like(logits)
        self._check(lib().etx_weighted_bce(self._h, _ptr(logits), _ptr(targets), _ptr(edge_offsets),
                                           edge_offsets.shape[0] - 1, float(pos_weight), _ptr(loss),
                                           _ptr(dlogits), _stream(stream)))
        return loss, dlogits

    def focal_loss(self, logits, targets, edge_offsets, alpha: float = 0.25, gamma: float = 2.0,
                   stream=None):
        """(loss [1], dlogits [len(logits)]) of the sigmoid focal loss (Eq. 5)."""
        dev = self.device
        _need(logits, torch.float32, "logits", dev)
        _need(targets, torch.float32, "targets", dev)
        _need(edge_offsets, torch.int32, "edge_offsets", dev)
        loss = torch.empty(1, dtype=torch.float32, device=dev)
        dlogits = torch.zeros_like(logits)
        self._check(lib().etx_focal_loss(self._h, _ptr(logits), _ptr(targets), _ptr(edge_offsets),
                                         edge_offsets.shape[0] - 1, float(alpha), float(gamma),
                                         _ptr(loss), _ptr(dlogits), _stream(stream)))
        return loss, dlogits

    def adam_step(self, params, grads, m, v, step: int, lr: float = 1e-3, beta1: float = 0.9,
                  beta2: float = 0.999, eps: float = 1e-8, stream=None):
        for t, n in ((params, "params"), (grads, "grads"), (m, "m"), (v, "v")):
            _need(t, torch.float32, n, self.device)
        self._check(lib().etx_adam_step(self._h, _ptr(params), _ptr(grads), _ptr(m), _ptr(v),
                                        params.numel(), float(lr), float(beta1), float(beta2),
                                        float(eps), int(step), _stream(stream)))

    def edges_to_tracks(self, src, dst, logits, threshold_logit: float, edge_offsets, hit_offsets,
                        min_hits: int = 3, labels=None, n_tracks=None, stream=None):
        dev = self.device
        _need(src, torch.int32, "src", dev)
        _need(dst, torch.int32, "dst", dev)
        _need(logits, torch.float32, "logits", dev)
        _need(edge_offsets, torch.int32, "edge_offsets", dev)
        _need(hit_offsets, torch.int32, "hit_offsets", dev)
        n_events = hit_offsets.shape[0] - 1
        n_hits = None
        if labels is None:
            n_hits = int(hit_offsets[-1].item())
            labels = torch.empty(n_hits, dtype=torch.int32, device=dev)
        n_hits = labels.shape[0]
        if n_tracks is None:
            n_tracks = torch.empty(max(n_events, 1), dtype=torch.int32, device=dev)
        self._check(lib().etx_edges_to_tracks(self._h, _ptr(src), _ptr(dst), _ptr(logits),
                                              float(threshold_logit), _ptr(edge_offsets),
                                              _ptr(hit_offsets), n_events, n_hits, int(min_hits),
                                              _ptr(labels), _ptr(n_tracks), _stream(stream)))
        return labels, n_tracks
