"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point include/etx.h declares; pure host functions agree
with the blob format; context creation fails cleanly without a device."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

from velo_synth import WORKLOADS, ModelConfig, blob_size

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def etx():
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import etx as m
    return m


def declared_entry_points():
    text = (ROOT / "include" / "etx.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(etx_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_pipeline():
    names = declared_entry_points()
    for n in ("etx_embed", "etx_build_graph", "etx_gnn_forward", "etx_gnn_backward",
              "etx_edges_to_tracks"):
        assert n in names


def test_library_exports_every_declared_symbol(etx):
    lib = ctypes.CDLL(str(etx.library_path()))
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    assert sorted(etx.EXPORTED) == declared_entry_points()


@pytest.mark.parametrize("name", ["plain", "batch500", "train64", "pileup4x"])
def test_weights_size_matches_blob_format(etx, name):
    model = WORKLOADS[name].model
    assert etx.weights_size(model) == blob_size(model)


def test_weights_size_rejects_bad_configs(etx):
    L = etx.lib()
    for bad in [ModelConfig(hidden=48), ModelConfig(emb_widths=(2, 32, 4)),
                ModelConfig(emb_widths=(3, 32, 64, 4)), ModelConfig(emb_widths=(3, 4))]:
        c = etx.make_config(bad, 1, 1, 1)
        assert L.etx_weights_size(ctypes.byref(c)) == -1


def test_ctx_create_without_device_fails_cleanly(etx):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(etx.EtxError):
        etx.Context(WORKLOADS["plain"].model, 1, 100, 100)


def test_null_handles(etx):
    L = etx.lib()
    assert L.etx_ctx_destroy(None) == 0
    assert L.etx_embed(None, None, None, None, 0, None, None) == etx.ETX_ERR_ARG
    assert L.etx_launch_count(None) == -1
    assert L.etx_last_error(None) == b"no context"


def test_workspace_sizes_are_host_functions(etx):
    """The workspace-size calls run on the host: they grow with their sizes,
    cover at least the arrays the call keeps there, and refuse negative sizes."""
    L = etx.lib()
    w = lambda n, cap: int(L.etx_hinge_loss_workspace(n, cap))
    # per pair: a coefficient and the pair's id in two key indices (3 x 4 bytes);
    # per hit: a count and two offset arrays of n + 1 entries (3 x 4 bytes)
    for n, cap in [(0, 0), (1, 1), (1000, 52000), (100000, 5200000)]:
        assert w(n, cap) >= 12 * cap + 12 * (n + 1)
        assert w(n, cap) % 16 == 0
    assert w(1000, 52000) <= w(1001, 52000) <= w(1001, 52001) < w(1101, 53000)
    assert w(-1, 10) == 0 and w(10, -1) == 0
    t = lambda b, n: int(L.etx_track_metrics_workspace(b, n))
    assert t(10, 1000) <= t(10, 2000) and t(-1, 5) == 0
