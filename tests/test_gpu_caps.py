"""Failure detection on the device without faulting the GPU: a bounded
union-find loop that reaches its iteration cap records ETX_ERR_TIMEOUT in the
context's error word and returns (no trap, no endless spin); the host reads
the status at etx_ctx_sync and the context stays usable.

The cap is the context's ``uf_iter_cap`` (etx_config).  A chain of hits
joined by kept edges puts every hit but the first below a parent, so with a
cap of one step any find on such a hit runs out: the timeout is certain, not
a race.
"""
import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import WORKLOADS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def etx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import etx as m
    return m


def _chain(n_hits):
    src = np.arange(n_hits - 1, dtype=np.int32)
    dst = src + 1
    hoff = np.array([0, n_hits], np.int32)
    eo = np.array([0, n_hits - 1], np.int32)
    logits = np.ones(n_hits - 1, np.float32)
    return src, dst, hoff, eo, logits


def test_union_find_cap_reports_timeout_and_returns(etx):
    model = WORKLOADS["plain"].model
    n = 4096
    src, dst, hoff, eo, logits = _chain(n)
    t = lambda a: torch.from_numpy(a).cuda()
    args = (t(src), t(dst), t(logits), 0.0, t(eo), t(hoff))
    capped = etx.Context(model, 1, n, n, uf_iter_cap=1)
    capped.edges_to_tracks(*args)
    with pytest.raises(etx.EtxError) as ei:
        capped.sync()
    assert ei.value.status == etx.ETX_ERR_TIMEOUT
    capped.sync()  # the error word was read and cleared: the context is usable again
    # the same context on a graph whose finds end at once (no kept edge) reports nothing
    none_kept = (t(src), t(dst), t(-logits), 0.0, t(eo), t(hoff))
    lab, _ = capped.edges_to_tracks(*none_kept)
    capped.sync()
    np.testing.assert_array_equal(lab.cpu().numpy(), np.arange(n))
    # with the default caps the chain is one component labelled 0
    ref = O.connected_components(src, dst, logits > 0, hoff)
    ctx = etx.Context(model, 1, n, n)
    lab, nt = ctx.edges_to_tracks(*args)
    ctx.sync()
    np.testing.assert_array_equal(lab.cpu().numpy(), ref)
    assert int(nt[0].item()) == 1


def test_negative_cap_is_rejected(etx):
    model = WORKLOADS["plain"].model
    with pytest.raises(etx.EtxError) as ei:
        etx.Context(model, 1, 16, 16, uf_iter_cap=-1)
    assert ei.value.status == etx.ETX_ERR_ARG
