"""Pins of the oracle's mixed-precision readings (the BF16 and e4m3 forms of
``gnn_forward``): WHICH operands are rounded.

The reading (design notes r12, r13): the activation and weight operands of
every matrix product with a hidden-width input are rounded -- the edge
encoder's two products, both products of every node and edge network, the
classifier's first product -- while the node encoder (3 inputs), biases,
LayerNorm, residual adds, message sums and the classifier's last dot product
stay exact.

Each case is a hand-built network with H = 2 and one message-passing step on
a two-hit, one-edge event, in which exactly one site carries a value that
the format cannot hold: v = 1 + 2^-9 for BF16 (8 significand bits: v rounds
to 1) or v = 1 + 2^-5 for e4m3 (4 bits), and the bias beside it is
-(1 + t) with t = v - 1 halved (2^-10, 2^-6).  In exact arithmetic that
layer's first pre-activation is +t, rounded it is -t.  With H = 2, LayerNorm
and ReLU turn the sign of (a_0 - a_1) into the one-hot pattern [c, 0] or
[0, c] (c = 0.15 to 0.9998 here), and the layers after it carry that pattern
to the logit's sign with margins far above any other rounding; every other
site holds exactly representable values (0, 1, 2, one-hot patterns) or
multiplies inexact values by zero.  So the logit's sign flips between the
exact and the rounded reading iff the reading rounds that site.  Biases of
-(1 + t) are themselves not representable in either format: were biases
rounded, the "kept exact" cases would flip too.
"""
import numpy as np
import pytest

from oracle import etx_oracle as O

H = 2
FMT = {"bf16": (1.0 + 2.0 ** -9, 2.0 ** -10), "fp8": (1.0 + 2.0 ** -5, 2.0 ** -6)}


def _block(k_in, W1=None, b1=None, g1=1.0, be1=None, W2=None, b2=None, g2=1.0, be2=None):
    z = lambda *s: np.zeros(s)
    return {"W1": z(H, k_in) if W1 is None else np.asarray(W1, float),
            "b1": z(H) if b1 is None else np.asarray(b1, float),
            "g1": np.full(H, g1), "be1": z(H) if be1 is None else np.asarray(be1, float),
            "W2": z(H, H) if W2 is None else np.asarray(W2, float),
            "b2": z(H) if b2 is None else np.asarray(b2, float),
            "g2": np.full(H, g2), "be2": z(H) if be2 is None else np.asarray(be2, float)}


def emitter(k_in, const):
    """Output relu(const) for every row, whatever the input (LayerNorm gains 0)."""
    return _block(k_in, g1=0.0, g2=0.0, be2=const)


PASS2 = [[1.0, -1.0], [-1.0, 1.0]]   # second layer: keep the one-hot pattern, c -> ~1


def signpass(k_in, p, q):
    """[~1, 0] if X[p] > X[q], else [0, ~1]."""
    W1 = np.zeros((H, k_in))
    W1[0, p], W1[0, q], W1[1, p], W1[1, q] = 1.0, -1.0, -1.0, 1.0
    return _block(k_in, W1=W1, W2=PASS2)


def threshold(k_in, p, thr, w=1.0, spare=None):
    """[~1, 0] if w * X[p] > thr, else [0, ~1].  ``spare`` = (row, col) of an
    extra weight 2 on an input that is zero (it sets the e4m3 weight scale)."""
    W1 = np.zeros((H, k_in))
    W1[0, p] = w
    if spare is not None:
        W1[spare] = 2.0
    return _block(k_in, W1=W1, b1=[-thr, 0.0], W2=PASS2)


def mid_detector(k_in, v, t):
    """Second product's operand = [v, 0] (first layer's gains 0, shift v);
    pre-activation v - 1 - t."""
    return _block(k_in, g1=0.0, be1=[v, 0.0], W2=[[1.0, 0.0], [0.0, 0.0]], b2=[-1.0 - t, 0.0])


def cls_sign():
    return {"W1": np.array(PASS2), "b1": np.zeros(H), "g1": np.ones(H), "be1": np.zeros(H),
            "W2": np.array([[1.0, -1.0]]), "b2": np.zeros(1)}


def cls_threshold(p, thr):
    W1 = np.zeros((H, H))
    W1[0, p] = 1.0
    return {"W1": W1, "b1": np.array([-thr, 0.0]), "g1": np.ones(H), "be1": np.zeros(H),
            "W2": np.array([[1.0, -1.0]]), "b2": np.zeros(1)}


def zero(k_in):
    return emitter(k_in, [0.0, 0.0])


def build(site, v, t):
    """(weights, x of the two hits) for the detector of ``site``."""
    x = np.ones(2)
    node_enc, edge_enc = emitter(3, [0.0, 0.0]), emitter(2 * H, [0.0, 0.0])
    node0, edge0, cls = zero(3 * H), zero(3 * H), cls_sign()
    if site == "edge_enc.in":        # [h_i, h_j] = [v, 0, v, 0]
        node_enc = emitter(3, [v, 0.0])
        edge_enc = threshold(2 * H, 0, 1.0 + t)
    elif site == "edge_enc.mid":
        edge_enc = mid_detector(2 * H, v, t)
    elif site == "edge_enc.W1":      # weight v on the input h_i[0] = 1
        node_enc = emitter(3, [1.0, 0.0])
        edge_enc = threshold(2 * H, 0, 1.0 + t, w=v, spare=(1, 3))
    elif site == "node0.in":         # [h, m_out, m_in] with h = [v, 0]
        node_enc = emitter(3, [v, 0.0])
        node0 = threshold(3 * H, 0, 1.0 + t)
        edge0 = threshold(3 * H, 3, 0.5)        # h_i[1]: 0 exact, ~1 if flipped
    elif site == "node0.mid":
        node0 = mid_detector(3 * H, v, t)
        edge0 = signpass(3 * H, 2, 3)           # h_i[0] vs h_i[1]
    elif site == "edge0.in":         # [e, h_i, h_j] with e = [v, 0]
        edge_enc = emitter(2 * H, [v, 0.0])
        edge0 = threshold(3 * H, 0, 1.0 + t)
        cls = cls_threshold(1, 0.5)             # e[1]: 0 exact, ~1 if flipped
    elif site == "edge0.mid":
        edge0 = mid_detector(3 * H, v, t)
    elif site == "edge0.W1":         # weight v on the input e[0] = 1
        edge_enc = emitter(2 * H, [1.0, 0.0])
        edge0 = threshold(3 * H, 0, 1.0 + t, w=v, spare=(1, 5))
        cls = cls_threshold(1, 0.5)
    elif site == "cls.in":           # e = [v, 0]
        edge_enc = emitter(2 * H, [v, 0.0])
        cls = cls_threshold(0, 1.0 + t)
    elif site == "node_enc.in":      # normalised x = v
        x = np.full(2, v)
        node_enc = threshold(3, 0, 1.0 + t)
        edge_enc = signpass(2 * H, 0, 1)
    elif site == "node_enc.mid":
        node_enc = mid_detector(3, v, t)
        edge_enc = signpass(2 * H, 0, 1)
    elif site == "node_enc.W1":      # weight v on x = 1
        node_enc = threshold(3, 0, 1.0 + t, w=v, spare=(1, 2))
        edge_enc = signpass(2 * H, 0, 1)
    elif site == "cls.W2":           # the last dot product: r = [1, 0], w = [v, 2]
        edge_enc = emitter(2 * H, [1.0, 0.0])
        cls = {"W1": np.zeros((H, H)), "b1": np.zeros(H), "g1": np.zeros(H),
               "be1": np.array([1.0, 0.0]), "W2": np.array([[v, 2.0]]),
               "b2": np.array([-1.0 - t])}
    else:
        raise ValueError(site)
    W = {"gnn_mu": np.zeros(3), "gnn_sigma": np.ones(3)}
    for prefix, blk in (("node_enc", node_enc), ("edge_enc", edge_enc), ("node0", node0),
                        ("edge0", edge0), ("cls", cls)):
        for k, a in blk.items():
            W[f"{prefix}.{k}"] = np.asarray(a, np.float32)
    return W, x


ROUNDED = ["edge_enc.in", "edge_enc.mid", "edge_enc.W1", "node0.in", "node0.mid", "edge0.in",
           "edge0.mid", "edge0.W1", "cls.in"]
EXACT = ["node_enc.in", "node_enc.mid", "node_enc.W1", "cls.W2"]


def _logits(W, x, gemm, act_scales=None):
    z = np.zeros(2)
    kw = {"act_scales": act_scales} if act_scales is not None else {}
    return O.gnn_forward(W, 1, x, z, z, np.array([0]), np.array([1]), gemm=gemm, **kw)[0]


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
@pytest.mark.parametrize("site", ROUNDED + EXACT)
def test_reading_rounds_exactly_the_hidden_width_products(fmt, site):
    v, t = FMT[fmt]
    # the chosen values really are outside / inside the format
    rnd = O.round_bf16 if fmt == "bf16" else O.round_e4m3
    assert rnd(v) == 1.0 and rnd(1.0) == 1.0 and rnd(2.0) == 2.0
    W, x = build(site, v, t)
    z64, zr = _logits(W, x, "fp64"), _logits(W, x, fmt)
    # a clear sign either way (the last dot product has no LayerNorm after it: +-t there)
    margin = t / 2 if site == "cls.W2" else 0.1
    assert abs(z64) > margin and abs(zr) > margin
    flipped = np.sign(z64) != np.sign(zr)
    assert flipped == (site in ROUNDED), (site, z64, zr)


@pytest.mark.parametrize("site", ROUNDED)
def test_power_of_two_activation_scales_keep_the_rounding(site):
    """A power-of-two activation scale moves e4m3's range but not its relative
    spacing: with every scale 2^-3 the same sites flip (and only they)."""
    v, t = FMT["fp8"]
    W, x = build(site, v, t)
    sc = [2.0 ** -3] * O.n_act_scales(1)
    z64, z8 = _logits(W, x, "fp64"), _logits(W, x, "fp8", sc)
    assert np.sign(z64) != np.sign(z8)


def test_activation_scale_values_and_saturation():
    """quant_act_e4m3 and fp8_act_scale by hand: 600 saturates to 448 at scale
    1 and is 576 at scale 2 (300 lies between e4m3 neighbours 288 and 320);
    0.001 is subnormal at scale 1 (spacing 2^-9: 2^-9) and normal at scale
    2^-6 (0.064 -> 0.0625, times 2^-6)."""
    assert O.quant_act_e4m3(np.array([600.0]), 1.0)[0] == 448.0
    assert O.quant_act_e4m3(np.array([600.0]), 2.0)[0] == 576.0
    assert O.quant_act_e4m3(np.array([0.001]), 1.0)[0] == 2.0 ** -9
    assert O.quant_act_e4m3(np.array([0.001]), 2.0 ** -6)[0] == 0.0625 * 2.0 ** -6
    assert O.fp8_act_scale(448.0) == 1.0 and O.fp8_act_scale(448.5) == 2.0
    assert O.fp8_act_scale(3.5) == 2.0 ** -7 and O.fp8_act_scale(3.51) == 2.0 ** -6
    assert O.fp8_act_scale(0.0) == 1.0
    with pytest.raises(ValueError):
        O.quant_act_e4m3(np.array([1.0]), 3.0)


def test_stored_edge_stream_rounds_where_it_is_written():
    """edge_store="bf16": the residual edge stream is rounded where it is
    written.  e0 = [v, 0] from the edge encoder (v = 1 + 2^-9), the edge
    network adds w = 1 + 2^-7 - 2^-10 (a constant emitter): exact e1 = 2 +
    2^-7 + 2^-10, which BF16 (spacing 2^-6 in [2, 4)) rounds up to 2 + 2^-6;
    stored, e0 is already 1 and 1 + w = 2 + 2^-7 - 2^-10 rounds down to 2.
    The classifier's threshold at 2 + 2^-7 sees the difference, which the
    plain BF16 reading (only operands rounded) does not have."""
    v, t = FMT["bf16"]
    w = 1.0 + 2.0 ** -7 - 2.0 ** -10
    W, x = build("cls.in", v, t)            # edge encoder emits [v, 0]
    for k, a in emitter(3 * H, [w, 0.0]).items():
        W[f"edge0.{k}"] = np.asarray(a, np.float32)
    for k, a in cls_threshold(0, 2.0 + 2.0 ** -7).items():
        W[f"cls.{k}"] = np.asarray(a, np.float32)
    z = np.zeros(2)
    run = lambda **kw: O.gnn_forward(W, 1, x, z, z, np.array([0]), np.array([1]), **kw)[0]
    z64, z16 = run(), run(gemm="bf16")
    z16s = run(gemm="bf16", edge_store="bf16")
    assert z64 > 0.1 and z16 > 0.1 and z16s < -0.1
    with pytest.raises(ValueError):
        run(gemm="fp8", edge_store="bf16")
