"""Training path on the GPU: weighted BCE, hand-written backward and Adam,
checked against the FP64 oracle (its gradient and central finite
differences) and torch's Adam."""
import numpy as np
import pytest
import torch

from oracle import etx_oracle as O
from velo_synth import (WORKLOADS, ModelConfig, global_particle_ids, make_batch, make_weights,
                        pack_blob, truth_edge_labels, unpack_blob, blob_layout)

pytestmark = pytest.mark.gpu
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def etx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_12119_gb300 import build as b
    b.build()
    from paper_2407_12119_gb300 import etx as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def problem(H, L, n_events, seed=0, perturb=0.3):
    cfg = ModelConfig(emb_widths=(3, 32, 32, 4), hidden=H, n_iters=L, radius=1.5, k_max=16)
    wl = WORKLOADS["plain"]
    b = make_batch(wl.recipe, n_events, 5000 + seed)
    W = make_weights(cfg, wl.calibration(), seed=seed, perturb=perturb)
    emb = O.embed(W, 3, b.x, b.y, b.z)
    s, d, eo = O.build_graph(emb, b.plane, b.hit_offsets, cfg.radius, cfg.k_max)
    y = truth_edge_labels(global_particle_ids(b), b.plane, s, d)
    return cfg, b, W, s, d, eo, y


def gnn_names(cfg):
    names = [n for n, _ in blob_layout(cfg)]
    return names[names.index("node_enc.W1"):]


def gpu_grads(etx, cfg, b, W, s, d, eo, y, dtype="f32"):
    ctx = etx.Context(cfg, b.n_events, b.n_hits, max(s.size, 1), train=True)
    ctx.load_weights(pack_blob(cfg, W))
    x, yy, z = cuda(b.x), cuda(b.y), cuda(b.z)
    st, dt, eot = cuda(s.astype(np.int32)), cuda(d.astype(np.int32)), cuda(eo.astype(np.int32))
    logits = ctx.gnn_forward(x, yy, z, st, dt, eot, dtype=dtype)
    loss, dl = ctx.weighted_bce(logits, cuda(y.astype(np.float32)), eot, 10.0)
    g = ctx.gnn_backward(dl)
    ctx.sync()
    flat = g.cpu().numpy().astype(np.float64)
    out, o = {}, 0
    shapes = dict(blob_layout(cfg))
    for n in gnn_names(cfg):
        k = int(np.prod(shapes[n]))
        out[n] = flat[o:o + k].reshape(shapes[n])
        o += k
    return float(loss.item()), out, logits.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)


@pytest.mark.parametrize("H,L,n_events", [(16, 2, 1), (32, 3, 2), (128, 2, 2)])
def test_backward_matches_oracle_gradient(etx, H, L, n_events):
    cfg, b, W, s, d, eo, y = problem(H, L, n_events)
    cache = {}
    z = O.gnn_forward(W, L, b.x, b.y, b.z, s, d, cache)
    loss_ref, dz = O.weighted_bce(z, y, 10.0)
    ref = O.gnn_backward(W, cache, dz)
    loss, g, _ = gpu_grads(etx, cfg, b, W, s, d, eo, y)
    assert abs(loss - loss_ref) <= 1e-5 * max(1.0, abs(loss_ref))
    worst = max((rel(g[n], ref[n]), n) for n in ref)
    print(f"H={H} L={L}: E={s.size}, worst per-tensor relative L2 {worst[0]:.2e} ({worst[1]})")
    assert worst[0] <= GRAD_RTOL, worst


def test_backward_matches_finite_differences(etx):
    # FP64 central differences (h = 1e-6) of the oracle loss on a 1-event,
    # hidden-16 copy, against the GPU gradient
    cfg, b, W, s, d, eo, y = problem(16, 2, 1, seed=3)
    _, g, _ = gpu_grads(etx, cfg, b, W, s, d, eo, y)
    Wd = {k: np.asarray(v, np.float64) for k, v in W.items()}
    rng = np.random.default_rng(1)
    h = 1e-6
    for name in ["node_enc.W1", "node_enc.b2", "edge_enc.W1", "node0.W1", "node1.g1", "edge0.W2",
                 "edge1.be2", "cls.W1", "cls.W2", "cls.b2"]:
        flat = Wd[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(5, flat.size), replace=False)
        fd = []
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp, _ = O.weighted_bce(O.gnn_forward(Wd, 2, b.x, b.y, b.z, s, d), y)
            flat[i] = old - h
            lm, _ = O.weighted_bce(O.gnn_forward(Wd, 2, b.x, b.y, b.z, s, d), y)
            flat[i] = old
            fd.append((lp - lm) / (2 * h))
        fd = np.array(fd)
        got = g[name].reshape(-1)[idx]
        assert rel(got, fd) <= GRAD_RTOL or np.abs(got - fd).max() <= 1e-7, (name, got, fd)


def test_adam_matches_torch(etx):
    cfg = WORKLOADS["plain"].model
    ctx = etx.Context(cfg, 1, 16, 16)
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=1000).astype(np.float32)
    p = cuda(p0.copy())
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    ref = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([ref], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 4):
        gr = rng.normal(size=1000).astype(np.float32)
        ctx.adam_step(p, cuda(gr), m, v, t)
        ref.grad = torch.from_numpy(gr)
        opt.step()
    ctx.sync()
    np.testing.assert_allclose(p.cpu().numpy(), ref.detach().numpy(), rtol=1e-5, atol=1e-6)


def test_training_steps_reduce_the_loss(etx):
    from paper_2407_12119_gb300.train import Trainer
    wl = WORKLOADS["train64"]
    cfg = wl.model
    b = wl.batch(8)
    W = wl.weights()
    emb = O.embed(W, 3, b.x, b.y, b.z)
    s, d, eo = O.build_graph(emb, b.plane, b.hit_offsets, cfg.radius, cfg.k_max)
    y = truth_edge_labels(global_particle_ids(b), b.plane, s, d).astype(np.float32)
    tr = Trainer(cfg, pack_blob(cfg, W), b.n_events, b.n_hits, s.size, dtype="bf16")
    args = [cuda(a) for a in (b.x, b.y, b.z, s.astype(np.int32), d.astype(np.int32),
                              eo.astype(np.int32), y)]
    losses = [float(tr.step(*args).item()) for _ in range(8)]
    tr.ctx.sync()
    print("losses", [round(l, 4) for l in losses])
    assert losses[-1] < losses[0]


def test_autograd_function_matches_backward(etx):
    from paper_2407_12119_gb300.train import InteractionNetworkFn
    cfg, b, W, s, d, eo, y = problem(32, 2, 1)
    ctx = etx.Context(cfg, b.n_events, b.n_hits, s.size, train=True)
    blob = pack_blob(cfg, W)
    ctx.load_weights(blob)
    theta = cuda(blob[blob.size - ctx.gnn_param_count:]).requires_grad_(True)
    args = (cuda(b.x), cuda(b.y), cuda(b.z), cuda(s.astype(np.int32)), cuda(d.astype(np.int32)),
            cuda(eo.astype(np.int32)))
    logits = InteractionNetworkFn.apply(theta, ctx, *args, "f32")
    w_h = np.linspace(-1.0, 1.0, logits.numel())             # upstream gradient, made on the host
    (logits * cuda(w_h.astype(np.float32))).sum().backward()
    cache = {}
    O.gnn_forward(W, 2, b.x, b.y, b.z, s, d, cache)
    ref = O.gnn_backward(W, cache, w_h.astype(np.float32).astype(np.float64))
    flat = np.concatenate([ref[n].reshape(-1) for n in gnn_names(cfg)])
    assert rel(theta.grad.cpu().numpy().astype(np.float64), flat) <= GRAD_RTOL


def test_gradients_and_loss_are_bit_reproducible(etx):
    """The weight gradients and the loss are sums over edges split across
    blocks; every split writes its partial and the partials are added in a
    fixed order, so two runs give the same bits (no atomics)."""
    cfg, b, W, s, d, eo, y = problem(128, 3, 8, seed=3)
    runs = [gpu_grads(etx, cfg, b, W, s, d, eo, y, dtype="bf16") for _ in range(2)]
    assert runs[0][0] == runs[1][0]
    for n in runs[0][1]:
        np.testing.assert_array_equal(runs[0][1][n], runs[1][1][n], err_msg=n)


def test_device_weight_update_equals_a_reload(etx):
    """etx_set_gnn_params (the device repack of a parameter vector) leaves the
    context exactly as loading the same values from the host would: the same
    logits (FP32 and BF16 tensor-core paths) and the same gradients; the e4m3
    images are not rebuilt, so FP8 is refused until the next load."""
    cfg, b, W, s, d, eo, y = problem(128, 2, 4, seed=5)
    blob = pack_blob(cfg, W)
    ctx_dev = etx.Context(cfg, b.n_events, b.n_hits, max(s.size, 1), train=True)
    ctx_dev.load_weights(blob)
    n = ctx_dev.gnn_param_count
    rng = np.random.default_rng(9)
    new = blob.copy()
    new[-n:] += (0.01 * rng.normal(size=n)).astype(np.float32)
    ctx_dev.set_gnn_params(cuda(new[-n:]))
    ctx_host = etx.Context(cfg, b.n_events, b.n_hits, max(s.size, 1), train=True)
    ctx_host.load_weights(new)
    x, yy, z = cuda(b.x), cuda(b.y), cuda(b.z)
    st, dt, eot = cuda(s.astype(np.int32)), cuda(d.astype(np.int32)), cuda(eo.astype(np.int32))
    tgt = cuda(y.astype(np.float32))
    for dtype in ("f32", "bf16"):
        outs = []
        for c in (ctx_dev, ctx_host):
            logits = c.gnn_forward(x, yy, z, st, dt, eot, dtype=dtype)
            _, dl = c.weighted_bce(logits, tgt, eot, 10.0)
            g = c.gnn_backward(dl)
            c.sync()
            outs.append((logits.cpu().numpy(), g.cpu().numpy()))
        np.testing.assert_array_equal(outs[0][0], outs[1][0], err_msg=dtype)
        np.testing.assert_array_equal(outs[0][1], outs[1][1], err_msg=dtype)
    with pytest.raises(etx.EtxError) as ei:
        ctx_dev.gnn_forward(x, yy, z, st, dt, eot, dtype="fp8")
    assert ei.value.status == etx.ETX_ERR_STATE


def test_bf16_forward_gradient_matches_the_oracle_reading(etx):
    """The training path with a BF16 tensor-core forward: the GPU's gradient
    against the oracle's reading of it (BF16-operand forward keeping the
    residual streams, exact recomputation of every block in the backward,
    ``gnn_backward(recompute=True)``), on the same logits gradient."""
    cfg, b, W, s, d, eo, y = problem(128, 2, 2, seed=1)
    loss, g, logits = gpu_grads(etx, cfg, b, W, s, d, eo, y, dtype="bf16")
    cache = {}
    z = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d, cache=cache, gemm="bf16")
    _, dz = O.weighted_bce(z, y, 10.0)
    ref = O.gnn_backward(W, cache, dz, recompute=True)
    devs = {n: rel(g[n], ref[n]) for n in g}
    worst = max(devs, key=devs.get)
    print(f"bf16-forward gradient vs the oracle's reading: worst relative L2 {devs[worst]:.2e} "
          f"({worst}), median {np.median(list(devs.values())):.2e}; logits max diff "
          f"{np.abs(logits - z).max():.2e}")
    # the BF16 forward itself moves these gradients by ~5% from the exact ones, so
    # rounding-boundary differences between the two BF16 forwards show at the % level
    assert devs[worst] <= 5e-2 and np.median(list(devs.values())) <= 2e-2


def test_bf16_forward_gradient_stage_isolated(etx):
    """The same BF16-forward training path, stage-isolated: the oracle's reverse
    pass (exact recomputation of every block) taken at the GPU's own
    checkpointed residual streams and the GPU's own logits gradient must give
    the GPU's gradient within 1e-3 relative per tensor."""
    cfg, b, W, s, d, eo, y = problem(128, 2, 2, seed=1)
    ctx = etx.Context(cfg, b.n_events, b.n_hits, max(s.size, 1), train=True)
    ctx.load_weights(pack_blob(cfg, W))
    x, yy, z = cuda(b.x), cuda(b.y), cuda(b.z)
    st, dt, eot = cuda(s.astype(np.int32)), cuda(d.astype(np.int32)), cuda(eo.astype(np.int32))
    logits = ctx.gnn_forward(x, yy, z, st, dt, eot, dtype="bf16")
    _, dl = ctx.weighted_bce(logits, cuda(y.astype(np.float32)), eot, 10.0)
    hs, es = [], []
    for k in range(cfg.n_iters + 1):
        h, e = ctx.gnn_checkpoints(k, b.n_hits, s.size)
        hs.append(h.cpu().numpy())
        es.append(e.cpu().numpy())
    g = ctx.gnn_backward(dl)
    ctx.sync()
    flat = g.cpu().numpy().astype(np.float64)
    cache = O.forward_cache_from_streams(W, cfg.n_iters, b.x, b.y, b.z, s, d, hs, es)
    ref = O.gnn_backward(W, cache, dl.cpu().numpy().astype(np.float64), recompute=True)
    shapes = dict(blob_layout(cfg))
    o, worst_m, worst_v = 0, (0.0, ""), (0.0, "")
    for n in gnn_names(cfg):
        k = int(np.prod(shapes[n]))
        r = (rel(flat[o:o + k].reshape(shapes[n]), ref[n]), n)
        if len(shapes[n]) > 1:
            worst_m = max(worst_m, r)
        else:
            worst_v = max(worst_v, r)
        o += k
    print(f"bf16-forward gradient, stage-isolated: worst relative L2 {worst_m[0]:.2e} ({worst_m[1]}) "
          f"of the matrices, {worst_v[0]:.2e} ({worst_v[1]}) of the vectors")
    assert worst_m[0] <= GRAD_RTOL
    # A ReLU mask decided differently by the FP32 and the FP64 recomputation (a
    # pre-activation within rounding of zero) moves a bias/gain column sum by one
    # term; the class-weighted BCE gradient cancels ~25x in those sums, so one such
    # term is ~1e-3 of the vector's norm on this problem.
    assert worst_v[0] <= 3 * GRAD_RTOL


def test_backward_several_tiles_per_cta(etx):
    """H = 128 on ~45k edges: more than twice as many 128-row tiles as SMs, so
    every persistent tensor-core backward CTA takes two or three tiles and
    alternates its two accumulators; gradients against the FP64 oracle as in
    the small cases."""
    cfg, b, W, s, d, eo, y = problem(128, 2, 24, seed=4)
    assert s.size > 2 * 152 * 128
    cache = {}
    z = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d, cache)
    loss_ref, dz = O.weighted_bce(z, y, 10.0)
    ref = O.gnn_backward(W, cache, dz)
    loss, g, _ = gpu_grads(etx, cfg, b, W, s, d, eo, y)
    assert abs(loss - loss_ref) <= 1e-5 * max(1.0, abs(loss_ref))
    worst = max((rel(g[n], ref[n]), n) for n in ref)
    print(f"H=128 L=2: E={s.size}, worst per-tensor relative L2 {worst[0]:.2e} ({worst[1]})")
    assert worst[0] <= GRAD_RTOL, worst


def test_backward_with_no_edges(etx):
    """A batch whose graph has no edge: the loss does not depend on any
    parameter, every gradient is exactly zero (the edge-row launches have no
    tile; their column-sum partials are written as zeros)."""
    cfg, b, W, s, d, eo, y = problem(128, 2, 2, seed=5)
    # one unused edge slot (the library takes no NULL array); every edge offset
    # is 0, so the batch has no edge
    s0 = np.zeros(1, np.int64)
    eo0 = np.zeros_like(eo)
    _, g, _ = gpu_grads(etx, cfg, b, W, s0, s0, eo0, np.zeros(1))
    for n, v in g.items():
        assert np.all(np.isfinite(v)) and not np.any(v), n


@pytest.mark.parametrize("alpha,gamma", [(0.25, 2.0), (0.5, 0.0), (0.9, 1.5)])
def test_focal_loss_matches_oracle(etx, alpha, gamma):
    """The sigmoid focal loss (Eq. 5) on the GPU: loss and d loss / d logit
    against the FP64 oracle on the logits the GPU computed (stage-isolated)."""
    cfg, b, W, s, d, eo, y = problem(32, 2, 2, seed=6)
    ctx = etx.Context(cfg, b.n_events, b.n_hits, max(s.size, 1), train=True)
    ctx.load_weights(pack_blob(cfg, W))
    eot = cuda(eo.astype(np.int32))
    logits = ctx.gnn_forward(cuda(b.x), cuda(b.y), cuda(b.z), cuda(s.astype(np.int32)),
                             cuda(d.astype(np.int32)), eot)
    loss, dl = ctx.focal_loss(logits, cuda(y.astype(np.float32)), eot, alpha, gamma)
    ctx.sync()
    z = logits.cpu().numpy().astype(np.float64)
    lr, dr = O.focal_loss(z, y, alpha=alpha, gamma=gamma)
    assert abs(float(loss.item()) - lr) <= 1e-5 * max(abs(lr), 1e-12)
    got = dl.cpu().numpy().astype(np.float64)
    assert np.abs(got - dr).max() <= 1e-5 * np.abs(dr).max() + 1e-12


def test_training_with_the_focal_loss(etx):
    """A few training steps with the focal loss lower it, and the gradient of
    one step matches the oracle's reverse pass of the focal loss."""
    cfg, b, W, s, d, eo, y = problem(128, 2, 2, seed=7)
    cache = {}
    z = O.gnn_forward(W, cfg.n_iters, b.x, b.y, b.z, s, d, cache)
    _, dz = O.focal_loss(z, y)
    ref = O.gnn_backward(W, cache, dz)
    ctx = etx.Context(cfg, b.n_events, b.n_hits, max(s.size, 1), train=True)
    ctx.load_weights(pack_blob(cfg, W))
    # the forward's inputs stay alive until the backward (it reads them again)
    x, yy, zz = cuda(b.x), cuda(b.y), cuda(b.z)
    st, dt, eot = cuda(s.astype(np.int32)), cuda(d.astype(np.int32)), cuda(eo.astype(np.int32))
    logits = ctx.gnn_forward(x, yy, zz, st, dt, eot)
    _, dl = ctx.focal_loss(logits, cuda(y.astype(np.float32)), eot)
    flat = ctx.gnn_backward(dl).cpu().numpy().astype(np.float64)
    shapes = dict(blob_layout(cfg))
    o, worst = 0, (0.0, "")
    for n in gnn_names(cfg):
        k = int(np.prod(shapes[n]))
        worst = max(worst, (rel(flat[o:o + k].reshape(shapes[n]), ref[n]), n))
        o += k
    assert worst[0] <= GRAD_RTOL, worst
    from paper_2407_12119_gb300.train import Trainer
    tr = Trainer(cfg, pack_blob(cfg, W), b.n_events, b.n_hits, max(s.size, 1), dtype="f32",
                 lr=1e-3, loss="focal")
    args = (x, yy, zz, st, dt, eot, cuda(y.astype(np.float32)))
    losses = [float(tr.step(*args).item()) for _ in range(8)]
    assert losses[-1] < losses[0], losses
