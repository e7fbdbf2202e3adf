"""Learned scan weights / initial marginals: the GPU features, MLP forward, loss gradient, backward
and heads against the fp64 CPU reference (oracle/mlp.py) on the same bf16-rounded parameters, and
a trained model's effect on the decoder (needs a GB300).

Tolerances: features are fp32 roundings of fp64 values (relative 1e-6); forward outputs and
gradients are fp32 accumulations of the same bf16 weights and fp32 inputs (relative 2e-4 of the
largest magnitude in each array, which bounds a few thousand fp32 roundings)."""
import numpy as np
import pytest

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_30239_gb300 import build, mcpd
    build.build()
    c = mcpd.Context(0)
    yield c
    c.close()


def _instances(count=6, seed=0):
    return [synth.make_instance(200 + 37 * i, 17 + i, 3 + (i % 5), 1 + (i % 3), 0.05 + 0.01 * i,
                                0.1 + 0.02 * i, (1 + (i % 3)) / (200 + 37 * i), 300 + i + seed,
                                400 + i + seed) for i in range(count)]


def _close(a, b, rel):
    scale = max(np.abs(b).max(), 1e-30)
    assert np.max(np.abs(a - b)) <= rel * scale, np.max(np.abs(a - b)) / scale


def test_features_match_reference(ctx):
    from paper_2608_30239_gb300 import learned
    insts = _instances() + [synth.high_noise_config()]
    F = learned.features(ctx, insts).cpu().numpy()
    ref = np.concatenate([mlp.features(inst) for inst in insts])
    assert F.shape == ref.shape
    assert np.allclose(F, ref, rtol=1e-6, atol=1e-6)


def test_forward_loss_backward_heads_match_reference(ctx):
    import torch
    from paper_2608_30239_gb300 import learned
    insts = _instances()
    seg = learned.segments(insts)
    X = learned.features(ctx, insts)
    model = learned.MLP(ctx, seed=5)
    theta = mlp.bf16_round(model.master.cpu().numpy())
    assert np.array_equal(mlp.bf16_round(model.W.cpu().numpy().view(np.uint16).astype(np.uint32).__lshift__(16)
                                         .astype(np.uint32).view(np.float32)), theta)
    layers = mlp.unpack(theta)
    Xn = X.cpu().numpy().astype(np.float64)
    cache = mlp.forward(Xn, layers)
    out = model.forward(X).cpu().numpy()
    _close(out, cache[-1], 2e-4)
    rng = np.random.default_rng(1)
    p = rng.random(len(Xn))
    tw = mlp.weight_target(rng.random(len(Xn)), seg)
    dev = X.device
    seg_d = torch.from_numpy(seg).to(dev)
    tw_d = torch.from_numpy(tw.astype(np.float32)).to(dev)
    p_d = torch.from_numpy(p.astype(np.float32)).to(dev)
    loss, out_d, dout = model.loss_grad(X, seg_d, tw_d, p_d)
    ref_loss, ref_dO = mlp.loss_and_dO(out_d.cpu().numpy().astype(np.float64), seg,
                                       tw_d.cpu().numpy().astype(np.float64), p_d.cpu().numpy().astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    _close(dout.cpu().numpy(), ref_dO, 1e-4)
    g_ref = mlp.backward(Xn, layers, cache, dout.cpu().numpy().astype(np.float64))
    _close(model.grad.cpu().numpy(), g_ref, 2e-4)
    w, nu = model.heads(X, seg_d)
    w_ref, nu_ref = mlp.heads(model.forward(X).cpu().numpy().astype(np.float64), seg)
    assert np.allclose(w.cpu().numpy(), w_ref, rtol=1e-12, atol=0)
    assert np.allclose(nu.cpu().numpy(), nu_ref, rtol=1e-12, atol=0)


def test_training_reduces_loss(ctx):
    import torch
    from paper_2608_30239_gb300 import learned
    insts = _instances(24, seed=3)
    seg = learned.segments(insts)
    X = learned.features(ctx, insts)
    rng = np.random.default_rng(2)
    # a learnable target: marginals that depend on the features
    Fh = X.cpu().numpy()
    p = 1.0 / (1.0 + np.exp(-(8.0 * Fh[:, 3] - 5.0 + 2.0 * Fh[:, 7])))
    tw = mlp.weight_target(p, seg)
    dev = X.device
    model = learned.MLP(ctx, seed=1)
    hist = model.fit(X, seg, torch.from_numpy(tw.astype(np.float32)).to(dev),
                     torch.from_numpy(p.astype(np.float32)).to(dev), epochs=25, batch_segments=8,
                     lr=3e-3, seed=rng.integers(1 << 30))
    # cross-entropies are bounded below by the targets' entropies: the excess must shrink
    floor = 0.0
    for a, b in zip(seg[:-1], seg[1:]):
        t = tw[a:b]
        pp = np.clip(p[a:b], 1e-12, 1 - 1e-12)
        floor += (-(t * np.log(t)).sum() - np.mean(pp * np.log(pp) + (1 - pp) * np.log(1 - pp))) / (len(seg) - 1)
    assert hist[-1] - floor < 0.5 * (hist[0] - floor), (hist, floor)


def test_learned_initial_marginals_gain(ctx):
    """What the trained network gains: trained on the method's own estimates for 256 generated
    high-noise 1298 x 97 instances, its initial marginals (with the paper's score weights kept)
    lower the largest per-clone standard error and the mean meeting time on 8 held-out instances
    at equal slots and horizon, while the estimator stays unbiased (Theorem 1)."""
    import torch
    from paper_2608_30239_gb300 import learned, learned_ab
    rng = np.random.default_rng(0)
    train = [learned_ab.high_noise_like(int(i), 100000) for i in rng.permutation(256)]
    held = [learned_ab.high_noise_like(i, 900000) for i in range(8)]
    p_hat, _, _ = learned.plain_marginals(ctx, train, slots=1024, sweeps=10)
    seg = learned.segments(train)
    X = learned.features(ctx, train)
    model = learned.MLP(ctx, seed=0)
    dev = X.device
    model.fit(X, seg, torch.tensor(learned.weight_target(p_hat, seg, mode="positive"), dtype=torch.float32, device=dev),
              torch.tensor(np.clip(p_hat, 0, 1), dtype=torch.float32, device=dev), epochs=30, batch_segments=64)
    hseg = learned.segments(held)
    _, nu = learned.learned_inputs(model, learned.features(ctx, held), hseg, nu_floor=0.02)
    plain_se, _, plain_st = learned_ab._per_instance_max_se(ctx, held, 4096, 29.4, 7)
    nu_se, _, nu_st = learned_ab._per_instance_max_se(ctx, held, 4096, 29.4, 7, init=nu)
    tau = lambda st: st["sum_tau"] / st["reps_retained"]   # noqa: E731
    print("max SE plain", plain_se.max(), "learned nu", nu_se.max(), "mean tau", tau(plain_st), tau(nu_st))
    assert nu_se.max() < plain_se.max()
    assert tau(nu_st) < 0.5 * tau(plain_st)


def test_forward_on_the_hand_worked_network(ctx):
    """The GPU forward pass on the integer network of the oracle's hand-worked pin gives exactly the
    numbers read off that network (every value is a small integer or half-integer: exact in fp32)."""
    import torch
    from test_learned_oracle import _readable_network
    from paper_2608_30239_gb300 import learned
    model = learned.MLP(ctx, seed=0)
    model.master.copy_(torch.from_numpy(_readable_network().astype(np.float32)))
    model.cast()
    X = torch.tensor([[(k + 1) * (-1) ** k for k in range(16)], [0.5] * 16], dtype=torch.float32,
                     device=f"cuda:{ctx.device}")
    O = model.forward(X).cpu().numpy()
    assert np.array_equal(O, np.array([[-14.5, -8.0], [2.0, -6.0]], dtype=np.float32))
