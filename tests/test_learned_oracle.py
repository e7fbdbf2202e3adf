"""CPU pins of the learned-model reference (oracle/mlp.py) and of unbiasedness under arbitrary
fixed scan weights and initial marginals (Proposition 1, Theorem 1)."""
import numpy as np
import pytest

import synth
from oracle import exact, mlp


def _theta(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.n_params())


def test_bf16_rounding_matches_definition():
    x = np.array([1.0, 1.00390625, 1.0078125, -3.14159, 1e-8, 65504.0, 1.0 + 2 ** -8 + 2 ** -9],
                 dtype=np.float32)
    r = mlp.bf16_round(x)
    # bf16 keeps 8 significand bits: representable values survive, others round to the nearest
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12
    assert r[6] == 1.0078125                      # above the halfway point rounds up
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)


def test_gradient_matches_central_differences():
    """The analytic gradient of the loss equals central finite differences (fp64)."""
    rng = np.random.default_rng(3)
    seg = np.array([0, 7, 19, 30])
    X = rng.normal(size=(30, mlp.N_FEATURES))
    p = rng.random(30)
    tw = mlp.weight_target(rng.random(30), seg)
    theta = _theta(1)

    def loss(th):
        layers = mlp.unpack(th)
        cache = mlp.forward(X, layers)
        return mlp.loss_and_dO(cache[-1], seg, tw, p)[0]

    layers = mlp.unpack(theta)
    cache = mlp.forward(X, layers)
    _, dO = mlp.loss_and_dO(cache[-1], seg, tw, p)
    g = mlp.backward(X, layers, cache, dO)
    idx = rng.choice(len(theta), 60, replace=False)
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = 1e-6
        fd = (loss(theta + e) - loss(theta - e)) / 2e-6
        assert g[k] == pytest.approx(fd, rel=2e-5, abs=1e-8)


def test_heads_are_valid_scan_weights_and_marginals():
    rng = np.random.default_rng(0)
    seg = np.array([0, 5, 105])
    O = rng.normal(scale=30.0, size=(105, 2))
    w, nu = mlp.heads(O, seg)
    for s in range(2):
        ws = w[seg[s]:seg[s + 1]]
        assert ws.sum() == pytest.approx(1.0, abs=1e-12)
        assert ws.min() >= mlp.ALPHA_W / len(ws) - 1e-15     # every site keeps weight >= 0.5/n
    assert nu.min() >= mlp.NU_MIN and nu.max() <= mlp.NU_MAX


def test_features_on_a_hand_built_design():
    """Two pools, four clones: clone 0 in both (both positive), clone 1 in pool 0, clone 2 in
    pool 1, clone 3 in a negative pool 2."""
    inst = synth.Instance(n=4, m=3, clone_ptr=np.array([0, 2, 3, 4, 5], np.int32),
                          clone_pools=np.array([0, 1, 0, 1, 2], np.int32),
                          y=np.array([1, 1, 0], np.uint8), positives=np.array([0], np.int32),
                          fp=0.1, fn=0.2, q=0.25)
    F = mlp.features(inst)
    # all-positive clones: 0, 1, 2 (clone 3's only pool is negative) -> ap = [2, 2, 0], NAP = 3
    assert F[0, 7] == 1 and F[1, 7] == 1 and F[2, 7] == 1 and F[3, 7] == 0
    assert F[0, 8] == pytest.approx(0.2) and F[0, 9] == pytest.approx(0.5)
    assert F[0, 10] == 0 and F[3, 11] == 0
    assert np.all(F[:, 12] == pytest.approx(0.03))
    assert F[0, 0] == pytest.approx(2 / 8) and F[3, 2] == pytest.approx(1 / 8)
    dbar = 5 / 3
    assert F[0, 5] == pytest.approx(((2 + 2) / 2) / dbar) and F[3, 6] == 0
    lam = np.log(0.25 / 0.75)
    ap = np.log(0.8 / 0.1)
    assert F[1, 4] == pytest.approx((lam + ap) / 10)


@pytest.mark.parametrize("what", ["weights", "init", "both"])
def test_unbiased_with_arbitrary_learned_inputs(oracle_lib, what):
    """Theorem 1 and Proposition 1: any fixed positive scan weights and any initial marginals
    leave theta_CT unbiased.  z-test against the 2^20 enumeration with random w and nu."""
    inst = synth.make_instance(20, 8, 3, 2, 0.1, 0.2, 0.05, 1001, 2001)
    _, p = exact.posterior(inst)
    rng = np.random.default_rng(7)
    w = rng.random(inst.n) + 0.3 if what in ("weights", "both") else None
    nu = rng.random(inst.n) if what in ("init", "both") else None
    res = oracle_lib.decode(inst, 100000, 3, 20, 60, seed=41, scan=oracle_lib.SCAN_CUSTOM if w is not None else 0,
                            custom_w=w, init_marginals=nu)
    assert res["status"] == 0
    z = np.abs(res["est"] - p) / res["se"]
    assert z.max() < 4.5, z
