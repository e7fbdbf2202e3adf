"""CPU pins of the learned-model reference (oracle/mlp.py) and of unbiasedness under arbitrary
fixed scan weights and initial marginals (Proposition 1, Theorem 1)."""
import math

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


# ---------------------------------------------------------------------------------------------
# The forward pass, the loss and the heads against hand-worked examples (their definitions, not a
# second implementation): a network whose integer weights compute a function one can read off.
def _readable_network():
    """W1 copies x_k to hidden unit k and -x_k to unit 16 + k (ReLU keeps the positive and the
    negative parts), unit 40 is the constant relu(b1 = 2); W2 shifts by one, Z2[k] = H1[k + 1]
    (Z2[63] = H1[0]), with b2[5] = -1; W3 gives O_0 = H2[0] + H2[1] + H2[2] - 3 H2[20] + 0.5 and
    O_1 = 2 H2[39] - H2[16] - 10.  So O_0 = relu(x1) + relu(x2) + relu(x3) - 3 relu(-x5) + 0.5 and
    O_1 = 4 - relu(-x1) - 10.  Layout: weights row-major [out][in]."""
    W1 = np.zeros((64, 16)); b1 = np.zeros(64)
    for k in range(16):
        W1[k, k] = 1.0
        W1[16 + k, k] = -1.0
    b1[40] = 2.0
    W2 = np.zeros((64, 64)); b2 = np.zeros(64)
    for k in range(64):
        W2[k, (k + 1) % 64] = 1.0
    b2[5] = -1.0
    W3 = np.zeros((2, 64)); b3 = np.array([0.5, -10.0])
    W3[0, [0, 1, 2]] = 1.0
    W3[0, 20] = -3.0
    W3[1, 39] = 2.0
    W3[1, 16] = -1.0
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def test_forward_on_a_hand_worked_network():
    """Row A = (1, -2, 3, -4, 5, -6, ...): O_0 = 0 + 3 + 0 - 3 * 6 + 0.5 = -14.5, O_1 = 4 - 2 - 10 = -8.
    Row B = 0.5 everywhere: O_0 = 1.5 + 0.5 = 2, O_1 = -6.  A transposed W2 (a shift the other way),
    a ReLU on the output layer or a missing bias gives other numbers."""
    theta = _readable_network()
    assert theta.size == mlp.n_params()
    X = np.array([[(k + 1) * (-1) ** k for k in range(16)], [0.5] * 16], dtype=np.float64)
    layers = mlp.unpack(mlp.bf16_round(theta))           # small integers: exact in bf16
    O = mlp.forward(X, layers)[-1]
    assert np.array_equal(O, np.array([[-14.5, -8.0], [2.0, -6.0]]))


def test_loss_and_gradient_on_hand_worked_segments():
    """Two instances.  Instance 1, rows (o_1, o_2) = (0, 0), (ln 3, 0), target w (1/2, 1/2), target p
    (1, 0): softmax = (1/4, 3/4), cross-entropy = ln 4 - (ln 3)/2, mean BCE = ln 2 (softplus(0));
    gradients (softmax - t) = (-1/4, 1/4) and (sigmoid - p) / 2 = (-1/4, 1/4).  Instance 2, one row
    (0, ln 3), target w 1, p 1/4: cross-entropy 0 with gradient 0, BCE = ln 4 - (ln 3)/4 with
    gradient 3/4 - 1/4 = 1/2.  The loss is the mean over the two instances, so every gradient
    entry is halved."""
    L3 = math.log(3.0)
    O = np.array([[0.0, 0.0], [L3, 0.0], [0.0, L3]])
    seg = np.array([0, 2, 3])
    tw = np.array([0.5, 0.5, 1.0])
    tp = np.array([1.0, 0.0, 0.25])
    loss, dO = mlp.loss_and_dO(O, seg, tw, tp)
    want = ((math.log(4.0) - L3 / 2 + math.log(2.0)) + (math.log(4.0) - L3 / 4)) / 2
    assert loss == pytest.approx(want, rel=1e-14)
    assert np.allclose(dO, np.array([[-0.25, -0.25], [0.25, 0.25], [0.0, 0.5]]) / 2, rtol=0, atol=1e-15)


def test_heads_on_hand_worked_outputs():
    """o_1 = (0, ln 3) gives softmax (1/4, 3/4) and w = 0.5 softmax + 0.5 / 2 = (3/8, 5/8);
    o_2 = (0, 100) gives sigmoid (1/2, ~1), clamped to (1/2, 1 - 1e-6)."""
    O = np.array([[0.0, 0.0], [math.log(3.0), 100.0]])
    w, nu = mlp.heads(O, np.array([0, 2]))
    assert np.allclose(w, [0.375, 0.625], rtol=0, atol=1e-15)
    assert nu[0] == 0.5 and nu[1] == 1.0 - 1e-6
