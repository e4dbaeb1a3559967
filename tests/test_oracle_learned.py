"""Pins of the FP64 reference of the learned correction (oracle/learned.py):
its gradient against central finite differences, GELU against its integral
definition, and the feature vector against its definition on a tiny state."""
import math

import numpy as np
import pytest

import oracle
from oracle import learned
from synth import traffic

SEED = 0x9E3779B97F4A7C15


def test_gelu_matches_definition_and_derivative():
    z = np.linspace(-6, 6, 101)
    # the tanh form approximates GELU(z) = z * Phi(z), Phi the normal CDF,
    # to within 1e-3 everywhere (Hendrycks & Gimpel 2016)
    phi = np.array([0.5 * (1 + math.erf(t / math.sqrt(2))) for t in z])
    np.testing.assert_allclose(learned.gelu_exact(z), z * phi, rtol=1e-12, atol=1e-15)
    assert np.abs(learned.gelu(z) - z * phi).max() < 1e-3
    t = np.tanh(math.sqrt(2 / math.pi) * (z + 0.044715 * z ** 3))
    np.testing.assert_allclose(learned.gelu(z), 0.5 * z * (1 + t), rtol=1e-14, atol=1e-15)
    h = 1e-6
    num = (learned.gelu(z + h) - learned.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(learned.gelu_grad(z), num, rtol=1e-7, atol=1e-8)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    theta = rng.normal(0, 0.3, learned.N_PARAMS)
    X = rng.random((7, learned.IN))
    y = rng.normal(0, 1, 7)
    g = learned.gradient(theta, X, y)
    idx = rng.choice(learned.N_PARAMS, 200, replace=False)
    idx = np.concatenate([idx, [learned.N_PARAMS - 1, 0]])  # b3, W1[0][0]
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num = (learned.loss(tp, X, y) - learned.loss(tm, X, y)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_zero_network_predicts_bias_and_correct_is_identity():
    theta = np.zeros(learned.N_PARAMS)
    theta[-1] = 0.25
    d, _ = learned.forward(theta, np.random.default_rng(1).random((5, learned.IN)))
    np.testing.assert_allclose(d, 0.25)
    n = np.array([0.0, 1.0, 10.0, 1e6])
    np.testing.assert_allclose(learned.correct(n, np.zeros(4)), n, rtol=1e-12)


def test_features_follow_their_definition():
    """Histogram bins count the host's virtual registers by value (Alg. 3 +
    Alg. 2 per index), the extra inputs are the stated statistics."""
    rng = np.random.default_rng(6)
    aips = traffic.distinct_u32(rng, 30)
    o = oracle.Oracle("gfast", k=4, Z=5003, b=5, seed=SEED)
    for _ in range(3):
        o.scan(traffic.uniform_pairs(rng, 4000, aips))
        o.slide()
    X, n_plain = o.features(aips)
    reg = o.registers()
    S_Z, V_Z = o.pool_sums()
    np.testing.assert_allclose(n_plain, o.estimate(aips))
    for h, a in enumerate(aips[:10]):
        M = np.array([reg[o.phy_idx(int(a), i)] for i in range(32)])
        np.testing.assert_allclose(X[h, :64], np.bincount(M, minlength=64)[:64] / 32.0)
        S = int(sum(2 ** (32 - int(m)) for m in M))
        V = int((M == 0).sum())
        assert X[h, 64] == 5 / 16
        assert X[h, 65] == pytest.approx(math.log1p(n_plain[h]) / 16)
        assert X[h, 66] == pytest.approx(math.log1p(oracle.hll(32, S, V)) / 16)
        assert X[h, 67] == pytest.approx(math.log1p(oracle.hll(5003, S_Z, V_Z) / 5003))
        assert X[h, 68] == pytest.approx(V_Z / 5003)
        assert X[h, 69] == pytest.approx(V / 32)
        assert not X[h, 70:].any()
    assert not X[:, 32:64].any()  # registers never exceed 31


def test_compact_network_is_the_full_network_restricted_to_its_inputs():
    """The compact network embedded in the 80-input one (its ten inputs wired
    to columns 0..3 and 64..69, its 16 units as the first 16 of each hidden
    layer, every other weight and bias 0 so the other units output GELU(0) =
    0) gives the same delta: pins the compact reference's input columns,
    parameter layout and layer order to the pinned full network."""
    rng = np.random.default_rng(21)
    tc = rng.normal(0, 0.4, learned.C_N_PARAMS)
    o = 0
    pc = {}
    for name, shape in learned.C_SIZES:
        k = int(np.prod(shape))
        pc[name] = tc[o:o + k].reshape(shape)
        o += k
    cols = [0, 1, 2, 3, 64, 65, 66, 67, 68, 69]
    W1 = np.zeros((learned.HID, learned.IN))
    W1[:16][:, cols] = pc["W1"]
    b1 = np.zeros(learned.HID)
    b1[:16] = pc["b1"]
    W2 = np.zeros((learned.HID, learned.HID))
    W2[:16, :16] = pc["W2"]
    b2 = np.zeros(learned.HID)
    b2[:16] = pc["b2"]
    w3 = np.zeros(learned.HID)
    w3[:16] = pc["w3"]
    tf = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, pc["b3"]])
    X80 = rng.random((9, learned.IN))
    X80[:, 70:] = 0.0
    d_full, _ = learned.forward(tf, X80)
    Xc = learned.compact_features(X80)
    np.testing.assert_array_equal(Xc, X80[:, cols])
    np.testing.assert_allclose(learned.compact_forward(tc, Xc), d_full, rtol=1e-13, atol=1e-14)


def test_compact_zero_network_predicts_its_bias():
    theta = np.zeros(learned.C_N_PARAMS)
    theta[-1] = -0.5
    d = learned.compact_forward(theta, np.random.default_rng(2).random((4, learned.C_IN)))
    np.testing.assert_allclose(d, -0.5)
