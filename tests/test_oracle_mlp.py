"""Pins of the oracle's network (learned form): BF16 rounding against
PyTorch's conversion, the backward pass against finite differences, the
placement of the roundings against a hand-worked network, and Adam against
its closed form for constant gradients (Kingma and Ba, 2015)."""
import numpy as np
import pytest

from oracle import mlp
from paper_0705_4371_gb300 import inputs
from tests._common import mlp_random_params, mlp_random_features


random_params = mlp_random_params
random_features = mlp_random_features


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    v = np.concatenate([
        inputs.uniform(5, (4000,), -3.0, 3.0),
        np.ldexp(inputs.uniform(6, (1000,), 1.0, 2.0), (inputs.uniform(7, (1000,), -140, 120)).astype(int)),
        # ties: halfway between adjacent BF16 values, both parities
        1.0 + np.arange(0, 64) * 2.0 ** -8,
        -(1.0 + np.arange(0, 64) * 2.0 ** -8),
        [0.0, -0.0, np.inf, -np.inf, 3.0e38, 1e-45],
    ]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = mlp.bf16(v)
    assert np.array_equal(got, ref)


def test_backward_matches_finite_differences():
    p = random_params(41)
    feat = random_features(42, 24)
    dmu = 0.05 * inputs.uniform(43, (24, 4))
    loss, g = mlp.loss_and_grad(p, feat, dmu, round=False)
    h = 1e-6
    idx = np.concatenate([np.arange(mlp.N_PARAMS - 12)[::37], np.arange(4736, 4740)])
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, feat, dmu, round=False)[0] -
              mlp.loss_and_grad(pm, feat, dmu, round=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
    # normalisation entries are not trained
    assert not g[4740:].any()


def test_rounding_points_on_a_hand_worked_network():
    # one path through the network: input 0 -> hidden 0 -> hidden 0 -> output 0
    d = mlp.unpack(np.zeros(mlp.N_PARAMS))
    d["mean"] = np.zeros(4)
    d["inv_std"] = np.ones(4)
    d["out_scale"] = np.ones(4)
    d["W1"][0, 0] = 1 + 2.0 ** -9     # rounds to 1
    d["b1"][0] = 2.0 ** -10           # bias kept exact: z1 = 1 + 2^-10, h1 rounds to 1
    d["W2"][0, 0] = 3.0
    d["W3"][0, 0] = 1 + 2.0 ** -12    # rounds to 1
    d["b3"][0] = 2.0 ** -20           # bias kept exact
    p = mlp.pack(d)
    feat = np.array([[1 + 2.0 ** -9, 0.0, 0.0, 0.0]])   # standardised input rounds to 1
    y, c = mlp.forward(p, feat, round=True)
    assert y[0, 0] == 3.0 + 2.0 ** -20
    assert c["x"][0, 0] == 1.0 and c["h1"][0, 0] == 1.0 and c["h2"][0, 0] == 3.0
    y64, _ = mlp.forward(p, feat, round=False)
    x = 1 + 2.0 ** -9
    assert y64[0, 0] == pytest.approx((x * (1 + 2.0 ** -9) + 2.0 ** -10) * 3.0 * (1 + 2.0 ** -12)
                                      + 2.0 ** -20, rel=1e-15)


def test_rounding_free_network_equals_exact_network():
    # weights on a coarse grid and inputs in {0, +-1/2, +-1}: every rounded
    # quantity is a BF16 value already, so both paths must agree exactly,
    # gradients included (they use the same formulas on the same numbers)
    g = inputs.SplitMix64(44)
    d = mlp.unpack(np.zeros(mlp.N_PARAMS))
    d["W1"] = np.round(g.uniform(256, -8, 8)).reshape(64, 4) / 8
    d["b1"] = np.round(g.uniform(64, -8, 8)) / 8
    W2 = np.zeros((64, 64))
    cols = (g.uniform(64) * 64).astype(int)
    W2[np.arange(64), cols] = np.round(g.uniform(64, -2, 2)) / 2
    d["W2"] = W2
    d["b2"] = np.round(g.uniform(64, -8, 8)) / 16
    d["W3"] = np.round(g.uniform(256, -4, 4)).reshape(4, 64) / 4
    d["b3"] = np.round(g.uniform(4, -4, 4)) / 4
    d["mean"], d["inv_std"], d["out_scale"] = np.zeros(4), np.ones(4), np.ones(4)
    p = mlp.pack(d)
    feat = np.round(g.uniform(4 * 32, -2, 2)).reshape(32, 4) / 2
    dmu = np.round(g.uniform(4 * 32, -8, 8)).reshape(32, 4) / 8
    y1, c1 = mlp.forward(p, feat, round=True)
    y0, c0 = mlp.forward(p, feat, round=False)
    assert np.array_equal(c1["h1"], c0["h1"]) and np.array_equal(c1["h2"], c0["h2"])
    assert np.array_equal(y1, y0)
    l1, g1 = mlp.loss_and_grad(p, feat, dmu, round=True)
    l0, g0 = mlp.loss_and_grad(p, feat, dmu, round=False)
    assert l1 == l0 and np.array_equal(g1, g0)


def test_adam_closed_form_for_constant_gradients():
    # with m = v = 0 and the same gradient g at every step, the bias-corrected
    # moments are g and g^2, so every step moves by lr g / (|g| + eps)
    p = random_params(45)
    g = inputs.uniform(46, (mlp.N_PARAMS,), -1e-2, 1e-2)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lr = 1e-3
    q = p.copy()
    for t in range(1, 4):
        q, m, v = mlp.adam_step(q, g, m, v, t, lr)
        step = lr * g / (np.abs(g) + 1e-8)
        tr = slice(0, 4740)
        assert np.allclose(q[tr], p[tr] - t * step[tr], rtol=0, atol=1e-15)
        assert np.array_equal(q[4740:], p[4740:])


def test_near_boundary_flags():
    # a z exactly on a BF16 midpoint is flagged; one a quarter-spacing away is not
    z = np.array([[1.0 + 2.0 ** -8, 1.0 + 2.0 ** -10, 0.0, -3.0]])
    mag = np.ones_like(z)
    f = mlp._near_boundary(z, mag, 1e-5)
    assert f.tolist() == [[True, False, True, False]]
