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


def _fp32_accumulated_forward(p, feat, seed):
    """The rounded network evaluated as a kernel would: products of BF16
    values (exact in FP32) and the FP32 bias summed in FP32 in a random order
    per unit, hidden values rounded to BF16 after the ReLU.  Also returns the
    largest error of a hidden pre-activation sum relative to the sum of the
    absolute values of its terms."""
    d = mlp.unpack(p)
    g = np.random.default_rng(seed)
    f32 = np.float32
    x = mlp.standardise(p, feat, True).astype(f32)
    worst = [0.0]

    def layer(h, W, b, hidden=True):
        terms = np.concatenate([h[:, None, :] * mlp.bf16(W).astype(f32)[None, :, :],
                                np.broadcast_to(b.astype(f32), (h.shape[0], b.size))[:, :, None]], axis=2)
        order = np.argsort(g.random(terms.shape), axis=2)
        terms = np.take_along_axis(terms, order, axis=2).astype(f32)
        s = np.zeros(terms.shape[:2], f32)
        for k in range(terms.shape[2]):
            s = (s + terms[:, :, k]).astype(f32)
        if hidden:
            t64 = terms.astype(np.float64)
            worst[0] = max(worst[0], float(np.max(np.abs(s - t64.sum(2)) / np.abs(t64).sum(2))))
        return s

    h1 = mlp.bf16(np.maximum(layer(x, d["W1"], d["b1"]), 0)).astype(f32)
    h2 = mlp.bf16(np.maximum(layer(h1, d["W2"], d["b2"]), 0)).astype(f32)
    return layer(h2, d["W3"], d["b3"], hidden=False).astype(np.float64), worst[0]


@pytest.mark.parametrize("band", [4e-6, 2.5e-7])
def test_forward_bounds_hold_every_fp32_accumulation_order(band):
    # Every order of the hidden sums whose error stays within band x the sum
    # of |terms| must give outputs inside the bounds (up to the output sum's
    # own FP32 error).  4e-6 covers the worst case of an FP32 sum of 65
    # terms (65 u / (1 - 65 u), u = 2^-24); 2.5e-7, the band of the GPU
    # check, covers the errors these orders make (asserted), and gives
    # bounds tight enough that a missing widening at either layer shows.
    p = random_params(51)
    feat = random_features(52, 1024)
    lo, hi = mlp.forward_bounds(p, feat, band)
    y, c = mlp.forward(p, feat, round=True)
    d = mlp.unpack(p)
    mag = c["h2"] @ np.abs(mlp.bf16(d["W3"])).T + np.abs(d["b3"])
    tol = 4e-6 * mag
    assert np.all(lo <= y + 1e-12 * mag) and np.all(y <= hi + 1e-12 * mag)
    moved = 0
    for seed in range(12):
        ys, worst = _fp32_accumulated_forward(p, feat, 600 + seed)
        assert worst <= band, (seed, worst)
        assert np.all(ys >= lo - tol) and np.all(ys <= hi + tol), seed
        moved += int(np.sum(np.abs(ys - y) > tol))
    # some orders flip a hidden rounding (the bounds are exercised, not trivial)
    assert moved > 0
    assert np.any(hi - lo > 10 * tol)


def test_forward_bounds_contain_every_perturbed_evaluation():
    # The bounds' definition by brute force: every hidden pre-activation
    # moved anywhere within band x the sum of its |terms| (uniformly inside,
    # and at both ends of the interval), the network evaluated in FP64 from
    # there; each output must lie inside the bounds.
    p = random_params(55)
    feat = random_features(56, 2048)
    band = 2.5e-7
    lo, hi = mlp.forward_bounds(p, feat, band)
    d = mlp.unpack(p)
    x = mlp.standardise(p, feat, True)
    W1, W2, W3 = mlp.bf16(d["W1"]), mlp.bf16(d["W2"]), mlp.bf16(d["W3"])
    g = np.random.default_rng(57)

    def shift(shape):
        u = g.uniform(-1.0, 1.0, shape)
        pick = g.random(shape)
        u[pick < 0.25] = -(1 - 1e-9)
        u[pick > 0.75] = 1 - 1e-9
        return u

    ymin, ymax = np.full(lo.shape, np.inf), np.full(lo.shape, -np.inf)
    outside = 0
    for _ in range(16):
        z1 = x @ W1.T + d["b1"]
        z1 = z1 + band * (np.abs(x) @ np.abs(W1).T + np.abs(d["b1"])) * shift(z1.shape)
        h1 = mlp.bf16(np.maximum(z1, 0.0))
        z2 = h1 @ W2.T + d["b2"]
        z2 = z2 + band * (h1 @ np.abs(W2).T + np.abs(d["b2"])) * shift(z2.shape)
        h2 = mlp.bf16(np.maximum(z2, 0.0))
        y = h2 @ W3.T + d["b3"]
        mag = h2 @ np.abs(W3).T + np.abs(d["b3"])
        outside += int(np.sum((y < lo - 1e-12 * mag) | (y > hi + 1e-12 * mag)))
        ymin, ymax = np.minimum(ymin, y), np.maximum(ymax, y)
    assert outside == 0
    # the perturbations reach far into the wide intervals (not point checks)
    assert (ymax - ymin).max() > 0.25 * (hi - lo).max() > 0


def test_forward_bounds_collapse_to_forward_without_band():
    p = random_params(53)
    feat = random_features(54, 256)
    y, _ = mlp.forward(p, feat, round=True)
    lo, hi = mlp.forward_bounds(p, feat, 0.0)
    assert np.allclose(lo, y, rtol=0, atol=1e-12) and np.allclose(hi, y, rtol=0, atol=1e-12)
