"""Learned form on the GPU against the oracle: the training data (Newton
multipliers), the network's forward pass, its loss gradient and Adam step,
training, the learned run's trajectory, and what the network gains.

The network's forward pass rounds hidden pre-activations accumulated in FP32
to BF16; where the oracle's FP64 value lies within a hair of a rounding
boundary the two sides may round differently, so the element-wise checks use
the samples the oracle flags as unambiguous, and every sample, the flagged
ones included, is held inside the oracle's bounds over all such roundings."""
import numpy as np
import pytest

from oracle import core as ora
from oracle import mlp as omlp
from paper_0705_4371_gb300 import inputs
from tests._common import (mlp_random_features, mlp_random_params, moment_errors, oracle_cfg,
                           rel_err)

pytestmark = pytest.mark.gpu

BAND = 2.5e-7   # half-width of the ambiguous band, relative to the sum of |terms| (4 FP32 ulps)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_0705_4371_gb300 import lbm
    lbm.load()
    assert torch.cuda.is_available()
    return torch, lbm


@pytest.fixture(scope="module")
def trained(env):
    from paper_0705_4371_gb300 import learned
    params, info = learned.train_energy_mlp(n=4_000_000, epochs=20, batch=4096, lr0=2e-3, lr1=2e-5)
    print("training: losses", ["%.3g" % x for x in info["losses"]], "data %.2fs train %.2fs"
          % (info["dataset_s"], info["train_s"]))
    return params, info


def dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def test_training_data_matches_oracle_newton(env):
    torch, lbm = env
    from paper_0705_4371_gb300 import learned
    n = 3000
    d = learned.make_dataset(n, seed=77, with_mu=True)
    it32, it64, samples, fails = d["stats"]
    assert samples == n and fails == 0
    mu_g = d["mu"].cpu().numpy()
    feat_g = d["feat"].cpu().numpy()
    dmu_g = d["dmu"].cpu().numpy()
    rho, ux, uy, es = inputs.energy_samples(77, n)
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    v2 = cx ** 2 + cy ** 2
    for i in range(n):
        fe = ora.feq_rho_u(ora.D2Q9, ora.EQ_ENTROPIC, rho[i], ux[i], uy[i])
        e2 = es[i] * float((fe * v2).sum())
        M = np.array([rho[i], rho[i] * ux[i], rho[i] * uy[i], e2])
        mu, it = ora.newton(ora.D2Q9, M)
        assert it >= 0
        mu, _ = ora.newton(ora.D2Q9, M, mu0=mu, tol=1e-15, maxit=2)
        assert np.abs(mu_g[i] - mu).max() <= 1e-10, (i, mu_g[i], mu)
        f = np.array([rho[i], ux[i], uy[i], e2 / rho[i] - ux[i] ** 2 - uy[i] ** 2], np.float32)
        assert np.all(np.abs(feat_g[i] - f) <= np.spacing(np.abs(f))), (i, feat_g[i], f)
        m0 = np.array([np.log(rho[i]) - 1.5 * (ux[i] ** 2 + uy[i] ** 2), 3 * ux[i], 3 * uy[i], 0.0])
        dm = mu - m0
        assert np.all(np.abs(dmu_g[i] - dm) <= 2e-10 + np.spacing(np.abs(dm).astype(np.float32))), i
    print("data set Newton: FP32 %.2f FP64 %.2f iterations per sample" % (it32 / n, it64 / n))


def test_forward_matches_oracle(env):
    torch, lbm = env
    n = 4096
    p = mlp_random_params(81)
    feat = mlp_random_features(82, n)
    y = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    pd, fd = dev(torch, p, np.float32), dev(torch, feat, np.float32)
    lbm.mlp_forward(pd.data_ptr(), fd.data_ptr(), n, y.data_ptr())
    torch.cuda.synchronize()
    yg = y.cpu().numpy().astype(np.float64)
    yo, c = omlp.forward(p, feat, round=True, band=BAND)
    amb = c["ambiguous"]
    d = omlp.unpack(p)
    mag = c["h2"] @ np.abs(omlp.bf16(d["W3"])).T + np.abs(d["b3"])
    ok = ~amb
    err = np.abs(yg - yo)[ok] / mag[ok]
    # every sample, the ambiguous ones included: inside the bounds of all
    # evaluations whose hidden sums stray by at most the band
    lo, hi = omlp.forward_bounds(p, feat, BAND)
    out = np.maximum(lo - yg, yg - hi) / mag
    width = (hi - lo) / mag
    print("forward: %d of %d samples ambiguous; max error / magnitude %.3g; all samples: "
          "worst excess over the bounds %.3g (interval width max %.3g, %d samples wider than 1e-5)"
          % (amb.sum(), n, err.max(), out.max(), width.max(), int(np.sum(width.max(1) > 1e-5))))
    assert amb.mean() < 0.3
    assert err.max() <= 1e-5
    assert out.max() <= 1e-5


def _clean_batch(p, seed, n):
    feat = mlp_random_features(seed, 2 * n)
    _, c = omlp.forward(p, feat, round=True, band=BAND)
    feat = feat[~c["ambiguous"]][:n]
    assert feat.shape[0] == n
    dmu = (0.05 * inputs.uniform(seed + 7, (n, 4))).astype(np.float32).astype(np.float64)
    return feat, dmu


def test_gradient_matches_oracle(env):
    torch, lbm = env
    n = 2000
    p = mlp_random_params(91)
    feat, dmu = _clean_batch(p, 92, n)
    grad = torch.zeros(omlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    pd, fd, dd = dev(torch, p, np.float32), dev(torch, feat, np.float32), dev(torch, dmu, np.float32)
    lbm.mlp_grad(pd.data_ptr(), fd.data_ptr(), dd.data_ptr(), n, grad.data_ptr(), loss.data_ptr())
    torch.cuda.synchronize()
    gg = grad.cpu().numpy().astype(np.float64)
    lo, go = omlp.loss_and_grad(p, feat, dmu, round=True)
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    gu, ou = omlp.unpack(gg), omlp.unpack(go)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        e = np.abs(gu[name] - ou[name]).max() / np.abs(ou[name]).max()
        print("grad %s: max error / max |g| = %.3g" % (name, e))
        assert e <= 1e-4, name
    assert np.linalg.norm(gg - go) <= 1e-5 * np.linalg.norm(go)
    assert not gg[omlp.N_PARAMS - 12:].any()


def test_adam_step_matches_oracle(env):
    torch, lbm = env
    P = omlp.N_PARAMS
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    p = f32(mlp_random_params(95))
    g = f32(inputs.uniform(96, (P,), -1e-2, 1e-2))
    m = f32(inputs.uniform(97, (P,), -1e-3, 1e-3))
    v = f32(inputs.uniform(98, (P,), 0.0, 1e-4))
    t, lr = 3, 2e-3
    tp, tg, tm, tv = (dev(torch, a, np.float32) for a in (p, g, m, v))
    lbm.mlp_adam(tp.data_ptr(), tg.data_ptr(), tm.data_ptr(), tv.data_ptr(), t, lr)
    torch.cuda.synchronize()
    po, mo, vo = omlp.adam_step(p, g, m, v, t, lr)
    tr = slice(0, P - 12)
    # FP32 evaluation of b1 m + (1 - b1) g: a few ulps of its terms
    assert (np.abs(tm.cpu().numpy()[tr] - mo[tr]) <= 2.0 ** -21 * (0.9 * np.abs(m) + 0.1 * np.abs(g))[tr]).all()
    assert np.allclose(tv.cpu().numpy()[tr], vo[tr], rtol=4e-7, atol=0)
    dp = np.abs(tp.cpu().numpy().astype(np.float64) - po)
    assert (dp <= 2.0 ** -22 * np.abs(po) + 1e-5 * lr).all(), dp.max()


def test_training_is_deterministic_and_learns(env):
    torch, lbm = env
    from paper_0705_4371_gb300 import learned
    a, ia = learned.train_energy_mlp(n=200_000, epochs=10, batch=4096)
    b, ib = learned.train_energy_mlp(n=200_000, epochs=10, batch=4096)
    assert np.array_equal(a, b)
    assert ia["losses"] == ib["losses"]
    print("losses per epoch", ia["losses"])
    assert ia["losses"][-1] < 0.1 * ia["losses"][0]
    assert np.isfinite(a).all()


def _energy_fields(w, seed, smooth=False):
    """rho, u of the cylinder recipe and 2E = isothermal 2E x a factor: a
    random U[0.9, 1.1] per site, or (smooth) 1 + 0.1 sin(2 pi y / ny)
    cos(2 pi x / nx) (the isothermal energy from the oracle's entropic
    equilibrium)."""
    cfg = oracle_cfg(w)
    rho, ux, uy = inputs.cylinder_fields(w, noise=1e-2)
    E = ora.moment_fields(cfg, ora.init_field(cfg, rho, ux, uy))[3]
    fac = inputs.energy_factor(w, smooth=True) if smooth else inputs.uniform(seed, E.shape, 0.9, 1.1)
    return rho, ux, uy, E * fac


def test_learned_run_matches_oracle(env, trained):
    # the warm start changes the Newton path, not its root: the learned run
    # follows the oracle's energy-form trajectory (replayed selection)
    torch, lbm = env
    params, _ = trained
    w = inputs.cylinder(200, 72, 8, 5000.0, delta=2e-6, k=16, eq=inputs.EQ_ENERGY)
    cfg = oracle_cfg(w)
    rho, ux, uy, e2 = _energy_fields(w, 101)
    f0 = ora.init_field(cfg, rho, ux, uy, e2)
    n = 100
    fo, log = ora.run(cfg, f0.copy(), n)
    ro, uo, vo, Eo = ora.moment_fields(cfg, fo)
    m = cfg.solid_mask()
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        g = lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[prec],
                                      equilibrium=lbm.LB_EQ_ENTROPIC_ENERGY_MLP)
        g.set_mlp(params)
        g.init_equilibrium(rho, ux, uy, e2)
        g.replay_selection(log.selected)
        g.step(n)
        g.sync()
        rg, ug, vg, Eg = g.moments()
        e_M, _, _ = moment_errors((rg, ug, vg), (ro, uo, vo), m, w.u_in[0])
        e_E = float(np.abs(Eg[~m] - Eo[~m]).max() / np.abs(Eo[~m]).max())
        it32, it64, sites, fails = g.newton_stats()
        print("learned form %s: M %.3g 2E %.3g; Newton FP32 %.2f FP64 %.2f per site"
              % (prec, e_M, e_E, it32 / sites, it64 / sites))
        assert fails == 0
        assert max(e_M, e_E) < tol, prec
        g.close()


def test_warm_start_gain(env, trained):
    # the same run with and without the network: the same f* (to the Newton
    # tolerance), fewer FP32 iterations with it
    torch, lbm = env
    params, _ = trained
    w = inputs.cylinder(512, 256, 16, 5000.0, k=0, eq=inputs.EQ_ENERGY)
    rho, ux, uy, e2 = _energy_fields(w, 102, smooth=True)
    stats, times, states = {}, {}, {}
    for name, eq in (("newton", lbm.LB_EQ_ENTROPIC_ENERGY), ("mlp", lbm.LB_EQ_ENTROPIC_ENERGY_MLP)):
        g = lbm.Lattice.from_workload(w, precision=lbm.LB_F32, equilibrium=eq)
        if eq == lbm.LB_EQ_ENTROPIC_ENERGY_MLP:
            g.set_mlp(params)
        g.init_equilibrium(rho, ux, uy, e2)
        g.newton_stats(reset=True)
        g.step(10)
        g.sync()
        stats[name] = g.newton_stats(reset=True)
        states[name] = g.get_state()
        g.set_timing(True)
        g.step(40)
        g.sync()
        ms = g.kernel_times(reset=True)
        times[name] = w.nx * w.ny * 40 / (ms["collide_ms"] * 1e-3) / 1e6
        g.close()
    per = {k: (s[0] / s[2], s[1] / s[2]) for k, s in stats.items()}
    print("Newton iterations per site (FP32, FP64): plain %.3f %.3f, warm-started %.3f %.3f"
          % (per["newton"] + per["mlp"]))
    print("MLUPS: plain %.0f, warm-started %.0f" % (times["newton"], times["mlp"]))
    assert stats["newton"][3] == 0 and stats["mlp"][3] == 0
    assert per["mlp"][0] <= 0.75 * per["newton"][0]
    assert per["mlp"][1] <= per["newton"][1] + 0.05
    assert rel_err(states["mlp"], states["newton"]) < 2e-6


def test_learned_run_needs_its_network(env):
    torch, lbm = env
    w = inputs.cylinder(64, 40, 6, 5000.0, eq=inputs.EQ_ENERGY)
    g = lbm.Lattice.from_workload(w, precision=lbm.LB_F32, equilibrium=lbm.LB_EQ_ENTROPIC_ENERGY_MLP)
    with pytest.raises(lbm.LBError) as e:
        g.step(1)
    assert e.value.code == lbm.LB_ERR_STATE
    bad = np.zeros(lbm.mlp_param_count(), np.float32)
    bad[5] = np.nan
    with pytest.raises(lbm.LBError) as e:
        g.set_mlp(bad)
    assert e.value.code == lbm.LB_ERR_ARG
    g.close()
