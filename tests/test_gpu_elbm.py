"""ELBM (elbmLB) on the GPU against the oracle, and the shock-tube figure
of Sec. 4.1 (nine panels: LBGK with polynomial or entropic f*, ELBM, each
without and with Ehrenfests' steps)."""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs
from tests._common import moment_errors, oracle_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_0705_4371_gb300 import lbm as m
    m.load()
    return m


@pytest.mark.parametrize("nu,reg", [(1.0 / 30.0, None), (1e-9, (4, 1e-4))])
def test_elbm_shock_tube_matches_oracle(lbm, nu, reg):
    k, delta = reg if reg else (0, 1e30)
    w = inputs.shock_tube(nu=nu, delta=delta, k=k, steps=400)
    cfg = oracle_cfg(w, elbm=True)
    rho, ux, _ = inputs.shock_tube_fields(w)
    f0 = ora.init_field(cfg, rho, ux)
    fo, log = ora.run(cfg, f0.copy(), 400)
    g = lbm.Lattice.from_workload(w, precision=lbm.LB_F64)
    g.set_collision(lbm.LB_COLLISION_ELBM)
    g.init_equilibrium(rho, ux)
    g.replay_selection(log.selected)
    g.step(400)
    g.sync()
    rg, ug, _, _ = g.moments()
    ro, uo, _, _ = ora.moment_fields(cfg, fo)
    e_rho = np.abs(rg - ro).max()
    e_u = np.abs(ug - uo).max()
    print("ELBM shock tube nu=%g: |d rho| %.3g |d u| %.3g, Ehrenfests' sites %d" % (nu, e_rho, e_u, log.counts.sum()))
    assert e_rho < 1e-12 and e_u < 1e-12


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_elbm_cylinder_matches_oracle(lbm, prec, tol):
    w = inputs.cylinder(200, 72, 8, 5000.0, delta=1e-5, k=16, eq=inputs.EQ_ENTROPIC)
    cfg = oracle_cfg(w, elbm=True)
    rho, ux, uy = inputs.cylinder_fields(w, noise=2e-2)
    f0 = ora.init_field(cfg, rho, ux, uy)
    n = 100
    fo, log = ora.run(cfg, f0.copy(), n)
    g = lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[prec])
    g.set_collision(lbm.LB_COLLISION_ELBM)
    g.init_equilibrium(rho, ux, uy)
    g.replay_selection(log.selected)
    g.step(n)
    g.sync()
    rg, ug, vg, _ = g.moments()
    ro, uo, vo, _ = ora.moment_fields(cfg, fo)
    e_M, _, _ = moment_errors((rg, ug, vg), (ro, uo, vo), cfg.solid_mask(), w.u_in[0])
    print("ELBM cylinder %s: e_M %.3g" % (prec, e_M))
    assert e_M < tol


def test_elbm_needs_the_entropic_equilibrium(lbm):
    w = inputs.cylinder(64, 40, 6, 1000.0, eq=inputs.EQ_POLY)
    g = lbm.Lattice.from_workload(w, precision=lbm.LB_F32)
    with pytest.raises(lbm.LBError) as e:
        g.set_collision(lbm.LB_COLLISION_ELBM)
    assert e.value.code == lbm.LB_ERR_ARG
    g.close()


def test_shock_tube_figure(lbm):
    # Sec. 4.1: at nu = 1e-9, LBGK (panels d, e) shows spurious post-shock
    # oscillations that Ehrenfests' steps (g, h; (k, delta) = (4, 1e-4)) subdue
    from paper_0705_4371_gb300 import experiments
    osc, sites = {}, {}
    for p in "abcdefghi":
        r, u, c = experiments.shock_panel(p)
        assert np.isfinite(r).all()
        osc[p] = experiments.oscillation(r)
        sites[p] = int(c.sum())
    print("excess total variation of rho: " + ", ".join("%s %.4f" % (p, osc[p]) for p in "abcdefghi"))
    print("Ehrenfests' sites over 400 steps: g %d h %d i %d" % (sites["g"], sites["h"], sites["i"]))
    assert osc["g"] < 0.5 * osc["d"]
    assert osc["h"] < 0.5 * osc["e"]
    assert osc["i"] <= osc["f"]
    assert max(osc["a"], osc["b"], osc["c"]) < osc["d"]     # high viscosity: smooth profiles
    assert sites["g"] > 0 and sites["h"] > 0 and sites["i"] > 0
