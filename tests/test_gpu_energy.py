"""GPU energy-constrained entropic quasiequilibrium (D2Q9, M = (rho, rho u, 2E),
(argmax) with the Lagrange form of Sec. 3.3) against the oracle's Newton solve.

The GPU eliminates the density multiplier by normalisation and solves for
the other three (FP32 iterations, FP64 final steps); the root is unique, so
the quasiequilibrium must agree with the oracle's to the Newton tolerance.
"""

import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs
from tests._common import oracle_cfg, rel_err, moment_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_0705_4371_gb300 import lbm as m
    m.load()
    return m


def energy_cylinder(nx=200, ny=72, L=8, re=5000.0, delta=1e-3, k=16):
    return inputs.cylinder(nx, ny, L, re, delta=delta, k=k, eq=inputs.EQ_ENERGY)


def energy_fields(w, seed, spread=0.1, noise=1e-2):
    """rho, u from the cylinder recipe and 2E = isothermal 2E x U[1-s, 1+s]."""
    rho, ux, uy = inputs.cylinder_fields(w, noise=noise)
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    e2 = np.zeros_like(rho)
    r = inputs.uniform(seed, rho.shape, 1 - spread, 1 + spread)
    for j in range(w.ny):
        for i in range(w.nx):
            fe = ora.feq_rho_u(ora.D2Q9, ora.EQ_ENTROPIC, rho[j, i], ux[j, i], uy[j, i])
            e2[j, i] = (fe * (cx ** 2 + cy ** 2)).sum() * r[j, i]
    return rho, ux, uy, e2


def test_energy_equilibrium_state_matches_oracle(lbm):
    w = energy_cylinder(nx=64, ny=40, L=6)
    cfg = oracle_cfg(w)
    rho, ux, uy, e2 = energy_fields(w, 11)
    fo = ora.init_field(cfg, rho, ux, uy, e2)
    for prec, tol in (("f64", 1e-12), ("f32", 2e-6)):
        g = lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[prec])
        g.init_equilibrium(rho, ux, uy, e2)
        fg = g.get_state()
        assert rel_err(fg, fo) < tol, prec
        r, u, v, E = g.moments()
        m = cfg.solid_mask()
        assert np.abs(E[~m] - e2[~m]).max() / e2[~m].max() < tol


def test_energy_delta_s_and_one_step_match_oracle(lbm):
    w = energy_cylinder(nx=64, ny=40, L=6)
    cfg = oracle_cfg(w)
    rho, ux, uy, e2 = energy_fields(w, 12)
    f0 = ora.init_field(cfg, rho, ux, uy, e2)
    f0 = f0 * (1 + 0.02 * inputs.uniform(13, f0.shape))
    f0[:, cfg.solid_mask()] = 0.0
    _, ds_o = ora.fields(cfg, f0)
    g = lbm.Lattice.from_workload(w, precision=lbm.LB_F64)
    g.set_state(f0)
    ds_g = g.delta_s()
    m = cfg.solid_mask()
    d = np.abs(ds_g[~m] - ds_o[~m])
    assert (d <= 1e-11 * np.abs(ds_o[~m]) + 1e-15).all(), d.max()
    fo, log = ora.run(cfg, f0.copy(), 3)
    g.step(3)
    assert rel_err(g.get_state(), fo) < 1e-12
    assert np.array_equal(g.selected(), log.selected[-1])
    it32, it64, sites, fails = g.newton_stats()
    assert sites > 0 and fails == 0


def test_isothermal_energy_reduces_to_product_form(lbm):
    # Given the isothermal energy of the product formula, the GPU Newton solve
    # must return the entropic product formula of Sec. 4.2 (energy multiplier
    # zero).  (The two schemes then evolve differently: the energy form
    # conserves 2E in the collision, the isothermal one relaxes it.)
    w = energy_cylinder(nx=64, ny=40, L=6)
    rho, ux, uy = inputs.cylinder_fields(w, noise=2e-2)
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    e2 = np.zeros_like(rho)
    for j in range(w.ny):
        for i in range(w.nx):
            fe = ora.feq_rho_u(ora.D2Q9, ora.EQ_ENTROPIC, rho[j, i], ux[j, i], uy[j, i])
            e2[j, i] = (fe * (cx ** 2 + cy ** 2)).sum()
    a = lbm.Lattice.from_workload(w, precision=lbm.LB_F64)
    a.init_equilibrium(rho, ux, uy, e2)        # Newton at the isothermal energy
    wp = inputs.cylinder(64, 40, 6, 5000.0, eq=inputs.EQ_ENTROPIC)
    b = lbm.Lattice.from_workload(wp, precision=lbm.LB_F64)
    b.init_equilibrium(rho, ux, uy)
    assert rel_err(a.get_state(), b.get_state()) < 1e-13


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_energy_run_replayed_selection(lbm, prec):
    w = energy_cylinder(re=5000.0, delta=2e-6, k=16)
    cfg = oracle_cfg(w)
    rho, ux, uy, e2 = energy_fields(w, 14, spread=0.05, noise=1e-3)
    f0 = ora.init_field(cfg, rho, ux, uy, e2)
    n = 200
    fo, log = ora.run(cfg, f0.copy(), n)
    g = lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[prec])
    g.init_equilibrium(rho, ux, uy, e2)
    g.replay_selection(log.selected)
    g.step(n)
    g.sync()
    ro, uo, vo, Eo = ora.moment_fields(cfg, fo)
    rg, ug, vg, Eg = g.moments()
    e_M, e_rho, e_u = moment_errors((rg, ug, vg), (ro, uo, vo), cfg.solid_mask(), w.u_in[0])
    m = cfg.solid_mask()
    e_E = float(np.abs(Eg[~m] - Eo[~m]).max() / np.abs(Eo[~m]).max())
    print("energy form %s after %d steps: M %.3g rho %.3g u %.3g 2E %.3g" % (prec, n, e_M, e_rho, e_u, e_E))
    tol = {"f64": 1e-12, "f32": 1e-5}[prec]
    assert max(e_M, e_E) < tol
    it32, it64, sites, fails = g.newton_stats()
    assert fails == 0
    print("Newton iterations per site: FP32 %.2f FP64 %.2f" % (it32 / sites, it64 / sites))


@pytest.mark.parametrize("prec", ["f32", "f16dev", "f64"])
def test_energy_tile_shapes_give_identical_results(lbm, prec):
    # the energy forms' register-fed shapes (0: 128 registers, 1: 64) and the
    # staged shapes 4 and 5 run the same per-site arithmetic; a noisy start puts
    # many sites near delta, so the pending lists fill and drain in the loop
    w = energy_cylinder(nx=328, ny=150, L=12, delta=1e-7, k=64)
    rho, ux, uy, e2 = energy_fields(w, 21, noise=2e-2)
    states = {}
    for shape in (0, 1, 4, 5):
        g = lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[prec])
        g.set_tile_shape(shape)
        g.init_equilibrium(rho, ux, uy, e2)
        g.step(12)
        states[shape] = (g.get_state(), g.counts(12))
        g.close()
    for shape in (1, 4):
        assert np.array_equal(states[0][0], states[shape][0]), shape
        assert np.array_equal(states[0][1], states[shape][1]), shape
    assert states[0][1].sum() > 0
