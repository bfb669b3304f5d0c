"""Pins of the oracle's time step (collision, free flight, boundary rules,
Ehrenfests' steps) against closed forms, invariants and special cases."""
import math
import os

import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cfg(w, beta=None, **kw):
    d = dict(lattice=w.lattice, nx=w.nx, ny=w.ny, eq=w.eq,
             beta=ora.beta_of_nu(w.nu) if beta is None else beta,
             delta=w.delta, k=w.k, bc=w.bc, rho_in=w.rho_in, u_in=w.u_in,
             obstacle=w.obstacle)
    d.update(kw)
    return ora.Config(**d)


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_free_flight_and_bounce_back_hand_example():
    # Pure free flight (beta = 0 makes the LBGK step the identity, Sec. 3 map
    # Theta_tau) on 5 D1Q3 sites with half-way bounce-back ends.  The golden
    # file holds the hand-derived populations after each step.
    g = _load_golden("d1q3_free_flight_5sites.txt")
    cfg = ora.Config(ora.D1Q3, 5, 1, ora.EQ_POLY, beta=0.0, delta=1e9, k=0)
    f = g[0:3].reshape(3, 1, 5).copy()
    for t in range(1, 5):
        f, _ = ora.run(cfg, f, 1)
        assert np.array_equal(f.reshape(3, 5), g[3 * t:3 * t + 3]), t


def test_shear_wave_decay_pins_beta_of_nu():
    # Transverse shear wave in a periodic box decays as exp(-nu k^2 t)
    # (incompressible Navier-Stokes limit); checks beta = 1/(1+6 nu).
    for nu in (0.02, 0.1):
        w = inputs.shear_wave(n=64, nu=nu, amp=1e-4, steps=300)
        cfg = _cfg(w)
        rho, ux, uy = inputs.shear_wave_fields(w)
        f = ora.init_field(cfg, rho, ux, uy)
        _, ux0, _, _ = ora.moment_fields(cfg, f)
        t = 300
        f, _ = ora.run(cfg, f, t, log_selection=False)
        _, ux1, _, _ = ora.moment_fields(cfg, f)
        mode = np.sin(2 * math.pi * np.arange(64) / 64)[:, None]
        a0 = (ux0 * mode).sum()
        a1 = (ux1 * mode).sum()
        kw = 2 * math.pi / 64
        assert abs(a1 / a0 / math.exp(-nu * kw * kw * t) - 1) < 0.01


def test_closed_box_conserves_mass_with_ehrenfest_steps():
    w = inputs.cylinder(40, 30, 6, 2000.0, delta=1e-9, k=5)
    cfg = _cfg(w, bc=(ora.BC_BB,) * 4)
    rho, ux, uy = inputs.cylinder_fields(w, noise=2e-2)
    f = ora.init_field(cfg, rho, ux, uy)
    m0 = f.sum()
    f, log = ora.run(cfg, f, 1000)
    assert log.counts.sum() > 0
    # round-off only: ~1e-16 per site update accumulates as a random walk
    # over 1e3 sites x 1e3 steps
    assert abs(f.sum() - m0) / m0 < 1e-12


def test_periodic_box_conserves_mass_and_momentum():
    cfg = ora.Config(ora.D2Q9, 24, 16, ora.EQ_POLY, beta=ora.beta_of_nu(1e-4), delta=1e-7, k=4,
                     bc=(ora.BC_PERIODIC,) * 4)
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    r = inputs.uniform(21, (3, 16, 24), -1, 1)
    f = ora.init_field(cfg, 1 + 0.05 * r[0], 0.05 * r[1], 0.05 * r[2])
    m0 = f.sum(); jx0 = (f * cx[:, None, None]).sum(); jy0 = (f * cy[:, None, None]).sum()
    f, log = ora.run(cfg, f, 1000)
    assert log.counts.sum() > 0
    assert abs(f.sum() - m0) / m0 < 1e-12
    assert abs((f * cx[:, None, None]).sum() - jx0) < 1e-12
    assert abs((f * cy[:, None, None]).sum() - jy0) < 1e-12


@pytest.mark.parametrize("eq", [ora.EQ_POLY, ora.EQ_ENTROPIC])
def test_collision_conserves_mass_momentum_per_site(eq):
    w = inputs.cylinder(30, 20, 4, 1000.0, eq=eq)
    cfg = _cfg(w, beta=0.97)
    rho, ux, uy = inputs.cylinder_fields(w, noise=5e-2)
    f = ora.init_field(cfg, rho, ux, uy)
    f *= 1 + 0.05 * inputs.uniform(22, f.shape)
    sel = [3, 77, 401]
    fp = ora.collide(cfg, f, sel)
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    for F in (f, fp):
        pass
    d_rho = np.abs(fp.sum(0) - f.sum(0)).max()
    d_jx = np.abs((fp * cx[:, None, None]).sum(0) - (f * cx[:, None, None]).sum(0)).max()
    d_jy = np.abs((fp * cy[:, None, None]).sum(0) - (f * cy[:, None, None]).sum(0)).max()
    assert max(d_rho, d_jx, d_jy) < 1e-15 * 8
    # Ehrenfests' step lands on the manifold: dS = 0 there
    fs2, ds2 = ora.fields(cfg, fp)
    for s in sel:
        assert abs(ds2.ravel()[s]) < 1e-15


def test_beta_half_everywhere_equals_ehrenfest_step_everywhere():
    # Sec. 3.2: beta = 1/2 makes the LBGK step land exactly on f*, i.e. an
    # Ehrenfests' step at every site.
    w = inputs.cylinder(32, 24, 4, 1000.0)
    cfg_lbgk = _cfg(w, beta=0.5, k=0, delta=1e9)
    cfg_ehr = _cfg(w, beta=0.5, k=w.n_sites, delta=-1.0)
    rho, ux, uy = inputs.cylinder_fields(w, noise=3e-2)
    f0 = ora.init_field(cfg_lbgk, rho, ux, uy) * (1 + 0.02 * inputs.uniform(23, (9, 24, 32)))
    a, _ = ora.run(cfg_lbgk, f0.copy(), 50, log_selection=False)
    b, log = ora.run(cfg_ehr, f0.copy(), 50)
    assert (log.counts == w.n_sites - 16).all()   # every fluid site selected
    assert np.abs(a - b).max() < 1e-14


def test_k_zero_is_plain_lbgk():
    w = inputs.cylinder(32, 24, 4, 5000.0)
    rho, ux, uy = inputs.cylinder_fields(w, noise=3e-2)
    c0 = _cfg(w, k=0, delta=1e-9)
    c1 = _cfg(w, k=7, delta=1e30)
    f0 = ora.init_field(c0, rho, ux, uy)
    a, la = ora.run(c0, f0.copy(), 40)
    b, lb = ora.run(c1, f0.copy(), 40)
    assert np.array_equal(a, b) and la.counts.sum() == 0 and lb.counts.sum() == 0


def test_uniform_flow_through_open_channel_stays_uniform():
    # Free-slip walls, free-stream inlet and either outlet (the quasiequilibrium
    # of the penultimate column, or the zero-gradient copy) preserve a uniform
    # free stream (no obstacle).
    for eq, outlet in ((ora.EQ_POLY, inputs.BC_OUTLET), (ora.EQ_ENTROPIC, inputs.BC_OUTLET),
                       (ora.EQ_POLY, inputs.BC_OUTLET_COPY), (ora.EQ_ENTROPIC, inputs.BC_OUTLET_COPY)):
        w = inputs.cylinder(48, 20, 4, 1000.0, eq=eq, outlet=outlet)
        cfg = _cfg(w, obstacle=(0, 0, 0, 0))
        rho = np.ones((20, 48)); ux = np.full((20, 48), 0.05); uy = np.zeros((20, 48))
        f = ora.init_field(cfg, rho, ux, uy)
        f0 = f.copy()
        f, _ = ora.run(cfg, f, 100)
        assert np.abs(f - f0).max() < 1e-13   # round-off of recomputed f* only


def test_mirror_symmetry_about_the_centreline():
    w = inputs.cylinder(64, 32, 8, 1000.0, delta=1e30, k=0)
    assert w.obstacle[1] * 2 + w.obstacle[3] == w.ny   # centred
    cfg = _cfg(w)
    rho, ux, uy = np.ones((32, 64)), np.full((32, 64), 0.05), np.zeros((32, 64))
    f = ora.init_field(cfg, rho, ux, uy)
    f, _ = ora.run(cfg, f, 200, log_selection=False)
    r, u, v, _ = ora.moment_fields(cfg, f)
    assert np.abs(r - r[::-1]).max() < 1e-13
    assert np.abs(u - u[::-1]).max() < 1e-13
    assert np.abs(v + v[::-1]).max() < 1e-13
    assert np.abs(v).max() > 1e-4   # the flow is not trivially symmetric


def test_equilibrium_start_selects_nothing_at_t0():
    w = inputs.cylinder(64, 32, 8, 20000.0, delta=1e-3, k=16)
    cfg = _cfg(w)
    f = ora.init_field(cfg, *inputs.cylinder_fields(w))
    _, ds = ora.fields(cfg, f)
    assert np.nanmax(np.abs(ds)) < 1e-15


def test_regulariser_damps_post_shock_oscillation():
    # Sec. 4.1: unregularised LBGK at nu = 1e-9 with polynomial equilibria
    # oscillates behind the shock; Ehrenfests' steps subdue it.
    w = inputs.shock_tube(eq=ora.EQ_POLY, delta=1e-4, k=4)
    rho, ux, _ = inputs.shock_tube_fields(w)
    res = {}
    for k in (0, 4):
        cfg = _cfg(w, k=k)
        f = ora.init_field(cfg, rho, ux)
        f, log = ora.run(cfg, f, 400)
        r, _, _, _ = ora.moment_fields(cfg, f)
        res[k] = (np.abs(np.diff(r[0])).sum(), log.counts)
    assert res[4][0] < 0.8 * res[0][0]           # total variation of rho
    assert res[4][1].max() <= 4 and res[4][1].sum() > 0


def test_zero_gradient_outlet_copies_the_outlet_column():
    # With the copy outlet, the populations entering the last column equal the
    # outgoing ones of that column one row along the population's direction:
    # a field that is uniform along x near the outlet (any profile in y) keeps
    # the last column's incoming populations equal to those of its neighbour
    # column, which also receives them from a column with the same values.
    w = inputs.cylinder(40, 16, 4, 1000.0, eq=ora.EQ_POLY, outlet=inputs.BC_OUTLET_COPY, delta=1e30, k=0)
    cfg = _cfg(w, obstacle=(0, 0, 0, 0), bc=(inputs.BC_PERIODIC, inputs.BC_PERIODIC, inputs.BC_FREESLIP,
                                                inputs.BC_FREESLIP))
    cfg_copy = _cfg(w, obstacle=(0, 0, 0, 0), bc=(inputs.BC_OUTLET_COPY, inputs.BC_OUTLET_COPY,
                                                     inputs.BC_FREESLIP, inputs.BC_FREESLIP))
    y = np.arange(16)[:, None]
    rho = np.ones((16, 40))
    ux = np.broadcast_to(0.03 + 0.02 * np.sin(2 * np.pi * y / 16), (16, 40)).copy()
    uy = np.zeros((16, 40))
    f = ora.init_field(cfg, rho, ux, uy)
    # x-independent fields: periodic wrap and zero-gradient copy see the same neighbours
    fa, _ = ora.run(cfg, f.copy(), 5, log_selection=False)
    fb, _ = ora.run(cfg_copy, f.copy(), 5, log_selection=False)
    assert np.abs(fa - fb).max() < 1e-15
    # a field that varies along x does see the difference at the ends only
    ux2 = ux * (1 + 0.1 * np.cos(2 * np.pi * np.arange(40)[None, :] / 40))
    f2 = ora.init_field(cfg, rho, ux2, uy)
    ga, _ = ora.run(cfg, f2.copy(), 1, log_selection=False)
    gb, _ = ora.run(cfg_copy, f2.copy(), 1, log_selection=False)
    d = np.abs(ga - gb).max(axis=(0, 1))
    assert d[0] > 0 and d[-1] > 0 and d[1:-1].max() == 0
