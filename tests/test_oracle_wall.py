"""Pins of the oracle's diffuse kinetic wall on the obstacle's faces (the
wall rule the paper leaves to the kinetic boundary conditions it cites in
Sec. 4.2): Maxwell's diffuse reflection on a wall at rest.  The properties
that define it are checked, not its formula: what the wall emits has the
shape of a rest quasiequilibrium (f_i / W_i the same on every wall link),
the wall is impermeable (it emits exactly what it absorbed), it emits no
tangential momentum, and every other link streams as before."""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs

CX, CY, W = ora.lattice_tables(ora.D2Q9)[:3]


def _box(nx=18, ny=14, obstacle=(6, 4, 4, 5), wall=ora.WALL_DIFFUSE, beta=0.0, k=0):
    # beta = 0, k = 0: the collision is the identity, so one step is pure
    # free flight with the boundary rules
    return ora.Config(ora.D2Q9, nx, ny, ora.EQ_POLY, beta, 1e30, k, (ora.BC_BB,) * 4,
                      obstacle=obstacle, wall=wall)


def _random_field(cfg, seed):
    f = 0.05 + inputs.uniform(seed, (9, cfg.ny, cfg.nx)) * 0.04 + 0.05
    f = f * W[:, None, None] * 9.0
    f[:, cfg.solid_mask()] = 0.0
    return np.ascontiguousarray(f)


def _wall_links(cfg, x, y):
    """Directions i whose source x - v_i lies in the obstacle (from the geometry)."""
    m = cfg.solid_mask()
    out = []
    for i in range(9):
        sx, sy = x - CX[i], y - CY[i]
        if 0 <= sx < cfg.nx and 0 <= sy < cfg.ny and m[sy, sx]:
            out.append(i)
    return out


def test_wall_emits_a_rest_quasiequilibrium_of_the_absorbed_mass():
    cfg_d = _box()
    cfg_b = _box(wall=ora.WALL_BOUNCE_BACK)
    fp = _random_field(cfg_d, 11)
    fd, _ = ora.run(cfg_d, fp.copy(), 1, log_selection=False)
    fb, _ = ora.run(cfg_b, fp.copy(), 1, log_selection=False)
    solid = cfg_d.solid_mask()
    seen = {1: 0, 2: 0, 3: 0}
    for y in range(cfg_d.ny):
        for x in range(cfg_d.nx):
            if solid[y, x]:
                continue
            B = _wall_links(cfg_d, x, y)
            other = [i for i in range(9) if i not in B]
            # every link that does not cross the obstacle's face streams as before
            assert np.array_equal(fd[other, y, x], fb[other, y, x])
            if not B:
                continue
            seen[len(B)] += 1
            # bounce-back returns f'_{-i}(x) on these links: the absorbed mass
            absorbed = fb[B, y, x].sum()
            assert fd[B, y, x].sum() == pytest.approx(absorbed, rel=1e-14)
            ratio = fd[B, y, x] / W[B]
            assert np.ptp(ratio) <= 1e-14 * ratio.max()
            if len(B) > 1:
                # the random field is not a rest quasiequilibrium: the rule acts
                assert np.abs(fd[B, y, x] - fb[B, y, x]).max() > 1e-6
    # faces (3 links), the sites next to a corner (2) and the convex corners (1)
    assert seen[3] > 0 and seen[2] == 8 and seen[1] == 4


def test_wall_emits_no_tangential_momentum():
    cfg = _box()
    fp = _random_field(cfg, 12)
    f, _ = ora.run(cfg, fp, 1, log_selection=False)
    x0, y0, w, h = cfg.obstacle
    checked = 0
    for y in range(cfg.ny):
        for x in range(cfg.nx):
            B = _wall_links(cfg, x, y)
            if len(B) != 3:
                continue
            # the face's normal is the common velocity component of its links
            vx, vy = CX[B], CY[B]
            tang = vy if np.all(vx == vx[0]) else vx
            assert abs((tang * f[B, y, x]).sum()) < 1e-16
            checked += 1
    assert checked == 2 * (w - 2) + 2 * (h - 2)


def test_closed_box_conserves_mass_with_the_diffuse_obstacle():
    cfg = _box(nx=32, ny=20, obstacle=(10, 7, 6, 5), beta=0.9)
    w = inputs.cylinder(32, 20, 6, 1000.0, delta=1e30, k=0)
    rho, ux, uy = inputs.cylinder_fields(w, noise=2e-2)
    f = ora.init_field(cfg, rho, ux, uy)
    f[:, cfg.solid_mask()] = 0.0
    m0 = f.sum()
    f, _ = ora.run(cfg, f, 300, log_selection=False)
    assert abs(f.sum() - m0) <= 1e-13 * m0
    # the diffuse wall takes momentum out of the flow (bounce-back too, but
    # differently): the two states part
    g = ora.init_field(cfg, rho, ux, uy)
    g[:, cfg.solid_mask()] = 0.0
    cfg_b = _box(nx=32, ny=20, obstacle=(10, 7, 6, 5), beta=0.9, wall=ora.WALL_BOUNCE_BACK)
    g, _ = ora.run(cfg_b, g, 300, log_selection=False)
    assert np.abs(f - g).max() > 1e-5


def test_rest_state_is_stationary():
    cfg = _box(nx=24, ny=16, obstacle=(8, 5, 5, 6), beta=0.97)
    f = ora.init_field(cfg, np.full((16, 24), 1.3), np.zeros((16, 24)), np.zeros((16, 24)))
    f0 = f.copy()
    f, _ = ora.run(cfg, f, 50, log_selection=False)
    assert np.abs(f - f0).max() < 1e-13   # round-off of the recomputed f* only


def test_mirror_symmetry_about_the_centreline():
    w = inputs.cylinder(64, 32, 8, 1000.0, delta=1e30, k=0, wall=inputs.WALL_DIFFUSE)
    assert w.obstacle[1] * 2 + w.obstacle[3] == w.ny
    cfg = ora.Config(w.lattice, w.nx, w.ny, w.eq, ora.beta_of_nu(w.nu), w.delta, w.k, w.bc,
                     w.rho_in, w.u_in, w.obstacle, wall=w.wall)
    f = ora.init_field(cfg, np.ones((32, 64)), np.full((32, 64), 0.05), np.zeros((32, 64)))
    f, _ = ora.run(cfg, f, 200, log_selection=False)
    r, u, v, _ = ora.moment_fields(cfg, f)
    assert np.abs(r - r[::-1]).max() < 1e-13
    assert np.abs(u - u[::-1]).max() < 1e-13
    assert np.abs(v + v[::-1]).max() < 1e-13
    assert np.abs(v).max() > 1e-4
