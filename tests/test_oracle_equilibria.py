"""Pins of the oracle's lattices, quasiequilibria and energy Newton solve
against facts the paper and the mathematics fix (not against the oracle's
own formulas)."""
import math

import numpy as np
import pytest
from scipy import optimize

from oracle import core as ora
from paper_0705_4371_gb300 import inputs


# --- lattices (Sec. 4.1, Sec. 4.2) -------------------------------------------

def test_d2q9_velocities_follow_the_trigonometric_definition():
    # Sec. 4.2: v_0 = 0; v_i = (cos((i-1) pi/2), sin((i-1) pi/2)), i = 1..4;
    # v_i = sqrt2 (cos((i-5) pi/2 + pi/4), sin(...)), i = 5..8.
    cx, cy, w = ora.lattice_tables(ora.D2Q9)
    for i in range(9):
        if i == 0:
            v = (0.0, 0.0)
        elif i <= 4:
            a = (i - 1) * math.pi / 2
            v = (math.cos(a), math.sin(a))
        else:
            a = (i - 5) * math.pi / 2 + math.pi / 4
            v = (math.sqrt(2) * math.cos(a), math.sqrt(2) * math.sin(a))
        assert (cx[i], cy[i]) == (round(v[0]), round(v[1]))
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-17)


@pytest.mark.parametrize("lattice", [ora.D1Q3, ora.D2Q9])
def test_lattice_quadrature_moments(lattice):
    # Gauss-Hermite view (Sec. 2): sum W = 1, sum W v = 0, sum W v v = I/3.
    cx, cy, w = ora.lattice_tables(lattice)
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * cx).sum()) < 1e-16 and abs((w * cy).sum()) < 1e-16
    assert abs((w * cx * cx).sum() - 1 / 3) < 1e-15
    if lattice == ora.D2Q9:
        assert abs((w * cy * cy).sum() - 1 / 3) < 1e-15
        assert abs((w * cx * cy).sum()) < 1e-16
        # fourth moments of the Maxwellian with c_s^2 = 1/3: <vx^4> = 3/9, <vx^2 vy^2> = 1/9
        assert abs((w * cx ** 4).sum() - 1 / 3) < 1e-15
        assert abs((w * cx ** 2 * cy ** 2).sum() - 1 / 9) < 1e-15


def test_d1q3_order_is_rest_left_right():
    cx, _, w = ora.lattice_tables(ora.D1Q3)
    assert list(cx) == [0, -1, 1]          # {v1, v2, v3} = {0, -1, 1}, Sec. 4.1
    assert np.allclose(w, [2 / 3, 1 / 6, 1 / 6])


def _random_states(seed, n, umax=0.2):
    r = inputs.uniform(seed, (n, 3), 0.0, 1.0)
    rho = 0.5 + 1.5 * r[:, 0]
    ang = 2 * math.pi * r[:, 1]
    mag = umax * np.sqrt(r[:, 2])
    return rho, mag * np.cos(ang), mag * np.sin(ang)


# --- polynomial quasiequilibria ------------------------------------------------

def test_poly_d2q9_matches_maxwellian_moments_to_second_order():
    # The polynomial quasiequilibrium is defined by matching the moments of the
    # Maxwellian (Sec. 3.3): rho, rho u, and the pressure tensor rho u u + rho/3 I.
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    for rho, ux, uy in zip(*_random_states(1, 50)):
        fs = ora.feq_rho_u(ora.D2Q9, ora.EQ_POLY, rho, ux, uy)
        assert abs(fs.sum() - rho) <= 1e-15 * rho * 4
        assert abs((fs * cx).sum() - rho * ux) <= 1e-15 * 4
        assert abs((fs * cy).sum() - rho * uy) <= 1e-15 * 4
        assert abs((fs * cx * cx).sum() - (rho * ux * ux + rho / 3)) < 1e-14
        assert abs((fs * cy * cy).sum() - (rho * uy * uy + rho / 3)) < 1e-14
        assert abs((fs * cx * cy).sum() - rho * ux * uy) < 1e-14


def test_poly_d1q3_is_the_one_dimensional_restriction():
    # Sec. 4.1 prints f1* = 2rho/3 (1 - 3u^2/2), f2,3* = rho/6 (1 -/+ 3u + 3u^2);
    # mass, momentum and 2E = rho (1/3 + u^2) follow.
    for rho, ux, _ in zip(*_random_states(2, 30)):
        fs = ora.feq_rho_u(ora.D1Q3, ora.EQ_POLY, rho, ux)
        assert abs(fs.sum() - rho) < 1e-15 * 4
        assert abs(fs[2] - fs[1] - rho * ux) < 1e-15 * 4
        assert abs(fs[1] + fs[2] - rho * (1 / 3 + ux * ux)) < 1e-15 * 4


# --- entropic quasiequilibria ------------------------------------------------

def _maxent_d1q3_bisection(rho, u):
    """Maximise H-entropy of Sec. 4.1 on the constraint line by solving the
    stationarity condition with a bracketing root finder."""
    j = rho * u
    # parametrise by f1: f2 = (rho - f1 - j)/2, f3 = (rho - f1 + j)/2
    def dS(f1):
        f2 = (rho - f1 - j) / 2
        f3 = (rho - f1 + j) / 2
        return -math.log(f1 / 4) + 0.5 * (math.log(f2) + math.log(f3))
    hi = rho - abs(j)
    f1 = optimize.brentq(dS, 1e-300, hi * (1 - 1e-15), xtol=1e-17, rtol=9e-16, maxiter=500)
    return np.array([f1, (rho - f1 - j) / 2, (rho - f1 + j) / 2])


def test_entropic_d1q3_is_the_maxent_point():
    for rho, ux, _ in zip(*_random_states(3, 40, umax=0.5)):
        fs = ora.feq_rho_u(ora.D1Q3, ora.EQ_ENTROPIC, rho, ux)
        ref = _maxent_d1q3_bisection(rho, ux)
        assert np.allclose(fs, ref, rtol=1e-13, atol=0)


def test_entropic_d1q3_conservation_and_label_reading():
    # momentum must be +rho u (the printed labels give -rho u, see the reading)
    for rho, ux, _ in zip(*_random_states(4, 40, umax=0.5)):
        fs = ora.feq_rho_u(ora.D1Q3, ora.EQ_ENTROPIC, rho, ux)
        assert abs(fs.sum() - rho) < 4e-15 * rho
        assert abs(fs[2] - fs[1] - rho * ux) < 4e-15
        # MaxEnt with H = f1 log(f1/4) + f2 log f2 + f3 log f3: ln f_i/W_i is
        # linear in v_i, hence f2 f3 = (f1 / 4)^2.
        assert abs(fs[1] * fs[2] - (fs[0] / 4) ** 2) < 1e-15


def test_entropic_agrees_with_poly_to_second_order():
    # both match rho, rho u and the second moment at u -> 0: difference O(u^3)
    for lattice in (ora.D1Q3, ora.D2Q9):
        prev = None
        for u in (0.08, 0.04, 0.02, 0.01):
            a = ora.feq_rho_u(lattice, ora.EQ_ENTROPIC, 1.0, u, 0.3 * u if lattice else 0.0)
            b = ora.feq_rho_u(lattice, ora.EQ_POLY, 1.0, u, 0.3 * u if lattice else 0.0)
            d = np.abs(a - b).max()
            if prev is not None:
                # halving u divides the gap by >= 8: agreement through O(u^2)
                assert prev / d > 6.0
            prev = d


def test_entropic_d2q9_is_tensor_product_of_d1q3():
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    cx1, _, _ = ora.lattice_tables(ora.D1Q3)
    pos = {v: i for i, v in enumerate(cx1)}
    for rho, ux, uy in zip(*_random_states(5, 30, umax=0.3)):
        fs = ora.feq_rho_u(ora.D2Q9, ora.EQ_ENTROPIC, rho, ux, uy)
        gx = ora.feq_rho_u(ora.D1Q3, ora.EQ_ENTROPIC, 1.0, ux)
        gy = ora.feq_rho_u(ora.D1Q3, ora.EQ_ENTROPIC, 1.0, uy)
        for i in range(9):
            assert abs(fs[i] - rho * gx[pos[cx[i]]] * gy[pos[cy[i]]]) <= 1e-15 * rho


def test_entropic_d2q9_is_the_maxent_point():
    # Brute-force MaxEnt (argmax) by minimising the convex dual with a generic
    # optimiser, independent of the closed form of Sec. 4.2.
    cx, cy, w = ora.lattice_tables(ora.D2Q9)
    m = np.stack([np.ones(9), cx, cy])
    for rho, ux, uy in zip(*_random_states(6, 10, umax=0.3)):
        M = np.array([rho, rho * ux, rho * uy])
        phi = lambda mu: (w * np.exp(mu @ m)).sum() - mu @ M
        grad = lambda mu: m @ (w * np.exp(mu @ m)) - M
        hess = lambda mu: (m * (w * np.exp(mu @ m))) @ m.T
        res = optimize.minimize(phi, np.zeros(3), jac=grad, hess=hess, method="trust-exact")
        sol = optimize.root(grad, res.x, jac=hess, method="hybr", options={"xtol": 1e-15})
        ref = w * np.exp(sol.x @ m)
        fs = ora.feq_rho_u(ora.D2Q9, ora.EQ_ENTROPIC, rho, ux, uy)
        assert np.allclose(fs, ref, rtol=1e-11, atol=0)


# --- energy-constrained quasiequilibrium (Newton) ------------------------------

def test_newton_isothermal_energy_reproduces_product_form():
    # With 2E equal to the isothermal energy of the product form, the energy
    # multiplier vanishes and f* is the closed form of Sec. 4.2.
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    for rho, ux, uy in zip(*_random_states(7, 40, umax=0.2)):
        fe = ora.feq_rho_u(ora.D2Q9, ora.EQ_ENTROPIC, rho, ux, uy)
        e2 = (fe * (cx ** 2 + cy ** 2)).sum()
        mu, it = ora.newton(ora.D2Q9, [rho, rho * ux, rho * uy, e2])
        assert it >= 0
        assert abs(mu[3]) < 1e-12
        fs = ora.equilibrium(ora.D2Q9, ora.EQ_ENERGY, [rho, rho * ux, rho * uy, e2])
        assert np.allclose(fs, fe, rtol=1e-12, atol=0)


def test_newton_d1q3_energy_is_determined_by_moments():
    # Three populations and three constraints: f0 = rho - 2E, f+- = (2E +- j)/2.
    g = inputs.uniform(8, (40, 3), 0.0, 1.0)
    for a, b, c in g:
        rho = 0.5 + 1.5 * a
        u = 0.4 * (b - 0.5)
        e2 = rho * (u * u + 1 / 3) * (0.9 + 0.2 * c)
        fs = ora.equilibrium(ora.D1Q3, ora.EQ_ENERGY, [rho, rho * u, 0.0, e2])
        ref = np.array([rho - e2, (e2 - rho * u) / 2, (e2 + rho * u) / 2])
        assert np.allclose(fs, ref, rtol=1e-12, atol=0)


def test_newton_converges_on_training_distribution_and_root_is_unique():
    cx, cy, _ = ora.lattice_tables(ora.D2Q9)
    r = inputs.uniform(9, (200, 4), 0.0, 1.0)
    for a, b, c, d in r:
        rho = 0.5 + 1.5 * a
        ang, mag = 2 * math.pi * b, 0.2 * math.sqrt(c)
        ux, uy = mag * math.cos(ang), mag * math.sin(ang)
        fe = ora.feq_rho_u(ora.D2Q9, ora.EQ_ENTROPIC, rho, ux, uy)
        e2 = (fe * (cx ** 2 + cy ** 2)).sum() * (0.9 + 0.2 * d)
        Mn = [rho, rho * ux, rho * uy, e2]
        mu, it = ora.newton(ora.D2Q9, Mn)
        assert 0 <= it <= 30
        fs = ora.equilibrium(ora.D2Q9, ora.EQ_ENERGY, [rho, rho * ux, rho * uy, e2])
        M = np.array([fs.sum(), (fs * cx).sum(), (fs * cy).sum(), (fs * (cx ** 2 + cy ** 2)).sum()])
        assert np.abs(M - Mn).max() / rho <= 1e-12
        # a distant start point lands on the same multipliers (strict convexity)
        mu2, it2 = ora.newton(ora.D2Q9, Mn, mu0=mu + np.array([0.3, -0.2, 0.2, 0.4]))
        assert it2 >= 0 and np.allclose(mu2, mu, rtol=0, atol=1e-10)
        # warm start at the solution needs no iteration
        _, it3 = ora.newton(ora.D2Q9, Mn, mu0=mu)
        assert it3 == 0
