"""Pins of the oracle's ELBM collision (elbmLB): alpha solves the
constant-entropy condition S(f + alpha (f* - f)) = S(f), nontrivial root."""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs


def _state(lattice, seed, eps):
    q = ora.q_of(lattice)
    if lattice == ora.D2Q9:
        base = ora.feq_rho_u(lattice, ora.EQ_ENTROPIC, 1.1, 0.06, -0.03)
    else:
        base = ora.feq_rho_u(lattice, ora.EQ_ENTROPIC, 0.9, 0.07)
    f = base * (1 + eps * inputs.uniform(seed, (q,)))
    M = ora.moments(lattice, f)
    uy = M[2] / M[0] if lattice == ora.D2Q9 else 0.0
    fs = ora.feq_rho_u(lattice, ora.EQ_ENTROPIC, M[0], M[1] / M[0], uy)
    return f, fs


@pytest.mark.parametrize("lattice", [ora.D1Q3, ora.D2Q9])
def test_entropy_is_constant_at_alpha(lattice):
    for seed in range(20):
        for eps in (1e-3, 0.05, 0.3):
            f, fs = _state(lattice, 100 + seed, eps)
            a = ora.elbm_alpha(lattice, f, fs)
            g = f + a * (fs - f)
            dS = ora.perfect_entropy(lattice, g) - ora.perfect_entropy(lattice, f)
            assert abs(dS) < 1e-13, (seed, eps, a, dS)
            # the nontrivial root: the entropy exceeds S(f) strictly inside (0, alpha)
            h = f + 0.5 * a * (fs - f)
            assert ora.perfect_entropy(lattice, h) > ora.perfect_entropy(lattice, f)
            assert a > 1.0


@pytest.mark.parametrize("lattice", [ora.D1Q3, ora.D2Q9])
def test_alpha_tends_to_lbgk_value_near_equilibrium(lattice):
    prev = None
    for eps in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        f, fs = _state(lattice, 7, eps)
        d = abs(ora.elbm_alpha(lattice, f, fs) - 2.0)
        if prev is not None:
            assert d < prev * 0.2      # first order in eps
        prev = d
    f, fs = _state(lattice, 7, 0.0)
    assert ora.elbm_alpha(lattice, f, fs) == 2.0     # f = f*: the LBGK value


def test_alpha_matches_a_brute_force_scan():
    # sign change of S(f + a D) - S(f) on a fine grid, evaluated directly
    lattice = ora.D2Q9
    for seed in range(5):
        f, fs = _state(lattice, 300 + seed, 0.4)
        D = fs - f
        amax = min(f[i] / -D[i] for i in range(9) if D[i] < 0)
        grid = np.linspace(1.0, min(amax, 4.0), 300001)
        S0 = ora.perfect_entropy(lattice, f)
        vals = np.array([ora.perfect_entropy(lattice, f + a * D) - S0 for a in grid[::100]])
        j = int(np.argmax(vals < 0))
        assert j > 0
        fine = grid[(j - 1) * 100:(j * 100) + 1]
        fv = np.array([ora.perfect_entropy(lattice, f + a * D) - S0 for a in fine])
        k = int(np.argmax(fv < 0))
        a = ora.elbm_alpha(lattice, f, fs)
        assert fine[k - 1] - 1e-12 <= a <= fine[k] + 1e-12


def test_positivity_limit():
    # a population far above its equilibrium: the entropy stays above S(f)
    # until f + a (f* - f) reaches the boundary of the positive cone
    lattice = ora.D1Q3
    f = np.array([0.02, 0.49, 0.49])   # rho = 1, u = 0; f* = (2/3, 1/6, 1/6)
    fs = ora.feq_rho_u(lattice, ora.EQ_ENTROPIC, 1.0, 0.0)
    D = fs - f
    amax = min(f[i] / -D[i] for i in range(3) if D[i] < 0)
    a = ora.elbm_alpha(lattice, f, fs)
    g = f + a * D
    S0 = ora.perfect_entropy(lattice, f)
    if a == amax:
        # on the boundary (one population zero up to rounding); the entropy
        # just inside it is still above S(f).  (The collision moves by
        # alpha beta < alpha, so its populations stay positive.)
        assert g.min() == pytest.approx(0.0, abs=1e-15)
        assert ora.perfect_entropy(lattice, f + a * (1 - 1e-9) * D) > S0
    else:
        assert abs(ora.perfect_entropy(lattice, g) - S0) < 1e-13
    assert 1.0 < a <= amax
    # outside the positive cone the solve reports -1
    assert ora.elbm_alpha(lattice, np.array([-0.1, 0.6, 0.5]), fs) == -1.0


def test_elbm_shock_tube_conserves_mass_and_stays_bounded():
    w = inputs.shock_tube(nu=1.0 / 30.0, delta=1e-4, k=4, steps=400)
    cfg = ora.Config(w.lattice, w.nx, w.ny, w.eq, ora.beta_of_nu(w.nu), w.delta, w.k, w.bc,
                     elbm=True)
    rho, ux, uy = inputs.shock_tube_fields(w)
    f = ora.init_field(cfg, rho, ux)
    m0 = f.sum()
    f, log = ora.run(cfg, f, 400)
    assert abs(f.sum() - m0) < 1e-11 * m0
    r, u, _, _ = ora.moment_fields(cfg, f)
    assert 0.45 < r.min() and r.max() < 1.05
