"""Pins of the oracle's entropies (PerfEnt, DelS) and of the Ehrenfests'
site selection (Sec. 3.2) against invariants and brute force."""
import itertools
import math

import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs


def _near_eq_states(seed, n, lattice, eq, eps=0.05, umax=0.15):
    r = inputs.uniform(seed, (n, 3), 0.0, 1.0)
    q = 3 if lattice == ora.D1Q3 else 9
    pert = inputs.uniform(seed + 1000, (n, q), -1.0, 1.0)
    out = []
    for (a, b, c), p in zip(r, pert):
        rho = 0.5 + 1.5 * a
        ang, mag = 2 * math.pi * b, umax * math.sqrt(c)
        ux, uy = mag * math.cos(ang), (mag * math.sin(ang) if lattice else 0.0)
        fs = ora.feq_rho_u(lattice, eq, rho, ux, uy)
        out.append(fs * (1 + eps * p))
    return out


@pytest.mark.parametrize("lattice", [ora.D1Q3, ora.D2Q9])
@pytest.mark.parametrize("eq", [ora.EQ_POLY, ora.EQ_ENTROPIC])
def test_delta_s_is_nonnegative_gibbs(lattice, eq):
    # dS = sum f ln(f/f*) with sum f = sum f* is a Kullback divergence >= 0.
    for f in _near_eq_states(11, 300, lattice, eq, eps=0.2):
        fs = ora.equilibrium(lattice, eq, ora.moments(lattice, f))
        assert ora.delta_s(lattice, f, fs) >= -1e-15 * f.sum()


@pytest.mark.parametrize("lattice", [ora.D1Q3, ora.D2Q9])
def test_delta_s_equals_entropy_gap_for_entropic_equilibrium(lattice):
    # (DelS): for the entropic f* with m(f) = m(f*), S(f*) - S(f) with the
    # perfect entropy (PerfEnt) equals sum f ln(f/f*).
    for f in _near_eq_states(12, 200, lattice, ora.EQ_ENTROPIC, eps=0.1):
        fs = ora.equilibrium(lattice, ora.EQ_ENTROPIC, ora.moments(lattice, f))
        gap = ora.perfect_entropy(lattice, fs) - ora.perfect_entropy(lattice, f)
        ds = ora.delta_s(lattice, f, fs)
        assert abs(ds - gap) < 2e-14 * max(1.0, f.sum())
        assert gap >= -1e-15   # the Ehrenfests' step raises the perfect entropy


def test_delta_s_second_order_limit():
    # Near equilibrium dS -> sum (f - f*)^2 / (2 f*) (Taylor of x ln x).
    f0 = ora.feq_rho_u(ora.D2Q9, ora.EQ_POLY, 1.1, 0.05, -0.02)
    p = inputs.uniform(13, (9,), -1, 1)
    p -= p.mean()  # keep mass fixed to first order
    for eps in (1e-2, 1e-3):
        f = f0 * (1 + eps * p)
        fs = ora.equilibrium(ora.D2Q9, ora.EQ_POLY, ora.moments(ora.D2Q9, f))
        ds = ora.delta_s(ora.D2Q9, f, fs)
        quad = ((f - fs) ** 2 / (2 * fs)).sum()
        assert abs(ds / quad - 1) < 20 * eps


def test_delta_s_zero_on_equilibrium_and_inf_outside_cone():
    fs = ora.feq_rho_u(ora.D2Q9, ora.EQ_POLY, 1.0, 0.1, 0.05)
    assert abs(ora.delta_s(ora.D2Q9, fs, fs)) == 0.0
    f = fs.copy()
    f[3] = -1e-6
    assert ora.delta_s(ora.D2Q9, f, fs) == math.inf
    g = fs.copy()
    g[0] = 0.0   # 0 ln 0 = 0
    assert math.isfinite(ora.delta_s(ora.D2Q9, g, fs))


# --- selection -------------------------------------------------------------------

def _brute_force_select(ds, delta, k, eligible=None):
    """Enumerate every subset of the qualifying sites of the right size and
    keep the one whose dS multiset is largest (ties to lower indices)."""
    n = len(ds)
    cand = [i for i in range(n) if (eligible is None or eligible[i]) and ds[i] > delta]
    m = min(k, len(cand))
    best, best_key = None, None
    for sub in itertools.combinations(cand, m):
        # lexicographic key: sorted dS descending, then indices ascending
        key = (sorted((ds[i] for i in sub), reverse=True), [-i for i in sorted(sub)])
        if best_key is None or key > best_key:
            best, best_key = sub, key
    return np.array(sorted(best), dtype=np.int64)


@pytest.mark.parametrize("seed", range(40))
def test_select_matches_brute_force_on_tiny_inputs(seed):
    r = inputs.uniform(100 + seed, (4,), 0.0, 1.0)
    n = 1 + int(r[0] * 12)
    k = int(r[1] * 7)
    ds = inputs.random_ds_with_ties(200 + seed, n, n_ties=int(r[2] * 4),
                                    frac_inf=0.2 if seed % 5 == 0 else 0.0)
    if seed % 3 == 0:
        ds = np.round(ds * 1e3) / 1e3  # many exact ties
    fin = ds[np.isfinite(ds)]
    delta = float(np.quantile(fin, r[3])) if (seed % 4 and fin.size) else -1.0
    elig = None
    if seed % 7 == 0:
        elig = (inputs.uniform(300 + seed, (n,), 0, 1) > 0.3).astype(np.uint8)
    got = ora.select(ds, delta, k, elig)
    ref = _brute_force_select(ds, delta, k, elig)
    assert np.array_equal(got, ref)


def test_select_takes_all_when_fewer_than_k_qualify_and_is_strict():
    ds = np.array([0.5, 1e-3, 2e-3, 0.0, 1e-3])
    assert list(ora.select(ds, 1e-3, 10)) == [0, 2]       # strict dS > delta
    assert list(ora.select(ds, 1e-3, 1)) == [0]
    assert list(ora.select(ds, -1.0, 3)) == [0, 1, 2]     # ties 1e-3 at 1 and 4: lower index
    assert list(ora.select(ds, 0.0, 0)) == []
