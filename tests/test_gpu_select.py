"""GPU selection (block top-k + global radix select) against the oracle's
selection rule, bit-exact on the same dS arrays (Sec. 3.2)."""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_0705_4371_gb300 import lbm as m
    m.load()
    return m


CASES = [
    # n, k, n_ties, frac_inf, delta quantile (None: -1)
    (1, 1, 0, 0.0, None),
    (5, 3, 0, 0.0, 0.5),
    (12, 4, 3, 0.0, 0.2),
    (1000, 16, 0, 0.0, 0.5),
    (1023, 16, 50, 0.0, 0.1),
    (1024, 1024, 0, 0.0, None),
    (1025, 7, 0, 0.3, 0.5),
    (5000, 64, 400, 0.0, 0.0),
    (100000, 16, 0, 0.0, 0.9),
    (100000, 840, 10000, 0.05, 0.3),
    (300000, 4, 0, 0.0, 0.999),
    (300000, 9000, 0, 0.0, None),      # more candidates than shared-memory staging
    (2048, 3000, 0, 0.0, 0.5),         # k larger than the qualifying set
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_select_only_bit_exact(lbm, case):
    n, k, ties, finf, q = CASES[case]
    ds = inputs.random_ds_with_ties(1000 + case, n, n_ties=ties, frac_inf=finf)
    fin = ds[np.isfinite(ds)]
    delta = -1.0 if q is None else float(np.quantile(fin, q))
    got = lbm.select_only(ds, delta, k)
    ref = ora.select(ds, delta, k)
    assert np.array_equal(got, ref)


def test_select_only_all_equal_keys(lbm):
    ds = np.full(5000, 0.25)
    for k in (1, 17, 1024, 4999, 5000, 6000):
        assert np.array_equal(lbm.select_only(ds, 0.0, k), ora.select(ds, 0.0, k))


def test_select_only_strict_threshold(lbm):
    ds = np.array([1e-3, 2e-3, 1e-3, 5e-4, np.inf, 0.0])
    assert list(lbm.select_only(ds, 1e-3, 10)) == [1, 4]
    assert list(lbm.select_only(ds, 1e-3, 0)) == []


def test_select_only_empty_input(lbm):
    ds = np.zeros(0)
    for k in (0, 1, 16):
        assert lbm.select_only(ds, 0.0, k).size == 0
        assert ora.select(ds, 0.0, k).size == 0
