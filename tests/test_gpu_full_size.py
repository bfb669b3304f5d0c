"""Parity at the full size of the roofline workload (square cylinder
4096 x 2048, L = 128, Re = 20000, delta = 1e-3, k = 16) in the launch
configuration the benchmark times (default staged tile shape, steps replayed
as CUDA graphs of 32): the oracle takes whole steps of the full grid from
the GPU's exported state (OpenMP over the host cores, well under a second
per step), and the GPU replays the oracle's selections so that both sides
take the same Ehrenfests' steps.  A second threshold (delta = 1e-6) makes
the selection itself work at this size; the selected sets are compared
exactly."""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs
from tests._common import oracle_cfg, rel_err

pytestmark = pytest.mark.gpu

SPIN_UP = 200      # the benchmark's spin-up: leaves the equilibrium start
STEPS = 4


@pytest.fixture(scope="module")
def lbm():
    from paper_0705_4371_gb300 import lbm as m
    m.load()
    return m


def _spun_up(lbm, w, prec):
    g = lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[prec])
    assert g.info()["tile_shape"] == 4
    g.init_equilibrium(*inputs.cylinder_fields(w, noise=1e-2))
    g.step(SPIN_UP)
    g.sync()
    return g


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
@pytest.mark.parametrize("delta", [1e-3, 1e-6])
def test_full_size_steps_match_the_oracle(lbm, prec, tol, delta):
    w = inputs.workload_c3()
    w.delta = delta
    cfg = oracle_cfg(w)
    g = _spun_up(lbm, w, prec)
    try:
        f0 = g.get_state()                  # pre-collision populations, FP64
        fo, log = ora.run(cfg, f0.copy(), STEPS)
        # the GPU's own selection on the same state, then the oracle's replayed
        g.step(1)
        g.sync()
        if prec == "f64":
            assert np.array_equal(g.selected(), log.selected[0])
        g.set_state(f0)
        g.replay_selection(log.selected)
        g.step(STEPS)
        g.sync()
        fg = g.get_state()
        mask = cfg.solid_mask()
        e = rel_err(fg, fo, mask)
        print("full size %s delta %g: max |df| / max |f| %.3g, Ehrenfests' sites per step %s"
              % (prec, delta, e, list(log.counts)))
        assert e < tol
        if delta < 1e-4:
            assert log.counts.sum() > 0          # the regulariser acts
    finally:
        g.close()


def test_full_size_delta_s_matches_the_oracle(lbm):
    w = inputs.workload_c3()
    cfg = oracle_cfg(w)
    g = _spun_up(lbm, w, "f64")
    try:
        f0 = g.get_state()
        _, ds_o = ora.fields(cfg, f0)
        ds_g = g.delta_s()
        m = cfg.solid_mask()
        assert np.isnan(ds_g[m]).all()
        d = np.abs(ds_g[~m] - ds_o[~m])
        assert (d <= 1e-11 * np.abs(ds_o[~m]) + 1e-15).all(), d.max()
        # the candidates above delta agree as a set
        assert np.array_equal(np.flatnonzero(ds_g[~m] > w.delta), np.flatnonzero(ds_o[~m] > w.delta))
    finally:
        g.close()
