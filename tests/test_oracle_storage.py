"""Pins of the oracle's storage option (the precision form: populations held
in FP32, or as deviations f - W_i rho0 in FP32 or FP16).

The oracle computes in FP64 and rounds the post-collision populations to the
storage type once per step, before the free flight.  Pinned here against
what fixes it independently of the oracle's code: IEEE binary32 / binary16
rounding as numpy performs it, the order of the step (collide, store,
stream) composed from the oracle's separate collide and stream calls, and
the size of the resulting drift (at most half a storage ulp per population
per step).
"""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs
from tests._common import oracle_cfg, initial_fields


def _samples():
    g = inputs.SplitMix64(424242)
    x = (g.uniform(4000, -1.0, 1.0) * 2.0 ** np.round(g.uniform(4000, -30, 18))).tolist()
    # ties of both formats (halfway between neighbours), subnormals, overflow
    x += [1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11,
          2.0 ** -130, 3 * 2.0 ** -150, 2.0 ** -149 * 0.5, 2.0 ** -20, 3 * 2.0 ** -25,
          65504.0, 65519.9, 65520.0, 3.4028234663852886e38, -0.1, 0.0, -0.0]
    return np.array(x)


def test_round_f32_is_ieee_binary32():
    x = _samples()
    got = np.array([ora.round_f32(v) for v in x])
    want = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want)


def test_round_f16_is_ieee_binary16():
    x = _samples()
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    got = np.array([ora.round_f16(v) for v in x])
    assert np.array_equal(got, want)


def _weights(cfg):
    _, _, w = ora.lattice_tables(cfg.lattice)
    return w[:, None, None]


@pytest.mark.parametrize("store", [ora.STORE_F32, ora.STORE_F32_DEV, ora.STORE_F16_DEV])
def test_storage_rounds_post_collision_populations(store):
    # run(store) equals, step by step, collide -> round every fluid
    # population to the storage type -> stream, composed by hand
    w = inputs.cylinder(90, 40, 6, 2000.0, delta=1e-6, k=6)
    cfg = oracle_cfg(w)
    rho, ux, uy = initial_fields(w, noise=1e-3)
    f = ora.init_field(cfg, rho, ux, uy)
    _, log = ora.run(cfg, f.copy(), 6)
    W = _weights(cfg)
    fluid = ~cfg.solid_mask()
    fh = f.copy()
    for t in range(6):
        fp = ora.collide(cfg, fh, log.selected[t])
        if store == ora.STORE_F32:
            r = fp.astype(np.float32).astype(np.float64)
        elif store == ora.STORE_F32_DEV:
            r = W + (fp - W).astype(np.float32).astype(np.float64)
        else:
            r = W + (fp - W).astype(np.float16).astype(np.float64)
        fp = np.where(fluid[None], r, fp)
        fh = ora.stream(cfg, fp)
    fr, _ = ora.run(oracle_cfg(w, store=store), f.copy(), 6, replay=log.selected)
    assert np.array_equal(fr, fh)


@pytest.mark.parametrize("store,half_ulp", [(ora.STORE_F32_DEV, 2.0 ** -24 * 0.125),
                                            (ora.STORE_F16_DEV, 2.0 ** -11 * 0.125)])
def test_storage_drift_is_bounded_by_half_an_ulp_per_step(store, half_ulp):
    # closed box, no inflow: total mass moves only by the storage rounding,
    # at most half an ulp of each stored deviation (|g| < 1/8 here) per
    # population per step
    w = inputs.Workload("box", inputs.D2Q9, 40, 30, inputs.EQ_POLY, 1e-2, 1e-3, 4, 10,
                        (inputs.BC_BB,) * 4)
    cfg = oracle_cfg(w, store=store)
    rho, ux, uy = initial_fields(w, noise=1e-2)
    f0 = ora.init_field(cfg, rho, ux, uy)
    n = 20
    fr, _ = ora.run(cfg, f0.copy(), n)
    m0, m1 = f0.sum(), fr.sum()
    bound = n * 9 * cfg.n_sites * half_ulp
    assert abs(m1 - m0) <= bound
    assert abs(m1 - m0) > 0.0            # the rounding does act
    # FP64 storage conserves mass to round-off
    f64, _ = ora.run(oracle_cfg(w), f0.copy(), n)
    assert abs(f64.sum() - m0) < 1e-11
