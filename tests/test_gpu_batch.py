"""Batched form: many runs advanced together (the batched kernel, one launch
per step over every run's tiles, or every run's own kernel in concurrent
graph branches).  Each run of a batch must evolve exactly as the same run
stepped alone (same per-site arithmetic, same selection), for every storage
type and launch strategy, and replayed selections must reproduce the
oracle's trajectories."""
import ctypes as C
import json

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


def mixed_runs():
    # sizes with ragged last tiles in x (not a multiple of 128) and in y
    # (not a multiple of the tile rows), thresholds that make the selection work
    return [inputs.cylinder(200, 72, 8, 1000.0, delta=1e-5, k=8, name="b0"),
            inputs.cylinder(130, 45, 6, 5000.0, delta=1e-6, k=4, name="b1"),
            inputs.cylinder(300, 150, 10, 20000.0, delta=1e-4, k=16, name="b2"),
            inputs.cylinder(64, 40, 6, 200.0, delta=1e-7, k=32, name="b3"),
            inputs.cylinder(520, 257, 12, 3000.0, delta=1e-5, k=8, name="b4")]


@pytest.mark.parametrize("prec,variant", [("f32dev", 0), ("f32dev", 1), ("f32dev", 2), ("f16dev", 0),
                                          ("f16dev", 2), ("f64", 1), ("f32", 0)])
def test_batch_equals_runs_stepped_alone(lbm, prec, variant):
    ws = mixed_runs()
    P = lbm.PRECISIONS[prec]
    b = lbm.Batch(ws, precision=P)
    b.set_variant(variant)
    alone = [lbm.Lattice.from_workload(w, precision=P) for w in ws]
    for r, w in enumerate(ws):
        f = inputs.cylinder_fields(w, noise=2e-2)
        b.run(r).init_equilibrium(*f)
        alone[r].init_equilibrium(*f)
    n = 45   # the fresh first step, one graph of 32, 12 direct launches
    b.step(n)
    b.sync()
    for a in alone:
        a.step(n)
        a.sync()
    total_sel = 0
    for r in range(len(ws)):
        fb, fa = b.run(r).get_state(), alone[r].get_state()
        assert np.array_equal(fb, fa), "run %d differs (max %.3g)" % (r, np.abs(fb - fa).max())
        cb, ca = b.run(r).counts(n), alone[r].counts(n)
        assert np.array_equal(cb, ca), r
        assert np.array_equal(b.run(r).selected(), alone[r].selected()), r
        total_sel += int(cb.sum())
    assert total_sel > 0   # the selections were exercised
    info = b.info()
    assert info["variant"] == variant and info["runs"] == len(ws)
    assert info["sites"] == sum(w.nx * w.ny for w in ws)
    b.close()


def test_batch_replays_oracle_trajectories(lbm):
    ws = [inputs.cylinder(96, 40, 6, 1000.0, delta=1e-6, k=8, name="o0"),
          inputs.cylinder(150, 60, 8, 5000.0, delta=1e-6, k=4, name="o1")]
    b = lbm.Batch(ws, precision=lbm.LB_F64)
    n = 60
    refs = []
    for r, w in enumerate(ws):
        cfg = oracle_cfg(w)
        rho, ux, uy = inputs.cylinder_fields(w, noise=2e-2)
        f0 = ora.init_field(cfg, rho, ux, uy)
        fo, log = ora.run(cfg, f0.copy(), n)
        refs.append((cfg, fo))
        b.run(r).init_equilibrium(rho, ux, uy)
        b.run(r).replay_selection(log.selected)
    b.step(n)
    b.sync()
    for r, (cfg, fo) in enumerate(refs):
        rg, ug, vg, _ = b.run(r).moments()
        ro, uo, vo, _ = ora.moment_fields(cfg, fo)
        e_M, _, _ = moment_errors((rg, ug, vg), (ro, uo, vo), cfg.solid_mask(), ws[r].u_in[0])
        assert e_M < 1e-12, (r, e_M)
    b.close()


def test_batch_rejects_mixed_runs_and_separate_steps(lbm):
    L = lbm.load()
    ws = mixed_runs()[:2]
    descs = (lbm.lb_run_desc * 2)()
    for d, w, prec in zip(descs, ws, (lbm.LB_F32, lbm.LB_F64)):
        d.lattice, d.nx, d.ny, d.equilibrium = lbm.LB_D2Q9, w.nx, w.ny, lbm.LB_EQ_POLY
        d.nu, d.delta, d.k, d.precision = w.nu, w.delta, w.k, prec
        d.bc = lbm.boundaries(w.bc, w.rho_in, w.u_in, w.obstacle)
    h = C.c_void_p()
    assert L.lb_batch_create(descs, 2, None, C.byref(h)) == lbm.LB_ERR_ARG
    descs[1].precision = lbm.LB_F32
    descs[1].equilibrium = lbm.LB_EQ_ENTROPIC_ENERGY
    assert L.lb_batch_create(descs, 2, None, C.byref(h)) == lbm.LB_ERR_ARG
    b = lbm.Batch(ws, precision=lbm.LB_F32)
    for r, w in enumerate(ws):
        b.run(r).init_equilibrium(*inputs.cylinder_fields(w))
    b.step(2)
    b.run(0).step(1)     # one run stepped alone: the buffers are out of step
    with pytest.raises(lbm.LBError) as e:
        b.step(1)
    assert e.value.code == lbm.LB_ERR_STATE
    b.close()


def test_autotuner_times_variants_and_caches_the_choice(lbm, tmp_path):
    ws = mixed_runs()
    b = lbm.Batch(ws, precision=lbm.LB_F32_DEV)
    for r, w in enumerate(ws):
        b.run(r).init_equilibrium(*inputs.cylinder_fields(w))
    cache = str(tmp_path / "autotune.json")
    v = b.autotune(steps=5, cache_path=cache)
    assert v in (0, 1, 2) and b.info()["variant"] == v
    d = json.load(open(cache))
    assert len(d) == 1
    (key, entry), = d.items()
    assert entry["variant"] == v and len(entry["ms_per_step"]) == 3
    assert min(entry["ms_per_step"]) == entry["ms_per_step"][v]
    # a second batch of the same runs reads the cached choice
    b2 = lbm.Batch(ws, precision=lbm.LB_F32_DEV)
    b2.set_variant((v + 1) % 3)
    assert b2.autotune(steps=5, cache_path=cache) == v
    assert len(json.load(open(cache))) == 1
    # the timing steps were real steps: runs stay consistent with each other
    b.sync()
    b.step(3)
    b.sync()
    b.close()
    b2.close()
