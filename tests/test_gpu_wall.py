"""The diffuse kinetic wall on the obstacle (LB_WALL_DIFFUSE) on the GPU:
element-by-element parity with the FP64 oracle, the same bits from every
tile shape and from the batched kernel, and the wall's impermeability."""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs
from tests._common import initial_fields, moment_errors, oracle_cfg, perturbed_state, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_0705_4371_gb300 import lbm as m
    m.load()
    return m


def diffuse_cylinder(re=20000.0, delta=2e-6, k=16, eq=inputs.EQ_POLY, outlet=inputs.BC_OUTLET_COPY,
                     nx=200, ny=72, L=8):
    # several 128 x 8 tiles with ragged tails; the cylinder's faces, the
    # sites beside its corners and its convex corners all inside staged tiles
    return inputs.cylinder(nx, ny, L, re, delta=delta, k=k, eq=eq, outlet=outlet,
                           wall=inputs.WALL_DIFFUSE)


@pytest.mark.parametrize("eq", [inputs.EQ_POLY, inputs.EQ_ENTROPIC])
def test_three_steps_fp64_match_the_oracle(lbm, eq):
    w = diffuse_cylinder(eq=eq, delta=1e-3)
    cfg = oracle_cfg(w)
    f0 = perturbed_state(cfg, w, seed=5, eps=0.02)
    g = lbm.Lattice.from_workload(w, precision=lbm.LB_F64)
    g.set_state(f0)
    fo, log = ora.run(cfg, f0.copy(), 3)
    g.step(3)
    g.sync()
    assert rel_err(g.get_state(), fo) < 1e-13
    assert np.array_equal(g.selected(), log.selected[-1])
    # the rule acts: bounce-back gives another state
    b = lbm.Lattice.from_workload(w, precision=lbm.LB_F64, wall=inputs.WALL_BOUNCE_BACK)
    b.set_state(f0)
    b.step(3)
    b.sync()
    assert rel_err(b.get_state(), fo) > 1e-6


TOL_M = {"f64": 1e-12, "f32": 1e-5}
TOL_U = {"f64": 1e-11, "f32": 2e-5}


@pytest.mark.parametrize("prec,re", [("f64", 20000.0), ("f32", 1000.0)])
def test_1000_steps_replayed_selection(lbm, prec, re):
    # the FP32 bounds are those of the bounce-back cylinder (storage rounding
    # over 1000 steps); the wall adds one division per wall site
    w = diffuse_cylinder(re=re)
    cfg = oracle_cfg(w)
    rho, ux, uy = initial_fields(w, noise=1e-3)
    fo, log = ora.run(cfg, ora.init_field(cfg, rho, ux, uy), 1000)
    assert log.counts.sum() > 100
    g = lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[prec])
    g.init_equilibrium(rho, ux, uy)
    g.replay_selection(log.selected)
    g.step(1000)
    g.sync()
    ro, uo, vo, _ = ora.moment_fields(cfg, fo)
    e_M, e_rho, e_u = moment_errors(g.moments()[:3], (ro, uo, vo), cfg.solid_mask(), w.u_in[0])
    print("diffuse wall, 1000 steps vs oracle %s Re %g: M %.3g rho %.3g u %.3g" % (prec, re, e_M, e_rho, e_u))
    assert e_M < TOL_M[prec] and e_rho < TOL_M[prec], (e_M, e_rho)
    assert e_u < TOL_U[prec], e_u


@pytest.mark.parametrize("prec", ["f32", "f16dev", "f64"])
@pytest.mark.parametrize("shape", [0, 2, 3, 4, 5, 6])
def test_tile_shapes_give_identical_results(lbm, shape, prec):
    w = inputs.cylinder(328, 150, 12, 20000.0, delta=1e-6, k=16, outlet=inputs.BC_OUTLET_COPY,
                        wall=inputs.WALL_DIFFUSE)
    rho, ux, uy = initial_fields(w, noise=1e-3)
    P = lbm.PRECISIONS[prec]
    ref = lbm.Lattice.from_workload(w, precision=P)
    ref.set_tile_shape(1)
    ref.init_equilibrium(rho, ux, uy)
    ref.step(50)
    g = lbm.Lattice.from_workload(w, precision=P)
    g.set_tile_shape(shape)
    g.init_equilibrium(rho, ux, uy)
    g.step(50)
    assert np.array_equal(ref.get_state(), g.get_state())
    assert np.array_equal(ref.counts(50), g.counts(50))


@pytest.mark.parametrize("variant", [0, 2])
def test_batch_equals_runs_stepped_alone(lbm, variant):
    ws = [diffuse_cylinder(re=1000.0, delta=1e-5, k=8),
          inputs.cylinder(300, 150, 10, 20000.0, delta=1e-4, k=16, wall=inputs.WALL_DIFFUSE),
          inputs.cylinder(130, 45, 6, 5000.0, delta=1e-6, k=4)]      # bounce-back beside them
    P = lbm.LB_F32_DEV
    b = lbm.Batch(ws, precision=P)
    b.set_variant(variant)
    alone = [lbm.Lattice.from_workload(w, precision=P) for w in ws]
    for r, w in enumerate(ws):
        f = inputs.cylinder_fields(w, noise=2e-2)
        b.run(r).init_equilibrium(*f)
        alone[r].init_equilibrium(*f)
    b.step(40)
    b.sync()
    for r, a in enumerate(alone):
        a.step(40)
        a.sync()
        assert np.array_equal(b.run(r).get_state(), a.get_state()), r
    b.close()
    for a in alone:
        a.close()


def test_closed_box_conserves_mass(lbm):
    w = inputs.Workload("box_diffuse", inputs.D2Q9, 131, 37, inputs.EQ_POLY, 1e-3, 1e-4, 8, 10,
                        (inputs.BC_BB,) * 4, obstacle=(40, 10, 9, 7), wall=inputs.WALL_DIFFUSE)
    cfg = oracle_cfg(w)
    f0 = perturbed_state(cfg, w, seed=9, eps=0.05)
    g = lbm.Lattice.from_workload(w, precision=lbm.LB_F64)
    g.set_state(f0)
    m0 = f0.sum()
    g.step(500)
    g.sync()
    assert abs(g.get_state().sum() - m0) <= 1e-12 * m0


def test_unknown_wall_rule_is_rejected(lbm):
    w = diffuse_cylinder()
    with pytest.raises(lbm.LBError) as e:
        lbm.Lattice.from_workload(w, precision=lbm.LB_F64, wall=7)
    assert e.value.code == lbm.LB_ERR_ARG
