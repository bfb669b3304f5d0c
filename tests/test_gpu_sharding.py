"""One run sharded in x, on the GPU: the slabs of a run (lb_set_slab ...
lb_slab_ghost) stepped together in one process (each kernel ordered by the
host; none waits for another) against the same run on one handle.  The
slabs' own columns and every step's selection must equal the unsharded
run's exactly: the per-site arithmetic is the same, the ghost columns carry
the neighbours' populations, and the merged candidates are the global
selection of Sec. 3.2."""
import numpy as np
import pytest

from paper_0705_4371_gb300 import inputs, sharding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_0705_4371_gb300 import lbm as m
    m.load()
    return m


@pytest.mark.parametrize("prec,nslabs", [("f64", 2), ("f32", 3), ("f32dev", 2), ("f16dev", 2)])
def test_slabs_step_like_one_run(lbm, prec, nslabs):
    # 328 x 150: staged tiles with ragged tails in each slab; Re 5000 and a
    # perturbed start put Ehrenfests' sites (more candidates than k) in every
    # step, some next to the slab boundaries
    w = inputs.cylinder(328, 150, 12, 5000.0, delta=1e-7, k=24)
    rho, ux, uy = inputs.cylinder_fields(w, noise=3e-2)
    P = lbm.PRECISIONS[prec]
    one = lbm.Lattice.from_workload(w, precision=P)
    one.init_equilibrium(rho, ux, uy)
    grp = sharding.SlabGroup(w, nslabs, P)
    grp.init_equilibrium(rho, ux, uy)
    steps = 50
    try:
        sels = grp.step(steps)
        total = 0
        for t in range(steps):
            one.step(1)
            ref = one.selected()
            assert np.array_equal(sels[t], ref), t
            total += len(ref)
        assert total > steps
        assert np.array_equal(grp.get_state(), one.get_state())
    finally:
        grp.close()
        one.close()


def test_slab_calls_are_checked(lbm):
    w = inputs.cylinder(200, 72, 8, 1000.0)
    slab = sharding.slab_plan(w.nx, 2, w.obstacle)[0]
    g = lbm.Lattice.from_workload(sharding.slab_workload(w, slab), precision=lbm.LB_F32_DEV)
    try:
        with pytest.raises(lbm.LBError):
            g.set_slab(1, 1, 0, w.nx)               # a ghost column on the grid's own edge
        g.set_slab(slab.ghost_left, slab.ghost_right, slab.x0, w.nx)
        g.init_equilibrium(*(sharding.local_field(a, slab) for a in inputs.cylinder_fields(w)))
        with pytest.raises(lbm.LBError) as e:
            g.step(1)                               # a slab steps through the slab calls
        assert e.value.code == lbm.LB_ERR_STATE
        with pytest.raises(lbm.LBError):
            g.slab_apply([])                        # nothing collided yet
        g.slab_collide()
        with pytest.raises(lbm.LBError):
            g.slab_collide()                        # the selection must be applied first
        g.slab_apply([])
        with pytest.raises(lbm.LBError):
            g.slab_ghost(0, 1, 0)                   # no neighbour on the left of slab 0
    finally:
        g.close()
