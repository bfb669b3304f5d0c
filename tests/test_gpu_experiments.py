"""Long runs against the oracle (Sec. 4): the Strouhal number of the
square-cylinder wake (Sec. 4.2.1; probe at (4L, -2L) from the centre, the
dominant frequency of the final 25 % of u_x) must agree within 1 %, in FP64
and FP32 storage.  The runs are free (no replayed selection): the two
trajectories drift apart at round-off level, the shedding frequency must not.
"""
import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs, strouhal
from tests._common import oracle_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_0705_4371_gb300 import lbm as m
    m.load()
    return m


@pytest.fixture(scope="module")
def oracle_strouhal():
    # 30L x 15L channel, L = 8, Re = 200: periodic (laminar) shedding, so the
    # frequency is sharply defined (at Re ~ 1000 in this small channel the wake
    # sheds irregularly and the estimate itself varies by a few per cent with
    # the window).  Inflow noise 1e-2 starts the shedding early; 40000 steps
    # leave about ten periods in the final quarter.
    w = inputs.cylinder(240, 120, 8, 200.0)
    steps = 40000
    cfg = oracle_cfg(w)
    rho, ux, uy = inputs.cylinder_fields(w, noise=1e-2)
    f0 = ora.init_field(cfg, rho, ux, uy)
    _, log = ora.run(cfg, f0, steps, log_selection=False, probe=w.probe)
    assert np.isfinite(log.probe).all()
    return w, steps, strouhal.strouhal(log.probe, w.L, w.u_in[0])


@pytest.mark.parametrize("prec", ["f64", "f32", "f32dev"])
def test_strouhal_matches_oracle(lbm, oracle_strouhal, prec):
    from paper_0705_4371_gb300 import experiments
    w, steps, st_o = oracle_strouhal
    r = experiments.cylinder_run(w, steps, precision=lbm.PRECISIONS[prec], noise=1e-2, chunk=4000)
    assert r["diverged_at"] is None
    st_g = r["strouhal"]
    print("Strouhal %s: GPU %.5f oracle %.5f (%.3f %%)" % (prec, st_g, st_o, 100 * abs(st_g - st_o) / st_o))
    assert abs(st_g - st_o) <= 0.01 * st_o
    assert 0.1 < st_o < 0.3   # a shedding wake, not a start-up transient


def test_shock_tube_runner_conserves_mass(lbm):
    from paper_0705_4371_gb300 import experiments
    w = inputs.shock_tube()
    rho, u, counts = experiments.shock_tube(w)
    assert abs(rho.sum() - 0.75 * w.nx) < 1e-9 * w.nx
    assert counts.size == w.steps and counts.max() <= w.k


def test_paper_cylinder_setup_runs(lbm):
    # the Sec. 4.2 layout at L = 8 (240 x 200), a short run of each collision
    from paper_0705_4371_gb300 import experiments
    for coll in (lbm.LB_COLLISION_LBGK, lbm.LB_COLLISION_ELBM):
        r = experiments.paper_cylinder(1000.0, k=4, delta=1e-4, steps=3000, L=8, collision=coll)
        assert r["diverged_at"] is None and r["steps"] == 3000
        assert r["collision"] == coll and r["strouhal"] is not None


def test_plain_lbgk_diverges_where_ehrenfests_steps_keep_the_run(lbm):
    # Sec. 4.2, end of the cylinder results: at L = 20 plain LBGK diverges
    # near Re = 1000, while a handful of Ehrenfests' steps per time step keep
    # the same run finite.  The paper's layout (30L x 25L, cylinder centre at
    # 10.5L, entropic f*, zero-gradient outflow), FP32 storage, 30000 steps.
    from paper_0705_4371_gb300 import experiments
    plain = experiments.paper_cylinder(1000.0, k=0, steps=30000)
    reg = experiments.paper_cylinder(1000.0, k=10, delta=1e-3, steps=30000)
    print("Re 1000, L 20: plain LBGK non-finite by step %s; with Ehrenfests' steps %s (%.2f sites per step)"
          % (plain["diverged_at"], reg["diverged_at"], reg["selected_per_step"]))
    assert plain["diverged_at"] is not None
    assert reg["diverged_at"] is None and reg["selected_per_step"] > 0


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as fh:
        return np.array([float(ln) for ln in fh if ln.strip() and not ln.startswith("#")])


def test_c2_re1000_probe_follows_the_oracle_trajectory(lbm):
    # The 600 x 500 channel of the cylinder workload (L = 20 at 5L,
    # polynomial f*, zero-gradient outflow, Re = 1000, k = 16, delta = 1e-3).
    # Its wake is aperiodic: the dominant frequency of the probe signal moves
    # between spectral peaks from one window to the next (the oracle's own
    # estimate over 25000-step windows ranges 0.05-0.26), so two runs agree
    # on a Strouhal number only by chance, and runs whose rounding differs
    # separate after about 5e4 steps.  Before that the trajectory is fixed:
    # the FP64 GPU run's probe u_x over the first 2e4 steps against the FP64
    # oracle's (tests/golden/c2_re1000_probe.txt, every 20th step), within
    # 1e-8 u_inf.
    from paper_0705_4371_gb300 import experiments
    ref = _golden("c2_re1000_probe.txt")
    w = inputs.workload_c2(1000.0)
    r = experiments.cylinder_run(w, 20000, precision=lbm.LB_F64, chunk=5000, tail=1.0)
    got = r["probe_tail"][19::20]
    assert got.shape == ref.shape
    err = np.abs(got - ref).max() / w.u_in[0]
    print("c2 Re 1000 FP64 probe, 2e4 steps: max |du| / u_inf = %.2e" % err)
    assert err <= 1e-8


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c2_re150_strouhal_matches_the_oracle_run(lbm, prec):
    # The same channel at Re = 150, where the wake sheds periodically: the
    # Strouhal number of the GPU's free run of 1e5 steps (seeded 1e-2 inflow
    # noise) against the FP64 oracle's (tests/golden/c2_re150_strouhal.txt),
    # within 1 %
    from paper_0705_4371_gb300 import experiments
    st_o = float(_golden("c2_re150_strouhal.txt")[0])
    w = inputs.workload_c2(150.0)
    r = experiments.cylinder_run(w, 100000, precision=lbm.PRECISIONS[prec], noise=1e-2, chunk=20000)
    assert r["diverged_at"] is None
    print("c2 Re 150 Strouhal %s: GPU %.5f oracle %.5f (%.3f %%)"
          % (prec, r["strouhal"], st_o, 100 * abs(r["strouhal"] - st_o) / st_o))
    assert abs(r["strouhal"] - st_o) <= 0.01 * st_o
