"""Writes the stored expected values of the 600 x 500 square-cylinder channel
(L = 20 with its upstream face at 5L, polynomial f*, free-slip walls,
zero-gradient outflow, u_inf = 0.05, delta = 1e-3, k = 16; probe at
(4L, -2L) from the cylinder centre, Sec. 4.2.1) from FP64 oracle runs only:

  re1000_probe    c2_re1000_probe.txt: u_x at the probe after every 20th of
                  the first 20000 steps at Re = 1000 (seeded 1e-4 inflow
                  noise).  The wake at this Re is aperiodic, and runs whose
                  arithmetic differs in rounding separate after about 5e4
                  steps; before that the trajectory is fixed.
  re150_strouhal  c2_re150_strouhal.txt: the Strouhal number of 1e5 steps at
                  Re = 150 (seeded 1e-2 noise to start the shedding), where
                  the wake sheds periodically; dominant frequency of the
                  final quarter with the oracle's own estimator.

    python tests/golden/make_c2_goldens.py re1000_probe     # minutes
    python tests/golden/make_c2_goldens.py re150_strouhal   # about half an hour on eight cores
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import core as ora  # noqa: E402
from oracle import strouhal as ost  # noqa: E402
from paper_0705_4371_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
PROBE_STEPS, PROBE_EVERY = 20000, 20
ST_STEPS, ST_NOISE = 100000, 1e-2


def oracle_run(w, steps, noise):
    cfg = ora.Config(w.lattice, w.nx, w.ny, w.eq, ora.beta_of_nu(w.nu), w.delta, w.k, w.bc,
                     w.rho_in, w.u_in, w.obstacle)
    rho, ux, uy = inputs.cylinder_fields(w, noise=noise)
    f = ora.init_field(cfg, rho, ux, uy)
    t0 = time.time()
    _, log = ora.run(cfg, f, steps, log_selection=False, probe=w.probe)
    return log, time.time() - t0


def re1000_probe():
    w = inputs.workload_c2(1000.0)
    log, sec = oracle_run(w, PROBE_STEPS, 1e-4)
    with open(os.path.join(HERE, "c2_re1000_probe.txt"), "w") as fh:
        fh.write("# u_x at the probe (4L, -2L) of %s after steps %d, %d, ... %d of the FP64 oracle's run\n"
                 "# (seeded 1e-4 inflow noise; Sec. 4.2.1 probe), written by tests/golden/make_c2_goldens.py;\n"
                 "# Ehrenfests' sites %d over the run; %.0f s on %d host threads\n"
                 % (w.name, PROBE_EVERY, 2 * PROBE_EVERY, PROBE_STEPS, int(log.counts.sum()), sec,
                    ora.num_threads()))
        for v in log.probe[PROBE_EVERY - 1::PROBE_EVERY]:
            fh.write("%.17g\n" % v)


def re150_strouhal():
    w = inputs.workload_c2(150.0)
    log, sec = oracle_run(w, ST_STEPS, ST_NOISE)
    st = ost.strouhal(log.probe, w.L, w.u_in[0])
    with open(os.path.join(HERE, "c2_re150_strouhal.txt"), "w") as fh:
        fh.write("# Strouhal number of the FP64 oracle's run of %s, %d steps, seeded %g inflow noise\n"
                 "# (Sec. 4.2.1 probe at (4L, -2L) from the cylinder centre, final quarter; oracle\n"
                 "# estimator), written by tests/golden/make_c2_goldens.py; %.0f s on %d host threads\n"
                 % (w.name, ST_STEPS, ST_NOISE, sec, ora.num_threads()))
        fh.write("%.8f\n" % st)
    print(st)


if __name__ == "__main__":
    parts = {"re1000_probe": re1000_probe, "re150_strouhal": re150_strouhal}
    for name in sys.argv[1:] or list(parts):
        parts[name]()
