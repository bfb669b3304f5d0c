"""Writes c2_re1000_strouhal.txt: the Strouhal number of the FP64 oracle's
free run of the 600 x 500 square-cylinder channel (L = 20 with its upstream
face at 5L, polynomial f*, free-slip walls, zero-gradient outflow,
u_inf = 0.05 with seeded 1e-4 inflow noise, Re = 1000, delta = 1e-3, k = 16),
2e5 steps, probe at (4L, -2L) from the cylinder centre (Sec. 4.2.1), St from
the final quarter (the oracle's own estimator).  Uses the oracle only; takes
about an hour on eight host cores.

    python tests/golden/make_c2_strouhal.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import core as ora  # noqa: E402
from oracle import strouhal as ost  # noqa: E402
from paper_0705_4371_gb300 import inputs  # noqa: E402

STEPS = 200000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_re1000_strouhal.txt")


def main():
    w = inputs.workload_c2(1000.0)
    cfg = ora.Config(w.lattice, w.nx, w.ny, w.eq, ora.beta_of_nu(w.nu), w.delta, w.k, w.bc,
                     w.rho_in, w.u_in, w.obstacle)
    rho, ux, uy = inputs.cylinder_fields(w)
    f = ora.init_field(cfg, rho, ux, uy)
    t0 = time.time()
    f, log = ora.run(cfg, f, STEPS, log_selection=False, probe=w.probe)
    st = ost.strouhal(log.probe, w.L, w.u_in[0])
    with open(OUT, "w") as fh:
        fh.write("# Strouhal number of the FP64 oracle's free run of %s (Sec. 4.2.1 probe at (4L, -2L)\n"
                 "# from the cylinder centre, final quarter of %d steps; oracle estimator), written by\n"
                 "# tests/golden/make_c2_strouhal.py; Ehrenfests' sites %d over the run; %.0f s on %d host threads\n"
                 % (w.name, STEPS, int(log.counts.sum()), time.time() - t0, ora.num_threads()))
        fh.write("%.8f\n" % st)
    print(st)


if __name__ == "__main__":
    main()
