"""The paper's experiments (Sec. 4) on the GPU path: the square-cylinder wake
(Strouhal number from the velocity probe of Sec. 4.2.1; stability with and
without Ehrenfests' steps) and the shock tube of Sec. 4.1 (density and
velocity profiles).  Every step runs in liblbm's kernels; these functions
only drive runs and read their logs.
"""
import time

import numpy as np

from . import inputs, lbm, strouhal


def cylinder_run(w, steps, precision=lbm.LB_F32, k=None, delta=None, noise=1e-4, chunk=2000,
                 tail=0.25, stream=None):
    """Run the square-cylinder workload w for `steps` steps.  Returns a dict
    with the step at which the run became non-finite (None if it did not),
    the Strouhal number of the probe signal's final `tail` fraction (None if
    the run diverged), the mean number of Ehrenfests' sites per step, and the
    wall time."""
    over = {}
    if k is not None:
        over["k"] = k
    if delta is not None:
        over["delta"] = delta
    keep = max(1, int(round(steps * tail))) + 1
    out = {"workload": w.name, "steps": steps, "k": over.get("k", w.k), "delta": over.get("delta", w.delta),
           "re": w.L * w.u_in[0] / w.nu}
    g = lbm.Lattice.from_workload(w, precision=precision, stream=stream, **over)
    try:
        g.set_log_capacity(max(keep, min(steps, 65536)))
        g.set_probe(*w.probe)
        g.init_equilibrium(*inputs.cylinder_fields(w, noise=noise))
        t0 = time.perf_counter()
        done, diverged, sel = 0, None, []
        cap = max(keep, min(steps, 65536))
        while done < steps:
            n = min(chunk, steps - done)
            try:
                g.step(n)
                g.sync()
            except lbm.LBError as e:
                if e.code != lbm.LB_ERR_NONFINITE:
                    raise
                diverged = done + n
                break
            sel.append(g.counts(min(n, cap)))
            done += n
        out["seconds"] = time.perf_counter() - t0
        out["diverged_at"] = diverged
        out["selected_per_step"] = float(np.mean(np.concatenate(sel))) if sel else 0.0
        if diverged is None:
            sig = g.probe(keep - 1)
            out["strouhal"] = strouhal.strouhal(sig, w.L, w.u_in[0], tail=1.0)
            out["probe_tail"] = sig
        else:
            out["strouhal"] = None
    finally:
        g.close()
    return out


def shock_tube(w, steps=None, precision=lbm.LB_F64, k=None, delta=None, nu=None):
    """Shock tube of Sec. 4.1: returns (rho, u) after `steps` steps and the
    per-step Ehrenfests' counts."""
    over = {}
    for name, v in (("k", k), ("delta", delta), ("nu", nu)):
        if v is not None:
            over[name] = v
    n = w.steps if steps is None else steps
    g = lbm.Lattice.from_workload(w, precision=precision, **over)
    try:
        rho, ux, _ = inputs.shock_tube_fields(w)
        g.init_equilibrium(rho, ux)
        g.step(n)
        g.sync()
        r, u, _, _ = g.moments()
        counts = g.counts(min(n, 65536))
    finally:
        g.close()
    return r[0], u[0], counts
