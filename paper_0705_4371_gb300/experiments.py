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
                 tail=0.25, stream=None, collision=lbm.LB_COLLISION_LBGK):
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
        if collision != lbm.LB_COLLISION_LBGK:
            g.set_collision(collision)
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


# The nine panels of the shock-tube figure (Sec. 4.1): (equilibrium,
# collision, nu, Ehrenfests' (k, delta) or None), 400 steps.
SHOCK_PANELS = {
    "a": (inputs.EQ_POLY, lbm.LB_COLLISION_LBGK, 1.0 / 30.0, None),
    "b": (inputs.EQ_ENTROPIC, lbm.LB_COLLISION_LBGK, 1.0 / 30.0, None),
    "c": (inputs.EQ_ENTROPIC, lbm.LB_COLLISION_ELBM, 1.0 / 30.0, None),
    "d": (inputs.EQ_POLY, lbm.LB_COLLISION_LBGK, 1e-9, None),
    "e": (inputs.EQ_ENTROPIC, lbm.LB_COLLISION_LBGK, 1e-9, None),
    "f": (inputs.EQ_ENTROPIC, lbm.LB_COLLISION_ELBM, 1e-9, None),
    "g": (inputs.EQ_POLY, lbm.LB_COLLISION_LBGK, 1e-9, (4, 1e-4)),
    "h": (inputs.EQ_ENTROPIC, lbm.LB_COLLISION_LBGK, 1e-9, (4, 1e-4)),
    "i": (inputs.EQ_ENTROPIC, lbm.LB_COLLISION_ELBM, 1e-9, (4, 1e-4)),
}


def shock_panel(name, steps=400, precision=lbm.LB_F64):
    """One panel: (rho, u, Ehrenfests' sites per step) after `steps` steps."""
    eq, coll, nu, reg = SHOCK_PANELS[name]
    k, delta = reg if reg else (0, 1e30)
    w = inputs.shock_tube(nu=nu, delta=delta, k=k, steps=steps, eq=eq)
    g = lbm.Lattice.from_workload(w, precision=precision)
    try:
        g.set_collision(coll)
        rho, ux, _ = inputs.shock_tube_fields(w)
        g.init_equilibrium(rho, ux)
        g.step(steps)
        g.sync()
        r, u, _, _ = g.moments()
        counts = g.counts(steps)
    finally:
        g.close()
    return r[0], u[0], counts


def oscillation(rho):
    """Total variation of rho in excess of that of a monotone profile with the
    same extremes (0 for a profile without spurious oscillations)."""
    rho = np.asarray(rho, np.float64)
    return float(np.abs(np.diff(rho)).sum() - (rho.max() - rho.min()))


# --------------------------------------------------------------------------
# Small cases for profiling (python -m paper_0705_4371_gb300.experiments ...)
# --------------------------------------------------------------------------

def energy_case(eq, steps=3, nx=512, ny=256, shape=None):
    """The energy-constrained cylinder (L = ny/16, Re 5000, k 64) with the
    smooth energy pattern, FP32 storage, `steps` directly launched steps; eq 3
    first trains a network on 2e6 samples; shape: tile shape (None: the
    default).  Prints the kernel time and Newton iterations."""
    w = inputs.cylinder(nx, ny, ny // 16, 5000.0, k=64, eq=inputs.EQ_ENERGY)
    rho, ux, uy = inputs.cylinder_fields(w, noise=1e-2)
    with lbm.Lattice.from_workload(w, precision=lbm.LB_F64) as iso:
        iso.init_equilibrium(rho, ux, uy)
        e2 = iso.moments()[3] * inputs.energy_factor(w)
    with lbm.Lattice.from_workload(w, precision=lbm.LB_F32, equilibrium=eq) as g:
        if eq == lbm.LB_EQ_ENTROPIC_ENERGY_MLP:
            from . import learned
            p, _ = learned.train_energy_mlp(n=2_000_000, epochs=10, batch=4096, lr0=2e-3, lr1=2e-5)
            g.set_mlp(p)
        if shape is not None:
            g.set_tile_shape(shape)
        g.init_equilibrium(rho, ux, uy, e2)
        g.set_timing(True)
        g.step(steps)
        g.sync()
        kt = g.kernel_times()
        s = g.newton_stats()
        print("energy case eq %d shape %d: %.4f ms per launch, FP32 / high-precision Newton iterations per site"
              " %.3f / %.3f" % (eq, g.info()["tile_shape"], kt["collide_ms"] / kt["collide_launches"], s[0] / s[2],
                               s[1] / s[2]))


def elbm_case(steps=44, nx=1024, ny=512, precision=lbm.LB_F32):
    """The entropic cylinder (L = ny/16, Re 20000, k 16) with the ELBM
    collision: 40 steps, then `steps - 40` directly launched (timed) steps.
    Prints the kernel time per step."""
    w = inputs.cylinder(nx, ny, ny // 16, 20000.0, eq=inputs.EQ_ENTROPIC)
    with lbm.Lattice.from_workload(w, precision=precision) as g:
        g.set_collision(lbm.LB_COLLISION_ELBM)
        g.init_equilibrium(*inputs.cylinder_fields(w, noise=1e-2))
        g.step(40)
        g.set_timing(True)
        g.step(max(1, steps - 40))
        g.sync()
        kt = g.kernel_times()
        ms = kt["collide_ms"] / kt["collide_launches"]
        print("elbm case %d x %d: %.4f ms per step, %.0f MLUPS" % (nx, ny, ms, w.n_sites / ms / 1e3))


def batch_case(nruns=24, steps=44, variant=0):
    """The first nruns runs of the 64-run batch (FP32 deviation storage):
    40 steps, then `steps - 40` directly launched (timed) steps."""
    ws = inputs.workload_c5()[:nruns]
    with lbm.Batch(ws, precision=lbm.LB_F32_DEV) as b:
        b.set_variant(variant)
        for r, w in enumerate(ws):
            b.run(r).init_equilibrium(*inputs.cylinder_fields(w))
        b.step(40)
        b.set_timing(True)
        b.step(max(1, steps - 40))
        b.sync()
        kt = b.kernel_times()
        print("batch case: %d runs, %d sites, %.4f ms per step" % (nruns, b.info()["sites"], kt["ms"] / kt["launches"]))


def paper_cylinder(re, k=10, delta=1e-3, wall=inputs.WALL_BOUNCE_BACK, steps=None, L=20,
                   eq=inputs.EQ_ENTROPIC, precision=lbm.LB_F32, collision=lbm.LB_COLLISION_LBGK):
    """The cylinder as Sec. 4.2 sets it up: 30L x 25L channel (600 x 500 at
    L = 20), cylinder centre at 10.5L, u_inf = 0.05, entropic f*, run to
    t_max = 1250 L / u_inf (5e5 steps at L = 20), zero-gradient outflow, the
    Strouhal number from the probe at (4L, -2L) over the final quarter."""
    w = inputs.cylinder(30 * L, 25 * L, L, re, k=k, delta=delta, eq=eq, face_x=10 * L,
                        outlet=inputs.BC_OUTLET_COPY, wall=wall)
    n = int(1250 * L / w.u_in[0]) if steps is None else steps
    r = cylinder_run(w, n, precision=precision, chunk=10000, collision=collision)
    r.pop("probe_tail", None)
    r.update({"wall": wall, "eq": eq, "L": L, "collision": collision})
    return r


# One-at-a-time changes of the 600 x 500 cylinder workload (L = 20, face at
# 5L, polynomial f*, zero-gradient outflow, bounce-back cylinder, k = 16,
# delta = 1e-3): the outlet rule (the paper's equilibrium outlet instead of
# the zero-gradient copy), the cylinder wall (diffuse kinetic wall), the
# quasiequilibrium (the entropic f* the paper's cylinder runs use), the
# cylinder position (face at 10L, the paper's centre at 10.5L), and the
# regulariser (k = L/2 = 10 as in the paper; or k = 100 with delta = 1e-4).
C2_VARIANTS = {
    "c2": {},
    "equilibrium_outlet": {"outlet": inputs.BC_OUTLET},
    "diffuse_wall": {"wall": inputs.WALL_DIFFUSE},
    "entropic_f": {"eq": inputs.EQ_ENTROPIC},
    "face_at_10L": {"face_x": 200},
    "k10": {"k": 10},
    "k100_delta1e-4": {"k": 100, "delta": 1e-4},
}


def c2_variant(re, name, steps=200000, precision=lbm.LB_F32):
    """One C2_VARIANTS case at Reynolds number re, run for `steps` steps or
    until non-finite."""
    kw = dict(outlet=inputs.BC_OUTLET_COPY)
    kw.update(C2_VARIANTS[name])
    w = inputs.cylinder(600, 500, 20, re, name="c2_%s_Re%g" % (name, re), **kw)
    r = cylinder_run(w, steps, precision=precision, chunk=10000)
    r.pop("probe_tail", None)
    r["variant"] = name
    return r


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="GPU cases: profiling cases of the learned and batched forms "
                                             "and of ELBM; the paper's cylinder runs")
    sub = ap.add_subparsers(dest="case", required=True)
    e = sub.add_parser("energy")
    e.add_argument("--eq", type=int, default=2)
    e.add_argument("--steps", type=int, default=3)
    e.add_argument("--nx", type=int, default=512)
    e.add_argument("--ny", type=int, default=256)
    e.add_argument("--shape", type=int, default=None)
    el = sub.add_parser("elbm")
    el.add_argument("--steps", type=int, default=44)
    el.add_argument("--nx", type=int, default=1024)
    el.add_argument("--ny", type=int, default=512)
    c = sub.add_parser("cylinder")
    c.add_argument("--re", type=float, nargs="+", default=[500.0, 1000.0, 2000.0, 5000.0, 10000.0, 20000.0])
    c.add_argument("--k", type=int, default=10)
    c.add_argument("--delta", type=float, default=1e-3)
    c.add_argument("--wall", choices=["bounce-back", "diffuse"], default="bounce-back")
    c.add_argument("--steps", type=int, default=None)
    c.add_argument("--collision", choices=["lbgk", "elbm"], default="lbgk")
    sh = sub.add_parser("shock")
    sh.add_argument("--steps", type=int, default=400)
    ab = sub.add_parser("c2ablation")
    ab.add_argument("--re", type=float, nargs="+", default=[5000.0, 20000.0])
    ab.add_argument("--steps", type=int, default=200000)
    b = sub.add_parser("batch")
    b.add_argument("--runs", type=int, default=24)
    b.add_argument("--steps", type=int, default=44)
    b.add_argument("--variant", type=int, default=0)
    a = ap.parse_args(argv)
    lbm.load()
    if a.case == "energy":
        energy_case(a.eq, a.steps, a.nx, a.ny, a.shape)
    elif a.case == "elbm":
        elbm_case(a.steps, a.nx, a.ny)
    elif a.case == "shock":
        # the nine panels of the Sec. 4.1 figure: excess total variation of rho
        # and Ehrenfests' sites over the run
        for name in sorted(SHOCK_PANELS):
            r, _, counts = shock_panel(name, a.steps)
            print("panel %s: excess TV of rho %.4f, Ehrenfests' sites %d" % (name, oscillation(r), int(counts.sum())))
    elif a.case == "c2ablation":
        import json
        for re in a.re:
            for name in C2_VARIANTS:
                print(json.dumps(c2_variant(re, name, a.steps)), flush=True)
    elif a.case == "cylinder":
        import json
        wall = inputs.WALL_DIFFUSE if a.wall == "diffuse" else inputs.WALL_BOUNCE_BACK
        for re in a.re:
            coll = lbm.LB_COLLISION_ELBM if a.collision == "elbm" else lbm.LB_COLLISION_LBGK
            print(json.dumps(paper_cylinder(re, a.k, a.delta, wall, a.steps, collision=coll)), flush=True)
    else:
        batch_case(a.runs, a.steps, a.variant)


if __name__ == "__main__":
    main()
