"""Throughput of the Ehrenfest-regularised D2Q9 step on one GB300 (or N
replicas), printed as one JSON line.

Workload (default): square cylinder of side L = 128 in a 4096 x 2048
free-slip channel, Re = 20000, inflow u = 0.05 with seeded 1e-4 noise,
polynomial equilibrium, delta = 1e-3, k = 16, populations stored as FP32
deviations f - W_i rho0 (the precision workload's storage).  One bench step
= one lattice time step of the whole hot path in one launch: pull-stream +
collide + dS + each block's k best candidates, then, in the launch's last
block, the global select + Ehrenfests' step.  The forms beside it: plain
FP32 and FP16 deviation storage on the same grid, every site a candidate
(delta < 0), the 600 x 500 channel, the learned and the batched forms.

  python bench.py [--steps K] [--warmup W] [--precision f32|f32dev|f16dev|f64]
  python bench.py --impl reference     # the FP64 CPU oracle as the reference arm
  torchrun --nproc-per-node N bench.py --gpus N   # N independent replicas
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0705_4371_gb300 import inputs  # noqa: E402

METRIC = ("D2Q9 MLUPS incl. Ehrenfest filter, % HBM roofline; chosen vs plain at equal error")
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "source": "fallback"}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_collide_d2q9_cylinder4096x2048.md")
GRAPH_STEPS = 32   # steps per CUDA graph of the library (lb_step)


def warm_graphs(h):
    """Untimed: have the run capture its CUDA graphs for both buffer parities
    (lb_step builds a graph the first time it needs one), so that no capture
    falls inside a timed region."""
    h.set_timing(False)
    for _ in range(2):
        h.step(2 * GRAPH_STEPS)
        h.step(1)
    h.sync()


SPACER_CYCLES = 1_000_000   # about 0.5 ms of device time at 2 GHz


def device_spacer(stream):
    """Untimed, inside the synchronised brackets: a sleep kernel on the
    timed stream, so that the device is still busy while the host enqueues
    the first event and the timed launches, and the first event is stamped
    when the device can start the first step, not while it waits for the
    host's first submission (tens of microseconds through ctypes)."""
    import torch
    with torch.cuda.stream(stream):
        torch.cuda._sleep(SPACER_CYCLES)


def timed_steps(h, stream, n):
    """Milliseconds of n steps through the library's own path (CUDA graphs of
    programmatically dependent launches; direct launches for a remainder
    below a graph), CUDA events on the run's stream."""
    import torch
    h.set_timing(False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    device_spacer(stream)
    e0.record(stream)
    h.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    h.sync()
    return e0.elapsed_time(e1)


def bracketed_launch_ms(h, n):
    """Mean duration of n stream-collide launches each bracketed by its own
    pair of CUDA events (direct launches: the events keep a launch from
    overlapping the previous one's end)."""
    h.set_timing(True)
    h.step(3)
    h.sync()
    h.kernel_times(reset=True)
    h.step(n)
    h.sync()
    k = h.kernel_times(reset=True)
    h.set_timing(False)
    return k["collide_ms"] / max(k["collide_launches"], 1)


def kernel_source_hash():
    """Hash of the sources that decide the single-run stream-collide launch's
    DRAM traffic: the device headers and instantiation units the kernels are
    compiled from, and the host API (which sets the tile shape and the tiles'
    claim order); not the batched kernel's header, which they do not include."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0705_4371_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name == "lbm_batch_kernels.cuh":
            continue
        if name.endswith((".cuh", ".h")) or name == "lbm_api.cu" or \
                (name.startswith("lbm_kernels_") and name.endswith(".cu")):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    return h.hexdigest()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return {"hbm_gbs": float(p["hbm_gbs"]), "source": "measured"}
    return dict(PEAKS_FALLBACK)


def traffic_per_launch(precision, n_sites):
    """DRAM bytes per launch of the stream-collide kernel from the committed
    ncu summary (its traffic_per_site line), scaled to n_sites; None if absent
    or if the CUDA sources changed since the counters were taken."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    s = None
    with open(PROFILE_SUMMARY) as fh:
        for line in fh:
            if line.startswith("traffic_per_site:"):
                s = json.loads(line.split(":", 1)[1])
    if not s or s.get("source_sha256") != kernel_source_hash():
        return None
    e = s.get("precisions", {}).get(precision)
    if not e:
        return None
    return int(e["dram_bytes_per_site"] * n_sites)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.2)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        sm, mx, pw = [], [], []
        for r in rows:
            try:
                sm.append(float(r[1])); mx.append(float(r[2])); pw.append(float(r[3]))
            except ValueError:
                pass
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_by_name(name):
    table = {"c3": inputs.workload_c3, "c3_scaled": inputs.workload_c3_scaled,
             "c2": inputs.workload_c2}
    if name in table:
        return table[name]()
    raise SystemExit("unknown workload %s" % name)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def run_gpu(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_0705_4371_gb300 import lbm
    lbm.load()
    w = workload_by_name(args.workload)
    prec = lbm.PRECISIONS[args.precision]
    stream = torch.cuda.Stream()
    g = lbm.Lattice.from_workload(w, precision=prec, stream=stream.cuda_stream)
    if args.tile_shape >= 0:
        g.set_tile_shape(args.tile_shape)
    rho, ux, uy = inputs.cylinder_fields(w)
    g.init_equilibrium(rho, ux, uy)
    info = g.info()
    n_sites = w.n_sites

    # spin-up (untimed): leave the equilibrium start so the regulariser works;
    # then the graphs the timed steps use, and the warm-up steps
    g.step(args.spinup)
    warm_graphs(g)
    g.step(args.warmup)
    g.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        barrier()
        device_spacer(stream)
        ev0.record(stream)
        g.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    g.sync()
    ms = ev0.elapsed_time(ev1)
    launches = args.steps * info["launches_per_step"]
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    counts = g.counts(min(args.steps, 65536))
    value = world * n_sites * args.steps / (ms * 1e-3) / 1e6
    # one launch per step: the timed region's time per launch is the launches'
    # average duration, inter-launch gaps included (an upper bound)
    coll_ms = ms / launches
    bracketed_ms = bracketed_launch_ms(g, min(args.steps, 200)) if rank == 0 else None
    alg_bytes = info["bytes_per_site"] * n_sites
    peaks = load_peaks()
    achieved = alg_bytes / (coll_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": traffic_per_launch(args.precision, n_sites),
                "kernel": "k_collide_d2q9", "algorithmic_bytes_per_site": info["bytes_per_site"],
                "avg_launch_ms": round(coll_ms, 5),
                "avg_launch_ms_source": "timed region / launches (one launch per step, gaps included)",
                "event_bracketed_launch_ms": round(bracketed_ms, 5) if bracketed_ms else None,
                "step_frac_of_peak": round(alg_bytes * args.steps / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                "peak_source": peaks["source"] + " hbm_gbs",
                "frac_of_nominal_8TBps": round(achieved / 8000.0, 4)}

    # e2e through the public C ABI with host buffers: each step uploads the
    # populations from pinned host memory, advances one step, and reads the
    # moments back to pinned host memory, queued as a serving loop does
    # (lb_set_state_async, lb_step, lb_moments_async: a step's upload
    # overlaps the previous step's download); the timed region ends when the
    # last step's moments are on the host (lb_sync).
    f_host = torch.from_numpy(g.get_state()).pin_memory().numpy()
    outs = [torch.empty((w.ny, w.nx), dtype=torch.float64).pin_memory().numpy() for _ in range(4)]
    import ctypes as C
    lib = lbm.load()

    def e2e_step():
        lbm._check(lib.lb_set_state_async(g.h, lbm._ptr(f_host)))
        lbm._check(lib.lb_step(g.h, 1))
        lbm._check(lib.lb_moments_async(g.h, *(lbm._ptr(o) for o in outs)))

    g.set_timing(False)
    for _ in range(2):
        e2e_step()
    lbm._check(lib.lb_sync(g.h))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    lbm._check(lib.lb_sync(g.h))
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": round(world * n_sites * args.e2e_steps / e2e_s / 1e6, 2), "unit": "MLUPS",
           "h2d_bytes_per_step": int(f_host.nbytes),
           "d2h_bytes_per_step": int(sum(o.nbytes for o in outs)),
           "steps": args.e2e_steps,
           "api": "per step lb_set_state_async(host f64) + lb_step(1) + lb_moments_async(host); "
                  "lb_sync after the last"}

    # forms beside the headline (same workload, same timing method)
    forms = {}
    if args.forms and rank == 0:
        for fname in ("f32", "f32dev", "f16dev"):
            if fname == args.precision:
                continue
            with lbm.Lattice.from_workload(w, precision=lbm.PRECISIONS[fname],
                                           stream=stream.cuda_stream) as h2:
                h2.init_equilibrium(rho, ux, uy)
                h2.step(args.spinup)
                warm_graphs(h2)
                h2.step(args.warmup)
                h2.sync()
                fms = timed_steps(h2, stream, args.form_steps)
                inf2 = h2.info()
                cms = fms / (args.form_steps * inf2["launches_per_step"])
                ach = inf2["bytes_per_site"] * n_sites / (cms * 1e-3) / 1e9
                forms[fname] = {"MLUPS": round(n_sites * args.form_steps / (fms * 1e-3) / 1e6, 1),
                                "ms_per_step": round(fms / args.form_steps, 5),
                                "collide_GBps": round(ach, 1),
                                "collide_frac": round(ach / peaks["hbm_gbs"], 4),
                                "bytes_per_site": inf2["bytes_per_site"]}

    if args.forms and rank == 0:
        forms["select_stress"] = select_stress_form(args, stream, w)
        forms["c2"] = c2_form(args, stream)
    if args.forms and args.learned and rank == 0:
        forms["learned"] = learned_form(args, stream)
    if args.forms and args.batched:
        bf = batched_form(args, stream, peaks, world, rank)   # every rank takes its share of the runs
        if rank == 0:
            forms["batched"] = bf

    cpu = cpu_baseline(w, args) if (rank == 0 and world == 1 and not args.no_cpu) else None
    clk = clocks.summary()
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f32dev": "f32", "f16dev": "f32", "f64": "f64"}[args.precision],
        "data": "synthetic (seeded splitmix64 inflow noise; no dataset)",
        "config": {"workload": w.name, "lattice": "D2Q9", "nx": w.nx, "ny": w.ny, "L": w.L,
                   "Re": round(w.L * w.u_in[0] / w.nu, 3), "nu": w.nu,
                   "equilibrium": "polynomial", "storage": args.precision,
                   "delta": w.delta, "k": w.k, "spinup_steps": args.spinup,
                   "l2": "inputs larger than L2 (two population buffers of %d MB each)"
                         % (info["bytes_per_pop"] * 9 * info["nxp"] * w.ny // 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "timing": "CUDA events on the library stream around the timed steps, "
                             "which run through the library's own path (CUDA graphs of "
                             "programmatically dependent launches)"},
        "roofline": roofline,
        "ehrenfest_sites_per_step_mean": round(float(np.mean(counts)), 3),
        "fluid_site_MLUPS": round(value * (1.0 - float(w.solid_mask().sum()) / n_sites), 1),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "launch_structure": "one launch per step; global select + Ehrenfests' step in its last block",
        "clocks": clk,
        "cpu_baseline": cpu,
        "forms": forms or None,
    }
    if rank == 0:
        print(json.dumps(line))
    g.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def select_stress_form(args, stream, w):
    """The headline workload with delta < 0: every fluid site is a candidate
    (dS >= 0 > delta), each block keeps its k = 16 best and the last block
    ranks at most k x blocks of them.  Step time over 20 steps after the
    same spin-up, beside the headline's."""
    import torch
    from paper_0705_4371_gb300 import lbm
    from copy import copy
    ws = copy(w)
    ws.delta = -1.0
    with lbm.Lattice.from_workload(ws, precision=lbm.PRECISIONS[args.precision],
                                   stream=stream.cuda_stream) as h2:
        h2.init_equilibrium(*inputs.cylinder_fields(ws))
        h2.step(args.spinup)
        h2.step(3)
        h2.sync()
        n = 20
        ms = timed_steps(h2, stream, n)
        counts = h2.counts(n)
    return {"delta": -1.0, "k": ws.k, "ms_per_step": round(ms / n, 4),
            "MLUPS": round(ws.n_sites * n / (ms * 1e-3) / 1e6, 1),
            "sites_per_step": int(counts.max()), "steps": n,
            "note": "every fluid site's exact dS evaluated and ranked each step"}


def c2_form(args, stream):
    """The 600 x 500 cylinder (L = 20, Re = 1000, polynomial f*, zero-gradient
    outflow, delta = 1e-3, k = 16), FP32: MLUPS over form_steps steps after
    the same spin-up.  Its 21.6 MB state is L2-resident: no HBM claim."""
    import torch
    from paper_0705_4371_gb300 import lbm
    w = inputs.workload_c2(1000.0)
    with lbm.Lattice.from_workload(w, precision=lbm.LB_F32, stream=stream.cuda_stream) as h2:
        h2.init_equilibrium(*inputs.cylinder_fields(w))
        h2.step(args.spinup)
        h2.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        device_spacer(stream)
        e0.record(stream)
        h2.step(args.form_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    return {"workload": w.name, "storage": "f32", "MLUPS": round(w.n_sites * args.form_steps / (ms * 1e-3) / 1e6, 1),
            "ms_per_step": round(ms / args.form_steps, 5), "steps": args.form_steps,
            "note": "state is L2-resident (21.6 MB): not an HBM roofline figure"}


def learned_form(args, stream):
    """Energy-constrained entropic run (2048 x 1024 cylinder, L = 64,
    Re = 5000, delta = 1e-3, k = 64, FP32 storage; initial energy = the
    isothermal energy x (1 + 0.1 sin(2 pi y/ny) cos(2 pi x/nx))) with the
    Newton solve started from the polynomial point and from the trained
    network: MLUPS and Newton iterations per site of each, and the network's
    training cost (1e7 samples on the GPU)."""
    import torch
    from paper_0705_4371_gb300 import learned, lbm
    t0 = time.perf_counter()
    params, info = learned.train_energy_mlp(n=args.mlp_samples, epochs=args.mlp_epochs, batch=4096,
                                            lr0=2e-3, lr1=2e-5)
    train_s = time.perf_counter() - t0
    w = inputs.workload_c4()
    rho, ux, uy = inputs.cylinder_fields(w)
    with lbm.Lattice.from_workload(w, precision=lbm.LB_F64, stream=stream.cuda_stream) as iso:
        iso.init_equilibrium(rho, ux, uy)
        e2 = iso.moments()[3] * inputs.energy_factor(w)
    out = {"workload": w.name, "storage": "f32", "train": {
        "samples": args.mlp_samples, "epochs": args.mlp_epochs, "batch": 4096,
        "final_loss": info["losses"][-1], "seconds": round(train_s, 2),
        "dataset_newton_fp32_it_per_sample": round(info["dataset_stats"][0] / info["dataset_stats"][2], 3)}}
    for name, eq in (("newton", lbm.LB_EQ_ENTROPIC_ENERGY), ("mlp_warm_start", lbm.LB_EQ_ENTROPIC_ENERGY_MLP)):
        with lbm.Lattice.from_workload(w, precision=lbm.LB_F32, equilibrium=eq,
                                       stream=stream.cuda_stream) as h2:
            if eq == lbm.LB_EQ_ENTROPIC_ENERGY_MLP:
                h2.set_mlp(params)
            h2.init_equilibrium(rho, ux, uy, e2)
            h2.set_timing(True)
            h2.step(args.learned_warmup)
            h2.sync()
            h2.kernel_times(reset=True)
            h2.newton_stats(reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            device_spacer(stream)
            e0.record(stream)
            h2.step(args.learned_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            fms = e0.elapsed_time(e1)
            k2 = h2.kernel_times(reset=True)
            it32, it64, sites, fails = h2.newton_stats(reset=True)
            out[name] = {"MLUPS": round(w.n_sites * args.learned_steps / (fms * 1e-3) / 1e6, 1),
                         "ms_per_step": round(fms / args.learned_steps, 4),
                         "collide_ms": round(k2["collide_ms"] / max(k2["collide_launches"], 1), 4),
                         "newton_fp32_it_per_site": round(it32 / max(sites, 1), 4),
                         "newton_finish_it_per_site": round(it64 / max(sites, 1), 4),
                         "newton_fails": int(fails), "steps": args.learned_steps}
    out["speedup"] = round(out["mlp_warm_start"]["MLUPS"] / out["newton"]["MLUPS"], 4)
    return out


def batched_form(args, stream, peaks, world=1, rank=0):
    """64 cylinder runs (sizes 256 x 128 .. 2048 x 1024, Re, delta and k
    drawn per run, seeded) in FP32 deviation storage: aggregate MLUPS of
    every launch strategy of the batch (graphs of 32 steps), the
    autotuner's choice, and the same runs stepped one after another (each
    through its own graphs).  Under torchrun the runs are split whole over
    the ranks (sharding.assign_runs; no exchange), each timed region is
    bracketed by barriers and reduced with a max over ranks."""
    import tempfile
    import torch
    from paper_0705_4371_gb300 import lbm
    from paper_0705_4371_gb300.sharding import assign_runs, max_over_ranks
    ws_all = inputs.workload_c5()
    share = assign_runs([w.nx * w.ny for w in ws_all], world)[rank]
    ws = [ws_all[i] for i in share]
    total_sites = sum(w.nx * w.ny for w in ws_all)
    out = {"workload": "64 cylinder runs (c5 recipe, seed %d)" % inputs.SEED_CYLINDER, "storage": "f32dev",
           "ranks": world, "scaling": "strong" if world > 1 else None}

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    if not ws:
        raise SystemExit("rank %d has no runs of the batch" % rank)
    with lbm.Batch(ws, precision=lbm.LB_F32_DEV, stream=stream.cuda_stream) as b:
        for r, w in enumerate(ws):
            b.run(r).init_equilibrium(*inputs.cylinder_fields(w))
        b.step(args.batch_spinup)
        b.sync()
        cache = args.autotune_cache or os.path.join(tempfile.gettempdir(),
                                                    "lbm_gb300_autotune_rank%d.json" % rank)
        t0 = time.perf_counter()
        v = b.autotune(steps=96, cache_path=cache)
        info = b.info()
        out.update({"runs": len(ws_all), "sites": total_sites, "runs_rank0": info["runs"],
                    "autotuned_variant": v, "autotune_s": round(time.perf_counter() - t0, 3)})
        try:
            with open(cache) as fh:
                entries = list(json.load(fh).values())
            if len(entries) == 1:   # a fresh cache: this batch's timings of every variant
                out["autotune_ms_per_step"] = entries[0].get("ms_per_step")
        except (OSError, ValueError, AttributeError):
            pass

        def timed(fn, n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            barrier()
            device_spacer(stream)
            e0.record(stream)
            fn(n)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            return max_over_ranks(e0.elapsed_time(e1), device="cuda")

        n = args.batch_steps
        names = {0: "batched_kernel_8row", 1: "batched_kernel_4row", 2: "concurrent_run_kernels"}
        variants = {}
        for var in (0, 1, 2):
            b.set_variant(var)
            b.step(32)
            ms = timed(b.step, n)
            variants[names[var]] = {"variant": var, "MLUPS": round(total_sites * n / (ms * 1e-3) / 1e6, 1),
                                    "ms_per_step": round(ms / n, 4),
                                    "launches_per_step": 2 if var < 2 else len(ws)}
        b.set_variant(v)
        b.step(32)
        ms_b = timed(b.step, n)
        ms_s = timed(b.step_sequential, n)
        b.sync()
        bytes_site = 72
        ach = bytes_site * total_sites / (ms_b / n * 1e-3) / 1e9 / world
        out.update({
            "chosen": {"variant": v, "MLUPS": round(total_sites * n / (ms_b * 1e-3) / 1e6, 1),
                       "ms_per_step": round(ms_b / n, 4)},
            "variants": variants,
            "sequential": {"MLUPS": round(total_sites * n / (ms_s * 1e-3) / 1e6, 1),
                           "ms_per_step": round(ms_s / n, 4), "launches_per_step": len(ws)},
            "speedup_vs_sequential": round(ms_s / ms_b, 3), "steps": n,
            "roofline": {"bound": "hbm", "algorithmic_bytes_per_site": bytes_site,
                         "achieved_GBps": round(ach, 1), "peak": peaks["hbm_gbs"],
                         "frac": round(ach / peaks["hbm_gbs"], 4),
                         "note": "the chosen strategy's whole step (every launch of it): algorithmic "
                                 "bytes / step time, per GPU"}})
    return out


# --------------------------------------------------------------------------
# CPU oracle: the reported baseline and the reference arm
# --------------------------------------------------------------------------

def _oracle_setup(w):
    from oracle import core as ora
    cfg = ora.Config(w.lattice, w.nx, w.ny, w.eq, ora.beta_of_nu(w.nu), w.delta, w.k, w.bc,
                     w.rho_in, w.u_in, w.obstacle)
    rho, ux, uy = inputs.cylinder_fields(w)
    f = ora.init_field(cfg, rho, ux, uy)
    return ora, cfg, f


def cpu_baseline(w, args):
    """The oracle as it stands on the host cores, on a bounded sample of the
    same workload: whole steps of the full grid for ~args.cpu_seconds."""
    ora, cfg, f = _oracle_setup(w)
    ora.run(cfg, f, 1, log_selection=False)          # first touch
    n, t = 0, 0.0
    while t < args.cpu_seconds and n < 1000:
        t0 = time.perf_counter()
        f, _ = ora.run(cfg, f, 1, log_selection=False)
        t += time.perf_counter() - t0
        n += 1
    out = {"value": round(w.n_sites * n / t / 1e6, 3), "unit": "MLUPS",
           "cores": ora.num_threads(), "kind": "oracle",
           "sample": "%d whole time steps of the %dx%d grid (%.1f s)" % (n, w.nx, w.ny, t)}
    # the same on one core, on a short sample (a few steps)
    cores = ora.num_threads()
    try:
        ora.set_num_threads(1)
        n1, t1 = 0, 0.0
        while t1 < min(args.cpu_seconds, 6.0) and n1 < 100:
            t0 = time.perf_counter()
            f, _ = ora.run(cfg, f, 1, log_selection=False)
            t1 += time.perf_counter() - t0
            n1 += 1
        out["one_core"] = {"value": round(w.n_sites * n1 / t1 / 1e6, 3), "unit": "MLUPS",
                           "sample": "%d whole time steps (%.1f s)" % (n1, t1)}
    finally:
        ora.set_num_threads(cores)
    return out


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import core as ora
    w_full = workload_by_name(args.workload)
    # calibrate the oracle's rate on the 1/8-scaled layout, then take the
    # largest layout of the same workload family whose K + W steps fit in
    # --ref-seconds
    cal = inputs.workload_c3_scaled()
    o, cfg, f = _oracle_setup(cal)
    t0 = time.perf_counter()
    o.run(cfg, f, 3, log_selection=False)
    rate = cal.n_sites * 3 / (time.perf_counter() - t0)
    per_step_s = args.ref_seconds / max(1, args.steps + args.warmup)
    cands = [w_full] + [inputs.cylinder(w_full.nx // s, w_full.ny // s, max(4, w_full.L // s),
                                        20000.0, name="%s_scaled_1_%d" % (w_full.name, s))
                        for s in (2, 4, 8, 16, 32)]
    w = next((c for c in cands if c.n_sites / rate <= per_step_s), cands[-1])
    o, cfg, f = _oracle_setup(w)
    for _ in range(args.warmup):
        f, _ = o.run(cfg, f, 1, log_selection=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, _ = o.run(cfg, f, 1, log_selection=False)
    el = time.perf_counter() - t0
    value = w.n_sites * args.steps / el / 1e6
    sample = "each step = one whole oracle time step of the %dx%d layout (L=%d)" % (w.nx, w.ny, w.L)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded splitmix64 inflow noise; no dataset)",
        "config": {"workload": w_full.name, "lattice": "D2Q9", "nx": w_full.nx, "ny": w_full.ny,
                   "L": w_full.L, "delta": w_full.delta, "k": w_full.k,
                   "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": ora.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--spinup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3")
    ap.add_argument("--precision", default="f32dev", choices=["f64", "f32", "f32dev", "f16dev"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--tile-shape", type=int, default=-1)
    ap.add_argument("--forms", type=int, default=1)
    ap.add_argument("--form-steps", type=int, default=2000)
    ap.add_argument("--learned", type=int, default=1)
    ap.add_argument("--batched", type=int, default=1)
    ap.add_argument("--batch-steps", type=int, default=400)
    ap.add_argument("--batch-spinup", type=int, default=64)
    ap.add_argument("--autotune-cache", default="")
    ap.add_argument("--learned-steps", type=int, default=400)
    ap.add_argument("--learned-warmup", type=int, default=20)
    ap.add_argument("--mlp-samples", type=int, default=10_000_000)
    ap.add_argument("--mlp-epochs", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
