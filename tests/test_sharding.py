"""Host side of the multi-GPU layout (CPU, gloo, two ranks): the batched
form's runs are split across ranks whole and deterministically, and the
timed region is reduced with a max over ranks."""
import os
import socket

import pytest

from paper_0705_4371_gb300 import inputs
from paper_0705_4371_gb300.sharding import assign_runs, max_over_ranks


def test_assignment_is_a_balanced_partition():
    sites = [w.nx * w.ny for w in inputs.workload_c5()]
    for world in (1, 2, 3, 4, 8):
        share = assign_runs(sites, world)
        flat = sorted(r for s in share for r in s)
        assert flat == list(range(len(sites)))
        loads = [sum(sites[r] for r in s) for s in share]
        # longest-first greedy: no rank exceeds another by more than the largest run
        assert max(loads) - min(loads) <= max(sites)
    assert assign_runs([5, 5, 5], 2) == [[0, 2], [1]]
    assert assign_runs([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        assign_runs([1], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sites = [w.nx * w.ny for w in inputs.workload_c5()]
        mine = assign_runs(sites, world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = max_over_ranks(1.5 + rank)
        dist.barrier()
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
            fh.write(repr((got, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_split_and_the_max(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    results = [eval(open(tmp_path / ("rank%d.txt" % r)).read()) for r in range(world)]
    sites = [w.nx * w.ny for w in inputs.workload_c5()]
    expect = assign_runs(sites, world)
    for got, t in results:
        assert got == expect               # every rank computed the same split
        assert t == 2.5                    # max over ranks of 1.5 + rank
    assert sorted(sum(expect, [])) == list(range(len(sites)))


# --------------------------------------------------------------------------
# One run sharded in x (slabs), host side on CPU: each gloo rank steps its
# slab with the oracle (test side) while the candidates' merge and the ghost
# exchange go through the library's sharding functions; the sharded run must
# equal the unsharded oracle run bit for bit (states and selections).
# --------------------------------------------------------------------------
from paper_0705_4371_gb300 import sharding  # noqa: E402

SLAB_STEPS = 60


def _slab_case():
    # Re 5000 at L = 6 with a perturbed start: Ehrenfests' sites at every
    # step, more candidates than k, the obstacle inside one slab
    w = inputs.cylinder(120, 48, 6, 5000.0, delta=1e-6, k=6)
    return w


def _perturbed(w):
    from oracle import core as ora
    from tests._common import oracle_cfg, perturbed_state
    cfg = oracle_cfg(w)
    return perturbed_state(cfg, w, seed=41, eps=0.02)


def _slab_worker(rank, world, port, out_dir):
    import numpy as np
    import torch
    import torch.distributed as dist
    from oracle import core as ora
    from tests._common import oracle_cfg
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _slab_case()
        slab = sharding.slab_plan(w.nx, world, w.obstacle)[rank]
        wl = sharding.slab_workload(w, slab)
        cfg = oracle_cfg(wl)
        f = sharding.local_field(_perturbed(w), slab)
        nxl, ny = slab.nx_local, w.ny
        own = np.zeros((ny, nxl), bool)
        own[:, slab.own_columns()] = True
        own &= ~cfg.solid_mask()
        first, last = slab.ghost_left, slab.ghost_left + slab.own - 1
        bufs = [torch.zeros(3 * ny, dtype=torch.float64) for _ in range(4)]
        sels = []
        for _ in range(SLAB_STEPS):
            _, ds = ora.fields(cfg, f)
            loc = ora.select(ds.ravel(), w.delta, w.k, eligible=own.ravel())
            gidx = (loc // nxl) * w.nx + (loc % nxl) + slab.lx0
            sel = sharding.allgather_candidates(ds.ravel()[loc], gidx, w.k)
            gx, gy = sel % w.nx, sel // w.nx
            mine = (gx >= slab.x0) & (gx < slab.x1)
            fp = ora.collide(cfg, f, gy[mine] * nxl + gx[mine] - slab.lx0)
            to_left = torch.from_numpy(np.ascontiguousarray(fp[list(sharding.LEFT_PLANES), :, first]).ravel())
            to_right = torch.from_numpy(np.ascontiguousarray(fp[list(sharding.RIGHT_PLANES), :, last]).ravel())
            sharding.exchange_ghosts(slab, to_left, to_right, bufs[0], bufs[1])
            if slab.ghost_left:
                fp[list(sharding.RIGHT_PLANES), :, 0] = bufs[0].numpy().reshape(3, ny)
            if slab.ghost_right:
                fp[list(sharding.LEFT_PLANES), :, nxl - 1] = bufs[1].numpy().reshape(3, ny)
            f = ora.stream(cfg, fp)
            sels.append(sel)
        np.save(os.path.join(out_dir, "f%d.npy" % rank), f[..., slab.own_columns()])
        np.save(os.path.join(out_dir, "sel%d.npy" % rank), np.array([list(s) + [-1] * (w.k - len(s)) for s in sels]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_run_equals_the_unsharded_oracle_run(tmp_path, world):
    pytest.importorskip("torch")
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import core as ora
    from tests._common import oracle_cfg
    w = _slab_case()
    plan = sharding.slab_plan(w.nx, world, w.obstacle)
    assert sum(s.own for s in plan) == w.nx
    mp.spawn(_slab_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    f_ref, log = ora.run(oracle_cfg(w), _perturbed(w), SLAB_STEPS)
    f_sh = np.concatenate([np.load(tmp_path / ("f%d.npy" % r)) for r in range(world)], axis=-1)
    assert np.array_equal(f_sh, f_ref)
    assert sum(len(s) for s in log.selected) > SLAB_STEPS          # Ehrenfests' steps all along
    for r in range(world):
        sels = np.load(tmp_path / ("sel%d.npy" % r))
        for t in range(SLAB_STEPS):
            got = sels[t][sels[t] >= 0]
            assert np.array_equal(got, log.selected[t]), (r, t)


def test_slab_plan_keeps_the_obstacle_in_one_slab():
    w = inputs.cylinder(200, 72, 8, 1000.0)
    for world in (2, 3, 4, 7):
        plan = sharding.slab_plan(w.nx, world, w.obstacle)
        ox0, _, ow, _ = w.obstacle
        holders = [s for s in plan if s.x0 <= ox0 and ox0 + ow <= s.x1]
        assert len(holders) == 1 and all(s.own >= 3 for s in plan)
        assert [s.x0 for s in plan][1:] == [s.x1 for s in plan][:-1]
        for s in plan:
            sharding.slab_workload(w, s)       # every slab's local run is valid
    with pytest.raises(ValueError):
        sharding.slab_plan(10, 4)


def test_merge_keeps_the_k_best_with_ties_to_the_lower_index():
    import numpy as np
    keys = np.array([5, 9, 9, 1, 9], np.uint64)
    idx = np.array([10, 40, 7, 3, 12], np.int64)
    assert list(sharding.merge_topk(keys, idx, 3)) == [7, 12, 40]
    assert list(sharding.merge_topk(keys, idx, 2)) == [7, 12]
    assert list(sharding.merge_topk(np.array([0.5, 0.7]), np.array([3, 2]), 5)) == [2, 3]
