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
