"""Multi-GPU layout of the batched form: independent runs are assigned whole
to ranks (no exchange between ranks on the data path); the only collective
is the max over ranks of the timed region.

assign_runs is deterministic, so every rank computes the same assignment
without communicating.
"""


def assign_runs(sites, world):
    """Longest-first greedy assignment of runs (by site count) to `world`
    ranks: each run, largest first (ties: lower index), goes to the rank
    with the fewest sites so far (ties: lower rank).  Returns one sorted
    list of run indices per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    share = [[] for _ in range(world)]
    for r in sorted(range(len(sites)), key=lambda i: (-int(sites[i]), i)):
        k = min(range(world), key=lambda q: (load[q], q))
        share[k].append(r)
        load[k] += int(sites[r])
    return [sorted(s) for s in share]


def max_over_ranks(value, device=None):
    """The largest `value` over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# One run sharded in x: slabs of columns, one per rank.  The selection of
# Sec. 3.2 is global (the k sites of the whole grid with the largest
# dS > delta), so every step gathers each slab's k best candidates and every
# rank keeps the k best of the union, the same set on every rank and the
# same set one unsharded run selects (the order is total: dS descending,
# global site index ascending).  Free flight moves three populations across
# each face (v_x = +1: 1, 5, 8 to the right; v_x = -1: 3, 6, 7 to the left),
# so each slab keeps one ghost column per neighbour, refreshed after every
# step from the neighbour's boundary column.
# --------------------------------------------------------------------------
from dataclasses import dataclass

import numpy as np

RIGHT_PLANES = (1, 5, 8)      # D2Q9 populations moving toward +x
LEFT_PLANES = (3, 6, 7)       # ... toward -x


@dataclass
class Slab:
    """Columns [x0, x1) of the global grid, with a ghost column on each side
    that faces another slab."""
    rank: int
    x0: int
    x1: int
    ghost_left: int
    ghost_right: int

    @property
    def own(self):
        return self.x1 - self.x0

    @property
    def nx_local(self):
        return self.own + self.ghost_left + self.ghost_right

    @property
    def lx0(self):
        """Global x of the slab's local column 0."""
        return self.x0 - self.ghost_left

    def own_columns(self):
        """Local column range of the slab's own sites."""
        return slice(self.ghost_left, self.ghost_left + self.own)


def slab_plan(nx, ranks, obstacle=(0, 0, 0, 0), min_cols=3):
    """Split nx columns into `ranks` slabs as evenly as possible; a cut that
    would fall within two columns of the obstacle moves past it, so that the
    obstacle (and its neighbouring columns) lies inside one slab.  Every slab
    owns at least min_cols columns."""
    if ranks < 1:
        raise ValueError("ranks must be >= 1")
    cuts = [round(nx * r / ranks) for r in range(ranks + 1)]
    ox0, _, ow, _ = obstacle
    if ow > 0:
        for r in range(1, ranks):
            if ox0 - 2 <= cuts[r] <= ox0 + ow + 2:
                cuts[r] = ox0 + ow + 3
        for r in range(1, ranks + 1):
            cuts[r] = max(cuts[r], cuts[r - 1] + min_cols)
    if cuts[-1] != nx or any(cuts[r + 1] - cuts[r] < min_cols for r in range(ranks)):
        raise ValueError("cannot split %d columns into %d slabs of at least %d" % (nx, ranks, min_cols))
    return [Slab(r, cuts[r], cuts[r + 1], 1 if r > 0 else 0, 1 if r < ranks - 1 else 0) for r in range(ranks)]


def slab_workload(w, slab):
    """The slab's local run: its columns and ghost columns, the run's
    boundary kinds on its outer sides (bounce-back, never read by an own
    site, on a side facing another slab), the obstacle in local coordinates,
    the probe if it lies in the slab."""
    from copy import copy
    from .inputs import BC_BB
    s = copy(w)
    s.nx = slab.nx_local
    s.name = "%s_slab%d" % (w.name, slab.rank)
    bc = list(w.bc)
    if slab.ghost_left:
        bc[0] = BC_BB
    if slab.ghost_right:
        bc[1] = BC_BB
    s.bc = tuple(bc)
    ox0, oy0, ow, oh = w.obstacle
    if ow > 0 and slab.x0 <= ox0 and ox0 + ow <= slab.x1:
        s.obstacle = (ox0 - slab.lx0, oy0, ow, oh)
    else:
        if ow > 0 and ox0 < slab.x1 and ox0 + ow > slab.x0:
            raise ValueError("the obstacle crosses a slab boundary")
        s.obstacle = (0, 0, 0, 0)
    if w.probe is not None and slab.x0 <= w.probe[0] < slab.x1:
        s.probe = (w.probe[0] - slab.lx0, w.probe[1])
    else:
        s.probe = None
    return s


def local_field(a, slab):
    """Columns of a global field [.., ny, nx] that the slab's local grid holds."""
    return np.ascontiguousarray(a[..., slab.lx0:slab.lx0 + slab.nx_local])


def merge_topk(keys, idx, k):
    """The k best of the gathered candidates: key descending, global index
    ascending (every rank computes the same set).  Returns sorted indices."""
    keys = np.asarray(keys)
    idx = np.asarray(idx, np.int64)
    if k <= 0 or idx.size == 0:
        return np.zeros(0, np.int64)
    order = np.lexsort((idx, -keys.astype(np.float64) if keys.dtype.kind == "f" else ~keys.astype(np.uint64)))
    return np.sort(idx[order[:k]])


def allgather_candidates(keys, idx, k, group=None):
    """Gather every rank's candidates (host arrays) and merge them."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, (np.asarray(keys).tolist(), np.asarray(idx, np.int64).tolist()), group=group)
    all_keys = np.concatenate([np.asarray(g[0], np.asarray(keys).dtype) for g in got])
    all_idx = np.concatenate([np.asarray(g[1], np.int64) for g in got])
    return merge_topk(all_keys, all_idx, k)


def exchange_ghosts(slab, to_left, to_right, from_left, from_right, group=None):
    """Neighbour exchange of one step (torch tensors, on the devices of the
    process group's backend): to_left goes to the slab on the left, whose
    to_right arrives in from_left, and so on.  Sends and receives are posted
    together (no ordering between ranks can deadlock)."""
    import torch.distributed as dist
    ops = []
    world = dist.get_world_size(group)
    if slab.ghost_left:
        ops.append(dist.P2POp(dist.isend, to_left, slab.rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, from_left, slab.rank - 1, group))
    if slab.ghost_right:
        assert slab.rank + 1 < world
        ops.append(dist.P2POp(dist.isend, to_right, slab.rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, from_right, slab.rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()




def _torch_dtype(precision):
    import torch
    from . import lbm
    return {lbm.LB_F64: torch.float64, lbm.LB_F32: torch.float32, lbm.LB_F32_DEV: torch.float32,
            lbm.LB_F16_DEV: torch.float16}[precision]


class SlabGroup:
    """All slabs of one run in one process, on the current GPU (ranks
    emulated in turn: every kernel of a step is ordered by the host, none
    waits for another).  Steps like one unsharded run."""

    def __init__(self, w, nslabs, precision, stream=None):
        import torch
        from . import lbm
        self.w, self.k = w, w.k
        self.plan = slab_plan(w.nx, nslabs, w.obstacle)
        self.runs = []
        for s in self.plan:
            g = lbm.Lattice.from_workload(slab_workload(w, s), precision=precision, stream=stream)
            g.set_slab(s.ghost_left, s.ghost_right, s.x0, w.nx)
            self.runs.append(g)
        dt = _torch_dtype(precision)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.buf = [[torch.zeros(3 * w.ny, dtype=dt, device=dev) for _ in range(2)] for _ in self.plan]

    def init_equilibrium(self, rho, ux, uy):
        for s, g in zip(self.plan, self.runs):
            g.init_equilibrium(local_field(rho, s), local_field(ux, s), local_field(uy, s))

    def step(self, n=1):
        """n steps; returns the global selection of each (sorted indices)."""
        import torch
        sels = []
        for _ in range(n):
            for g in self.runs:
                g.slab_collide()
            cand = [g.slab_candidates(self.k) for g in self.runs]
            keys = np.concatenate([c[0] for c in cand]) if cand else np.zeros(0, np.uint64)
            idx = np.concatenate([c[1] for c in cand]) if cand else np.zeros(0, np.int64)
            sel = merge_topk(keys, idx, self.k)
            for g in self.runs:
                g.slab_apply(sel)
            # ghost exchange: pack every slab's outgoing columns, then unpack
            for s, g, b in zip(self.plan, self.runs, self.buf):
                if s.ghost_left:
                    g.slab_ghost(0, b[0].data_ptr(), 0)
                if s.ghost_right:
                    g.slab_ghost(1, b[1].data_ptr(), 0)
            torch.cuda.synchronize()
            for r, (s, g) in enumerate(zip(self.plan, self.runs)):
                if s.ghost_left:
                    g.slab_ghost(0, self.buf[r - 1][1].data_ptr(), 1)
                if s.ghost_right:
                    g.slab_ghost(1, self.buf[r + 1][0].data_ptr(), 1)
            torch.cuda.synchronize()
            sels.append(sel)
        return sels

    def get_state(self):
        """Pre-collision populations of the whole grid [Q][ny][nx] (FP64)."""
        return np.concatenate([g.get_state()[..., s.own_columns()] for s, g in zip(self.plan, self.runs)],
                              axis=-1)

    def close(self):
        for g in self.runs:
            g.close()


class SlabRun:
    """This rank's slab of a run sharded in x over the ranks of the default
    process group (one GPU per rank; NCCL carries the ghost columns and the
    candidates)."""

    def __init__(self, w, precision, stream=None):
        import torch
        import torch.distributed as dist
        from . import lbm
        self.w, self.k = w, w.k
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.plan = slab_plan(w.nx, self.world, w.obstacle)
        self.slab = self.plan[self.rank]
        self.g = lbm.Lattice.from_workload(slab_workload(w, self.slab), precision=precision, stream=stream)
        self.g.set_slab(self.slab.ghost_left, self.slab.ghost_right, self.slab.x0, w.nx)
        dt = _torch_dtype(precision)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.send = [torch.zeros(3 * w.ny, dtype=dt, device=dev) for _ in range(2)]
        self.recv = [torch.zeros(3 * w.ny, dtype=dt, device=dev) for _ in range(2)]

    def init_equilibrium(self, rho, ux, uy):
        s = self.slab
        self.g.init_equilibrium(local_field(rho, s), local_field(ux, s), local_field(uy, s))

    def step(self, n=1):
        import torch
        sels = []
        for _ in range(n):
            self.g.slab_collide()
            keys, idx = self.g.slab_candidates(self.k)
            sel = allgather_candidates(keys, idx, self.k)
            self.g.slab_apply(sel)
            s = self.slab
            if s.ghost_left:
                self.g.slab_ghost(0, self.send[0].data_ptr(), 0)
            if s.ghost_right:
                self.g.slab_ghost(1, self.send[1].data_ptr(), 0)
            torch.cuda.synchronize()
            exchange_ghosts(s, self.send[0], self.send[1], self.recv[0], self.recv[1])
            if s.ghost_left:
                self.g.slab_ghost(0, self.recv[0].data_ptr(), 1)
            if s.ghost_right:
                self.g.slab_ghost(1, self.recv[1].data_ptr(), 1)
            sels.append(sel)
        return sels

    def close(self):
        self.g.close()
