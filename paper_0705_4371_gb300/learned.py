"""Learned form: build the training set and train the warm-start network
on the GPU (every computation in liblbm's kernels; PyTorch only holds the
device buffers).

    params, info = train_energy_mlp(n=1_000_000, seed=..., epochs=4)
    run = lbm.Lattice(..., equilibrium=lbm.LB_EQ_ENTROPIC_ENERGY_MLP, ...)
    run.set_mlp(params)
"""
import time

import numpy as np

from . import inputs, lbm


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the learned form trains on the GPU; no CUDA device is available")
    return torch


def make_dataset(n, seed=inputs.SEED_ENERGY_SAMPLES, with_mu=False, device=0, stream=None):
    """Samples drawn by inputs.energy_samples, uploaded, and solved on the
    GPU (lb_energy_dataset).  Returns dict of device tensors feat, dmu (and
    mu) and the Newton statistics (it32, it64, samples, fails)."""
    torch = _torch()
    dev = torch.device("cuda", device)
    rho, ux, uy, es = inputs.energy_samples(seed, n)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
         for k, v in (("rho", rho), ("ux", ux), ("uy", uy), ("es", es))}
    feat = torch.empty((n, 4), dtype=torch.float32, device=dev)
    dmu = torch.empty((n, 4), dtype=torch.float32, device=dev)
    mu = torch.empty((n, 4), dtype=torch.float64, device=dev) if with_mu else None
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    lbm.energy_dataset(t["rho"].data_ptr(), t["ux"].data_ptr(), t["uy"].data_ptr(), t["es"].data_ptr(),
                       n, feat.data_ptr(), dmu.data_ptr(), mu.data_ptr() if mu is not None else None,
                       stats.data_ptr(), st)
    torch.cuda.synchronize(dev)
    out = dict(feat=feat, dmu=dmu, stats=tuple(int(x) for x in stats.cpu().numpy()))
    if mu is not None:
        out["mu"] = mu
    return out


def train_energy_mlp(n=1_000_000, seed=inputs.SEED_ENERGY_SAMPLES, init_seed=1, epochs=4, batch=8192,
                     lr0=3e-3, lr1=1e-4, device=0):
    """Training set of n samples, lb_mlp_normalise, lb_mlp_train.  Returns
    (params as a host FP32 array, info dict with the per-epoch losses, the
    data set's Newton statistics and the wall times)."""
    torch = _torch()
    dev = torch.device("cuda", device)
    t0 = time.perf_counter()
    data = make_dataset(n, seed, device=device)
    t1 = time.perf_counter()
    p = torch.from_numpy(lbm.mlp_init(init_seed)).to(dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    lbm.mlp_normalise(p.data_ptr(), data["feat"].data_ptr(), data["dmu"].data_ptr(), n, st)
    losses = torch.zeros(max(1, epochs), dtype=torch.float32, device=dev)
    lbm.mlp_train(p.data_ptr(), data["feat"].data_ptr(), data["dmu"].data_ptr(), n, batch, epochs,
                  lr0, lr1, losses.data_ptr(), st)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    info = dict(losses=losses.cpu().numpy()[:epochs].tolist(), dataset_stats=data["stats"],
                dataset_s=t1 - t0, train_s=t2 - t1, n=n, epochs=epochs, batch=batch)
    return p.cpu().numpy(), info
