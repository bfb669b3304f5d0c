"""Helpers shared by the tests: build oracle configs and GPU runs from the
same seeded workload description."""
import numpy as np

from oracle import core as ora
from paper_0705_4371_gb300 import inputs

PREC_TOL = {  # relative tolerance of moments after 1000 steps (replayed selection)
    "f64": 1e-12,
    "f32": 1e-5,
}


def oracle_cfg(w, **over):
    d = dict(lattice=w.lattice, nx=w.nx, ny=w.ny, eq=w.eq, beta=ora.beta_of_nu(w.nu),
             delta=w.delta, k=w.k, bc=w.bc, rho_in=w.rho_in, u_in=w.u_in, obstacle=w.obstacle,
             wall=w.wall)
    if "nu" in over:
        d["beta"] = ora.beta_of_nu(over.pop("nu"))
    d.update(over)
    return ora.Config(**d)


def initial_fields(w, noise=1e-4):
    if w.lattice == inputs.D1Q3:
        return inputs.shock_tube_fields(w)
    return inputs.cylinder_fields(w, noise=noise)


def perturbed_state(cfg, w, seed, eps, noise=1e-2):
    """Oracle equilibrium of the workload's fields times (1 + eps U[-1,1])."""
    rho, ux, uy = initial_fields(w, noise=noise)
    f = ora.init_field(cfg, rho, ux, uy)
    f = f * (1.0 + eps * inputs.uniform(seed, f.shape))
    f[:, cfg.solid_mask()] = 0.0
    return f


def rel_err(a, b, mask=None):
    """max |a - b| / max |b| over fluid sites."""
    if mask is not None:
        a, b = a[..., ~mask], b[..., ~mask]
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def moment_errors(got, ref, mask, u_ref):
    """Errors of the moment fields over fluid sites.

    e_M:   max over sites of |M_got - M_ref| / |M_ref|, M = (rho, rho u_x, rho u_y)
           (the conserved moments of Sec. 2, compared as a vector per site);
    e_rho: max |d rho| / max rho;
    e_u:   max |d u| / u_ref (u_ref: the free-stream speed).
    """
    (rg, ug, vg), (ro, uo, vo) = got, ref
    f = ~mask
    Mg = np.stack([rg[f], rg[f] * ug[f], rg[f] * vg[f]])
    Mo = np.stack([ro[f], ro[f] * uo[f], ro[f] * vo[f]])
    e_M = float((np.linalg.norm(Mg - Mo, axis=0) / np.linalg.norm(Mo, axis=0)).max())
    e_rho = float(np.abs(rg[f] - ro[f]).max() / np.abs(ro[f]).max())
    e_u = float(max(np.abs(ug[f] - uo[f]).max(), np.abs(vg[f] - vo[f]).max()) / u_ref)
    return e_M, e_rho, e_u


def mlp_random_params(seed, scale=0.5):
    """Network parameters for parity tests: uniform weights and biases, the
    normalisation of the learned form's sample distribution."""
    from oracle import mlp
    u = inputs.uniform(seed, (mlp.N_PARAMS,)) * scale
    d = mlp.unpack(u)
    d["mean"] = np.array([1.25, 0.0, 0.0, 0.66])
    d["inv_std"] = np.array([2.3, 10.0, 10.0, 30.0])
    d["out_scale"] = np.array([0.05, 0.02, 0.02, 0.1])
    return mlp.pack(d).astype(np.float32).astype(np.float64)


def mlp_random_features(seed, n):
    rho, ux, uy, es = inputs.energy_samples(seed, n)
    th = (2.0 / 3.0) * es + 0.01 * inputs.uniform(seed + 1, (n,))
    return np.stack([rho, ux, uy, th], axis=1).astype(np.float32).astype(np.float64)
