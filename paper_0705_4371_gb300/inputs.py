"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.

This module holds none of the method's arithmetic: no equilibria, no
entropies, no collision, no streaming.  It only produces random numbers
(splitmix64, Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014, written from that published definition), the
initial macroscopic fields of the two experiments of Sec. 4, and the
geometry / parameter sets of the workloads.  Both the CUDA path and the
oracle receive the same arrays from here.
"""
from dataclasses import dataclass, field
import math

import numpy as np

MASK64 = (1 << 64) - 1
SEED_CYLINDER = 20070302


class SplitMix64:
    """splitmix64 stream: state += golden gamma; output = mix(state)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64_array(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = np.uint64(self.state) + idx * np.uint64(self.GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * self.GAMMA) & MASK64
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n doubles in [lo, hi): the top 53 bits of each output / 2^53."""
        u = (self.next_u64_array(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u


# --------------------------------------------------------------------------
# Boundary kinds (same numbering on both sides of the parity tests).
# --------------------------------------------------------------------------
BC_BB, BC_FREESLIP, BC_INLET, BC_OUTLET, BC_PERIODIC, BC_OUTLET_COPY = 0, 1, 2, 3, 4, 5
WALL_BOUNCE_BACK, WALL_DIFFUSE = 0, 1      # rule on the obstacle's faces
D1Q3, D2Q9 = 0, 1
EQ_POLY, EQ_ENTROPIC, EQ_ENERGY, EQ_ENERGY_MLP = 0, 1, 2, 3
SEED_ENERGY_SAMPLES = 20070531


@dataclass
class Workload:
    """Parameters of one run (no derived method quantities)."""
    name: str
    lattice: int
    nx: int
    ny: int
    eq: int
    nu: float
    delta: float
    k: int
    steps: int
    bc: tuple
    rho_in: float = 1.0
    u_in: tuple = (0.0, 0.0)
    obstacle: tuple = (0, 0, 0, 0)      # x0, y0, w, h
    probe: tuple = None                 # (x, y)
    L: int = 0
    seed: int = SEED_CYLINDER
    extra: dict = field(default_factory=dict)
    wall: int = WALL_BOUNCE_BACK

    @property
    def n_sites(self):
        return self.nx * self.ny

    def solid_mask(self):
        m = np.zeros((self.ny, self.nx), bool)
        x0, y0, w, h = self.obstacle
        if w > 0:
            m[y0:y0 + h, x0:x0 + w] = True
        return m


def shock_tube(n=800, nu=1e-9, delta=1e-3, k=4, steps=500, eq=EQ_ENTROPIC):
    """1:2 isothermal shock tube of Sec. 4.1 (800 sites, split at x = 400)."""
    return Workload("d1q3_shock_tube", D1Q3, n, 1, eq, nu, delta, k, steps,
                    (BC_BB, BC_BB, BC_BB, BC_BB))


def shock_tube_fields(w: Workload):
    x = np.arange(w.nx)
    rho = np.where(x < w.nx // 2, 1.0, 0.5)[None, :]
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def cylinder(nx=600, ny=500, L=20, re=1000.0, u_inf=0.05, delta=1e-3, k=16,
             steps=200000, eq=EQ_POLY, face_x=None, name=None, seed=SEED_CYLINDER, outlet=BC_OUTLET,
             wall=WALL_BOUNCE_BACK):
    """Square cylinder of side L in a free-slip channel (Sec. 4.2).

    Upstream face at x = 5L (face_x), centred in y; inlet at x = 0,
    zero-gradient (quasiequilibrium of the penultimate column) outlet at
    x = nx-1, free-slip walls at y = 0 and y = ny-1.  nu = L u_inf / Re.
    Probe at (4L, -2L) from the cylinder centre (Sec. 4.2.1).  wall: half-way
    bounce-back or the diffuse kinetic wall on the cylinder's faces.
    """
    fx = 5 * L if face_x is None else face_x
    oy0 = (ny - L) // 2
    cxc, cyc = fx + L // 2, oy0 + L // 2
    probe = (min(cxc + 4 * L, nx - 3), max(cyc - 2 * L, 1))
    nu = L * u_inf / re
    return Workload(name or "d2q9_cylinder_%dx%d_L%d_Re%g" % (nx, ny, L, re), D2Q9, nx, ny, eq,
                    nu, delta, k, steps, (BC_INLET, outlet, BC_FREESLIP, BC_FREESLIP),
                    1.0, (u_inf, 0.0), (fx, oy0, L, L), probe, L, seed, wall=wall)


def cylinder_fields(w: Workload, noise=1e-4):
    """rho = 1, u = (u_inf, 0) plus U[-noise, noise] on both components at
    every site (drawn in site order, u_x then u_y), seeded splitmix64."""
    g = SplitMix64(w.seed)
    r = g.uniform(2 * w.n_sites, -noise, noise).reshape(w.ny, w.nx, 2)
    rho = np.ones((w.ny, w.nx))
    ux = w.u_in[0] + r[..., 0]
    uy = w.u_in[1] + r[..., 1]
    m = w.solid_mask()
    ux[m] = 0.0  # solid sites hold no fluid; their values are never read
    uy[m] = 0.0
    return rho, ux, uy


def shear_wave(n=64, nu=0.05, amp=1e-3, steps=200):
    """Periodic box with u_x = amp sin(2 pi y / n): decays as exp(-nu k^2 t)."""
    w = Workload("d2q9_shear_wave", D2Q9, n, n, EQ_POLY, nu, 1e9, 0, steps,
                 (BC_PERIODIC,) * 4)
    w.extra["amp"] = amp
    return w


def shear_wave_fields(w: Workload):
    y = np.arange(w.ny)
    ux = w.extra["amp"] * np.sin(2.0 * math.pi * y / w.ny)[:, None] * np.ones((1, w.nx))
    return np.ones((w.ny, w.nx)), ux, np.zeros((w.ny, w.nx))


# Standard workloads ---------------------------------------------------------

def workload_c1():
    return shock_tube()


def workload_c2(re=1000.0):
    """600 x 500 channel, L = 20 at 5L from the inlet, zero-gradient outflow."""
    return cylinder(600, 500, 20, re, outlet=BC_OUTLET_COPY,
                    name="d2q9_cylinder_600x500_L20_Re%g_zero_gradient_outlet" % re)


def workload_c3():
    """4096 x 2048 channel, L = 128, Re = 20000 (the roofline workload)."""
    return cylinder(4096, 2048, 128, 20000.0, name="d2q9_cylinder_4096x2048_L128_Re20000")


def workload_c3_scaled():
    """The same layout scaled by 1/8 (512 x 256, L = 16), oracle-sized."""
    return cylinder(512, 256, 16, 20000.0, name="d2q9_cylinder_512x256_L16_Re20000")


def workload_c4():
    return cylinder(2048, 1024, 64, 5000.0, k=64, eq=EQ_ENERGY,
                    name="d2q9_energy_cylinder_2048x1024_L64_Re5000")


def workload_c5(nruns=64, seed=SEED_CYLINDER):
    """64 cylinder runs: scale s ~ logU[1, 8], nx = round8(256 s), ny = nx/2,
    L = round(ny/25), Re ~ logU[100, 20000], delta in {1e-4, 1e-3, 1e-2},
    k = max(1, round(1e-4 nx ny))."""
    g = SplitMix64(seed)
    u = g.uniform(4 * nruns).reshape(nruns, 4)
    runs = []
    for r in range(nruns):
        s = math.exp(u[r, 0] * math.log(8.0))
        nx = max(256, int(round(256 * s / 8.0)) * 8)
        ny = nx // 2
        L = max(4, int(round(ny / 25.0)))
        re = math.exp(math.log(100.0) + u[r, 1] * (math.log(20000.0) - math.log(100.0)))
        delta = (1e-4, 1e-3, 1e-2)[min(2, int(u[r, 2] * 3))]
        k = max(1, int(round(1e-4 * nx * ny)))
        w = cylinder(nx, ny, L, re, delta=delta, k=k, name="batch%02d_%dx%d" % (r, nx, ny),
                     seed=seed + r + 1)
        runs.append(w)
    return runs


def energy_factor(w, smooth=True, amplitude=0.1, seed=SEED_CYLINDER):
    """Factor applied to the isothermal energy of the initial field of the
    energy-constrained runs: 1 + a sin(2 pi y / ny) cos(2 pi x / nx) (a
    smooth temperature pattern), or 1 + a U[-1, 1] per site."""
    if not smooth:
        return 1.0 + amplitude * uniform(seed, (w.ny, w.nx))
    y = np.arange(w.ny)[:, None]
    x = np.arange(w.nx)[None, :]
    return 1.0 + amplitude * np.sin(2 * np.pi * y / w.ny) * np.cos(2 * np.pi * x / w.nx)


def energy_samples(seed, n, rho=(0.5, 2.0), u_max=0.2, escale=(0.9, 1.1)):
    """Moments for the learned form's training set: rho ~ U[rho], u uniform
    in the disc |u| < u_max, and an energy factor ~ U[escale] that multiplies
    the isothermal energy 2E(rho, u).  Returns (rho, ux, uy, escale)."""
    g = SplitMix64(seed)
    u = g.uniform(4 * n).reshape(4, n)
    r = rho[0] + (rho[1] - rho[0]) * u[0]
    rad = u_max * np.sqrt(u[1])
    ang = 2.0 * np.pi * u[2]
    es = escale[0] + (escale[1] - escale[0]) * u[3]
    return r, rad * np.cos(ang), rad * np.sin(ang), es


# Generic random arrays for parity tests -----------------------------------

def uniform(seed, shape, lo=-1.0, hi=1.0):
    n = int(np.prod(shape))
    return SplitMix64(seed).uniform(n, lo, hi).reshape(shape)


def random_ds_with_ties(seed, n, n_ties=0, tie_value=None, frac_inf=0.0):
    """Random non-negative dS values; optional forced ties and +inf entries."""
    g = SplitMix64(seed)
    ds = g.uniform(n, 0.0, 1.0) ** 3 * 1e-2
    if n_ties and n:
        pick = (g.uniform(n_ties) * n).astype(np.int64)
        ds[pick] = ds[pick[0]] if tie_value is None else tie_value
    if frac_inf > 0 and n:
        pick = (g.uniform(max(1, int(frac_inf * n))) * n).astype(np.int64)
        ds[pick] = np.inf
    return ds
