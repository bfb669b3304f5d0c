"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

Arrays are numpy float64 in the layout [Q][ny][nx] (population planes,
x fastest), populations in the paper's numbering (Sec. 4.1 for D1Q3,
Sec. 4.2 for D2Q9).  Nothing here imports the CUDA library.
"""
import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

D1Q3, D2Q9 = 0, 1
EQ_POLY, EQ_ENTROPIC, EQ_ENERGY = 0, 1, 2
BC_BB, BC_FREESLIP, BC_INLET, BC_OUTLET, BC_PERIODIC = 0, 1, 2, 3, 4
WALL_BOUNCE_BACK, WALL_DIFFUSE = 0, 1
# storage of the populations (precision form): FP64, FP32, FP32 and FP16
# deviations f - W rho0 (rho0 = 1)
STORE_F64, STORE_F32, STORE_F32_DEV, STORE_F16_DEV = 0, 1, 2, 3

_lib = None


class _Cfg(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("eq", C.c_int), ("beta", C.c_double), ("delta", C.c_double),
                ("k", C.c_long), ("bc", C.c_int * 4), ("rho_in", C.c_double),
                ("ux_in", C.c_double), ("uy_in", C.c_double), ("ox0", C.c_int),
                ("oy0", C.c_int), ("ow", C.c_int), ("oh", C.c_int), ("elbm", C.c_int),
                ("wall", C.c_int), ("store", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        cfgp = C.POINTER(_Cfg)
        L.ora_q.argtypes = [C.c_int]
        L.ora_lattice.argtypes = [C.c_int, ip, ip, dp]
        L.ora_moments.argtypes = [C.c_int, dp, dp]
        L.ora_equilibrium.argtypes = [C.c_int, C.c_int, dp, dp]
        L.ora_feq_rho_u.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp]
        L.ora_mu_guess.argtypes = [C.c_int, dp, dp]
        L.ora_newton.argtypes = [C.c_int, dp, dp, C.c_double, C.c_int]
        L.ora_perfect_entropy.argtypes = [C.c_int, dp]
        L.ora_perfect_entropy.restype = C.c_double
        L.ora_delta_s.argtypes = [C.c_int, dp, dp]
        L.ora_elbm_alpha.argtypes = [C.c_int, dp, dp]
        L.ora_elbm_alpha.restype = C.c_double
        L.ora_delta_s.restype = C.c_double
        L.ora_select.argtypes = [dp, C.c_void_p, C.c_long, C.c_double, C.c_long, lp]
        L.ora_select.restype = C.c_long
        L.ora_fields.argtypes = [cfgp, dp, C.c_void_p, C.c_void_p]
        L.ora_fields.restype = C.c_long
        L.ora_moment_fields.argtypes = [cfgp, dp, dp, dp, C.c_void_p, C.c_void_p]
        L.ora_init.argtypes = [cfgp, dp, dp, C.c_void_p, C.c_void_p, dp]
        L.ora_run.argtypes = [cfgp, dp, C.c_long, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_long, C.c_void_p, C.c_int, C.c_int]
        L.ora_collide.argtypes = [cfgp, dp, C.c_void_p, C.c_long, dp]
        L.ora_stream.argtypes = [cfgp, dp, dp]
        L.ora_round_f32.argtypes = [C.c_double]
        L.ora_round_f32.restype = C.c_double
        L.ora_round_f16.argtypes = [C.c_double]
        L.ora_round_f16.restype = C.c_double
        L.ora_num_threads.restype = C.c_int
        L.ora_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def q_of(lattice):
    return 3 if lattice == D1Q3 else 9


def lattice_tables(lattice):
    q = q_of(lattice)
    cx = np.zeros(q, np.int32)
    cy = np.zeros(q, np.int32)
    w = np.zeros(q, np.float64)
    lib().ora_lattice(lattice, cx, cy, w)
    return cx, cy, w


@dataclass
class Config:
    """One run: lattice, grid, equilibrium, beta, (delta, k), boundaries.

    bc = (x0, x1, y0, y1) kinds; obstacle = (x0, y0, w, h), w == 0: none.
    """
    lattice: int
    nx: int
    ny: int
    eq: int
    beta: float
    delta: float
    k: int
    bc: tuple = (BC_BB, BC_BB, BC_BB, BC_BB)
    rho_in: float = 1.0
    u_in: tuple = (0.0, 0.0)
    obstacle: tuple = (0, 0, 0, 0)
    elbm: bool = False        # collision (elbmLB) instead of (lbgkLB)
    wall: int = 0             # rule on the obstacle's faces: WALL_BOUNCE_BACK / WALL_DIFFUSE
    store: int = 0            # storage of the populations: STORE_F64 / _F32 / _F32_DEV / _F16_DEV

    @property
    def q(self):
        return q_of(self.lattice)

    @property
    def n_sites(self):
        return self.nx * self.ny

    def c_struct(self):
        s = _Cfg()
        s.lattice, s.nx, s.ny, s.eq = self.lattice, self.nx, self.ny, self.eq
        s.beta, s.delta, s.k = self.beta, self.delta, self.k
        for i in range(4):
            s.bc[i] = self.bc[i]
        s.rho_in, s.ux_in, s.uy_in = self.rho_in, self.u_in[0], self.u_in[1]
        s.ox0, s.oy0, s.ow, s.oh = self.obstacle
        s.elbm = 1 if self.elbm else 0
        s.wall = self.wall
        s.store = self.store
        return s

    def solid_mask(self):
        m = np.zeros((self.ny, self.nx), bool)
        x0, y0, w, h = self.obstacle
        if w > 0:
            m[y0:y0 + h, x0:x0 + w] = True
        return m


def beta_of_nu(nu):
    """LBGK parameter from the kinematic viscosity.

    The paper writes the LBGK step as f + 2 beta (f* - f) (lbgkLB), i.e. the
    BGK rate omega = 2 beta, but does not state nu(beta).  The standard
    lattice relation nu = c_s^2 (1/omega - 1/2) with c_s^2 = 1/3 gives
    beta = 1 / (1 + 6 nu); it reproduces the paper's pairs (nu = 1/30,
    beta = 5/6) and (nu = 1e-9, beta -> 1).  Pinned by the shear-wave test.
    """
    return 1.0 / (1.0 + 6.0 * nu)


def moments(lattice, f):
    M = np.zeros(4)
    lib().ora_moments(lattice, np.ascontiguousarray(f, np.float64), M)
    return M


def equilibrium(lattice, eq, M):
    """Quasiequilibrium for M = (rho, rho ux, rho uy, 2E)."""
    fs = np.zeros(q_of(lattice))
    Mv = np.zeros(4)
    Mv[:len(M)] = M
    rc = lib().ora_equilibrium(lattice, eq, Mv, fs)
    if rc != 0:
        raise RuntimeError("oracle Newton solve failed for M=%r" % (M,))
    return fs


def feq_rho_u(lattice, eq, rho, ux, uy=0.0):
    fs = np.zeros(q_of(lattice))
    lib().ora_feq_rho_u(lattice, eq, rho, ux, uy, fs)
    return fs


def mu_guess(lattice, Mn):
    mu = np.zeros(3 if lattice == D1Q3 else 4)
    lib().ora_mu_guess(lattice, np.ascontiguousarray(Mn, np.float64), mu)
    return mu


def newton(lattice, Mn, mu0=None, tol=1e-12, maxit=100):
    """Energy-constrained multipliers for Mn = (rho, j[, jy], 2E).

    Returns (mu, iterations); iterations = -1 when not converged.
    """
    Mn = np.ascontiguousarray(Mn, np.float64)
    mu = mu_guess(lattice, Mn) if mu0 is None else np.array(mu0, np.float64)
    it = lib().ora_newton(lattice, Mn, mu, tol, maxit)
    return mu, it


def elbm_alpha(lattice, f, fs):
    """ELBM parameter alpha of (elbmLB): S(f + alpha (f* - f)) = S(f)."""
    return lib().ora_elbm_alpha(lattice, np.ascontiguousarray(f, np.float64),
                                np.ascontiguousarray(fs, np.float64))


def perfect_entropy(lattice, f):
    return lib().ora_perfect_entropy(lattice, np.ascontiguousarray(f, np.float64))


def delta_s(lattice, f, fs):
    return lib().ora_delta_s(lattice, np.ascontiguousarray(f, np.float64),
                             np.ascontiguousarray(fs, np.float64))


def select(ds, delta, k, eligible=None):
    """Indices (ascending) of the k largest ds > delta (ties: lower index)."""
    ds = np.ascontiguousarray(ds, np.float64)
    out = np.zeros(max(int(k), 1), np.int64)
    el = None if eligible is None else np.ascontiguousarray(eligible, np.uint8)
    m = lib().ora_select(ds, _ptr(el), ds.size, delta, int(k), out)
    return out[:m].copy()


def fields(cfg, f):
    """(f*, dS) at every site of a pre-collision field."""
    fs = np.zeros_like(f)
    ds = np.zeros(cfg.n_sites)
    s = cfg.c_struct()
    fails = lib().ora_fields(C.byref(s), np.ascontiguousarray(f), _ptr(fs), _ptr(ds))
    if fails:
        raise RuntimeError("oracle Newton failed at %d sites" % fails)
    return fs, ds.reshape(cfg.ny, cfg.nx)


def moment_fields(cfg, f):
    N = cfg.n_sites
    rho, ux, uy, e2 = (np.zeros(N) for _ in range(4))
    s = cfg.c_struct()
    lib().ora_moment_fields(C.byref(s), np.ascontiguousarray(f), rho, ux, _ptr(uy), _ptr(e2))
    sh = (cfg.ny, cfg.nx)
    return rho.reshape(sh), ux.reshape(sh), uy.reshape(sh), e2.reshape(sh)


def init_field(cfg, rho, ux, uy=None, e2=None):
    f = np.zeros((cfg.q, cfg.ny, cfg.nx))
    s = cfg.c_struct()
    rho = np.ascontiguousarray(rho, np.float64).ravel()
    ux = np.ascontiguousarray(ux, np.float64).ravel()
    uyp = None if uy is None else np.ascontiguousarray(uy, np.float64).ravel()
    e2p = None if e2 is None else np.ascontiguousarray(e2, np.float64).ravel()
    rc = lib().ora_init(C.byref(s), rho, ux, _ptr(uyp), _ptr(e2p), f)
    if rc != 0:
        raise RuntimeError("oracle init failed")
    return f


@dataclass
class RunLog:
    counts: np.ndarray
    selected: list = field(default_factory=list)
    probe: np.ndarray = None


def run(cfg, f, nsteps, replay=None, log_selection=True, probe=None):
    """Advance the pre-collision field f (modified in place) by nsteps.

    replay: list of index arrays, one per step, to force the selection.
    probe: (x, y) site whose pre-collision u_x is logged each step.
    """
    f = np.ascontiguousarray(f, np.float64)
    s = cfg.c_struct()
    cnt = np.zeros(nsteps, np.int64)
    cap = max(1, nsteps * max(cfg.k, 0)) if log_selection else 0
    if replay is not None:
        rc_arr = np.array([len(r) for r in replay[:nsteps]], np.int64)
        ri = np.concatenate([np.asarray(r, np.int64) for r in replay[:nsteps]] +
                            [np.zeros(0, np.int64)])
        cap = max(cap, int(rc_arr.sum()) + 1)
    else:
        rc_arr = ri = None
    sel = np.zeros(cap, np.int64) if log_selection else None
    pr = np.zeros(nsteps) if probe is not None else None
    px, py = probe if probe is not None else (0, 0)
    rc = lib().ora_run(C.byref(s), f, nsteps, _ptr(rc_arr), _ptr(ri), _ptr(cnt),
                       _ptr(sel), cap, _ptr(pr), px, py)
    if rc != 0:
        raise RuntimeError("oracle run failed with status %d" % rc)
    out = RunLog(counts=cnt, probe=pr)
    if log_selection:
        off = 0
        for t in range(nsteps):
            out.selected.append(sel[off:off + cnt[t]].copy())
            off += cnt[t]
    return f, out


def collide(cfg, f, sel=()):
    sel = np.ascontiguousarray(np.asarray(sel, np.int64))
    fp = np.zeros_like(f)
    s = cfg.c_struct()
    rc = lib().ora_collide(C.byref(s), np.ascontiguousarray(f), _ptr(sel), sel.size, fp)
    if rc != 0:
        raise RuntimeError("oracle collide failed")
    return fp


def stream(cfg, fp):
    f = np.zeros_like(fp)
    s = cfg.c_struct()
    lib().ora_stream(C.byref(s), np.ascontiguousarray(fp), f)
    return f


def round_f32(x):
    """x rounded to the nearest IEEE binary32 value (ties to even)."""
    return lib().ora_round_f32(float(x))


def round_f16(x):
    """x rounded to the nearest IEEE binary16 value (ties to even)."""
    return lib().ora_round_f16(float(x))


def num_threads():
    return lib().ora_num_threads()


def set_num_threads(n):
    lib().ora_set_num_threads(int(n))
