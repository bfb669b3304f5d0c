"""Thin ctypes binding of liblbm.so (declared in include/lbm.h).

Argument marshalling only: every step of the lattice Boltzmann path runs in
the library's CUDA kernels.  ``load()`` raises if the library is missing or
cannot be loaded; there is no fallback.  Array arguments are numpy FP64
arrays on the host, or (where the C function takes ``on_device``) CUDA
device pointers given as integers (e.g. ``torch.Tensor.data_ptr()``).
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LB_D1Q3, LB_D2Q9 = 0, 1
LB_EQ_POLY, LB_EQ_ENTROPIC, LB_EQ_ENTROPIC_ENERGY, LB_EQ_ENTROPIC_ENERGY_MLP = 0, 1, 2, 3
LB_F64, LB_F32, LB_F32_DEV, LB_F16_DEV = 0, 1, 2, 3
LB_BB, LB_FREESLIP, LB_INLET_EQ, LB_OUTLET_EQ, LB_PERIODIC, LB_OUTLET_COPY = 0, 1, 2, 3, 4, 5
LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_NONFINITE, LB_ERR_NEWTON, LB_ERR_TIMEOUT, LB_ERR_OOM, \
    LB_ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7

PRECISIONS = {"f64": LB_F64, "f32": LB_F32, "f32dev": LB_F32_DEV, "f16dev": LB_F16_DEV}
LB_COLLISION_LBGK, LB_COLLISION_ELBM = 0, 1
LB_WALL_BOUNCE_BACK, LB_WALL_DIFFUSE = 0, 1


class LBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("liblbm error %d: %s" % (code, msg))
        self.code = code


class lb_boundaries(C.Structure):
    _fields_ = [("kind_x0", C.c_int), ("kind_x1", C.c_int), ("kind_y0", C.c_int),
                ("kind_y1", C.c_int), ("rho_in", C.c_double), ("u_in", C.c_double * 2),
                ("obstacle_x0", C.c_int), ("obstacle_y0", C.c_int), ("obstacle_w", C.c_int),
                ("obstacle_h", C.c_int), ("obstacle_wall", C.c_int)]


class lb_run_desc(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("equilibrium", C.c_int),
                ("nu", C.c_double), ("delta", C.c_double), ("k", C.c_int), ("bc", lb_boundaries),
                ("precision", C.c_int)]


_lib = None


def load(path=None):
    """Load liblbm.so (raises OSError if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError("liblbm.so not built at %s (run paper_0705_4371_gb300/build.py)" % path)
    L = C.CDLL(path)
    vp, ip, dp, fp = C.c_void_p, C.c_int, C.c_double, C.c_float
    H = C.c_void_p
    sig = {
        "lb_create": ([ip, ip, ip, ip, dp, dp, ip, C.POINTER(lb_boundaries), ip, vp, C.POINTER(H)], ip),
        "lb_destroy": ([H], None),
        "lb_init_equilibrium": ([H, vp, vp, vp, vp], ip),
        "lb_get_state": ([H, vp], ip),
        "lb_set_state": ([H, vp], ip),
        "lb_step": ([H, ip], ip),
        "lb_sync": ([H], ip),
        "lb_moments": ([H, vp, vp, vp, vp, ip], ip),
        "lb_set_state_async": ([H, vp], ip),
        "lb_moments_async": ([H, vp, vp, vp, vp], ip),
        "lb_selected": ([H, vp, ip, C.POINTER(ip)], ip),
        "lb_counts": ([H, vp, ip], ip),
        "lb_set_probe": ([H, ip, ip], ip),
        "lb_probe": ([H, vp, ip], ip),
        "lb_set_log_capacity": ([H, ip], ip),
        "lb_delta_s": ([H, vp, ip], ip),
        "lb_select_only": ([vp, ip, dp, ip, vp, C.POINTER(ip)], ip),
        "lb_replay_selection": ([H, vp, vp, ip], ip),
        "lb_mlp_param_count": ([], ip),
        "lb_set_mlp": ([H, vp, ip], ip),
        "lb_set_collision": ([H, ip], ip),
        "lb_newton_stats": ([H, vp, vp, vp, vp, ip], ip),
        "lb_set_timing": ([H, ip], ip),
        "lb_kernel_times": ([H, vp, vp, vp, vp, ip], ip),
        "lb_info": ([H, vp, vp], ip),
        "lb_set_tile_shape": ([H, ip], ip),
        "lb_select_only_noalloc": ([vp, ip, dp, ip, vp, vp, vp], ip),
        "lb_mlp_init": ([vp, ip, C.c_ulonglong], ip),
        "lb_batch_create": ([C.POINTER(lb_run_desc), ip, vp, C.POINTER(vp)], ip),
        "lb_batch_destroy": ([vp], None),
        "lb_batch_run": ([vp, ip], vp),
        "lb_batch_step": ([vp, ip], ip),
        "lb_batch_step_sequential": ([vp, ip], ip),
        "lb_batch_sync": ([vp], ip),
        "lb_batch_set_variant": ([vp, ip], ip),
        "lb_batch_autotune": ([vp, ip, C.c_char_p, C.POINTER(ip)], ip),
        "lb_batch_set_timing": ([vp, ip], ip),
        "lb_batch_kernel_times": ([vp, C.POINTER(dp), C.POINTER(C.c_longlong), ip], ip),
        "lb_batch_info": ([vp, vp], ip),
        "lb_energy_dataset": ([vp, vp, vp, vp, C.c_longlong, vp, vp, vp, vp, vp], ip),
        "lb_mlp_normalise": ([vp, vp, vp, C.c_longlong, vp], ip),
        "lb_mlp_forward": ([vp, vp, C.c_longlong, vp, vp], ip),
        "lb_mlp_grad": ([vp, vp, vp, ip, vp, vp, vp], ip),
        "lb_mlp_adam": ([vp, vp, vp, vp, C.c_longlong, dp, vp], ip),
        "lb_mlp_train": ([vp, vp, vp, C.c_longlong, ip, ip, dp, dp, vp, vp], ip),
        "lb_set_slab": ([H, ip, ip, ip, ip], ip),
        "lb_slab_collide": ([H], ip),
        "lb_slab_candidates": ([H, vp, vp, ip, C.POINTER(ip)], ip),
        "lb_slab_apply": ([H, vp, ip], ip),
        "lb_slab_ghost": ([H, ip, vp, ip], ip),
        "lb_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def last_error():
    """Message of the calling thread's last failed library call (lb_last_error)."""
    return load().lb_last_error().decode()


def _check(rc):
    if rc != LB_OK:
        raise LBError(rc, last_error())
    return rc


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return C.c_void_p(a)
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def boundaries(kinds=(LB_BB,) * 4, rho_in=1.0, u_in=(0.0, 0.0), obstacle=(0, 0, 0, 0), wall=0):
    """An lb_boundaries struct: side kinds (x0, x1, y0, y1), inlet state, obstacle rectangle (x0,
    y0, w, h; w = 0: none) and its wall rule."""
    b = lb_boundaries()
    b.kind_x0, b.kind_x1, b.kind_y0, b.kind_y1 = kinds
    b.rho_in = rho_in
    b.u_in[0], b.u_in[1] = u_in
    b.obstacle_x0, b.obstacle_y0, b.obstacle_w, b.obstacle_h = obstacle
    b.obstacle_wall = wall
    return b


def select_only(ds, delta, k):
    """lb_select_only: indices (sorted) of the k largest ds > delta."""
    L = load()
    ds = np.ascontiguousarray(ds, np.float64)
    out = np.zeros(max(1, min(int(k), ds.size)), np.int32)
    cnt = C.c_int(0)
    _check(L.lb_select_only(_ptr(ds), ds.size, float(delta), int(k), _ptr(out), C.byref(cnt)))
    return np.sort(out[:cnt.value].astype(np.int64))


NOALLOC_MAX_N = 262144


def select_only_noalloc(ds_ptr, n, delta, k, idx_ptr, count_ptr, stream=None):
    """lb_select_only_noalloc on device pointers (integers); asynchronous on
    `stream` (a cudaStream_t as an integer, or None).  Allocates nothing."""
    L = load()
    _check(L.lb_select_only_noalloc(C.c_void_p(ds_ptr), int(n), float(delta), int(k),
                                    C.c_void_p(idx_ptr), C.c_void_p(count_ptr),
                                    C.c_void_p(stream) if stream else None))


def mlp_param_count():
    """Number of FP32 parameters of the 4-64-64-4 network (lb_mlp_param_count)."""
    return load().lb_mlp_param_count()


# Learned form (device pointers are integers, streams cudaStream_t integers
# or None; every call is asynchronous on its stream) ----------------------

def _vp(x):
    return C.c_void_p(x) if x else None


def mlp_init(seed):
    """Initial parameters (host FP32 array), lb_mlp_init."""
    L = load()
    p = np.zeros(L.lb_mlp_param_count(), np.float32)
    _check(L.lb_mlp_init(_ptr(p), p.size, int(seed) & ((1 << 64) - 1)))
    return p


def energy_dataset(rho, ux, uy, escale, n, feat, dmu, mu=None, stats=None, stream=None):
    """lb_energy_dataset: features and multiplier targets of n samples by the GPU Newton solve."""
    _check(load().lb_energy_dataset(_vp(rho), _vp(ux), _vp(uy), _vp(escale), int(n), _vp(feat),
                                    _vp(dmu), _vp(mu), _vp(stats), _vp(stream)))


def mlp_normalise(params, feat, dmu, n, stream=None):
    """lb_mlp_normalise: fold the training set's standardisation into the parameters."""
    _check(load().lb_mlp_normalise(_vp(params), _vp(feat), _vp(dmu), int(n), _vp(stream)))


def mlp_forward(params, feat, n, y, stream=None):
    """lb_mlp_forward: network outputs y[n][4] for features feat[n][4]."""
    _check(load().lb_mlp_forward(_vp(params), _vp(feat), int(n), _vp(y), _vp(stream)))


def mlp_grad(params, feat, dmu, n, grad, loss=None, stream=None):
    """lb_mlp_grad: gradient (and optionally the loss) of the mean squared error."""
    _check(load().lb_mlp_grad(_vp(params), _vp(feat), _vp(dmu), int(n), _vp(grad), _vp(loss),
                              _vp(stream)))


def mlp_adam(params, grad, m, v, t, lr, stream=None):
    """lb_mlp_adam: one Adam update of the parameters."""
    _check(load().lb_mlp_adam(_vp(params), _vp(grad), _vp(m), _vp(v), int(t), float(lr), _vp(stream)))


def mlp_train(params, feat, dmu, n, batch, epochs, lr0, lr1, loss_log=None, stream=None):
    """lb_mlp_train: epochs of mini-batch Adam with a geometric learning-rate decay."""
    _check(load().lb_mlp_train(_vp(params), _vp(feat), _vp(dmu), int(n), int(batch), int(epochs),
                               float(lr0), float(lr1), _vp(loss_log), _vp(stream)))


class Lattice:
    """One run (a lb_handle).  Mirrors the C calls one to one."""

    def __init__(self, lattice, nx, ny, equilibrium, nu, delta, k, bc=None, precision=LB_F32,
                 stream=None):
        self.L = load()
        self.lattice, self.nx, self.ny = lattice, nx, ny
        self.q = 3 if lattice == LB_D1Q3 else 9
        h = C.c_void_p()
        bptr = C.byref(bc) if bc is not None else None
        st = C.c_void_p(stream) if stream else None
        _check(self.L.lb_create(lattice, nx, ny, equilibrium, float(nu), float(delta), int(k),
                                bptr, precision, st, C.byref(h)))
        self.h = h

    @classmethod
    def _borrow(cls, handle, lattice, nx, ny):
        """A run owned by someone else (a batch): close() does not destroy it."""
        self = cls.__new__(cls)
        self.L = load()
        self.lattice, self.nx, self.ny = lattice, nx, ny
        self.q = 3 if lattice == LB_D1Q3 else 9
        self.h = C.c_void_p(handle)
        self._borrowed = True
        return self

    @classmethod
    def from_workload(cls, w, precision=LB_F32, stream=None, **over):
        """Create from a paper_0705_4371_gb300.inputs.Workload."""
        p = dict(nu=w.nu, delta=w.delta, k=w.k, equilibrium=w.eq)
        p.update(over)
        bc = boundaries(w.bc, w.rho_in, w.u_in, w.obstacle, p.get("wall", w.wall))
        return cls(w.lattice, w.nx, w.ny, p["equilibrium"], p["nu"], p["delta"], p["k"], bc, precision,
                   stream)

    def close(self):
        """Destroy the run (lb_destroy); a run borrowed from a batch is left to the batch."""
        if getattr(self, "h", None):
            if not getattr(self, "_borrowed", False):
                self.L.lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shape(self):
        """(ny, nx) of the site fields."""
        return (self.ny, self.nx)

    def init_equilibrium(self, rho, ux, uy=None, e2=None):
        """Quasiequilibrium of the given host fields at every fluid site (lb_init_equilibrium); e2
        (2E) for the energy forms."""
        rho, ux, uy, e2 = _f64(rho), _f64(ux), _f64(uy), _f64(e2)
        _check(self.L.lb_init_equilibrium(self.h, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(e2)))

    def get_state(self):
        """Pre-collision populations of the current step, FP64 [Q][ny][nx] in the paper's numbering
        (lb_get_state)."""
        f = np.zeros((self.q, self.ny, self.nx))
        _check(self.L.lb_get_state(self.h, _ptr(f)))
        return f

    def set_state(self, f):
        """Load populations (FP64 [Q][ny][nx]); the next step starts from them (lb_set_state)."""
        f = _f64(f)
        assert f.size == self.q * self.nx * self.ny
        _check(self.L.lb_set_state(self.h, _ptr(f)))

    def step(self, n=1):
        """Queue n time steps on the run's stream (lb_step; graphs of 32 steps where possible);
        raises on a sticky error of earlier work."""
        return _check(self.L.lb_step(self.h, int(n)))

    def sync(self):
        """Wait for the run's queued work (lb_sync)."""
        return _check(self.L.lb_sync(self.h))

    def moments(self):
        """(rho, ux, uy, 2E) of the current pre-collision state as FP64 host arrays [ny][nx]
        (lb_moments)."""
        rho, ux, uy, e2 = (np.zeros(self.shape) for _ in range(4))
        _check(self.L.lb_moments(self.h, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(e2), 0))
        return rho, ux, uy, e2

    def set_state_async(self, f):
        """lb_set_state_async: queue the upload of f (an FP64 [Q][ny][nx] C-contiguous array,
        kept unchanged by the caller until sync())."""
        assert f.dtype == np.float64 and f.flags.c_contiguous and f.size == self.q * self.nx * self.ny
        _check(self.L.lb_set_state_async(self.h, _ptr(f)))

    def moments_async(self, rho, ux, uy=None, e2=None):
        """lb_moments_async into caller-provided FP64 [ny][nx] host arrays, valid after sync()."""
        for a in (rho, ux, uy, e2):
            assert a is None or (a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.nx * self.ny)
        _check(self.L.lb_moments_async(self.h, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(e2)))

    def moments_device(self, rho_ptr, ux_ptr, uy_ptr=None, e2_ptr=None):
        """lb_moments into caller-provided device arrays (integer pointers; asynchronous)."""
        _check(self.L.lb_moments(self.h, _ptr(rho_ptr), _ptr(ux_ptr), _ptr(uy_ptr), _ptr(e2_ptr), 1))

    def delta_s(self):
        """Exact dS of every site of the current pre-collision state (NaN at solid sites;
        lb_delta_s)."""
        ds = np.zeros(self.shape)
        _check(self.L.lb_delta_s(self.h, _ptr(ds), 0))
        return ds

    def selected(self, cap=1 << 20):
        """Sorted indices y nx + x of the sites the last step moved to f* (lb_selected)."""
        idx = np.zeros(cap, np.int32)
        cnt = C.c_int(0)
        _check(self.L.lb_selected(self.h, _ptr(idx), cap, C.byref(cnt)))
        return np.sort(idx[:min(cnt.value, cap)].astype(np.int64))

    def counts(self, n):
        """Ehrenfests' sites of each of the last n steps, oldest first (lb_counts)."""
        out = np.zeros(n, np.int32)
        _check(self.L.lb_counts(self.h, _ptr(out), int(n)))
        return out

    def set_probe(self, x, y):
        """Log u_x at site (x, y) every step (lb_set_probe)."""
        _check(self.L.lb_set_probe(self.h, int(x), int(y)))

    def probe(self, n):
        """The last n logged u_x values of the probe site, oldest first (lb_probe)."""
        out = np.zeros(n)
        _check(self.L.lb_probe(self.h, _ptr(out), int(n)))
        return out

    def set_log_capacity(self, n):
        """Steps kept by the count and probe rings (lb_set_log_capacity)."""
        _check(self.L.lb_set_log_capacity(self.h, int(n)))

    def replay_selection(self, selections):
        """Make the next len(selections) steps take the given sets as their Ehrenfests' sites
        (lb_replay_selection)."""
        counts = np.array([len(s) for s in selections], np.int32)
        idx = np.concatenate([np.asarray(s, np.int32) for s in selections] + [np.zeros(0, np.int32)])
        idx = np.ascontiguousarray(idx, np.int32)
        _check(self.L.lb_replay_selection(self.h, _ptr(counts), _ptr(idx), len(selections)))

    def set_collision(self, collision):
        """LB_COLLISION_LBGK or LB_COLLISION_ELBM (entropic f* only; lb_set_collision)."""
        _check(self.L.lb_set_collision(self.h, int(collision)))

    def set_mlp(self, params):
        """Load the learned form's network (host FP32 parameters; lb_set_mlp)."""
        p = np.ascontiguousarray(params, np.float32)
        _check(self.L.lb_set_mlp(self.h, _ptr(p), p.size))

    def newton_stats(self, reset=False):
        """(FP32 iterations, finishing iterations, sites solved, sites that missed 1e-12) of the
        energy forms (lb_newton_stats)."""
        v = [C.c_longlong(0) for _ in range(4)]
        _check(self.L.lb_newton_stats(self.h, *(C.byref(x) for x in v), int(reset)))
        return tuple(x.value for x in v)

    def set_timing(self, enable):
        """Time every stream-collide launch with CUDA events (direct launches instead of graphs;
        lb_set_timing)."""
        _check(self.L.lb_set_timing(self.h, int(bool(enable))))

    def kernel_times(self, reset=False):
        """Summed kernel milliseconds and launch counts since the last reset (lb_kernel_times)."""
        cm, sm = C.c_double(0), C.c_double(0)
        cn, sn = C.c_longlong(0), C.c_longlong(0)
        _check(self.L.lb_kernel_times(self.h, C.byref(cm), C.byref(cn), C.byref(sm), C.byref(sn),
                                      int(reset)))
        return {"collide_ms": cm.value, "collide_launches": cn.value,
                "select_ms": sm.value, "select_launches": sn.value}

    # slabs of a run sharded in x (lb_set_slab ... lb_slab_ghost)
    def set_slab(self, ghost_left, ghost_right, global_x0, global_nx):
        """Make the run a slab of a run sharded in x (lb_set_slab)."""
        _check(self.L.lb_set_slab(self.h, int(ghost_left), int(ghost_right), int(global_x0), int(global_nx)))

    def slab_collide(self):
        """Queue the slab's stream + collide launch (lb_slab_collide)."""
        _check(self.L.lb_slab_collide(self.h))

    def slab_candidates(self, cap):
        """The slab's best candidates of the collided step: (uint64 keys, int64 global site
        indices) (lb_slab_candidates)."""
        keys = np.zeros(max(1, cap), np.uint64)
        idx = np.zeros(max(1, cap), np.int64)
        cnt = C.c_int(0)
        _check(self.L.lb_slab_candidates(self.h, _ptr(keys), _ptr(idx), int(cap), C.byref(cnt)))
        m = min(cnt.value, cap)
        return keys[:m].copy(), idx[:m].copy()

    def slab_apply(self, global_idx):
        """Apply the step's global selection and complete the step (lb_slab_apply)."""
        g = np.ascontiguousarray(global_idx, np.int64)
        _check(self.L.lb_slab_apply(self.h, _ptr(g), g.size))

    def slab_ghost(self, side, buf_ptr, direction):
        """Pack (direction 0) or unpack (1) a side's crossing populations to / from a device
        buffer given as an integer pointer (lb_slab_ghost)."""
        _check(self.L.lb_slab_ghost(self.h, int(side), C.c_void_p(buf_ptr), int(direction)))

    def set_tile_shape(self, shape):
        """Tile shape of the D2Q9 stream-collide kernel (0-6; lb_set_tile_shape); results do not
        depend on it."""
        _check(self.L.lb_set_tile_shape(self.h, int(shape)))

    def info(self):
        """Run facts: populations, row padding, bytes per population and per site update, launches
        per step, grid, tile shape, beta (lb_info)."""
        out = np.zeros(8, np.int64)
        beta = C.c_double(0)
        _check(self.L.lb_info(self.h, _ptr(out), C.byref(beta)))
        return {"Q": int(out[0]), "nxp": int(out[1]), "bytes_per_pop": int(out[2]),
                "bytes_per_site": int(out[3]), "launches_per_step": int(out[4]),
                "grid_blocks": int(out[5]), "blocks_per_sm": int(out[6]),
                "tile_shape": int(out[7]), "beta": beta.value}


class Batch:
    """Many D2Q9 runs advanced together (lb_batch_*).  runs(r) gives run r as
    a Lattice (owned by the batch) for initialisation and reading."""

    def __init__(self, workloads, precision=LB_F32_DEV, stream=None, equilibrium=None):
        self.L = load()
        n = len(workloads)
        descs = (lb_run_desc * n)()
        for d, w in zip(descs, workloads):
            d.lattice, d.nx, d.ny = LB_D2Q9, w.nx, w.ny
            d.equilibrium = w.eq if equilibrium is None else equilibrium
            d.nu, d.delta, d.k = w.nu, w.delta, w.k
            d.bc = boundaries(w.bc, w.rho_in, w.u_in, w.obstacle, w.wall)
            d.precision = precision
        h = C.c_void_p()
        _check(self.L.lb_batch_create(descs, n, C.c_void_p(stream) if stream else None, C.byref(h)))
        self.h = h
        self.workloads = list(workloads)
        self._runs = [Lattice._borrow(self.L.lb_batch_run(h, r), LB_D2Q9, w.nx, w.ny)
                      for r, w in enumerate(workloads)]

    def run(self, r):
        """The r-th run as a Lattice (borrowed: its state, logs and exports; stepping goes through
        the batch)."""
        return self._runs[r]

    def __len__(self):
        return len(self._runs)

    def step(self, n=1):
        """Advance every run by n steps with the chosen launch strategy (lb_batch_step)."""
        _check(self.L.lb_batch_step(self.h, int(n)))

    def step_sequential(self, n=1):
        """Advance every run by n steps, one run after another through its own graphs
        (lb_batch_step_sequential)."""
        _check(self.L.lb_batch_step_sequential(self.h, int(n)))

    def sync(self):
        """Wait for the batch's queued work (lb_batch_sync)."""
        _check(self.L.lb_batch_sync(self.h))

    def set_variant(self, v):
        """Launch strategy: 0/1 batched kernel with 8- or 4-row tiles, 2 concurrent per-run kernels
        (lb_batch_set_variant)."""
        _check(self.L.lb_batch_set_variant(self.h, int(v)))

    def autotune(self, steps=20, cache_path=None):
        """Time every strategy (or read the cache) and keep the fastest; returns its number
        (lb_batch_autotune)."""
        v = C.c_int(-1)
        _check(self.L.lb_batch_autotune(self.h, int(steps), cache_path.encode() if cache_path else None,
                                        C.byref(v)))
        return v.value

    def set_timing(self, enable):
        """Time each step of the batch with CUDA events (lb_batch_set_timing)."""
        _check(self.L.lb_batch_set_timing(self.h, int(enable)))

    def kernel_times(self, reset=False):
        """Summed step milliseconds and step counts since the last reset (lb_batch_kernel_times)."""
        ms, n = C.c_double(0), C.c_longlong(0)
        _check(self.L.lb_batch_kernel_times(self.h, C.byref(ms), C.byref(n), int(reset)))
        return {"ms": ms.value, "launches": n.value}

    def info(self):
        """Batch facts: runs, sites, tiles, grid, blocks per SM, strategy, tile rows, graph steps
        (lb_batch_info)."""
        out = np.zeros(8, np.int64)
        _check(self.L.lb_batch_info(self.h, _ptr(out)))
        keys = ("runs", "sites", "tiles", "grid_blocks", "blocks_per_sm", "variant", "tile_rows",
                "graph_steps")
        return dict(zip(keys, (int(x) for x in out)))

    def close(self):
        """Destroy the batch and its runs (lb_batch_destroy)."""
        if getattr(self, "h", None):
            for r in self._runs:
                r.h = None
            self.L.lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
