"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function include/lbm.h declares, and rejects bad arguments on the host."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(lb_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0705_4371_gb300 import build, lbm
    build.build()
    return lbm.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lb_create", "lb_step", "lb_moments", "lb_destroy", "lb_select_only",
              "lb_replay_selection", "lb_get_state", "lb_set_state"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_0705_4371_gb300 import lbm
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (lb_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_host_argument_checks_need_no_gpu(lib):
    from paper_0705_4371_gb300 import lbm
    h = C.c_void_p()
    bad = [
        (7, 64, 32, 0, 0.1, 1e-3, 4),           # unknown lattice
        (1, 64, 32, 9, 0.1, 1e-3, 4),           # unknown equilibrium
        (1, 64, 32, 0, -0.1, 1e-3, 4),          # nu <= 0
        (1, 64, 32, 0, 0.1, 1e-3, -1),          # k < 0
        (0, 64, 2, 0, 0.1, 1e-3, 4),            # D1Q3 with ny != 1
        (1, 2, 32, 0, 0.1, 1e-3, 4),            # grid too small
        (1, 64, 32, 0, 0.1, float("nan"), 4),   # delta NaN
    ]
    for lat, nx, ny, eq, nu, delta, k in bad:
        rc = lib.lb_create(lat, nx, ny, eq, nu, delta, k, None, lbm.LB_F32, None, C.byref(h))
        assert rc == lbm.LB_ERR_ARG, (lat, nx, ny, eq, nu, delta, k)
        assert lbm.last_error()
    b = lbm.boundaries((lbm.LB_FREESLIP, lbm.LB_OUTLET_EQ, lbm.LB_BB, lbm.LB_BB))
    assert lib.lb_create(1, 64, 32, 0, 0.1, 1e-3, 4, C.byref(b), lbm.LB_F32, None, C.byref(h)) == lbm.LB_ERR_ARG
    b = lbm.boundaries((lbm.LB_INLET_EQ, lbm.LB_OUTLET_EQ, lbm.LB_FREESLIP, lbm.LB_FREESLIP),
                       u_in=(0.05, 0), obstacle=(60, 10, 4, 4))   # too close to the outlet
    assert lib.lb_create(1, 64, 32, 0, 0.1, 1e-3, 4, C.byref(b), lbm.LB_F32, None, C.byref(h)) == lbm.LB_ERR_ARG
    b = lbm.boundaries((lbm.LB_PERIODIC, lbm.LB_BB, lbm.LB_BB, lbm.LB_BB))
    assert lib.lb_create(1, 64, 32, 0, 0.1, 1e-3, 4, C.byref(b), lbm.LB_F32, None, C.byref(h)) == lbm.LB_ERR_ARG
    b = lbm.boundaries(obstacle=(20, 10, 4, 4), wall=7)                # unknown wall rule
    assert lib.lb_create(1, 64, 32, 0, 0.1, 1e-3, 4, C.byref(b), lbm.LB_F32, None, C.byref(h)) == lbm.LB_ERR_ARG
    # a population array of 2^31 values or more
    assert lib.lb_create(1, 65536, 4096, 0, 0.1, 1e-3, 4, None, lbm.LB_F32, None, C.byref(h)) == lbm.LB_ERR_ARG
    assert lib.lb_step(None, 1) == lbm.LB_ERR_ARG
    lib.lb_destroy(None)   # NULL-safe
    assert lib.lb_mlp_param_count() == 64 * 4 + 64 + 64 * 64 + 64 + 4 * 64 + 4 + 12
