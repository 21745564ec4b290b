"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every function that
include/*.h declares, and its pure-host calls behave (velocity set, workspace size, arguments)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1804_01918_gb300 import build, lb
    build.build()
    return lb


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lb_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15, names
    lib = L.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_velocity_set_matches_the_oracle_as_a_set(L, orc):
    cx, cy, w, r = L.velocity_set()
    ocx, ocy, ow, orr = orc.velocity_set()
    perm = orc.order_map(cx, cy)           # raises unless the same 37 vectors
    assert np.array_equal(ow[perm], w)     # same weights per vector
    assert r == orr
    # opposite pairs: population 18 + k moves opposite to k
    assert np.array_equal(cx[19:], -cx[1:19]) and np.array_equal(cy[19:], -cy[1:19])


def test_workspace_bytes_is_the_double_buffered_soa_footprint(L):
    """Table 1: 1024x8192 needs ~4.6 GB (two FP64 copies of 37 populations); the library adds
    3 halo rows per wall and a host-exchange staging area of 4 fields."""
    n = L.workspace_bytes(1024, 8192, "fp64")
    pops = 2 * 37 * 8 * 1024 * (8192 + 6)
    stage = 4 * 8 * 1024 * 8192
    assert pops <= n <= pops + stage + 4096
    assert pops / 2**30 == pytest.approx(4.6, abs=0.05)
    n32 = L.workspace_bytes(1024, 8192, "fp32dev")
    assert 2 * 37 * 4 * 1024 * (8192 + 6) <= n32 < n


def test_invalid_arguments_are_rejected_without_a_gpu(L):
    lib = L.lib()
    n = C.c_size_t()
    p = L.make_params(3, 100, 0.9)
    assert lib.lb_workspace_bytes(C.byref(p), C.byref(n)) == 1
    p = L.make_params(100, 100, 0.9, precision=0)
    p.precision = 7
    assert lib.lb_workspace_bytes(C.byref(p), C.byref(n)) == 1
    assert lib.lb_workspace_bytes(None, C.byref(n)) == 1
    ctx = C.c_void_p()
    p = L.make_params(64, 64, 0.5)  # tau must exceed 1/2
    z = np.zeros(64 * 64)
    assert lib.lb_init(C.byref(p), z.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                       C.byref(ctx)) == 1
    assert lib.lb_step(None, 1) == 1
    for field, value in (("wall_mode", 5), ("gx", float("nan")), ("T_top", 0.0), ("T_bottom", -1.0),
                         ("tau", float("inf"))):
        p = L.make_params(64, 64, 0.9)
        setattr(p, field, value)
        assert lib.lb_init(C.byref(p), z.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                           C.byref(ctx)) == 1, field
    lib.lb_free(None)
    # ensemble members get the single-lattice checks (no GPU needed: the workspace query validates)
    for field, value in (("tau", float("inf")), ("tau", 0.5), ("T_top", float("inf")),
                         ("T_bottom", float("nan")), ("gx", float("nan")), ("gy", float("-inf")),
                         ("wall_mode", 1)):
        members = (L.lb_params * 2)(L.make_params(64, 64, 0.9), L.make_params(32, 128, 0.8))
        setattr(members[1], field, value)
        assert lib.lb_ensemble_workspace_bytes(2, members, None, C.byref(n)) == 1, field
    members = (L.lb_params * 2)(L.make_params(64, 64, 0.9), L.make_params(32, 128, 0.8))
    assert lib.lb_ensemble_workspace_bytes(2, members, None, C.byref(n)) == 0
    assert lib.lb_status_str(4) == b"non-finite or non-positive density/temperature"
