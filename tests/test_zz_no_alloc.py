"""The allocation-free moments call (lb_moments_noalloc) against the context call (lb_moments).

lb_moments_noalloc serves callers that cannot allocate device memory: its staging area is a
static device array inside the library. It must give the same fields as lb_moments on the same
populations, call after call (the static array is shared and reused), and refuse lattices larger
than its fixed capacity. This file is collected last so that a failing run stopped at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1804_01918_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01918_gb300 import build, lb
    build.build()
    return lb


@pytest.mark.parametrize("Lx,Ly", [(64, 256), (256, 256)])   # 16384 sites; exactly the capacity
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32dev", 1e-14), ("fp32split", 1e-14)])
def test_noalloc_moments_match_context_moments_two_calls(L, precision, tol, Lx, Ly):
    assert Lx * Ly <= 65536
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9, precision=precision)
    base = lat._ws.data_ptr()             # population copy A: workspace offset 0
    for call in range(2):
        lat.step(2)                       # an even number of steps leaves the state in copy A
        lat.sync()
        want = lat.moments()
        got = L.moments_noalloc(Lx, Ly, base, precision=precision, stream=lat.stream)
        for g, w in zip(got, want):
            assert np.max(np.abs(g - w)) <= tol * max(1.0, float(np.max(np.abs(w)))), call
    lat.close()


def test_noalloc_rejects_lattices_beyond_capacity(L):
    import torch
    lib = L.lib()
    p = L.make_params(512, 256, 1.0)      # 131072 sites > 65536
    f = torch.zeros(37 * (256 + 6) * 512, dtype=torch.float64, device="cuda")
    out = np.empty((4, 256, 512), np.float64)
    st = lib.lb_moments_noalloc(C.byref(p), f.data_ptr(), *[o.ctypes.data for o in out])
    assert st == 1
    assert "exceeds the static scratch" in L.last_error()
