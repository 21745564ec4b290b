"""The C ABI used from plain C (tests/c_client/lb_client.c: no Python, no torch, library-owned
memory and stream), compared with the same run through the Python binding: both drive the same
kernels, so every printed sum must agree to the last digit."""
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01918_gb300 import build
    lib = build.build()
    exe = str(tmp_path_factory.mktemp("c_client") / "lb_client")
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "c_client", "lb_client.c"), "-o", exe, "-L", libdir, "-llb_d2q37",
                    "-Wl,-rpath," + libdir, "-lm"], check=True)
    return exe


def run_client(exe, steps, wall_mode):
    out = subprocess.run([exe, str(steps), str(wall_mode)], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


def python_run(steps, wall_mode):
    from paper_1804_01918_gb300 import lb
    Lx, Ly = 48, 40
    y, x = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    rho = 1.0 + 0.05 * np.sin(2.0 * np.pi * x / Lx) * np.cos(np.pi * y / Ly)
    ux = 0.01 * np.cos(2.0 * np.pi * y / Ly)
    uy = 0.005 * np.sin(2.0 * np.pi * x / Lx)
    T = 1.0 + 0.1 * (0.5 - y / (Ly - 1))
    lat = lb.Lattice(Lx, Ly, 0.8, rho, ux, uy, T, gy=-1e-4, T_top=0.95, T_bottom=1.05,
                     wall_mode=wall_mode)
    lat.step(steps)
    r, u, v, t = lat.moments()
    f = lat.get_populations()
    lat.close()
    return r, u, v, t, f


@pytest.mark.parametrize("wall_mode", [0, 1])
def test_c_client_matches_the_python_binding(client, wall_mode):
    c = run_client(client, 25, wall_mode)
    assert c["steps"] == 25
    r, u, v, t, f = python_run(25, wall_mode)
    # the same sums in the same order as the C program
    sums = {"sum_rho": 0.0, "sum_jx": 0.0, "sum_jy": 0.0, "sum_T": 0.0}
    for a, b, cc, d in zip(r.ravel(), u.ravel(), v.ravel(), t.ravel()):
        sums["sum_rho"] += a
        sums["sum_jx"] += a * b
        sums["sum_jy"] += a * cc
        sums["sum_T"] += d
    sum_f = 0.0
    for val in f.ravel():
        sum_f += val
    for k, val in sums.items():
        assert c[k] == val, k
    assert c["sum_f"] == sum_f
