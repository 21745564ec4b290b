"""One lattice cut into slabs on the GPU (include/lb_slab.h, paper_1804_01918_gb300/slabs.py): the
domain decomposition of the multi-GPU path, run here with every slab on the one GPU, exchanging
ghost rows device to device (lb_slab_exchange) or through packed buffers moved by a stand-in for
the rank-to-rank transport (lb_slab_pack / lb_slab_unpack, the split step that overlaps it).

Each slab runs the library's step kernel on its own rows, so the slabs together must equal the
single lattice bit for bit, and the FP64 oracle at the 1e-12 bar. The ghost rows of the cut sides
start as whatever the workspace held and only the 26 population-rows per cut and direction are ever
written; a schedule that read any other ghost entry would not reproduce the single lattice.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1804_01918_gb300 import inputs, slabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01918_gb300 import build, lb
    build.build()
    return lb


def fields_of(st):
    return (st.rho, st.ux, st.uy, st.T)


def single(L, st, tau, n, **kw):
    lat = L.Lattice.from_fields(st, tau=tau, **kw)
    lat.step(n)
    lat.sync()
    f = lat.get_populations()
    lat.close()
    return f


@pytest.mark.parametrize("wall_mode", ["rest", "mirror"])
@pytest.mark.parametrize("nslabs", [2, 4])
def test_slab_lattice_equals_single_lattice_and_oracle(L, orc, nslabs, wall_mode):
    Lx, Ly, tau, n = 64, 256, 0.9, 100
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    sl = slabs.SlabLattice(L, Lx, Ly, tau, fields_of(st), nslabs, gy=st.gy, T_top=st.T_top,
                           T_bottom=st.T_bottom, wall_mode=wall_mode)
    sl.step(n)
    sl.sync()
    got = sl.get_populations()
    sl.close()
    assert np.array_equal(got, single(L, st, tau, n, wall_mode=wall_mode))
    cx, cy, _, _ = L.velocity_set()
    want = orc.run(orc.init_fields(st), tau=tau, nsteps=n, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom, wall_mode=wall_mode)
    err = float(np.max(np.abs(orc.from_planes(got, cx, cy) - want) / np.abs(want)))
    print(f"{nslabs} slabs, {wall_mode} walls: max rel err vs oracle after {n} steps {err:.2e}")
    assert err <= 1e-12


@pytest.mark.parametrize("precision", ["fp32split", "fp32dev"])
def test_slab_lattice_fp32_forms_equal_single_lattice(L, precision):
    Lx, Ly, tau, n = 96, 120, 0.85, 40
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=3)
    sl = slabs.SlabLattice(L, Lx, Ly, tau, fields_of(st), 3, gy=st.gy, T_top=st.T_top,
                           T_bottom=st.T_bottom, precision=precision)
    sl.step(n)
    sl.sync()
    got = sl.get_populations()
    sl.close()
    assert np.array_equal(got, single(L, st, tau, n, precision=precision))


class LocalLinks:
    """Stand-in for the rank-to-rank transport with every rank in this process on one stream: a
    rank's receive buffers are copied from its neighbours' send buffers when it waits."""

    def __init__(self):
        self.ranks = []

    def transport_for(self, r):
        def transport(send_lo, send_hi, recv_lo, recv_hi):
            def wait():
                if r > 0:
                    recv_lo.copy_(self.ranks[r - 1].send_hi)
                if r < len(self.ranks) - 1:
                    recv_hi.copy_(self.ranks[r + 1].send_lo)
            return wait
        return transport


@pytest.mark.parametrize("overlap", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "fp32split"])
def test_slab_ranks_with_packed_transfers_equal_single_lattice(L, precision, overlap):
    """Three SlabRank objects: bands, pack, post, interior, wait, unpack -- the per-rank schedule of
    the multi-GPU path -- with buffers moved in process."""
    import torch
    Lx, Ly, tau, n, world = 64, 90, 0.9, 30, 3
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=5)
    stream = torch.cuda.Stream()
    links = LocalLinks()
    ranks = [slabs.SlabRank(L, Lx, Ly, tau, fields_of(st), r, world, links.transport_for(r), overlap=overlap,
                            gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom, precision=precision,
                            stream=stream) for r in range(world)]
    links.ranks = ranks
    for r in ranks:
        r.pack_ghosts()
    for r in ranks:
        r.receive_ghosts()
    for _ in range(n):
        for r in ranks:
            r.step_bands()
        for r in ranks:
            r.step_rest()
    for r in ranks:
        r.lat.sync()
    got = np.concatenate([r.lat.get_populations() for r in ranks], axis=1)
    for r in ranks:
        r.close()
    assert np.array_equal(got, single(L, st, tau, n, precision=precision))


def test_slab_pack_layout_is_the_ghost_table(L):
    """lb_slab_pack writes, row by row, the populations of ghost_table from the rows next to the cut."""
    import torch
    Lx, Ly = 40, 24
    st = inputs.random_state(Lx, Ly, seed=8)
    lat = L.Lattice(Lx, Ly, 0.9, *fields_of(st), cuts=3)
    buf = torch.empty(slabs.GHOST_ROWS * Lx, dtype=torch.float64, device="cuda")
    f = lat.get_populations()
    _, cy, _, _ = L.velocity_set()
    for side, up in ((0, False), (1, True)):
        with torch.cuda.stream(lat.stream):
            lat.slab_pack(side, buf)
        lat.sync()
        got = buf.cpu().numpy().reshape(slabs.GHOST_ROWS, Lx)
        want = np.stack([f[i, k - 1] if side == 0 else f[i, Ly - k] for i, k in slabs.ghost_table(cy, up)])
        assert np.array_equal(got, want), side
    lat.close()


def test_slab_argument_and_state_checks(L):
    import torch
    lib = L.lib()
    st = inputs.random_state(32, 16, seed=2)
    lo = L.Lattice(32, 16, 0.9, *fields_of(st), cuts=2)
    hi = L.Lattice(32, 16, 0.9, *fields_of(st), cuts=1)
    other = L.Lattice(40, 16, 0.9, *[np.zeros((16, 40)) + v for v in (1.0, 0.0, 0.0, 1.0)], cuts=1)
    L.slab_exchange(lo, hi)                                      # defined ghost rows for the steps below
    assert lib.lb_step(lo._ctx, 2) == 5                      # exchanges must come between steps
    buf = torch.empty(slabs.GHOST_ROWS * 32, dtype=torch.float64, device="cuda")
    assert lib.lb_slab_unpack(lo._ctx, 0, buf.data_ptr()) == 1   # side 0 of lo is a wall
    assert lib.lb_slab_exchange(lo._ctx, other._ctx) == 1        # Lx differs
    assert lib.lb_slab_exchange(hi._ctx, lo._ctx) == 1           # wrong sides
    assert lib.lb_slab_step(lo._ctx, 2) == 5                     # interior before bands
    assert lib.lb_slab_step(lo._ctx, 1) == 0
    assert lib.lb_slab_step(lo._ctx, 1) == 5                     # bands twice
    assert lib.lb_step(lo._ctx, 1) == 5                          # a split step is pending
    assert lib.lb_slab_step(lo._ctx, 2) == 0
    assert lib.lb_set_staging(lo._ctx, 1) == 5
    p = L.make_params(32, 5, 0.9)
    ctx = C.c_void_p()
    z = np.ones(32 * 5)
    assert lib.lb_init_slab(C.byref(p), 1, *(z.ctypes.data,) * 4, C.byref(ctx)) == 1   # Ly < 6
    assert lib.lb_init_slab(C.byref(p), 4, *(z.ctypes.data,) * 4, C.byref(ctx)) == 1   # bad cuts
    for lat in (lo, hi, other):
        lat.close()
