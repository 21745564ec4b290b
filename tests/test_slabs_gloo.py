"""The slab decomposition's exchange schedule (paper_1804_01918_gb300/slabs.py) on gloo ranks on
the CPU, against the single-lattice result of the oracle.

Each rank holds one slab of a Rayleigh-Taylor lattice (walls at the global top and bottom,
periodic x) and advances it with the oracle's own walls, pull and collide; after every step it packs
the rows it sends across its cuts in ghost_table order, exchanges them with its neighbours through
exchange_ghosts (torch.distributed point-to-point over gloo), and unpacks what arrived into its
ghost rows. Every ghost-row entry outside the 26 population-rows per cut and direction is NaN, so
a schedule that needed any other entry would spread NaN. The gathered slabs must equal the oracle's
run of the whole lattice bit for bit (the same per-site arithmetic in the same order).
"""
import os
import socket

import numpy as np
import pytest

from paper_1804_01918_gb300 import slabs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


LX, LY, TAU, STEPS = 24, 40, 0.8, 12


def _fields():
    from paper_1804_01918_gb300 import inputs
    st = inputs.random_state(LX, LY, seed=31, du=0.05, dT=0.15, drho=0.15)
    return inputs.RTFields(st.rho, st.ux, st.uy, st.T, T_top=0.9, T_bottom=1.1, gy=-1e-3)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from oracle import oracle as orc
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = _fields()
        y0, h = slabs.split_rows(LY, world)[rank]
        cuts = slabs.cuts_of(rank, world)
        _, cy, _, _ = orc.velocity_set()
        up, down = slabs.ghost_table(cy, True), slabs.ghost_table(cy, False)
        f = orc.equilibrium(*[a[y0:y0 + h] for a in (st.rho, st.ux, st.uy, st.T)])
        nan = np.full((3, LX, 37), np.nan)
        ghost_lo, ghost_hi = nan.copy(), nan.copy()   # padded rows 0..2 and h+3..h+5
        buf = lambda: torch.zeros(slabs.GHOST_ROWS * LX, dtype=torch.float64)
        send_lo, send_hi, recv_lo, recv_hi = buf(), buf(), buf(), buf()

        def exchange(f):
            if cuts & 1:   # rows sent down: populations moving down, from rows k - 1
                send_lo.copy_(torch.from_numpy(np.stack([f[k - 1, :, i] for i, k in down]).ravel()))
            if cuts & 2:   # rows sent up: populations moving up, from rows h - k
                send_hi.copy_(torch.from_numpy(np.stack([f[h - k, :, i] for i, k in up]).ravel()))
            slabs.exchange_ghosts(dist, rank, world, send_lo, send_hi, recv_lo, recv_hi)()
            if cuts & 1:   # arriving below: populations moving up, into ghost row -k (padded 3 - k)
                r = recv_lo.numpy().reshape(slabs.GHOST_ROWS, LX)
                for j, (i, k) in enumerate(up):
                    ghost_lo[3 - k, :, i] = r[j]
            if cuts & 2:   # arriving above: populations moving down, into ghost row h - 1 + k
                r = recv_hi.numpy().reshape(slabs.GHOST_ROWS, LX)
                for j, (i, k) in enumerate(down):
                    ghost_hi[k - 1, :, i] = r[j]

        exchange(f)
        for _ in range(STEPS):
            full = orc.with_walls(f, st.T_top, st.T_bottom)
            if cuts & 1:
                full[:3] = ghost_lo
            if cuts & 2:
                full[h + 3:] = ghost_hi
            f = orc.collide(orc.propagate(full, LX, h, False), TAU, 0.0, st.gy)
            exchange(f)
        q.put((rank, y0, f))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_exchange_on_gloo_ranks_equals_the_whole_lattice(orc, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([t[2] for t in parts], axis=0)
    assert [t[1] for t in parts] == [y0 for y0, _ in slabs.split_rows(LY, world)]
    st = _fields()
    want = orc.run(orc.init_fields(st), tau=TAU, nsteps=STEPS, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom)
    assert np.all(np.isfinite(got))
    assert np.array_equal(got, want)


def test_split_rows_and_cuts():
    assert slabs.split_rows(40, 3) == [(0, 14), (14, 13), (27, 13)]
    assert slabs.split_rows(12, 2) == [(0, 6), (6, 6)]
    with pytest.raises(ValueError):
        slabs.split_rows(11, 2)
    assert [slabs.cuts_of(k, 4) for k in range(4)] == [2, 3, 3, 1]
    assert slabs.cuts_of(0, 1) == 0


def test_ghost_table_has_15_8_3_rows_per_direction(orc):
    """Ghost row k of a cut is read by the pull for exactly the populations crossing the cut by at
    least k rows: 15, 8 and 3 of the 37 (brute force over the pull's reach)."""
    cx, cy, _, _ = orc.velocity_set()
    for up in (True, False):
        t = slabs.ghost_table(cy, up)
        assert [sum(1 for _, k in t if k == kk) for kk in (1, 2, 3)] == [15, 8, 3]
        # brute force: rows 0..2 pull population i from row y - c_y; collect the ghost rows reached
        needed = set()
        for y in range(3):
            for i in range(37):
                src = y - int(cy[i]) if up else y + int(cy[i])   # mirror for the side above
                if src < 0:
                    needed.add((i, -src))
        assert needed == set(t)
