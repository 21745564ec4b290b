"""One lattice cut into horizontal slabs (include/lb_slab.h): the plan and the drivers.

The paper runs on one KNL socket and leaves a hybrid MPI + OpenMP code over many nodes to future
work (Sec. 5). A D2Q37 step of a site reads sites at most three rows away (Sec. 3), so a lattice cut
along y into slabs needs, per step and per cut, only the populations that cross the cut: ghost row
k below a slab (k = 1, 2, 3) is read for populations with c_y >= k, ghost row k above it for
c_y <= -k -- 26 population-rows each way (``ghost_table``). x stays periodic inside every slab; the
global walls stay on the outer sides of the first and last slab (``cuts_of``).

Drivers:

* ``SlabLattice``: all slabs in this process on one device; after every step each cut is exchanged
  lattice to lattice (lb_slab_exchange).
* ``SlabRank``: one slab per rank. Each step writes the rows next to its cuts first, packs them,
  hands them to a transport (``exchange_ghosts`` over torch.distributed point-to-point, NCCL on
  GPUs), writes its interior rows while they travel, then unpacks what arrived into its ghost rows.

Every slab runs the library's own step kernel on its rows, so the result equals one lattice of all
the rows bit for bit.
"""
from __future__ import annotations

import numpy as np

HALO = 3
GHOST_ROWS = 26


def split_rows(Ly: int, n: int) -> list[tuple[int, int]]:
    """(first row, row count) of n slabs covering rows 0 .. Ly - 1, as even as possible (the first
    Ly % n slabs take one row more). Every slab of a cut lattice needs at least 2 * HALO rows."""
    if n < 1 or Ly < n * 2 * HALO and n > 1:
        raise ValueError(f"cannot cut {Ly} rows into {n} slabs of at least {2 * HALO} rows")
    base, extra = divmod(Ly, n)
    out, y0 = [], 0
    for k in range(n):
        h = base + (1 if k < extra else 0)
        out.append((y0, h))
        y0 += h
    return out


def cuts_of(k: int, n: int) -> int:
    """Cut bits of slab k of n (bit 0: a slab lies below it, bit 1: a slab lies above it)."""
    return (1 if k > 0 else 0) | (2 if k < n - 1 else 0)


def ghost_table(cy, up: bool) -> list[tuple[int, int]]:
    """The 26 (population, k) entries of one direction in the packed order of lb_slab_pack: k = 1,
    2, 3 outward from the cut, then the populations (in the order of cy) whose velocity crosses the
    cut by at least k rows -- moving up (c_y >= k, arriving below a slab) or down (c_y <= -k)."""
    out = [(i, k) for k in range(1, HALO + 1) for i in range(len(cy))
           if (int(cy[i]) if up else -int(cy[i])) >= k]
    assert len(out) == GHOST_ROWS
    return out


def slab_fields(fields, y0: int, h: int):
    """The rows y0 .. y0 + h - 1 of host fields (rho, ux, uy, T), each [Ly][Lx]."""
    return [np.ascontiguousarray(np.asarray(a)[y0:y0 + h]) for a in fields]


class SlabLattice:
    """One lattice of Lx x Ly sites as `nslabs` slab contexts in this process (one device), each
    step followed by the exchange across every cut (lb_slab_exchange). All slabs share one stream
    unless `streams` gives one per slab."""

    def __init__(self, lb, Lx, Ly, tau, fields, nslabs, streams=None, **kw):
        self.lb = lb
        self.Lx, self.Ly = Lx, Ly
        self.rows = split_rows(Ly, nslabs)
        if streams is None:
            import torch
            s = torch.cuda.Stream()
            streams = [s] * nslabs
        self.slabs = []
        for k, (y0, h) in enumerate(self.rows):
            sub = slab_fields(fields, y0, h)
            self.slabs.append(lb.Lattice(Lx, h, tau, *sub, stream=streams[k], cuts=cuts_of(k, nslabs), **kw))
        self.exchange()

    def exchange(self) -> None:
        for lo, hi in zip(self.slabs[:-1], self.slabs[1:]):
            self.lb.slab_exchange(lo, hi)

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            for s in self.slabs:
                s.step(1)
            self.exchange()

    def sync(self) -> None:
        for s in self.slabs:
            s.sync()

    def get_populations(self) -> np.ndarray:
        return np.concatenate([s.get_populations() for s in self.slabs], axis=1)

    def moments(self):
        parts = [s.moments() for s in self.slabs]
        return tuple(np.concatenate([p[j] for p in parts], axis=0) for j in range(4))

    def close(self) -> None:
        for s in self.slabs:
            s.close()
        self.slabs = []


def exchange_ghosts(dist, rank: int, world: int, send_lo, send_hi, recv_lo, recv_hi):
    """Post one step's ghost-row traffic between neighbouring ranks over torch.distributed: send_lo
    (the rows this rank packed across its cut below) to rank - 1 and send_hi to rank + 1; recv_lo
    from rank - 1 and recv_hi from rank + 1. All sends and receives are posted together, so no
    ordering between ranks can deadlock. Returns wait(): it completes the transfers (with NCCL it
    makes the current CUDA stream wait for them; work queued before it overlaps the transfer)."""
    ops = []
    if rank > 0:
        ops += [dist.P2POp(dist.isend, send_lo, rank - 1), dist.P2POp(dist.irecv, recv_lo, rank - 1)]
    if rank < world - 1:
        ops += [dist.P2POp(dist.isend, send_hi, rank + 1), dist.P2POp(dist.irecv, recv_hi, rank + 1)]
    reqs = dist.batch_isend_irecv(ops) if ops else []

    def wait():
        for req in reqs:
            req.wait()
    return wait


class SlabRank:
    """Slab `rank` of `world` of one Lx x Ly lattice, advanced with a transport that moves packed
    ghost rows between neighbours: transport(send_lo, send_hi, recv_lo, recv_hi) posts this rank's
    transfers and returns wait() (``exchange_ghosts`` bound to a process group; or an in-process
    stand-in). Buffers are CUDA tensors of 26 x Lx elements of the storage type. With overlap, each
    step writes the rows next to the cuts, packs them, posts the transfers, writes the interior rows
    while they travel, waits, and unpacks."""

    def __init__(self, lb, Lx, Ly, tau, fields, rank, world, transport, overlap=True, **kw):
        import torch
        self.lb = lb
        self.rank, self.world = rank, world
        self.transport = transport
        self.overlap = overlap
        y0, h = split_rows(Ly, world)[rank]
        self.y0, self.h = y0, h
        self.cuts = cuts_of(rank, world)
        self.lat = lb.Lattice(Lx, h, tau, *slab_fields(fields, y0, h), cuts=self.cuts, **kw)
        dtype = torch.float64 if kw.get("precision", lb.LB_FP64) in (lb.LB_FP64, "fp64") else torch.float32
        mk = lambda: torch.empty(GHOST_ROWS * Lx, dtype=dtype, device="cuda")
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()

    def _pack(self) -> None:
        if self.cuts & 1:
            self.lat.slab_pack(0, self.send_lo)
        if self.cuts & 2:
            self.lat.slab_pack(1, self.send_hi)

    def _post(self):
        import torch
        with torch.cuda.stream(self.lat.stream):
            return self.transport(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi)

    def _wait(self, wait) -> None:
        import torch
        with torch.cuda.stream(self.lat.stream):
            wait()

    def _unpack(self) -> None:
        if self.cuts & 1:
            self.lat.slab_unpack(0, self.recv_lo)
        if self.cuts & 2:
            self.lat.slab_unpack(1, self.recv_hi)

    def pack_ghosts(self) -> None:
        """Pack the rows this slab sends across its cuts, from its newest state."""
        self._pack()

    def receive_ghosts(self) -> None:
        """Post the transfers of the packed rows, wait for them and unpack into the ghost rows."""
        self._wait(self._post())
        self._unpack()

    def first_exchange(self) -> None:
        """Fill the ghost rows of the initial state (every rank calls it once before stepping)."""
        self.pack_ghosts()
        self.receive_ghosts()

    def step_bands(self) -> None:
        """First half of a step: the rows next to the cuts (all rows without overlap), packed."""
        self.lat.slab_step(1 if self.overlap else 0)
        self._pack()

    def step_rest(self) -> None:
        """Second half: post the packed rows, the interior rows while they travel, the ghost rows."""
        wait = self._post()
        if self.overlap:
            self.lat.slab_step(2)
        self._wait(wait)
        self._unpack()

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            self.step_bands()
            self.step_rest()

    def close(self) -> None:
        self.lat.close()
