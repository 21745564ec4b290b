"""Multi-rank host logic of bench.py (replicas, weak scaling) on 2 gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_1804_01918_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.rank_env()
    ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    worst = replicas.max_over_ranks(ms, dist)
    dist.barrier()
    value = replicas.aggregate_mlups(1000, 10, worst, w)
    q.put((r, w, lr, worst, value, replicas.replica_seed(r)))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 150.0 for o in out)                 # max over ranks
    assert all(o[4] == pytest.approx(2 * 1000 * 10 / 0.150 / 1e6) for o in out)
    assert out[0][5] != out[1][5]                          # distinct replicas


def test_single_process_needs_no_group():
    from paper_1804_01918_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.aggregate_mlups(100, 2, 1.0, 1) == pytest.approx(0.2)
    with pytest.raises(ValueError):
        replicas.aggregate_mlups(1, 1, 0.0, 1)
