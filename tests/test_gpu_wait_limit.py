"""The failure path of the library's asynchronous waits, made to run out on purpose without a GPU
fault: lb_probe_wait waits, with the same bounded wait the tensor-core and TMA kernels use, on a
shared-memory barrier that nothing ever completes (no asynchronous copy or product targets it, so
nothing is in flight when it gives up). The wait must give up after its time limit and report it,
and the context must stay usable for the next launch."""
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


def test_bounded_wait_gives_up_after_its_time_limit(L):
    limit = 2_000_000                       # 2 ms
    gave_up, ns = L.probe_wait(limit, arrive=False)
    assert gave_up
    assert limit <= ns < 500 * limit        # it waited the limit, and not much longer


def test_bounded_wait_succeeds_when_the_phase_completes(L):
    gave_up, ns = L.probe_wait(1_000_000_000, arrive=True)
    assert not gave_up and ns < 1_000_000


def test_context_usable_after_a_wait_gave_up(L):
    L.probe_wait(1_000_000, arrive=False)
    st = inputs.rayleigh_taylor(32, 32, R=2.0, seed=1)
    lat = L.Lattice.from_fields(st, tau=0.9)
    lat.step(3)
    lat.sync()
    assert np.all(np.isfinite(lat.get_populations()))
    lat.close()
