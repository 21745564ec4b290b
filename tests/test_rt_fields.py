"""The library's seeded Rayleigh-Taylor fields (lb_rt_fields, a host call: no GPU needed) against
the inputs module's implementation of the same recipe and the same published generator
(SplitMix64): equal up to the last-place rounding of cos, tanh and exp, which the C math library
and numpy may round differently."""
import numpy as np
import pytest

from paper_1804_01918_gb300 import inputs


@pytest.fixture(scope="module")
def L():
    from paper_1804_01918_gb300 import build, lb
    build.build()
    return lb


@pytest.mark.parametrize("Lx,Ly,R,seed", [(64, 256, 2.0, 0), (37, 21, 1.5, 7), (2304, 64, 3.0, 2**63 + 5)])
def test_c_fields_match_the_inputs_module(L, Lx, Ly, R, seed):
    c = L.rt_fields(Lx, Ly, R, seed)
    p = inputs.rayleigh_taylor_splitmix(Lx, Ly, R, seed)
    assert (c.T_top, c.T_bottom, c.gy) == (p.T_top, p.T_bottom, p.gy)
    for a, b in ((c.rho, p.rho), (c.T, p.T)):
        assert np.max(np.abs(a - b) / np.abs(b)) <= 4 * 2.0**-52
    assert not np.any(c.ux) and not np.any(c.uy)


def test_splitmix64_reference_values():
    """SplitMix64 from its published definition: outputs for seed 0 are the well-known sequence
    0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    s, out = 0, []
    for _ in range(3):
        s, z = inputs._splitmix64(s)
        out.append(z)
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_fields_are_seeded_and_physical(L):
    a = L.rt_fields(96, 128, 2.0, 1)
    b = L.rt_fields(96, 128, 2.0, 1)
    c = L.rt_fields(96, 128, 2.0, 2)
    assert np.array_equal(a.rho, b.rho) and not np.array_equal(a.rho, c.rho)
    assert a.T_top == pytest.approx(2 / 3) and a.T_bottom == pytest.approx(4 / 3)
    assert a.T[0].min() > 1.3 and a.T[-1].max() < 0.67          # hot below, cold above
    p = a.rho * a.T                                              # p = 1 on the interface
    assert p[64].mean() == pytest.approx(1.0, abs=2e-3)
    assert np.all(np.diff(p.mean(axis=1)) < 0)                  # and falls with height


def test_invalid_arguments(L):
    import ctypes as C
    z = np.zeros(4)
    assert L.lib().lb_rt_fields(0, 2, 2.0, 0, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                                z.ctypes.data, None, None, None) == 1
    assert L.lib().lb_rt_fields(2, 2, -1.0, 0, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                                z.ctypes.data, None, None, None) == 1
