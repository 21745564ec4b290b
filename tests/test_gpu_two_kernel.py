"""The paper's two-kernel structure on the GPU -- a propagate launch, then a collide launch (Sec. 3;
Table 1 times the two separately) -- against the FP64 oracle directly, not only against the fused
step: lb_propagate + lb_collide over 100 steps for both wall closures, and lb_collide alone on a
far-from-equilibrium state, then the wall halo rows it writes, as the next pull reads them.
Bar: 1e-12 relative per population (the FP64 parity bar of the fused step).
"""
import numpy as np
import pytest

from paper_1804_01918_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01918_gb300 import build, lb
    build.build()
    return lb


def rel_err(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


@pytest.mark.parametrize("wall_mode", ["rest", "mirror"])
def test_two_kernel_run_matches_oracle(L, orc, wall_mode):
    """100 x (lb_propagate, lb_collide) on the 64 x 256 Rayleigh-Taylor lattice vs oracle.run."""
    Lx, Ly, n, tau = 64, 256, 100, 0.9
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=tau, wall_mode=wall_mode)
    for _ in range(n):
        lat.propagate()
        lat.collide()
    lat.sync()
    cx, cy, _, _ = L.velocity_set()
    got = orc.from_planes(lat.get_populations(), cx, cy)
    lat.close()
    want = orc.run(orc.init_fields(st), tau=tau, nsteps=n, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom, wall_mode=wall_mode)
    err = rel_err(got, want)
    print(f"two-kernel {wall_mode}: max rel err after {n} steps {err:.2e}")
    assert err <= TOL


@pytest.mark.parametrize("wall_mode", ["rest", "mirror"])
def test_collide_alone_matches_oracle_collide_and_writes_the_halo(L, orc, wall_mode):
    """lb_collide on a far-from-equilibrium state (random fields' equilibria times 1 +- 5 % noise,
    gravity on both axes) equals oracle.collide per population; the halo rows it writes are the
    oracle's walls of the collided state, as the next lb_propagate reads them."""
    Lx, Ly, tau, gx, gy = 48, 40, 0.7, 1e-3, -2e-3
    st = inputs.random_state(Lx, Ly, seed=21, du=0.08, dT=0.15, drho=0.2)
    f0 = orc.equilibrium(st.rho, st.ux, st.uy, st.T)
    rng = np.random.default_rng(22)
    f0 = f0 * (1.0 + 0.05 * rng.uniform(-1, 1, f0.shape))
    cx, cy, _, _ = L.velocity_set()
    lat = L.Lattice(Lx, Ly, tau, st.rho, st.ux, st.uy, st.T, gx=gx, gy=gy, T_top=st.T_top,
                    T_bottom=st.T_bottom, wall_mode=wall_mode)
    lat.set_populations(orc.to_planes(f0, cx, cy))
    lat.collide()
    lat.sync()
    collided = orc.from_planes(lat.get_populations(), cx, cy)
    want = orc.collide(f0, tau, gx, gy)
    err = rel_err(collided, want)
    assert err <= TOL, err
    # the halo rows: one pull after the collide reads them in rows 0..2 and Ly-3..Ly-1
    lat.propagate()
    lat.sync()
    pulled = orc.from_planes(lat.get_populations(), cx, cy)
    lat.close()
    want_pull = orc.propagate(orc.with_walls(want, st.T_top, st.T_bottom, wall_mode), Lx, Ly, False)
    err_pull = rel_err(pulled, want_pull)
    print(f"collide alone {wall_mode}: {err:.2e}; after the next pull (halo rows) {err_pull:.2e}")
    assert err_pull <= TOL
