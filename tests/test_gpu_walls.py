"""GPU parity of the mirror wall closure and of the half-step fields (through the C ABI) against
the CPU oracle.

Bars as for the rest closure: FP64 within 1e-12 relative per population after 100 steps, the
two-kernel step equal to the fused step bit for bit, the FP32 forms within the stated L2 error
budget (n steps x 37 populations x 2^-24 x 0.35). Half-step fields: FP64 moments plus a shift,
within 1e-14.
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


def to_oracle(L, orc, f_planes):
    cx, cy, _, _ = L.velocity_set()
    return orc.from_planes(f_planes, cx, cy)


def to_gpu(L, orc, f_site):
    cx, cy, _, _ = L.velocity_set()
    return orc.to_planes(f_site, cx, cy)


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("Lx,Ly,steps", [(64, 256, 100), (70, 50, 100), (13, 5, 30)])
def test_fp64_mirror_walls_match_oracle_rayleigh_taylor(L, orc, Lx, Ly, steps):
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9, wall_mode="mirror")
    lat.step(steps)
    lat.sync()
    got = to_oracle(L, orc, lat.get_populations())
    want = orc.run(orc.init_fields(st), tau=0.9, nsteps=steps, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom, wall_mode="mirror")
    assert rel_err(got, want) <= TOL
    # the closure matters: the rest closure gives a different state
    rest = orc.run(orc.init_fields(st), tau=0.9, nsteps=steps, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom, wall_mode="rest")
    assert rel_err(got, rest) > 1e-9


def test_fp64_mirror_walls_strong_gravity_both_axes(L, orc):
    Lx, Ly = 33, 40
    st = inputs.random_state(Lx, Ly, seed=9, du=0.03, dT=0.1)
    lat = L.Lattice.from_fields(st, tau=0.7, gx=1e-3, gy=-2e-3, T_top=0.9, T_bottom=1.2,
                                wall_mode="mirror")
    lat.step(40)
    lat.sync()
    got = to_oracle(L, orc, lat.get_populations())
    want = orc.run(orc.init_fields(st), tau=0.7, nsteps=40, gx=1e-3, gy=-2e-3, T_top=0.9,
                   T_bottom=1.2, wall_mode="mirror")
    assert rel_err(got, want) <= TOL


@pytest.mark.parametrize("mode", ["rest", "mirror"])
def test_fp64_two_kernel_step_equals_fused_step(L, mode):
    st = inputs.rayleigh_taylor(96, 80, R=2.0, seed=5)
    a = L.Lattice.from_fields(st, tau=0.85, wall_mode=mode)
    b = L.Lattice.from_fields(st, tau=0.85, wall_mode=mode)
    for _ in range(7):
        a.propagate()
        a.collide()
    b.step(7)
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_set_populations_rewrites_mirror_halos(L, orc):
    """lb_set_populations rewrites the halo rows from the new interior state (halo kernel); one
    step then matches the oracle started from the same populations."""
    Lx, Ly = 40, 30
    rng = np.random.default_rng(5)
    st = inputs.random_state(Lx, Ly, seed=2)
    lat = L.Lattice.from_fields(st, tau=0.9, T_top=0.8, T_bottom=1.25, wall_mode="mirror")
    f0 = orc.equilibrium(st.rho, st.ux, st.uy, st.T) * (1 + 0.01 * rng.uniform(-1, 1, (Ly, Lx, 37)))
    lat.set_populations(to_gpu(L, orc, f0))
    lat.step(3)
    lat.sync()
    got = to_oracle(L, orc, lat.get_populations())
    want = orc.run(f0, tau=0.9, nsteps=3, T_top=0.8, T_bottom=1.25, wall_mode="mirror")
    assert rel_err(got, want) <= TOL


@pytest.mark.parametrize("form", ["fp32dev", "fp32split"])
def test_fp32_forms_mirror_walls_l2_error_vs_fp64_oracle(L, orc, form):
    Lx, Ly, steps = 64, 256, 100
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9, precision=form, wall_mode="mirror")
    lat.step(steps)
    rho, ux, uy, T = lat.moments()
    f = orc.run(orc.init_fields(st), tau=0.9, nsteps=steps, gy=st.gy, T_top=st.T_top,
                T_bottom=st.T_bottom, wall_mode="mirror")
    orho, _, _, oT = orc.moments(f)
    bound = steps * 37 * 2.0**-24 * 0.35
    e_rho, e_T = rel_l2(rho, orho), rel_l2(T, oT)
    print(f"{form} mirror walls 64x256 100 steps: rel L2 rho {e_rho:.3e}, T {e_T:.3e}")
    assert e_rho < bound and e_T < bound


@pytest.mark.parametrize("precision", ["fp64", "fp32split"])
def test_half_step_fields_match_oracle(L, orc, precision):
    Lx, Ly = 48, 64
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=3)
    gx = 2e-4
    lat = L.Lattice.from_fields(st, tau=0.9, gx=gx, precision=precision)
    lat.step(6)
    rho, ux, uy, T = lat.moments_half_step()
    f = to_oracle(L, orc, lat.get_populations())
    orho, oux, ouy, oT = orc.moments_half_step(f, gx, st.gy)
    tol = 1e-14 if precision == "fp64" else 1e-7
    assert rel_err(rho, orho) < tol and rel_err(T, oT) < tol
    assert np.max(np.abs(ux - oux)) < tol and np.max(np.abs(uy - ouy)) < tol
    # the shift itself: half-step minus plain fields
    prho, pux, puy, pT = lat.moments()
    assert np.allclose(pux - ux, 0.5 * gx, rtol=0, atol=1e-15)
    assert np.allclose(puy - uy, 0.5 * st.gy, rtol=0, atol=1e-15)
    assert np.allclose(T - pT, (gx**2 + st.gy**2) / 8.0, rtol=1e-6, atol=1e-18)


def test_non_positive_reflected_temperature_is_reported(L):
    """A mirror row hotter than twice the wall temperature cannot be reflected: the step flags it
    (LB_ERR_NONFINITE at the next sync) instead of writing a negative-temperature halo."""
    Lx, Ly = 32, 16
    one = np.ones((Ly, Lx))
    z = np.zeros((Ly, Lx))
    lat = L.Lattice(Lx, Ly, 0.9, one, z, z, one, T_top=0.4, T_bottom=1.0, wall_mode="mirror")
    with pytest.raises(L.NonFiniteError):
        lat.sync()  # the halo rows written at init already hit it


def test_ensemble_members_use_the_rest_closure(L):
    st = inputs.rayleigh_taylor(64, 64, R=2.0, seed=0)
    m = dict(Lx=64, Ly=64, tau=0.9, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom, rho=st.rho,
             ux=st.ux, uy=st.uy, T=st.T, wall_mode="mirror")
    with pytest.raises(L.LBError):
        L.Ensemble([m])


def test_invalid_wall_mode_is_rejected(L):
    st = inputs.rayleigh_taylor(32, 32, R=2.0, seed=0)
    with pytest.raises(L.LBError):
        L.Lattice.from_fields(st, tau=0.9, wall_mode=7)
