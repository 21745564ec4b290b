"""Pins of the oracle's alternative wall closure (mirror walls) and of its half-step fields.

The paper leaves walls and the reported fields to its references (Sec. 3). The oracle offers, next
to the rest-equilibrium walls, a mirror closure -- halo rows at the equilibrium of the mirror row's
density, opposite velocity and temperature reflected about the wall value -- and half-step fields
that average the pre- and post-collision momentum and energy. These tests pin both to their
defining properties and to channel physics.
"""
import numpy as np
import pytest

from paper_1804_01918_gb300 import inputs


def raw_sums(orc, f):
    """(sum f, sum f xi_x, sum f xi_y, sum f |xi|^2) per site, straight from the velocity set."""
    cx, cy, w, r = orc.velocity_set()
    xi_x, xi_y = r * cx, r * cy
    return (f.sum(-1), (f * xi_x).sum(-1), (f * xi_y).sum(-1), (f * (xi_x**2 + xi_y**2)).sum(-1))


@pytest.mark.parametrize("gx,gy", [(0.0, -0.02), (0.015, 0.01)])
def test_half_step_fields_average_pre_and_post_collision(orc, gx, gy):
    """rho_h u_h and rho_h (|u_h|^2 + D T_h) are the means of the pre- and post-collision momentum
    and energy sums (D = 2); rho_h is rho."""
    st = inputs.random_state(6, 5, seed=11)
    rng = np.random.default_rng(3)
    f_pre = orc.equilibrium(st.rho, st.ux, st.uy, st.T) * (1 + 0.02 * rng.uniform(-1, 1, (5, 6, 37)))
    f_post = orc.collide(f_pre, tau=0.85, gx=gx, gy=gy)
    m0, jx0, jy0, e0 = raw_sums(orc, f_pre)
    m1, jx1, jy1, e1 = raw_sums(orc, f_post)
    rho, ux, uy, T = orc.moments_half_step(f_post, gx, gy)
    assert np.allclose(rho, m0, rtol=1e-14, atol=0)
    assert np.allclose(rho * ux, 0.5 * (jx0 + jx1), rtol=0, atol=1e-15)
    assert np.allclose(rho * uy, 0.5 * (jy0 + jy1), rtol=0, atol=1e-15)
    assert np.allclose(rho * (ux * ux + uy * uy + 2.0 * T), 0.5 * (e0 + e1), rtol=1e-14, atol=0)


def test_half_step_fields_without_gravity_are_the_plain_moments(orc):
    st = inputs.random_state(5, 4, seed=2)
    f = orc.equilibrium(st.rho, st.ux, st.uy, st.T)
    a = orc.moments(f)
    b = orc.moments_half_step(f, 0.0, 0.0)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_mirror_halo_interpolates_to_zero_velocity_and_wall_temperature(orc):
    """Each halo row y = -1-k (y = Ly+k) holds the mirror row's density; the mean of a row's and its
    halo row's velocity is zero and the mean temperature is the wall temperature."""
    Lx, Ly, Tt, Tb = 7, 9, 0.8, 1.3
    st = inputs.random_state(Lx, Ly, seed=5, du=0.05, dT=0.2)
    f = orc.equilibrium(st.rho, st.ux, st.uy, st.T)
    full = orc.with_walls(f, Tt, Tb, wall_mode="mirror")
    rho, ux, uy, T = orc.moments(full)
    for k in range(3):
        for h, m, Tw in ((2 - k, 3 + k, Tb), (Ly + 3 + k, Ly + 2 - k, Tt)):
            assert np.allclose(rho[h], rho[m], rtol=1e-14, atol=0)
            assert np.max(np.abs(ux[h] + ux[m])) < 1e-15
            assert np.max(np.abs(uy[h] + uy[m])) < 1e-15
            assert np.allclose(0.5 * (T[h] + T[m]), Tw, rtol=1e-14, atol=0)
    # the interior rows are untouched
    assert np.array_equal(full[3:Ly + 3], f)


def test_rest_wall_mode_is_the_default_run(orc):
    st = inputs.rayleigh_taylor(8, 16, R=2.0, seed=1)
    f0 = orc.init_fields(st)
    a = orc.run(f0, tau=0.9, nsteps=5, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom, nthreads=1)
    b = orc.run(f0, tau=0.9, nsteps=5, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom, nthreads=1,
                wall_mode="rest")
    c = orc.run(f0, tau=0.9, nsteps=5, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom, nthreads=1,
                wall_mode="mirror")
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def _poiseuille(orc, wall_mode, Ly=32, tau=0.8, g=1e-6, steps=8000):
    Lx = 4
    one, z = np.ones((Ly, Lx)), np.zeros((Ly, Lx))
    f = orc.run(orc.equilibrium(one, z, z, one), tau=tau, nsteps=steps, gx=g, wall_mode=wall_mode)
    _, ux, _, _ = orc.moments_half_step(f, g, 0.0)
    c = np.polyfit(np.arange(Ly), ux.mean(axis=1), 2)
    lo, hi = np.sort(np.roots(c)).real
    return -c[0], lo, hi - (Ly - 1)


def test_poiseuille_channel_curvature_and_wall_position(orc):
    """Gravity along x between the walls: the steady half-step velocity is a parabola whose
    curvature is g / (2 nu), nu = T (tau - 1/2) / r^2 (both closures). The mirror closure puts the
    zero of the profile within a fraction of a site of the plane half a site outside the last row;
    the rest-equilibrium halo slips further out."""
    _, _, _, r = orc.velocity_set()
    g, tau = 1e-6, 0.8
    nu = (tau - 0.5) / r**2
    A, lo, hi = _poiseuille(orc, "mirror", tau=tau, g=g)
    assert A == pytest.approx(g / (2 * nu), rel=2e-3)
    assert abs(lo + 0.5) < 0.2 and abs(hi - 0.5) < 0.2
    A0, lo0, hi0 = _poiseuille(orc, "rest", tau=tau, g=g)
    assert A0 == pytest.approx(g / (2 * nu), rel=5e-3)
    assert lo0 < -0.7 and hi0 > 0.7


def test_conduction_between_mirror_walls(orc):
    """No gravity, walls at T_bottom = 1.01 and T_top = 0.99: the steady temperature profile is
    linear with slope within 2 % of (T_top - T_bottom) / Ly, and it reaches each wall temperature
    within a quarter site of the plane half a site outside the last row (the rest-equilibrium halo
    reaches it about a site out)."""
    Lx, Ly, tau = 4, 32, 0.8
    one, z = np.ones((Ly, Lx)), np.zeros((Ly, Lx))
    y = np.arange(Ly)
    for mode, tol in (("mirror", 0.25), ("rest", None)):
        f = orc.run(orc.equilibrium(one, z, z, one), tau=tau, nsteps=8000, T_top=0.99, T_bottom=1.01,
                    wall_mode=mode)
        _, _, _, T = orc.moments(f)
        slope, icpt = np.polyfit(y, T.mean(axis=1), 1)
        yb, yt = (1.01 - icpt) / slope, (0.99 - icpt) / slope
        if tol is not None:
            assert slope == pytest.approx(-0.02 / Ly, rel=0.02)
            assert abs(yb + 0.5) < tol and abs(yt - (Ly - 0.5)) < tol
        else:
            assert yb < -0.75 and yt > Ly - 0.25


def test_mirror_halo_falls_back_to_rest_where_not_reflectable(orc):
    """Where the mirror row is hotter than twice the wall temperature the reflected temperature
    would not be positive; that halo site holds the rest closure's value instead."""
    Lx, Ly, Tt, Tb = 4, 8, 0.3, 1.0
    one, z = np.ones((Ly, Lx)), np.zeros((Ly, Lx))
    T = one.copy()
    T[-1, 1] = 0.5  # reflectable at the top: 2 * 0.3 - 0.5 > 0
    f = orc.equilibrium(one, z, z, T)
    mirror = orc.with_walls(f, Tt, Tb, wall_mode="mirror")
    rest = orc.with_walls(f, Tt, Tb, wall_mode="rest")
    top = Ly + 3  # halo row above row Ly - 1
    cols = [0, 2, 3]
    assert np.array_equal(mirror[top][cols], rest[top][cols])
    _, _, _, Th = orc.moments(mirror[top])
    assert Th[1] == pytest.approx(2 * Tt - 0.5, rel=1e-14)
