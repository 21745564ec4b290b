"""Pins of the oracle's time step (propagate, walls, full step) against closed forms, library
routines and textbook hydrodynamics.

Sec. 3: populations propagate from site to site, then collide; no site depends on another.
Sec. 4, Fig. 3 listing: propagate is a pull, new[p][site] = old[p][site + OFF[p]].
"""
import math

import numpy as np
import pytest

from paper_1804_01918_gb300 import inputs


def test_propagate_is_a_cyclic_shift_per_population(orc):
    """y-periodic mode: every population plane is np.roll of its input by (c_y, c_x); the
    result is a permutation, so sums over the lattice are preserved exactly."""
    cx, cy, w, r = orc.velocity_set()
    Lx, Ly = 11, 9
    rng = np.random.default_rng(0)
    src = np.zeros((Ly + 6, Lx, 37))
    src[3:Ly + 3] = rng.integers(-2**20, 2**20, size=(Ly, Lx, 37)) / 2.0**10   # dyadic values
    out = orc.propagate(src, Lx, Ly, y_periodic=True)
    for i in range(37):
        expect = np.roll(src[3:Ly + 3, :, i], shift=(int(cy[i]), int(cx[i])), axis=(0, 1))
        assert np.array_equal(out[:, :, i], expect)
        assert np.sort(out[:, :, i], axis=None).tolist() == np.sort(src[3:Ly + 3, :, i], axis=None).tolist()
    assert out.sum() == src.sum()


def test_propagate_moves_a_population_along_its_velocity(orc):
    """A single population placed at (x0, y0) arrives at (x0 + c_x, y0 + c_y) (pull with
    OFF = -c): the direction convention."""
    cx, cy, w, r = orc.velocity_set()
    Lx, Ly, x0, y0 = 12, 12, 5, 6
    for i in range(37):
        src = np.zeros((Ly + 6, Lx, 37))
        src[y0 + 3, x0, i] = 1.0
        out = orc.propagate(src, Lx, Ly, y_periodic=False)
        ys, xs, ps = np.nonzero(out)
        assert (ys.tolist(), xs.tolist(), ps.tolist()) == ([y0 + cy[i]], [x0 + cx[i]], [i])


def test_propagate_reads_wall_halo_rows(orc):
    """With walls, populations with c_y > 0 entering rows 0..2 come from the halo rows below."""
    cx, cy, w, r = orc.velocity_set()
    Lx, Ly = 8, 10
    src = np.zeros((Ly + 6, Lx, 37))
    for h in range(3):
        src[h] = 1000.0 + h          # halo rows y = -3, -2, -1
        src[Ly + 3 + h] = 2000.0 + h  # halo rows y = Ly, Ly+1, Ly+2
    out = orc.propagate(src, Lx, Ly, y_periodic=False)
    for i in range(37):
        for y in range(Ly):
            ys = y - cy[i]
            want = 1000.0 + (ys + 3) if ys < 0 else (2000.0 + (ys - Ly) if ys >= Ly else 0.0)
            assert np.all(out[y, :, i] == want)


def test_walls_hold_rest_equilibrium_at_wall_temperature(orc):
    """Halo rows carry u = 0, T = T_wall and the mirror row's density (moment closed forms)."""
    rng = np.random.default_rng(1)
    Lx, Ly = 6, 9
    st = inputs.random_state(Lx, Ly, seed=4)
    f = orc.equilibrium(st.rho, st.ux, st.uy, st.T)
    f = f * (1 + 0.01 * rng.uniform(-1, 1, f.shape))
    full = orc.with_walls(f, T_top=0.7, T_bottom=1.3)
    for k in range(3):
        rb, uxb, uyb, Tb = orc.moments(full[2 - k])
        rt, uxt, uyt, Tt = orc.moments(full[Ly + 3 + k])
        assert np.allclose(rb, f[k].sum(-1), rtol=1e-14)
        assert np.allclose(rt, f[Ly - 1 - k].sum(-1), rtol=1e-14)
        assert np.max(np.abs(np.concatenate([uxb, uyb, uxt, uyt]))) < 1e-15
        assert np.allclose(Tb, 1.3, rtol=1e-14) and np.allclose(Tt, 0.7, rtol=1e-14)


def test_uniform_rest_state_with_walls_is_steady(orc):
    """rho = 1, T = T_top = T_bottom = 1, g = 0 stays fixed for 100 steps."""
    cx, cy, w, r = orc.velocity_set()
    Lx, Ly = 8, 16
    f0 = np.tile(w, (Ly, Lx, 1))
    f = orc.run(f0, tau=0.9, nsteps=100, gy=0.0, T_top=1.0, T_bottom=1.0)
    assert np.max(np.abs(f - f0)) < 1e-14


def test_global_conservation_periodic(orc):
    """Periodic in both directions and g = 0: total mass, momentum and energy are invariants."""
    cx, cy, w, r = orc.velocity_set()
    st = inputs.random_state(16, 12, seed=2)
    f0 = orc.equilibrium(st.rho, st.ux, st.uy, st.T)
    f = orc.run(f0, tau=0.8, nsteps=20, y_periodic=True)
    xi2 = (r * cx) ** 2 + (r * cy) ** 2
    for weight in (np.ones(37), r * cx, r * cy, xi2):
        a, b = float((f0 * weight).sum()), float((f * weight).sum())
        assert abs(a - b) <= 1e-12 * max(1.0, abs(a))


def test_gravity_adds_rho_g_per_step_to_total_momentum(orc):
    """Periodic box with gravity: total momentum grows by g * total mass each step."""
    cx, cy, w, r = orc.velocity_set()
    st = inputs.random_state(8, 8, seed=3)
    f0 = orc.equilibrium(st.rho, st.ux, st.uy, st.T)
    g = -1e-3
    n = 10
    f = orc.run(f0, tau=0.9, nsteps=n, gy=g, y_periodic=True)
    mass = f0.sum()
    jy0 = (f0 * r * cy).sum()
    jy1 = (f * r * cy).sum()
    assert jy1 - jy0 == pytest.approx(n * g * mass, rel=1e-11)


def _sine_mode(a, L):
    y = np.arange(L)
    return 2.0 / L * np.sum(a * np.sin(2 * np.pi * y / L))


def test_shear_wave_decays_at_bgk_viscosity(orc):
    """Physics pin: a small shear wave u_x = U sin(2 pi y / Ly) decays as exp(-nu k^2 t) with
    the BGK kinematic viscosity nu = T (tau - 1/2) / r^2 in lattice units (xi = r c, c_s^2 = T
    in thermal units)."""
    cx, cy, w, r = orc.velocity_set()
    Lx, Ly, U, tau, n = 4, 64, 1e-4, 0.8, 200
    y = np.arange(Ly)
    ux = np.tile((U * np.sin(2 * np.pi * y / Ly))[:, None], (1, Lx))
    f0 = orc.equilibrium(np.ones((Ly, Lx)), ux, np.zeros((Ly, Lx)), np.ones((Ly, Lx)))
    f = orc.run(f0, tau=tau, nsteps=n, y_periodic=True)
    rho, uxn, uyn, T = orc.moments(f)
    amp = _sine_mode(uxn.mean(axis=1), Ly)
    nu = (tau - 0.5) / r**2
    k = 2 * np.pi / Ly
    assert amp / U == pytest.approx(math.exp(-nu * k * k * n), rel=0.01)


def test_sound_wave_travels_at_adiabatic_speed(orc):
    """Physics pin: an isentropic density/temperature wave of a 2-D perfect gas (p = rho T,
    Sec. 3) oscillates at c = sqrt(gamma T) with gamma = (D + 2) / D = 2, i.e. c / r sites per
    step. Measured from the zero crossings of the standing wave's density mode."""
    cx, cy, w, r = orc.velocity_set()
    Lx, Ly, eps, tau, n = 2, 96, 1e-5, 0.6, 260
    y = np.arange(Ly)
    s = np.sin(2 * np.pi * y / Ly)
    rho = np.tile((1 + eps * s)[:, None], (1, Lx))
    T = np.tile((1 + eps * s)[:, None], (1, Lx))   # delta T / T = (gamma - 1) delta rho / rho
    f = orc.equilibrium(rho, np.zeros_like(rho), np.zeros_like(rho), T)
    a = [_sine_mode(rho[:, 0] - 1.0, Ly)]
    for _ in range(n):
        f = orc.run(f, tau=tau, nsteps=1, y_periodic=True, nthreads=1)
        a.append(_sine_mode(orc.moments(f)[0][:, 0] - 1.0, Ly))
    a = np.array(a)
    crossings = [t + a[t] / (a[t] - a[t + 1]) for t in range(n) if a[t] * a[t + 1] < 0]
    assert len(crossings) >= 3
    half_period = np.mean(np.diff(crossings))
    c_measured = Ly / (2 * half_period)
    assert c_measured == pytest.approx(math.sqrt(2.0) / r, rel=0.01)


def test_rt_inputs_are_seeded_and_hydrostatic():
    a = inputs.rayleigh_taylor(64, 256, R=2.0, seed=0)
    b = inputs.rayleigh_taylor(64, 256, R=2.0, seed=0)
    c = inputs.rayleigh_taylor(64, 256, R=2.0, seed=1)
    assert np.array_equal(a.rho, b.rho) and np.array_equal(a.T, b.T)
    assert not np.array_equal(a.rho, c.rho)
    assert a.T_top == pytest.approx(2 / 3) and a.T_bottom == pytest.approx(4 / 3)
    assert a.T[0].min() > 1.3 and a.T[-1].max() < 0.67           # hot below, cold above
    assert a.gy < 0 and abs(a.gy) * 256 / a.T_top == pytest.approx(0.1)
    # pressure p = rho T is 1 on the interface row and decreases upward
    p = a.rho * a.T
    assert np.all(np.diff(p.mean(axis=1)) < 0)
    assert p[128].mean() == pytest.approx(1.0, abs=2e-3)
