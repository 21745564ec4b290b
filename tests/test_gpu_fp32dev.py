"""GPU checks of the FP32-deviation forms against the FP64 oracle: populations stored in FP32 as
f - w with an FP32 collide, and the moment sums plus the conservation projection done either in
FP64 (fp32dev) or by an exact three-way FP32 split (fp32split).

The form is not expected to match FP64 bit for bit; the bar is a stated relative L2 error of the
density and temperature fields and conservation at the level of FP32 storage rounding.
Error budget used as the hard bound: each step rounds every stored deviation to FP32
(relative 2^-24); deviations of the Rayleigh-Taylor state are at most ~35% of the population, so
a linear (worst-case) accumulation over n steps and 37 populations gives
n * 37 * 2^-24 * 0.35 ~ 7.7e-5 at n = 100.
"""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


FORMS = ["fp32dev", "fp32split"]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("tau", [0.55, 2.5])
def test_fp32_forms_strong_flow_vs_fp64_oracle(L, orc, form, tau):
    """The FP64 step's strong-flow regime (uncorrelated velocities to 0.15, densities 0.7-1.3,
    temperatures 0.8-1.2, gravity 3e-3 on both axes): after 20 steps every population is within
    20 x 16 FP32 ulps of a unit deviation, relative to its weight, of the FP64 oracle (each step
    rounds every stored deviation once and the FP32 collide adds a few roundings more)."""
    Lx, Ly, n = 40, 36, 20
    st = inputs.random_state(Lx, Ly, seed=7, du=0.15, dT=0.2, drho=0.3)
    lat = L.Lattice(Lx, Ly, tau, st.rho, st.ux, st.uy, st.T, gx=3e-3, gy=-3e-3, T_top=0.9,
                    T_bottom=1.1, precision=form)
    lat.step(n)
    lat.sync()
    cx, cy, _, _ = L.velocity_set()
    got = orc.from_planes(lat.get_populations(), cx, cy)
    lat.close()
    want = orc.run(orc.init_fields(st), tau=tau, nsteps=n, gx=3e-3, gy=-3e-3, T_top=0.9,
                   T_bottom=1.1)
    _, _, w, _ = orc.velocity_set()
    err = float(np.max(np.abs(got - want) / w))
    print(f"{form} strong flow tau {tau}: max |f - f_oracle| / w = {err:.2e}")
    assert err <= n * 16 * 2.0**-24


@pytest.mark.parametrize("form", FORMS)
def test_fp32dev_rayleigh_taylor_l2_error_vs_fp64_oracle(L, orc, form):
    Lx, Ly, steps = 64, 256, 100
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9, precision=form)
    lat.step(steps)
    rho, ux, uy, T = lat.moments()
    f = orc.run(orc.init_fields(st), tau=0.9, nsteps=steps, gy=st.gy, T_top=st.T_top,
                T_bottom=st.T_bottom)
    orho, oux, ouy, oT = orc.moments(f)
    bound = steps * 37 * 2.0**-24 * 0.35
    e_rho, e_T = rel_l2(rho, orho), rel_l2(T, oT)
    print(f"{form} 64x256 100 steps: rel L2 rho {e_rho:.3e}, T {e_T:.3e} (bound {bound:.1e})")
    assert e_rho < bound and e_T < bound
    # and the FP32 form is far better than plain FP32 storage of absolute populations would be
    assert e_rho < 1e-5 and e_T < 1e-5


def test_fp32dev_init_and_moments(L, orc):
    st = inputs.rayleigh_taylor(40, 64, R=2.0, seed=2)
    lat = L.Lattice.from_fields(st, tau=0.9, precision="fp32dev")
    rho, ux, uy, T = lat.moments()
    # deviations of magnitude <= 0.35 w are stored with relative error 2^-24
    assert rel_l2(rho, st.rho) < 1e-7 and rel_l2(T, st.T) < 1e-7
    assert np.max(np.abs(ux)) < 1e-8


@pytest.mark.parametrize("form", FORMS)
def test_fp32dev_conserves_mass_momentum_energy_periodic(L, orc, form):
    Lx, Ly = 48, 40
    st = inputs.random_state(Lx, Ly, seed=3, du=0.02, dT=0.1, drho=0.1)
    lat = L.Lattice.from_fields(st, tau=0.8, y_periodic=True, precision=form)
    cx, cy, w, r = L.velocity_set()
    f0 = lat.get_populations()
    lat.step(50)
    f1 = lat.get_populations()
    xi2 = (r * cx) ** 2 + (r * cy) ** 2
    for weight, scale in ((np.ones(37), 1.0), (r * cx, 1.0), (r * cy, 1.0), (xi2, 2.0)):
        a = float(np.tensordot(weight, f0, 1).sum())
        b = float(np.tensordot(weight, f1, 1).sum())
        assert abs(a - b) <= 1e-8 * scale * Lx * Ly


def test_fp32dev_propagate_bit_exact(L):
    """The pull moves FP32 deviations unchanged: each plane is a cyclic shift."""
    Lx, Ly = 21, 17
    st = inputs.random_state(Lx, Ly, seed=5)
    lat = L.Lattice.from_fields(st, tau=0.9, y_periodic=True, precision="fp32dev")
    cx, cy, w, r = L.velocity_set()
    rng = np.random.default_rng(1)
    dev = (rng.uniform(-0.1, 0.1, (37, Ly, Lx)) * w[:, None, None]).astype(np.float32)
    f0 = w[:, None, None] + dev.astype(np.float64)
    lat.set_populations(f0)
    lat.propagate()
    got = lat.get_populations()          # w + (double) deviation, one rounding
    for i in range(37):
        want = w[i] + np.roll(dev[i], shift=(int(cy[i]), int(cx[i])), axis=(0, 1)).astype(np.float64)
        assert np.array_equal(got[i], want)


@pytest.mark.parametrize("form", FORMS)
def test_fp32dev_gravity_momentum_budget(L, form):
    """Periodic box with gravity: total momentum grows by g x mass per step (the projection
    targets rho u + rho g), to FP32 storage accuracy."""
    Lx, Ly, n, g = 32, 32, 20, -1e-4
    st = inputs.random_state(Lx, Ly, seed=8, du=0.01, dT=0.05, drho=0.05)
    lat = L.Lattice.from_fields(st, tau=0.9, y_periodic=True, gy=g, precision=form)
    cx, cy, w, r = L.velocity_set()
    f0 = lat.get_populations()
    lat.step(n)
    f1 = lat.get_populations()
    mass = f0.sum()
    jy0 = float(np.tensordot(r * cy, f0, 1).sum())
    jy1 = float(np.tensordot(r * cy, f1, 1).sum())
    assert jy1 - jy0 == pytest.approx(n * g * mass, rel=1e-4)


def test_fp32split_one_step_matches_fp64_accumulation(L):
    """One step from the same stored deviations: the split accumulation and the FP64 accumulation
    feed the same FP32 collide, so results agree to a few FP32 ulps of the weights."""
    Lx, Ly = 40, 36
    st = inputs.random_state(Lx, Ly, seed=11, du=0.03, dT=0.15, drho=0.15)
    a = L.Lattice.from_fields(st, tau=0.75, gy=-1e-3, precision="fp32dev")
    b = L.Lattice.from_fields(st, tau=0.75, gy=-1e-3, precision="fp32split")
    b.set_populations(a.get_populations())
    a.step(1)
    b.step(1)
    cx, cy, w, r = L.velocity_set()
    fa, fb = a.get_populations(), b.get_populations()
    assert np.max(np.abs(fa - fb) / w[:, None, None]) < 2.0**-19


def test_fp32split_reports_out_of_range_deviation(L):
    """A deviation |f - w| >= 1 (planted on the host) leaves the exact-split range: the step flags
    it and lb_sync reports LB_ERR_RANGE once."""
    st = inputs.rayleigh_taylor(32, 32, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9, precision="fp32split")
    f = lat.get_populations()
    f[3, 10, 7] += 6.0
    lat.set_populations(f)
    lat.step(1)
    with pytest.raises(L.RangeError):
        lat.sync()
    lat.sync()


@pytest.mark.parametrize("Lx,Ly,yp", [(36, 20, False), (68, 30, True), (256, 64, False), (64, 37, True),
                                      (2304, 64, False)])
def test_tma_staged_step_equals_plain_loads(L, Lx, Ly, yp):
    """The TMA-staged pull (boxes of 40 x 4, wrap-around read from global memory) gives the same
    populations, bit for bit, as plain loads: ragged tiles in x and y, walls and y-periodic."""
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=Lx + Ly)
    a = L.Lattice.from_fields(st, tau=0.8, y_periodic=yp, gy=st.gy * 3, precision="fp32split")
    b = L.Lattice.from_fields(st, tau=0.8, y_periodic=yp, gy=st.gy * 3, precision="fp32split")
    a.set_staging(True)
    b.set_staging(False)
    a.step(21)
    b.step(21)
    a.sync()
    b.sync()
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_tma_staging_unavailable_for_unaligned_rows(L):
    st = inputs.rayleigh_taylor(30, 20, R=2.0, seed=1)
    lat = L.Lattice.from_fields(st, tau=0.8, precision="fp32split")
    with pytest.raises(L.LBError):
        lat.set_staging(True)      # Lx = 30: rows are not 16-byte multiples
    lat.set_staging(False)


def _window_oracle(orc, st, x0, y0, n, half, tau):
    """FP64 oracle populations at (x0, y0) after n steps on a window around it (wrong values enter
    a window's cut edges at <= 3 sites per step, so the centre of a half-width >= 3 (n + 1) window
    is exact). Windows wrap in x and stop at real walls."""
    Ly, Lx = st.rho.shape
    xs = np.arange(x0 - half, x0 + half + 1) % Lx
    ylo, yhi = max(0, y0 - half), min(Ly, y0 + half + 1)
    sub = [a[ylo:yhi][:, xs] for a in (st.rho, st.ux, st.uy, st.T)]
    out = orc.run(orc.equilibrium(*sub), tau=tau, nsteps=n, gy=st.gy, T_top=st.T_top,
                  T_bottom=st.T_bottom, nthreads=1)
    return out[y0 - ylo, half]


def test_fp32split_full_size_2304x8192_sampled_sites_match_oracle(L, orc):
    """The FP32 split form at the bench size (2304 x 8192) in its launch configuration; sampled
    sites, including the x wrap and both walls, against the FP64 oracle on windows around them.
    Bound: n steps x 37 populations x 2^-24 x 0.35 relative to each population's weight."""
    Lx, Ly, n, tau = 2304, 8192, 4, 0.9
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=tau, precision="fp32split")
    lat.step(n)
    lat.sync()
    f = lat.get_populations()
    lat.close()
    cx, cy, w, _ = L.velocity_set()
    perm = orc.order_map(cx, cy)
    wo = np.empty(37)
    wo[perm] = w
    half = 3 * (n + 1)
    rng = np.random.default_rng(1)
    samples = [(0, 0), (Lx - 1, Ly - 1), (2, 1), (Lx - 3, Ly - 2), (1151, 4095), (7, Ly // 2)]
    samples += [(int(rng.integers(Lx)), int(rng.integers(Ly))) for _ in range(10)]
    bound = n * 37 * 2.0**-24 * 0.35
    worst = 0.0
    for (x0, y0) in samples:
        want = _window_oracle(orc, st, x0, y0, n, half, tau)
        got = np.empty(37)
        got[perm] = f[:, y0, x0]
        worst = max(worst, float(np.max(np.abs(got - want) / wo)))
    print(f"fp32split 2304x8192 sampled sites, {n} steps: max |f - f_oracle| / w = {worst:.2e}")
    assert worst < bound
