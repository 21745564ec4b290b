"""GPU parity of the FP64 path (through the C ABI) against the CPU oracle.

Bar: propagate bit-exact (a pure copy, Fig. 3 listing); the fused FP64 step within 1e-12
relative per population after 100 steps (the oracle and the kernel sum in different orders and
the kernel fuses multiply-adds, so results agree to rounding, not bit for bit).
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


def gpu_to_oracle(L, orc, f_planes):
    cx, cy, _, _ = L.velocity_set()
    return orc.from_planes(f_planes, cx, cy)


def oracle_to_gpu(L, orc, f_site):
    cx, cy, _, _ = L.velocity_set()
    return orc.to_planes(f_site, cx, cy)


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_init_is_the_equilibrium(L, orc):
    st = inputs.rayleigh_taylor(64, 256, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9)
    f = gpu_to_oracle(L, orc, lat.get_populations())
    assert rel_err(f, orc.init_fields(st)) < 1e-14


@pytest.mark.parametrize("Lx,Ly", [(11, 9), (64, 256), (70, 50)])
def test_propagate_is_bit_exact_periodic(L, orc, Lx, Ly):
    rng = np.random.default_rng(Lx * 1000 + Ly)
    st = inputs.random_state(Lx, Ly, seed=1)
    lat = L.Lattice.from_fields(st, tau=0.9, y_periodic=True)
    f0 = rng.uniform(0.0, 1.0, (37, Ly, Lx))
    lat.set_populations(f0)
    lat.propagate()
    got = lat.get_populations()
    src = np.zeros((Ly + 6, Lx, 37))
    src[3:Ly + 3] = gpu_to_oracle(L, orc, f0)
    want = oracle_to_gpu(L, orc, orc.propagate(src, Lx, Ly, y_periodic=True))
    assert np.array_equal(got, want)


def test_propagate_with_walls_bit_exact_away_from_walls(L, orc):
    """Rows 3..Ly-4 read no halo row: bit-exact. Rows next to a wall read halo values that both
    sides computed as a rest equilibrium (rounding-level agreement)."""
    Lx, Ly = 40, 30
    rng = np.random.default_rng(5)
    st = inputs.random_state(Lx, Ly, seed=2)
    lat = L.Lattice.from_fields(st, tau=0.9)
    f0 = orc.equilibrium(st.rho, st.ux, st.uy, st.T) * (1 + 0.01 * rng.uniform(-1, 1, (Ly, Lx, 37)))
    lat.set_populations(oracle_to_gpu(L, orc, f0))
    lat.propagate()
    got = gpu_to_oracle(L, orc, lat.get_populations())
    want = orc.propagate(orc.with_walls(f0, st.T_top, st.T_bottom), Lx, Ly, y_periodic=False)
    assert np.array_equal(got[3:Ly - 3], want[3:Ly - 3])
    assert rel_err(got, want) < 1e-14


@pytest.mark.parametrize("Lx,Ly,steps", [(64, 256, 100), (70, 50, 100), (13, 11, 30)])
def test_fused_step_matches_oracle_rayleigh_taylor(L, orc, Lx, Ly, steps):
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9)
    lat.step(steps)
    got = gpu_to_oracle(L, orc, lat.get_populations())
    want = orc.run(orc.init_fields(st), tau=0.9, nsteps=steps, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom)
    assert rel_err(got, want) <= TOL


def test_fused_step_matches_oracle_random_state_strong_gravity(L, orc):
    """Far-from-equilibrium start, strong gravity along both axes, walls at unequal temperature."""
    Lx, Ly = 33, 40
    st = inputs.random_state(Lx, Ly, seed=9)
    lat = L.Lattice.from_fields(st, tau=0.7, gx=1e-3, gy=-2e-3)
    lat.step(40)
    got = gpu_to_oracle(L, orc, lat.get_populations())
    want = orc.run(orc.init_fields(st), tau=0.7, nsteps=40, gx=1e-3, gy=-2e-3,
                   T_top=st.T_top, T_bottom=st.T_bottom)
    assert rel_err(got, want) <= TOL


def test_moments_match_oracle(L, orc):
    st = inputs.rayleigh_taylor(64, 256, R=2.0, seed=3)
    lat = L.Lattice.from_fields(st, tau=0.9)
    lat.step(7)
    rho, ux, uy, T = lat.moments()
    f = gpu_to_oracle(L, orc, lat.get_populations())
    orho, oux, ouy, oT = orc.moments(f)
    assert rel_err(rho, orho) < 1e-14 and rel_err(T, oT) < 1e-14
    assert np.max(np.abs(ux - oux)) < 1e-15 and np.max(np.abs(uy - ouy)) < 1e-15


def test_density_is_the_correctly_rounded_sum(L):
    """lb_moments' rho is the exact sum of a site's 37 populations rounded once to FP64 (round to
    nearest, ties to even): the moment sums are exact fixed-point sums, rounded on the integer
    pipe. Populations of mixed sign and magnitude in [2^-28, 16), including sites whose exact sum
    needs many more than 53 bits, and dyadic sites whose sums land on rounding ties. A site whose
    populations are symmetric under c -> -c has zero momentum exactly, and sites with rho = 1
    exactly and dyadic populations of either sign give u = r sum f c with a single rounding."""
    from fractions import Fraction
    Lx, Ly = 24, 10
    rng = np.random.default_rng(17)
    cx, cy, w, _ = L.velocity_set()
    f = w[:, None, None] * (1.0 + 0.3 * rng.uniform(-1, 1, (37, Ly, Lx)))
    # rows 2-3: magnitudes spread over 2^-28 .. 2^0 with random signs (positive site sums)
    spread = 2.0 ** rng.uniform(-28, 0, (37, 2, Lx)) * rng.choice([-1.0, 1.0], (37, 2, Lx))
    spread[0] = np.abs(spread[1:]).sum(axis=0) + 0.5
    assert spread[0].max() < 16.0
    f[:, 2:4] = spread
    # rows 4-5: dyadic values whose sums hit exact ties of the 53-bit rounding
    big = rng.integers(1, 2**20, (37, 2, Lx)).astype(np.float64)
    f[:, 4:6] = big * 2.0**-18
    s0 = f[:, 4:6].sum(axis=0)  # exact: every term is a multiple of 2^-18 below 2^2
    f[0, 4:6] += np.spacing(s0) * 0.5 * rng.choice([1.0, 3.0], (2, Lx))  # half an ulp, or 1.5
    # row 6: symmetric populations (zero momentum)
    half = w[1:19, None] * (1.0 + 0.2 * rng.uniform(-1, 1, (18, Lx)))
    f[1:19, 6] = half
    f[19:37, 6] = half
    # rows 7-8: dyadic populations of either sign with rho = 1 exactly, so that u = r sum f c is
    # one rounding of an exact value: checks the signed rounding of the momentum sums
    wq = np.round(w[1:] * 2.0**24)[:, None, None]
    k = rng.integers(-2**18, 2**18, (36, 2, Lx)).astype(np.float64)
    f[1:, 7:9] = (wq + k) * 2.0**-24
    f[0, 7:9] = 1.0 - f[1:, 7:9].sum(axis=0)  # exact: every term is a multiple of 2^-24 below 1
    lat = L.Lattice(Lx, Ly, 0.9, np.ones((Ly, Lx)), np.zeros((Ly, Lx)), np.zeros((Ly, Lx)),
                    np.ones((Ly, Lx)))
    lat.set_populations(f)
    rho, ux, uy, _ = lat.moments()
    for y in range(Ly):
        for x in range(Lx):
            exact = sum((Fraction(float(v)) for v in f[:, y, x]), Fraction(0))
            assert rho[y, x] == float(exact), (y, x, rho[y, x], float(exact))
    assert np.all(ux[6] == 0.0) and np.all(uy[6] == 0.0)
    _, _, _, r = L.velocity_set()
    assert np.all(rho[7:9] == 1.0)
    jx = np.einsum("i,iyx->yx", cx.astype(np.float64), f[:, 7:9])  # exact dyadic sums
    jy = np.einsum("i,iyx->yx", cy.astype(np.float64), f[:, 7:9])
    assert np.array_equal(ux[7:9], r * jx) and np.array_equal(uy[7:9], r * jy)


def test_graph_replay_equals_single_launches(L):
    st = inputs.rayleigh_taylor(64, 64, R=2.0, seed=4)
    a = L.Lattice.from_fields(st, tau=0.9)
    b = L.Lattice.from_fields(st, tau=0.9)
    a.step(37)                 # two 16-step graph replays + 5 single launches
    for _ in range(37):
        b.step(1)
    assert a.steps_done == b.steps_done == 37
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_checkpoint_resume_is_bit_identical(L):
    st = inputs.random_state(48, 40, seed=6)
    a = L.Lattice.from_fields(st, tau=0.8, y_periodic=True)
    a.step(20)
    b = L.Lattice.from_fields(st, tau=0.8, y_periodic=True)
    b.step(9)
    snap = b.get_populations()
    c = L.Lattice.from_fields(st, tau=0.8, y_periodic=True, own_memory=True)
    c.set_populations(snap)
    c.step(11)
    assert np.array_equal(a.get_populations(), c.get_populations())


def test_library_owned_memory_and_stream(L, orc):
    st = inputs.rayleigh_taylor(32, 64, R=2.0, seed=1)
    lat = L.Lattice.from_fields(st, tau=0.9, own_memory=True, stream=0)
    lat.step(5)
    got = gpu_to_oracle(L, orc, lat.get_populations())
    want = orc.run(orc.init_fields(st), tau=0.9, nsteps=5, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom)
    assert rel_err(got, want) <= TOL


def test_nonfinite_state_is_reported(L):
    """A NaN planted on the host is flagged by the step kernel and reported once by lb_sync."""
    st = inputs.rayleigh_taylor(32, 32, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9)
    f = lat.get_populations()
    f[5, 10, 7] = np.nan
    lat.set_populations(f)
    lat.step(1)
    with pytest.raises(L.NonFiniteError):
        lat.sync()
    lat.sync()  # the flag was cleared


def test_rest_state_with_walls_stays_at_rest(L):
    cx, cy, w, r = L.velocity_set()
    Lx, Ly = 40, 24
    lat = L.Lattice(Lx, Ly, 0.9, np.ones((Ly, Lx)), np.zeros((Ly, Lx)), np.zeros((Ly, Lx)),
                    np.ones((Ly, Lx)))
    lat.step(100)
    f = lat.get_populations()
    assert np.max(np.abs(f - w[:, None, None])) < 1e-14


def _window_oracle(orc, st, x0, y0, n, half, tau):
    """Oracle populations at (x0, y0) after n steps computed on a window of the lattice around it.
    Wrong values enter a window from its cut edges at <= 3 sites per step, so the centre of a
    window with half-width >= 3 (n + 1) is exact. Windows wrap in x and stop at real walls."""
    Ly, Lx = st.rho.shape
    xs = np.arange(x0 - half, x0 + half + 1) % Lx
    ylo, yhi = max(0, y0 - half), min(Ly, y0 + half + 1)
    sub = [a[ylo:yhi][:, xs] for a in (st.rho, st.ux, st.uy, st.T)]
    f0 = orc.equilibrium(*sub)
    out = orc.run(f0, tau=tau, nsteps=n, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom, nthreads=1)
    return out[y0 - ylo, half]


def test_full_size_2304x8192_sampled_sites_match_oracle(L, orc):
    """The bench workload (2304 x 8192, FP64, RT initial state) in the bench's launch
    configuration; sampled sites -- including the x wrap and both walls -- against the oracle
    run on windows around them."""
    Lx, Ly, n, tau = 2304, 8192, 4, 0.9
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=tau)
    lat.step(n)
    f = lat.get_populations()
    cx, cy, _, _ = L.velocity_set()
    perm = orc.order_map(cx, cy)
    half = 3 * (n + 1)
    rng = np.random.default_rng(0)
    samples = [(0, 0), (Lx - 1, Ly - 1), (1, 2), (Lx - 2, Ly - 3), (1151, 4095), (5, Ly // 2)]
    samples += [(int(rng.integers(Lx)), int(rng.integers(Ly))) for _ in range(10)]
    for (x0, y0) in samples:
        want = _window_oracle(orc, st, x0, y0, n, half, tau)
        got = f[:, y0, x0]
        got_o = np.empty(37)
        got_o[perm] = got
        assert rel_err(got_o, want) <= TOL, (x0, y0)


@pytest.mark.parametrize("y_periodic", [False, True])
def test_two_kernel_step_equals_fused_step(L, y_periodic):
    """The paper's two-kernel structure (propagate, then collide; Sec. 3, Table 1) gives the fused
    step's populations bit for bit."""
    st = inputs.rayleigh_taylor(96, 80, R=2.0, seed=5)
    a = L.Lattice.from_fields(st, tau=0.85, y_periodic=y_periodic)
    b = L.Lattice.from_fields(st, tau=0.85, y_periodic=y_periodic)
    for _ in range(7):
        a.propagate()
        a.collide()
    b.step(7)
    assert np.array_equal(a.get_populations(), b.get_populations())


@pytest.mark.parametrize("case", range(10))
def test_randomized_configurations_match_oracle(L, orc, case):
    """Seeded random configurations -- size (ragged, down to the 4 x 4 minimum), relaxation time,
    gravity on both axes, wall temperatures, wall closure, periodic or walled y -- each run 30 FP64
    steps from a random state and compared with the oracle at the 1e-12 bar."""
    rng = np.random.default_rng(1000 + case)
    Lx, Ly = (4, 4) if case == 0 else (int(rng.integers(4, 72)), int(rng.integers(4, 64)))
    tau = float(rng.uniform(0.65, 1.4))
    gx, gy = (float(v) for v in rng.uniform(-1.5e-3, 1.5e-3, 2))
    T_top, T_bottom = (float(v) for v in rng.uniform(0.85, 1.15, 2))
    y_periodic = bool(rng.integers(2))
    wall = "mirror" if rng.integers(2) else "rest"
    st = inputs.random_state(Lx, Ly, seed=case, du=0.02, dT=0.1, drho=0.1)
    lat = L.Lattice(Lx, Ly, tau, st.rho, st.ux, st.uy, st.T, gx=gx, gy=gy, T_top=T_top,
                    T_bottom=T_bottom, y_periodic=y_periodic, wall_mode=wall)
    lat.step(30)
    lat.sync()
    got = gpu_to_oracle(L, orc, lat.get_populations())
    lat.close()
    want = orc.run(orc.init_fields(st), tau=tau, nsteps=30, gx=gx, gy=gy, T_top=T_top,
                   T_bottom=T_bottom, y_periodic=y_periodic, wall_mode=wall)
    assert rel_err(got, want) <= TOL, (Lx, Ly, tau, gx, gy, y_periodic, wall)


@pytest.mark.parametrize("tau", [0.55, 0.7, 2.5])
def test_strong_flow_matches_oracle(L, orc, tau):
    """A harder regime than the Rayleigh-Taylor runs: spatially uncorrelated velocities up to 0.15
    per component, densities 0.7-1.3, temperatures 0.8-1.2, gravity 3e-3 on both axes, relaxation
    times from near the stability limit to strongly under-relaxed. After 20 steps every population
    agrees with the oracle within 1e-12 of its weight (the populations' scale at rest, so that
    populations that the flow drives towards zero are held to the same absolute standard)."""
    Lx, Ly = 40, 36
    st = inputs.random_state(Lx, Ly, seed=7, du=0.15, dT=0.2, drho=0.3)
    lat = L.Lattice(Lx, Ly, tau, st.rho, st.ux, st.uy, st.T, gx=3e-3, gy=-3e-3, T_top=0.9,
                    T_bottom=1.1)
    lat.step(20)
    lat.sync()
    got = gpu_to_oracle(L, orc, lat.get_populations())
    lat.close()
    want = orc.run(orc.init_fields(st), tau=tau, nsteps=20, gx=3e-3, gy=-3e-3, T_top=0.9,
                   T_bottom=1.1)
    _, _, w, _ = orc.velocity_set()
    assert np.max(np.abs(got - want) / w) <= TOL


@pytest.mark.parametrize("tau", [0.6, 1.7])
def test_fixed_point_domain_edge_and_fallback_match_oracle(L, orc, tau):
    """Sites on both sides of the fixed-point pair terms' domain (|u*| components <= 0.2, T* in
    [0.6, 1.4]; outside it the FP64 evaluation runs) mixed within every warp: uncorrelated
    velocities up to 0.3 per component and temperatures 0.45-1.55. After 5 steps every population
    agrees with the oracle within 1e-12 of its weight."""
    Lx, Ly = 64, 24
    st = inputs.random_state(Lx, Ly, seed=11, du=0.3, dT=0.55, drho=0.2)
    lat = L.Lattice(Lx, Ly, tau, st.rho, st.ux, st.uy, st.T, gx=1e-3, gy=-2e-3, T_top=0.8,
                    T_bottom=1.2)
    lat.step(5)
    lat.sync()
    got = gpu_to_oracle(L, orc, lat.get_populations())
    lat.close()
    want = orc.run(orc.init_fields(st), tau=tau, nsteps=5, gx=1e-3, gy=-2e-3, T_top=0.8, T_bottom=1.2)
    _, _, w, _ = orc.velocity_set()
    inside = (np.abs(st.ux) <= 0.2) & (np.abs(st.uy) <= 0.2) & (np.abs(st.T - 1.0) <= 0.4)
    assert 0.2 < inside.mean() < 0.8            # both paths, within warps
    err = float(np.max(np.abs(got - want) / w))
    print(f"fixed-point domain edge, tau {tau}: max |f - f_oracle| / w = {err:.2e}")
    assert err <= TOL


def test_exact_sums_outside_their_fast_range_match_oracle(L, orc):
    """The step's exact moment sums take a shorter path when every population of a batch is positive
    and in [2^-28, 16); planted negative, tiny (< 2^-28, truncated at the 2^-80 quantum) and large
    populations at scattered sites send those sites' batches through the general conversion. One
    step agrees with the oracle within 1e-12 of each population's weight everywhere."""
    Lx, Ly = 48, 20
    st = inputs.random_state(Lx, Ly, seed=13, du=0.05, dT=0.1, drho=0.1)
    f0 = orc.equilibrium(st.rho, st.ux, st.uy, st.T)
    rng = np.random.default_rng(14)
    f0 = f0 * (1.0 + 0.02 * rng.uniform(-1, 1, f0.shape))
    _, _, w, _ = orc.velocity_set()
    for k, (y, x) in enumerate([(2, 3), (5, 40), (9, 17), (13, 30), (17, 8), (11, 44)]):
        i = (7 * k + 3) % 37
        f0[y, x, i] = (-0.01, 1e-12, 3e-10, 2.5, -1e-9, 0.9)[k] * (w[i] if k != 3 else 1.0)
    cx, cy, _, _ = L.velocity_set()
    lat = L.Lattice(Lx, Ly, 0.8, st.rho, st.ux, st.uy, st.T, T_top=st.T_top, T_bottom=st.T_bottom,
                    y_periodic=True)
    lat.set_populations(orc.to_planes(f0, cx, cy))
    lat.step(1)
    lat.sync()
    got = orc.from_planes(lat.get_populations(), cx, cy)
    lat.close()
    want = orc.run(f0, tau=0.8, nsteps=1, y_periodic=True)
    err = float(np.max(np.abs(got - want) / w))
    print(f"planted populations outside the fast range: max |f - f_oracle| / w = {err:.2e}")
    assert err <= TOL


@pytest.mark.parametrize("wall_mode", ["rest", "mirror"])
def test_fused_step_matches_oracle_over_1000_steps(L, orc, wall_mode):
    """Ten times the bar's horizon: the rounding differences between the kernel (exact integer
    moment sums, fused multiply-adds, regrouped polynomials) and the oracle (table-order FP64 sums)
    grow slowly -- about 5e-13 relative after 1000 steps of the 64 x 256 Rayleigh-Taylor case -- and
    stay within 1e-12."""
    st = inputs.rayleigh_taylor(64, 256, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9, wall_mode=wall_mode)
    lat.step(1000)
    lat.sync()
    got = gpu_to_oracle(L, orc, lat.get_populations())
    lat.close()
    want = orc.run(orc.init_fields(st), tau=0.9, nsteps=1000, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom, wall_mode=wall_mode)
    assert rel_err(got, want) <= TOL


def test_device_allocation_failure_is_reported(L):
    """A lattice whose populations cannot fit in device memory (2e9 sites, ~1.2 TB): lb_init fails
    with LB_ERR_ALLOC before it reads any host field, names the failed allocation, and the device
    stays usable."""
    import ctypes as C
    lib = L.lib()
    ctx = C.c_void_p()
    p = L.make_params(40000, 50000, 0.9)
    z = np.zeros(4)
    assert lib.lb_init(C.byref(p), z.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                       C.byref(ctx)) == 2
    assert not ctx.value
    assert "cudaMalloc" in L.last_error()
    st = inputs.rayleigh_taylor(32, 32, R=2.0, seed=0)
    lat = L.Lattice.from_fields(st, tau=0.9)
    lat.step(3)
    lat.sync()
    lat.close()


def test_nan_in_the_initial_fields_is_reported(L):
    """A NaN planted in the host density field: the first step flags it and lb_sync reports
    LB_ERR_NONFINITE once."""
    st = inputs.rayleigh_taylor(32, 32, R=2.0, seed=0)
    rho = st.rho.copy()
    rho[17, 9] = np.nan
    lat = L.Lattice(32, 32, 0.9, rho, st.ux, st.uy, st.T, gy=st.gy, T_top=st.T_top,
                    T_bottom=st.T_bottom)
    lat.step(1)
    with pytest.raises(L.NonFiniteError):
        lat.sync()
    lat.sync()
    lat.close()


def test_api_edge_cases(L):
    """lb_step(0) is a no-op, a negative count is an argument error, moments accept NULL outputs,
    and a population round trip through the host is exact (FP64) or within FP32 storage rounding
    of the deviations (FP32 forms)."""
    import ctypes as C
    st = inputs.rayleigh_taylor(40, 48, R=2.0, seed=8)
    lat = L.Lattice.from_fields(st, tau=0.9)
    f0 = lat.get_populations()
    lat.step(0)
    assert lat.steps_done == 0 and np.array_equal(lat.get_populations(), f0)
    assert L.lib().lb_step(lat._ctx, -1) == 1
    rho = np.empty((48, 40))
    assert L.lib().lb_moments(lat._ctx, rho.ctypes.data, None, None, None) == 0
    assert np.allclose(rho, st.rho, rtol=1e-14, atol=0)
    lat.set_populations(f0)
    assert np.array_equal(lat.get_populations(), f0)
    lat.close()
    cx, cy, w, _ = L.velocity_set()
    for form in ("fp32dev", "fp32split"):
        lat = L.Lattice.from_fields(st, tau=0.9, precision=form)
        f = lat.get_populations()
        lat.set_populations(f)
        g = lat.get_populations()
        dev = np.abs(f - w[:, None, None])
        assert np.all(np.abs(g - f) <= dev * 2.0**-24 + 1e-300), form
        lat.close()
