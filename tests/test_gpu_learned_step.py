"""The learned LB step on the GPU (step_learned_kernel through lb_step) against the FP64 oracle of
the same step (oracle/learned.py), population by population, tile decision by tile decision.

Inputs are seeded on both sides: the fields from inputs.rayleigh_taylor / random_state, the
network's parameters and normalisation from inputs.mlp_params / mlp_norm. Each side builds its
own initial populations from the fields and takes one step.

Bounds. The network runs with BF16 operands and FP32 accumulation on the tensor cores; the oracle
evaluates the same network in FP64 with the BF16 rounding points (the bar of the forward-pass test:
1e-2 of the largest output). A difference dy in the normalised output moves the candidate by
sd_t dy, and the projection is the linear map P = I - W M^T (M W M^T)^-1 M on that difference, so a
kept population may differ by sum_j |P_ij| sd_t,j dy_max plus FP32 storage rounding (16 FP32 ulps
of a unit deviation times the weight, the one-step bar of the FP32 forms). A fallback population
is the FP32 exact-split plain collide against the oracle's FP64 collide. Its FP32 relaxation sums
terms of the shifted equilibrium that reach a few times the weight where the temperature is far
from 1 (on the |c| = 3 shells at theta = 1/3 the xi^4 theta^2 / 8 term alone is ~3 w), so each
rounding there is worth ~4 ulps of the weight: the bar is 64 FP32 ulps of the weight.
The residual difference of a tile is bounded by those population bounds over max |f_plain|; tile
decisions must agree wherever the oracle's residual is farther than that from the bound.
"""
import numpy as np
import pytest

from oracle import learned as olr
from paper_1804_01918_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_BAR = 16 * 2.0**-24     # one step, relative to the weight
FP32_PLAIN_BAR = 64 * 2.0**-24   # the FP32 plain collide far from T = 1, relative to the weight
Y_BAR = 1e-2                 # network output, relative to its largest value


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01918_gb300 import build, lb
    build.build()
    return lb


def projection_operator(orc):
    _, _, w, _ = orc.velocity_set()
    M = olr.moment_matrix()
    A = (M * w) @ M.T
    return np.eye(37) - (w[:, None] * M.T) @ np.linalg.solve(A, M)


def gap_bound(residuals):
    """A bound between the two tile residuals of the widest ratio gap (geometric mean), so that
    some tiles keep the network, some fall back, and none sits near the bound."""
    r = np.sort(np.asarray(residuals).ravel())
    k = int(np.argmax(r[1:] / r[:-1]))
    return float(np.sqrt(r[k] * r[k + 1]))


def run_case(L, orc, st, tau, bound, params, norm, y_periodic=False, gx=0.0):
    """One learned step on the GPU and in the oracle. bound="gap" picks the bound from the
    oracle's tile residuals (gap_bound) before the GPU runs."""
    Ly, Lx = st.rho.shape
    cxg, cyg, wg, _ = L.velocity_set()
    order = (cxg, cyg)

    def oracle(b):
        return olr.learned_step(orc.init_fields(st), tau, olr.network_change(params, norm, order), norm,
                                order, b, gx=gx, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom,
                                y_periodic=y_periodic)

    want = oracle(np.inf)
    if bound == "gap":
        bound = gap_bound(want["residual"])
        want = oracle(bound)
    want["bound"] = bound
    net = L.MLP(seed=0)
    net.set_params(params, norm)
    lat = L.Lattice.from_fields(st, tau=tau, precision="fp32split", y_periodic=y_periodic, gx=gx)
    lat.set_collide_learned(net, bound=bound)
    lat.step(1)
    lat.sync()
    got = orc.from_planes(lat.get_populations(), cxg, cyg)
    modes = lat.learned_tiles()
    stats = lat.learned_stats()
    lat.close()
    net.close()
    # per-population bounds in oracle order
    _, _, w, _ = orc.velocity_set()
    perm = orc.order_map(cxg, cyg)
    sd_t = np.empty(37)
    sd_t[perm] = np.asarray(norm, np.float64)[3]
    dy = Y_BAR * np.max(np.abs(want["y"]))
    tol_learned = np.abs(projection_operator(orc)) @ (sd_t * dy) + FP32_BAR * w
    tol_plain = FP32_PLAIN_BAR * w
    return got, modes, stats, want, tol_learned, tol_plain


def check_case(got, modes, stats, want, tol_learned, tol_plain, tile=32):
    nty, ntx = want["fallback"].shape
    margin_all = 0.0
    decided = 0
    for ty in range(nty):
        for tx in range(ntx):
            sl = (slice(ty * tile, (ty + 1) * tile), slice(tx * tile, (tx + 1) * tile))
            fp = want["f_plain"][sl]
            margin = 1.5 * np.max(tol_learned + tol_plain) / np.max(np.abs(fp))
            margin_all = max(margin_all, margin)
            res = want["residual"][ty, tx]
            if not np.isfinite(res) or abs(res - want["bound"]) > margin * max(1.0, res):
                assert bool(modes[ty, tx]) == bool(want["fallback"][ty, tx]), (ty, tx, res)
                decided += 1
            if modes[ty, tx]:
                err = np.abs(got[sl] - fp) / tol_plain
            else:
                err = np.abs(got[sl] - want["f_learned"][sl]) / tol_learned
            assert err.max() <= 1.0, (ty, tx, bool(modes[ty, tx]), float(err.max()))
    assert decided == nty * ntx, "a tile's oracle residual sits within rounding of the bound"
    assert stats["tiles_checked"] == nty * ntx
    assert stats["tiles_fallback"] == int(want["fallback"].sum())
    rmax = float(np.max(want["residual"]))
    assert abs(stats["max_residual"] - rmax) <= margin_all * rmax
    return margin_all


@pytest.mark.parametrize("bound", [np.inf, "gap"])
def test_learned_step_matches_oracle_rayleigh_taylor(L, orc, bound):
    """128 x 128 Rayleigh-Taylor lattice with walls: 16 tiles. The tiles along the interface
    (far from equilibrium after the first pull) have residuals ~0.1, those along the walls ~2e-4;
    with the bound in that gap the interface tiles fall back and the wall tiles keep the network,
    with an infinite bound every tile keeps it. Every population of every tile is held to its
    bar against the oracle's learned step (kept tiles) or plain step (fallback tiles)."""
    _, _, wg, _ = L.velocity_set()
    st = inputs.rayleigh_taylor(128, 128, R=2.0, seed=3)
    params = inputs.mlp_params(5)
    norm = inputs.mlp_norm(wg, seed=1, sd_t=1e-4, mu_t=2e-4)
    got, modes, stats, want, tl, tp = run_case(L, orc, st, 0.9, bound, params, norm)
    if bound == "gap":
        assert want["fallback"].any() and not want["fallback"].all()
    check_case(got, modes, stats, want, tl, tp)
    kept = ~want["fallback"]
    print(f"bound {want['bound']:.3e}: tiles kept {int(kept.sum())}/16, oracle residuals "
          f"{np.array2string(want['residual'].ravel(), formatter={'float': lambda v: '%.2e' % v})}")


def test_learned_step_matches_oracle_random_state_periodic(L, orc):
    """Uncorrelated random fields on a y-periodic 64 x 64 lattice with gravity on both axes and an
    infinite bound: the projection of the network's change is compared at every site."""
    _, _, wg, _ = L.velocity_set()
    st = inputs.random_state(64, 64, seed=9, du=0.03, dT=0.1, drho=0.1)
    st = inputs.RTFields(st.rho, st.ux, st.uy, st.T, st.T_top, st.T_bottom, gy=-2e-3)
    params = inputs.mlp_params(6, scale=1.5)
    norm = inputs.mlp_norm(wg, seed=4, sd_t=3e-4, mu_t=-2e-5)
    got, modes, stats, want, tl, tp = run_case(L, orc, st, 0.8, np.inf, params, norm, y_periodic=True,
                                               gx=1e-3)
    check_case(got, modes, stats, want, tl, tp)


@pytest.mark.parametrize("bound", [np.inf, "gap"])
def test_learned_step_with_constant_network_output_is_fp32_exact(L, orc, bound):
    """With the last weight matrix zero the network's output is its last bias b3 exactly (the
    third product adds zeros in FP32), so the kept tiles hold the projection of d + sd_t b3 + mu_t
    at the FP32 bar of the plain forms, with nothing left to the BF16 network: a dropped or
    mis-indexed b3, mu_t or sd_t, or an error in the addition or the projection fails here."""
    _, _, wg, _ = L.velocity_set()
    st = inputs.rayleigh_taylor(128, 96, R=2.0, seed=4)
    params = inputs.mlp_params(7)
    w3 = slice(128 * 37 + 128 + 128 * 128 + 128, 128 * 37 + 128 + 128 * 128 + 128 + 37 * 128)
    params[w3] = 0.0
    norm = inputs.mlp_norm(wg, seed=2, sd_t=1e-4, mu_t=2e-4)
    got, modes, stats, want, _, tp = run_case(L, orc, st, 0.9, bound, params, norm)
    _, _, w, _ = orc.velocity_set()
    assert np.max(np.abs(want["y"])) > 0.01          # the bias is there to be dropped
    check_case(got, modes, stats, want, FP32_BAR * w, tp)


def test_learned_step_full_size_sampled_tiles_match_oracle(L, orc):
    """The bench workload's size (2304 x 8192 Rayleigh-Taylor, FP32 split storage) in the bench's
    launch configuration (one CTA per SM, each warpgroup stepping ~40 tiles one after another):
    sampled tiles -- at both walls, at the x wrap, across the interface and at random -- against
    the oracle's learned step evaluated on a window around each (a tile pulls from at most 3 sites
    beyond its edges; the window wraps in x and stops at the real walls). Bound 1e-2: tiles across
    the interface fall back, the rest keep the network."""
    Lx, Ly, tau, bound = 2304, 8192, 0.9, 1e-2
    _, _, wg, _ = L.velocity_set()
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=0)
    params = inputs.mlp_params(5)
    norm = inputs.mlp_norm(wg, seed=1, sd_t=1e-4, mu_t=2e-4)
    net = L.MLP(seed=0)
    net.set_params(params, norm)
    lat = L.Lattice.from_fields(st, tau=tau, precision="fp32split")
    lat.set_collide_learned(net, bound=bound)
    lat.step(1)
    lat.sync()
    f1 = lat.get_populations()
    modes = lat.learned_tiles()
    stats = lat.learned_stats()
    lat.close()
    net.close()
    ntx, nty = Lx // 32, Ly // 32
    assert stats["tiles_checked"] == ntx * nty
    cxg, cyg, _, _ = L.velocity_set()
    perm = orc.order_map(cxg, cyg)
    _, _, w, _ = orc.velocity_set()
    nrm = np.empty((4, 37))
    nrm[:, perm] = np.asarray(norm, np.float64)
    predict = olr.network_change(params, norm, (cxg, cyg))
    P = np.abs(projection_operator(orc))
    rng = np.random.default_rng(7)
    tiles = [(0, 0), (ntx - 1, 0), (0, nty - 1), (ntx - 1, nty - 1), (5, nty // 2 - 1), (6, nty // 2),
             (ntx // 2, nty // 2 - 1), (ntx - 1, nty // 2)]
    tiles += [(int(rng.integers(ntx)), int(rng.integers(nty))) for _ in range(8)]
    kinds = set()
    for tx, ty in tiles:
        x0, y0 = 32 * tx, 32 * ty
        xs = np.arange(x0 - 3, x0 + 35) % Lx
        ylo, yhi = max(0, y0 - 3), min(Ly, y0 + 35)
        sub = [a[ylo:yhi][:, xs] for a in (st.rho, st.ux, st.uy, st.T)]
        fp = olr.pulled(orc.equilibrium(*sub), st.T_top, st.T_bottom)[y0 - ylo:y0 - ylo + 32, 3:35]
        d = (fp - w).reshape(-1, 37)
        y = predict(d)
        dl = olr.project(olr.add_change(d, y, nrm), olr.targets(d, 0.0, st.gy))
        f_learned = (dl + w).reshape(32, 32, 37)
        f_plain = orc.collide(fp, tau, 0.0, st.gy)
        res = olr.tile_residual(f_learned, f_plain)
        got = orc.from_planes(f1[:, y0:y0 + 32, x0:x0 + 32], cxg, cyg)
        tol_learned = P @ (nrm[3] * Y_BAR * np.max(np.abs(y))) + FP32_BAR * w
        tol_plain = FP32_PLAIN_BAR * w
        margin = 1.5 * np.max(tol_learned + tol_plain) / np.max(np.abs(f_plain))
        if abs(res - bound) > margin * max(1.0, res):
            assert bool(modes[ty, tx]) == olr.falls_back(res, bound), (tx, ty, res)
        if modes[ty, tx]:
            err = np.abs(got - f_plain) / tol_plain
        else:
            err = np.abs(got - f_learned) / tol_learned
        kinds.add(bool(modes[ty, tx]))
        assert err.max() <= 1.0, (tx, ty, bool(modes[ty, tx]), float(err.max()))
    assert kinds == {False, True}, "the sampled tiles should include kept and fallback ones"
