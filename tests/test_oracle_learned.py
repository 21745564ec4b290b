"""Pins of the learned-collide oracle (oracle/learned.py) against mathematics that does not come
from the oracle itself: the plain collide (pinned in test_oracle_model.py / test_oracle_step.py),
the defining properties of a weighted least-norm projection, and brute force on small cases.

The paper has no learned collide; the step is the Sec. 3 collide replaced by a network whose
output is projected onto the moments that collide conserves (mass, momentum, energy; gravity
through the shifted equilibrium), with a per-tile fallback to the plain collide.

Each pin is a helper taking the functions under test, so that the planted-mistake tests at the end
can run the same pin on a deliberately broken copy of the oracle and see it fail.
"""
import numpy as np
import pytest
from scipy.linalg import null_space

from oracle import learned as olr
from oracle import mlp as omlp
from paper_1804_01918_gb300 import inputs


def table(orc):
    cx, cy, w, r = orc.velocity_set()
    return cx.astype(float), cy.astype(float), w, r


def nonequilibrium_state(orc, n=64, seed=0, amp=0.05):
    """Site-major populations [n, 37]: equilibria of random fields times (1 + amp * noise), i.e.
    far from equilibrium, with positive density and temperature."""
    st = inputs.random_state(n, 1, seed=seed, du=0.1, dT=0.2, drho=0.2)
    f = orc.equilibrium(st.rho, st.ux, st.uy, st.T).reshape(-1, 37)
    rng = np.random.default_rng(seed + 100)
    return f * (1.0 + amp * rng.uniform(-1, 1, f.shape))


# ---- pins as helpers ---------------------------------------------------------------------------

def pin_projection_meets_targets(orc, project):
    _, _, w, _ = table(orc)
    rng = np.random.default_rng(1)
    dhat = 0.1 * w * rng.standard_normal((200, 37))
    tgt = 0.05 * rng.standard_normal((200, 4))
    M = olr.moment_matrix()
    got = project(dhat, tgt) @ M.T
    return float(np.max(np.abs(got - tgt)))


def pin_correction_in_weighted_quadratic_span(orc, project):
    """(project(x) - x)_i / w_i must be a combination of 1, c_x, c_y, |c|^2 (least-squares fit of
    the 37 ratios by those four columns leaves no residual)."""
    cx, cy, w, _ = table(orc)
    rng = np.random.default_rng(2)
    dhat = 0.1 * w * rng.standard_normal((50, 37))
    tgt = 0.05 * rng.standard_normal((50, 4))
    ratio = (project(dhat, tgt) - dhat) / w
    B = np.stack([np.ones(37), cx, cy, cx * cx + cy * cy], axis=1)
    coef, *_ = np.linalg.lstsq(B, ratio.T, rcond=None)
    return float(np.max(np.abs(B @ coef - ratio.T)) / np.max(np.abs(ratio)))


def pin_targets_match_plain_collide(orc, targets, gx, gy, tau=0.8):
    """The moments of the plain collide's output (an independently pinned function) are the
    targets computed from its input."""
    _, _, w, _ = table(orc)
    f = nonequilibrium_state(orc, seed=3)
    post = orc.collide(f, tau, gx, gy)
    M = olr.moment_matrix()
    return float(np.max(np.abs((post - w) @ M.T - targets(f - w, gx, gy))))


def pin_exact_predictor_gives_plain_step(orc, learned_step, norm_scale=(0.3, 2e-4, 1e-5, 3e-4)):
    """With a predictor that returns the exact normalised change of the plain collide, the
    learned candidate equals the plain collide and the full step equals the oracle's plain step."""
    _, _, w, _ = table(orc)
    Lx, Ly, tau, gy = 32, 64, 0.9, -2e-4
    st = inputs.rayleigh_taylor(Lx, Ly, R=2.0, seed=4)
    f0 = orc.init_fields(st)
    rng = np.random.default_rng(5)
    cxo, cyo, _, _ = orc.velocity_set()
    norm = np.stack([s * (1 + rng.random(37)) * (w if k else 1.0) for k, s in enumerate(norm_scale)])
    fp = olr.pulled(f0, st.T_top, st.T_bottom)
    exact = ((orc.collide(fp, tau, 0.0, gy) - fp).reshape(-1, 37) - norm[2]) / norm[3]

    def predict(d):
        return exact

    out = learned_step(f0, tau, predict, norm, (cxo, cyo), bound=1e-9, gy=gy, T_top=st.T_top,
                       T_bottom=st.T_bottom)
    plain = orc.run(f0, tau=tau, nsteps=1, gy=gy, T_top=st.T_top, T_bottom=st.T_bottom)
    return float(np.max(np.abs(out["f_learned"] - plain) / w)), out


def pin_residual_definition(tile_residual):
    """Relative max-norm error of the learned tile against the plain tile: a uniform relative
    perturbation eps gives eps; a spike of size s at any population gives s / max|f_plain|."""
    rng = np.random.default_rng(6)
    fp = rng.uniform(0.01, 0.3, (32, 32, 37))
    errs = [abs(tile_residual(fp, fp))]
    eps = 0.1
    errs.append(abs(tile_residual(fp * (1 + eps), fp) - eps) / eps)
    spike = fp.copy()
    spike[3, 7, 11] += 0.02
    errs.append(abs(tile_residual(spike, fp) - 0.02 / fp.max()) / 0.02)
    return max(errs)


# ---- the pins ----------------------------------------------------------------------------------

def test_projection_meets_targets(orc):
    assert pin_projection_meets_targets(orc, olr.project) < 1e-15


def test_projection_is_idempotent(orc):
    _, _, w, _ = table(orc)
    rng = np.random.default_rng(7)
    dhat = 0.1 * w * rng.standard_normal((100, 37))
    tgt = 0.05 * rng.standard_normal((100, 4))
    once = olr.project(dhat, tgt)
    assert np.max(np.abs(olr.project(once, tgt) - once) / w) < 1e-14


def test_projection_passes_changes_orthogonal_to_the_invariants(orc):
    """A change v with M v = 0 (orthogonal in the inner product sum a_i b_i / w_i to every
    correction w_i (l0 + lx c_x + ly c_y + le |c|^2)) passes the projection unchanged."""
    _, _, w, _ = table(orc)
    rng = np.random.default_rng(8)
    N = null_space(olr.moment_matrix())                       # 37 x 33 basis of {v : M v = 0}
    assert N.shape == (37, 33)
    dhat = 0.1 * w * rng.standard_normal((20, 37))
    v = (N @ rng.standard_normal((33, 20))).T * 1e-3
    tgt = 0.05 * rng.standard_normal((20, 4))
    assert np.max(np.abs(olr.project(dhat + v, tgt) - (olr.project(dhat, tgt) + v))) < 1e-15


def test_projection_correction_is_weight_times_quadratic_in_c(orc):
    assert pin_correction_in_weighted_quadratic_span(orc, olr.project) < 1e-12


def test_projection_has_least_weighted_norm(orc):
    """Brute force: adding any null-space change to the correction makes sum delta^2 / w larger."""
    _, _, w, _ = table(orc)
    rng = np.random.default_rng(9)
    dhat = 0.1 * w * rng.standard_normal(37)
    tgt = 0.05 * rng.standard_normal(4)
    delta = olr.project(dhat, tgt) - dhat
    base = np.sum(delta * delta / w)
    N = null_space(olr.moment_matrix())
    for _ in range(500):
        n = N @ rng.standard_normal(33) * 10.0 ** rng.uniform(-6, -2)
        assert np.sum((delta + n) ** 2 / w) > base


@pytest.mark.parametrize("g", [(0.0, 0.0), (0.0, -3e-3), (2e-3, 1e-3)])
def test_targets_are_the_plain_collides_moments(orc, g):
    assert pin_targets_match_plain_collide(orc, olr.targets, *g) < 1e-13


def test_plain_collide_is_a_fixed_point_of_the_projection(orc):
    """The plain collide already has the target moments, so projecting it changes nothing."""
    _, _, w, _ = table(orc)
    f = nonequilibrium_state(orc, seed=10)
    post = orc.collide(f, 0.7, 1e-3, -2e-3) - w
    again = olr.project(post, olr.targets(f - w, 1e-3, -2e-3))
    # the collide's own moments sit within ~2e-15 of the targets (its rounding)
    assert np.max(np.abs(again - post) / w) < 1e-13


def test_exact_predictor_reproduces_the_plain_step(orc):
    err, out = pin_exact_predictor_gives_plain_step(orc, olr.learned_step)
    assert err < 1e-12
    assert not out["fallback"].any() and out["residual"].max() < 1e-12


def test_tile_residual_definition():
    assert pin_residual_definition(olr.tile_residual) < 1e-14
    assert olr.tile_residual(np.full((2, 2), 0.5), np.zeros((2, 2))) == 0.5


def test_fallback_rule():
    assert not olr.falls_back(1e-4, 1e-4)
    assert olr.falls_back(np.nextafter(1e-4, 1.0), 1e-4)
    assert olr.falls_back(float("nan"), 1e-4)
    assert not olr.falls_back(0.0, 0.0)


def random_network(seed, out_scale):
    """Seeded parameters with the output layer scaled by out_scale (network order = any)."""
    p = inputs.mlp_params(seed)
    p[omlp.NPARAM - 37 - 37 * 128:] *= out_scale
    return p


def test_bound_zero_falls_back_everywhere_and_equals_the_plain_step(orc):
    _, _, w, _ = table(orc)
    cxo, cyo, _, _ = orc.velocity_set()
    st = inputs.rayleigh_taylor(32, 64, R=2.0, seed=11)
    f0 = orc.init_fields(st)
    norm = inputs.mlp_norm(w, seed=1)
    pred = olr.network_change(random_network(3, 1.0), norm, (cxo, cyo))
    out = olr.learned_step(f0, 0.9, pred, norm, (cxo, cyo), bound=0.0, gy=st.gy, T_top=st.T_top,
                           T_bottom=st.T_bottom)
    assert out["fallback"].all()
    plain = orc.run(f0, tau=0.9, nsteps=1, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom)
    assert np.array_equal(out["f"], plain)


def test_learned_step_conserves_and_keeps_moments_of_kept_tiles(orc):
    """Infinite bound: every tile keeps the network's result, whose mass, momentum and energy are
    those of the plain collide at every site (y-periodic lattice: the sums over the lattice are
    those of the pulled state plus the gravity terms)."""
    _, _, w, r = table(orc)
    cxo, cyo, _, _ = orc.velocity_set()
    st = inputs.random_state(32, 32, seed=12, du=0.02, dT=0.1, drho=0.1)
    f0 = orc.init_fields(st)
    norm = inputs.mlp_norm(w, seed=2)
    pred = olr.network_change(random_network(4, 1.0), norm, (cxo, cyo))
    out = olr.learned_step(f0, 0.8, pred, norm, (cxo, cyo), bound=np.inf, gy=-1e-3, y_periodic=True)
    assert not out["fallback"].any()
    M = olr.moment_matrix()
    a = (out["f"] - w) @ M.T
    b = (out["f_plain"] - w) @ M.T
    assert np.max(np.abs(a - b)) < 1e-14
    assert abs((out["f"].sum() - f0.sum()) / f0.sum()) < 1e-14


# ---- planted mistakes: each broken copy of the oracle fails a pin -----------------------------

def _unweighted_project(dhat, m_target):
    M = olr.moment_matrix()
    lam = np.linalg.solve(M @ M.T, (m_target - dhat @ M.T).T).T
    return dhat + lam @ M


def _targets_without_gravity_energy(d, gx=0.0, gy=0.0):
    t = olr.targets(d, gx, gy)
    return np.concatenate([t[..., :3], olr.targets(d)[..., 3:]], axis=-1)


def _targets_gravity_sign(d, gx=0.0, gy=0.0):
    return olr.targets(d, -gx, -gy)


def _residual_wrong_norm(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(a)))


def test_planted_unweighted_projection_fails(orc):
    assert pin_projection_meets_targets(orc, _unweighted_project) < 1e-15   # still on target
    assert pin_correction_in_weighted_quadratic_span(orc, _unweighted_project) > 1e-3


@pytest.mark.parametrize("bad", [_targets_without_gravity_energy, _targets_gravity_sign])
def test_planted_target_mistakes_fail(orc, bad):
    assert pin_targets_match_plain_collide(orc, bad, 2e-3, -3e-3) > 1e-8


def test_planted_residual_normalisation_fails():
    assert pin_residual_definition(_residual_wrong_norm) > 1e-3


@pytest.mark.parametrize("which", ["mu_t dropped", "sd_x for sd_t"])
def test_planted_change_mistakes_fail(orc, which, monkeypatch):
    def bad_add(d, y, norm):
        norm = np.asarray(norm, dtype=np.float64)
        return d + y * norm[3] if which == "mu_t dropped" else d + y * norm[1] + norm[2]
    monkeypatch.setattr(olr, "add_change", bad_add)
    err, _ = pin_exact_predictor_gives_plain_step(orc, olr.learned_step)
    assert err > 1e-6
