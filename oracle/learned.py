"""Plain FP64 oracle of the learned-collide step (test infrastructure only).

Only tests/, the package smoke check and the benchmark's CPU-baseline leg may import this module.
It never touches the CUDA path.

The paper has no learned collide: its collide (Sec. 3) relaxes every site toward the Hermite
equilibrium. The learned form replaces that relaxation by a small network and keeps the plain
collide as judge and fallback. This module states the step in the order the method takes it,
in FP64 on numpy arrays, so that the CUDA path can be held to it population by population:

  1. walls and pull: the oracle's own wall halo write and propagate (Sec. 3: populations
     propagate, then collide);
  2. deviations d_i = f_i - w_i of the pulled populations (the FP32 storage form the learned
     step runs on);
  3. normalised network inputs x_i = (d_i - mu_x,i) / sd_x,i;
  4. network output y = MLP(x) (``oracle.mlp.forward``; with bf16=True it rounds to bfloat16 at
     the points where a tensor-core evaluation with BF16 operands must);
  5. candidate post-collision deviations d^_i = d_i + sd_t,i y_i + mu_t,i (the network predicts
     the normalised collision change post - pre);
  6. projection of d^ onto the moments the plain collide produces (``targets``): among all
     corrections that put mass, momentum and energy at those values, the one of least
     weighted norm sum_i delta_i^2 / w_i (``project``);
  7. the plain collide of the same pulled populations (``oracle.collide``);
  8. per tile of 32 x 32 sites, the residual max_i |f_learned - f_plain| / max |f_plain|
     (``tile_residual``); a tile keeps the learned result when residual <= bound and falls back
     to the plain result otherwise, a residual that is not a number included (``falls_back``).

Velocity orders: the oracle works in its own population order (``oracle.velocity_set``); the
network's 37 inputs and outputs follow the caller's order, given as (cx, cy) tables and matched by
velocity vector.
"""
from __future__ import annotations

import numpy as np

from . import mlp as _mlp
from . import oracle as _orc

TILE = 32


def _table():
    cx, cy, w, r = _orc.velocity_set()
    return cx.astype(np.float64), cy.astype(np.float64), w, r


def moment_matrix():
    """M (4 x 37, oracle order): rows 1, c_x, c_y, |c|^2 -- the conserved moments of a population
    vector in lattice units (mass; momentum and energy up to the factors r and r^2)."""
    cx, cy, _, _ = _table()
    return np.stack([np.ones_like(cx), cx, cy, cx * cx + cy * cy])


def targets(d, gx: float = 0.0, gy: float = 0.0):
    """Moments M d' that the plain collide gives the post-collision deviations of a site whose
    pulled deviations are d[..., 37] (Sec. 3 collide, gravity through the shifted equilibrium):

      sum d'         = sum d                                   (mass),
      r sum d' c     = r sum d c + rho g                       (momentum gains rho g),
      r^2 sum d'|c|^2 = r^2 sum d |c|^2 + rho (|u + g|^2 - |u|^2)  (kinetic energy of the shift;
                                                                the temperature is unchanged),

    with rho = sum f = 1 + sum d (the weights sum to 1 and have zero odd moments) and
    rho u = r sum d c. Returns [..., 4] in lattice units (rows of ``moment_matrix``)."""
    d = np.asarray(d, dtype=np.float64)
    _, _, _, r = _table()
    m = d @ moment_matrix().T
    rho = 1.0 + m[..., 0]
    ux = r * m[..., 1] / rho
    uy = r * m[..., 2] / rho
    out = m.copy()
    out[..., 1] += rho * gx / r
    out[..., 2] += rho * gy / r
    out[..., 3] += rho * (((ux + gx) ** 2 + (uy + gy) ** 2) - (ux * ux + uy * uy)) / (r * r)
    return out


def project(dhat, m_target):
    """Weighted least-norm projection of candidate deviations dhat[..., 37] onto the moments
    m_target[..., 4]: dhat + W M^T (M W M^T)^-1 (m_target - M dhat), W = diag(w) -- the correction
    of least sum_i delta_i^2 / w_i that reaches the targets, so each population moves in
    proportion to its weight."""
    dhat = np.asarray(dhat, dtype=np.float64)
    _, _, w, _ = _table()
    M = moment_matrix()
    A = (M * w) @ M.T                                   # M W M^T (4 x 4)
    resid = np.asarray(m_target, dtype=np.float64) - dhat @ M.T
    lam = np.linalg.solve(A, resid.reshape(-1, 4).T).T.reshape(resid.shape)
    return dhat + (lam @ M) * w


def normalise(d, norm):
    """Network inputs (d - mu_x) / sd_x; norm[4][37] = mu_x, sd_x, mu_t, sd_t (network order)."""
    norm = np.asarray(norm, dtype=np.float64)
    return (d - norm[0]) / norm[1]


def add_change(d, y, norm):
    """Candidate post-collision deviations d + sd_t y + mu_t (network order)."""
    norm = np.asarray(norm, dtype=np.float64)
    return d + y * norm[3] + norm[2]


def tile_residual(f_learned, f_plain):
    """max |f_learned - f_plain| / max |f_plain| over one tile (any shape; absolute populations).
    A tile whose plain populations are all zero divides by nothing: the residual is then the
    largest difference itself."""
    a = np.asarray(f_learned, dtype=np.float64)
    b = np.asarray(f_plain, dtype=np.float64)
    num = np.max(np.abs(a - b))
    den = np.max(np.abs(b))
    return num / den if den > 0 else num


def falls_back(residual: float, bound: float) -> bool:
    """A tile falls back to the plain collide unless its residual is at most the bound (a
    residual that is not a number falls back)."""
    return not (residual <= bound)


def pulled(f, T_top: float, T_bottom: float, y_periodic: bool = False, wall_mode: str = "rest"):
    """Walls then pull of site-major populations f[Ly, Lx, 37] (oracle order)."""
    Ly, Lx, _ = f.shape
    full = _orc.with_walls(f, T_top, T_bottom, wall_mode) if not y_periodic else np.concatenate(
        [np.zeros((3, Lx, 37)), f, np.zeros((3, Lx, 37))])
    return _orc.propagate(full, Lx, Ly, y_periodic)


def network_change(params, norm, order, bf16: bool = True):
    """A predictor y(d) of the normalised change: the network of packed parameters `params` and
    normalisation norm[4][37], both in the velocity order `order` = (cx, cy), applied to oracle-order
    deviations d[n, 37]; returns y in oracle order."""
    perm = _orc.order_map(*order)   # oracle index of the network's population j

    def predict(d):
        x = normalise(d[:, perm], norm)
        y, _ = _mlp.forward(np.asarray(params, dtype=np.float64), x, bf16=bf16)
        out = np.empty_like(y)
        out[:, perm] = y
        return out
    return predict


def learned_step(f, tau: float, predict, norm, order, bound: float, gx: float = 0.0, gy: float = 0.0,
                 T_top: float = 1.0, T_bottom: float = 1.0, y_periodic: bool = False, tile: int = TILE):
    """One learned time step of site-major populations f[Ly, Lx, 37] (oracle order).

    predict(d) maps oracle-order deviations d[n, 37] to the network's normalised output in oracle
    order (``network_change``); norm[4][37] is the network's normalisation in velocity order
    `order`. Lx and Ly are multiples of `tile`. Returns a dict with the new populations `f`, the
    learned candidate `f_learned` and the plain result `f_plain` (all [Ly, Lx, 37]), the tile
    residuals `residual` and decisions `fallback` ([Ly/tile, Lx/tile], row-major by tile row)."""
    f = np.asarray(f, dtype=np.float64)
    Ly, Lx, npop = f.shape
    assert npop == 37 and Lx % tile == 0 and Ly % tile == 0
    _, _, w, _ = _table()
    perm = _orc.order_map(*order)
    nrm = np.empty((4, 37))
    nrm[:, perm] = np.asarray(norm, dtype=np.float64)       # normalisation in oracle order
    fp = pulled(f, T_top, T_bottom, y_periodic)             # 1. walls and pull
    d = (fp - w).reshape(-1, 37)                            # 2. deviations
    y = predict(d)                                          # 3-4. normalised inputs, network
    dhat = add_change(d, y, nrm)                            # 5. candidate
    dl = project(dhat, targets(d, gx, gy))                  # 6. projection
    f_learned = (dl + w).reshape(Ly, Lx, 37)
    f_plain = _orc.collide(fp, tau, gx, gy)                 # 7. plain collide
    nty, ntx = Ly // tile, Lx // tile
    res = np.empty((nty, ntx))
    fall = np.empty((nty, ntx), bool)
    out = f_learned.copy()
    for ty in range(nty):                                   # 8. tile residual and fallback
        for tx in range(ntx):
            sl = (slice(ty * tile, (ty + 1) * tile), slice(tx * tile, (tx + 1) * tile))
            res[ty, tx] = tile_residual(f_learned[sl], f_plain[sl])
            fall[ty, tx] = falls_back(res[ty, tx], bound)
            if fall[ty, tx]:
                out[sl] = f_plain[sl]
    return {"f": out, "f_learned": f_learned, "f_plain": f_plain, "residual": res, "fallback": fall,
            "y": y.reshape(Ly, Lx, 37)}
