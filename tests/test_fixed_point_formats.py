"""The number formats of the FP64 step's fixed-point pair terms (csrc/step_fp64.cu, namespace fxp),
checked on the host by evaluating the kernel's integer arithmetic exactly with Python integers:

* over the whole domain (|u*| components <= FX_UMAX, |T* - 1| / 2 <= FX_HB, density factor in
  [1, 2)) no intermediate leaves the 2^62 range the formats promise;
* in the Rayleigh-Taylor and strong-flow regimes the fixed-point G = WA0 + b^2 e2 +- b q (the
  shell coefficients themselves integer products of the host's rounded constants and the site
  terms), against exact rational arithmetic on the same FP64 constants and site terms, is as
  accurate as the FP64 evaluation of the same expression (the formats were chosen so).

The per-shell scales are read from the kernel header; weights and the thermal scale come from the
oracle's velocity set. Relaxation terms follow step_fp64.cu (relax_site_terms, shell_relax,
pair_base, relax_pair_fx).
"""
import os
import random
import re
import struct
from fractions import Fraction as Fr

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1804_01918_gb300", "csrc")
LAM = 0.25
KAPPA = [1, 1, 1, 2, 1, 2, 3, 1]
C2 = [0, 1, 2, 4, 5, 8, 9, 10]
# populations 1..18 of the library's table: (c_x, c_y, shell)
PAIRS = [(1, 0, 1), (0, 1, 1), (1, 1, 2), (1, -1, 2), (2, 0, 3), (0, 2, 3), (2, 1, 4), (2, -1, 4), (1, 2, 4),
         (1, -2, 4), (2, 2, 5), (2, -2, 5), (3, 0, 6), (0, 3, 6), (3, 1, 7), (3, -1, 7), (1, 3, 7), (1, -3, 7)]


def kernel_tables():
    hdr = open(os.path.join(CSRC, "d2q37_gpu.cuh")).read()
    def table(name):
        m = re.search(name + r"\(int s\) \{\s*constexpr int t\[NSHELL\] = \{([^}]*)\}", hdr)
        return [int(v) for v in m.group(1).split(",")]
    umax = float(re.search(r"FX_UMAX = ([0-9.]+);", hdr).group(1))
    hb = float(re.search(r"FX_HB = ([0-9.]+);", hdr).group(1))
    return table("fx_coarse_unit"), table("fx_fine_unit"), umax, hb


@pytest.fixture(scope="module")
def model(orc):
    cx, cy, w, r = orc.velocity_set()
    ws = {}
    for i in range(37):
        ws.setdefault(int(cx[i] ** 2 + cy[i] ** 2), w[i])
    return [ws[c] for c in C2], r


def bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def to_fixed(v, s):
    b = bits(v)
    e = (b >> 52) & 0x7FF
    m = (b & ((1 << 52) - 1)) | ((1 << 52) if e else 0)
    sh = e - 1075 + s
    v_int = (m << min(sh, 63)) if sh >= 0 else (m >> min(-sh, 63))
    return -v_int if b >> 63 else v_int


def from_fixed(g, s):
    """The kernel's rounding of g 2^-s to FP64: to nearest, ties away from zero."""
    if g == 0:
        return 0.0
    u = abs(g)
    z = 64 - u.bit_length()
    sig = ((((u << z) & ((1 << 64) - 1)) >> 10) + 1) >> 1
    val = sig * 2.0 ** (63 - z - s - 52)     # exact: sig has at most 54 bits, a power-of-two scale
    return -val if g < 0 else val


def test_from_fixed_rounds_to_nearest():
    """Against Python's correctly rounded int / float: equal except at exact ties, and never more
    than half an ulp away."""
    rng = random.Random(3)
    for _ in range(20000):
        g, s = rng.randint(-2 ** 62, 2 ** 62), rng.randint(40, 70)
        exact = Fr(g, 2 ** s)
        got = from_fixed(g, s)
        assert abs(Fr(got) - exact) <= Fr(abs(got)) * Fr(1, 2 ** 53)


class Overflow(AssertionError):
    pass


def fits(v):
    if not -2 ** 62 <= v < 2 ** 62:
        raise Overflow(v)
    return v


def site(ux, uy, h, rwm, r):
    U1, V1 = LAM * r * ux, LAM * r * uy
    m = 0.5 - (U1 * U1 + V1 * V1) / (4 * LAM * LAM * r * r)
    t = rwm * h
    bq = m - 2 * h
    Rb = rwm * bq
    P1, P2 = t * bq, t * h
    R0h = -2 * P2 + Rb * bq + rwm * 0.25 + t
    return U1, V1, t, Rb, P1, P2, R0h


def shell(S, w, r, rwm, t, Rb, P1, P2, R0h):
    k, X, ww = KAPPA[S], r * r * C2[S], w[S]
    WA0 = 0.5 * ww * X * X * P2 + 2 * ww * X * P1 + 2 * ww * R0h
    WB1 = 4 * k * ww * X * t + 8 * k * ww * Rb
    DA = -16 * k * k * ww * t + k * WB1
    CO = 32 * k ** 3 * ww / 3 * rwm
    return WA0, WB1, DA, CO


def pair_b(cx, cy, U, V):
    if cy == 0:
        return U
    if cx == 0:
        return V
    if cx == cy:
        return U + V
    if cx == -cy:
        return U - V
    if cx == 1:
        return U + cy * V
    return cx * U + (V if cy > 0 else -V)


def shell_constants(S, w, r):
    """shell_relax's FP64 constants q_a2, q_a1, q_a0, q_b1, q_b0, q_e0, q_co of shell S."""
    k, X, ww = KAPPA[S], r * r * C2[S], w[S]
    return (0.5 * ww * X * X, 2 * ww * X, 2 * ww, 4 * k * ww * X, 8 * k * ww, 16 * k * k * ww,
            32 * k ** 3 * ww / 3)


def fixed_G(coarse, fine, S, site_terms, w, r, U, V, cx, cy, rwm):
    """The kernel's integer arithmetic of one pair: (G(+c), G(-c)) as integers in the fine unit.
    WA0 is the FP64 evaluation rounded to the fine unit; k WB1, DA and k^3 C are high words of
    products of the host's rounded constants (d2q37_gpu.cuh, ShellFx) with the site terms."""
    t, Rb, P1, P2, R0h = site_terms
    sc, sf = coarse[S], fine[S]
    d, k = sf - sc, KAPPA[S]
    qa2, qa1, qa0, qb1, qb0, qe0, qco = shell_constants(S, w, r)
    c = [None, None, None, round(qb1 * 2.0 ** sc), round(qb0 * 2.0 ** (sc + 2)), round(qe0 * 2.0 ** sc),
         round(qco * 2.0 ** (sc + 2))]
    for v in c[3:]:
        fits(v)
    T, RB = to_fixed(t, 64), to_fixed(Rb, 62)
    mq = to_fixed(rwm, 62)
    WA0 = qa2 * P2 + (qa1 * P1 + qa0 * R0h)     # the kernel's FP64 WA0 (fma order; rounding aside)
    xa0 = fits(to_fixed(WA0, sf))
    xb1 = fits(((c[3] * T) >> 64) + ((c[4] * RB) >> 64))
    xda = fits(k * xb1 - ((c[5] * T) >> 64))
    xco = fits((c[6] * mq) >> 64)
    b = fits(pair_b(cx, cy, U, V))
    b2 = fits((b * b) >> 64)
    q = fits(xb1 + ((xco * b2) >> 64))
    e2 = fits(k * q + xda)
    we = fits(xa0 + fits((b2 * e2) >> (64 - d)))
    bq = fits((b * q) >> (64 - d))
    return fits(we + bq), fits(we - bq)


def test_no_intermediate_leaves_the_formats_over_the_domain(model):
    w, r = model
    coarse, fine, umax, hb = kernel_tables()
    g = np.linspace(-1.0, 1.0, 9)
    for ux in g * umax:
        for uy in g * umax:
            for h in g * hb:
                for rwm in (1.0, 1.999999):
                    U1, V1, t, Rb, P1, P2, R0h = site(ux, uy, h, rwm, r)
                    U, V = fits(to_fixed(U1, 64)), fits(to_fixed(V1, 64))
                    for cx, cy, S in PAIRS:
                        fixed_G(coarse, fine, S, (t, Rb, P1, P2, R0h), w, r, U, V, cx, cy, rwm)


@pytest.mark.parametrize("urange,Trange", [(0.05, (0.67, 1.33)), (0.16, (0.8, 1.2))])
def test_fixed_point_G_as_accurate_as_fp64(model, urange, Trange):
    w, r = model
    coarse, fine, _, _ = kernel_tables()
    rng = random.Random(5)
    worst_fx = worst_fp = 0.0
    for _ in range(300):
        ux, uy = rng.uniform(-urange, urange), rng.uniform(-urange, urange)
        h, rwm = (rng.uniform(*Trange) - 1.0) / 2.0, rng.uniform(1.0, 2.0)
        U1, V1, t, Rb, P1, P2, R0h = site(ux, uy, h, rwm, r)
        U, V = to_fixed(U1, 64), to_fixed(V1, 64)
        for cx, cy, S in PAIRS:
            WA0, WB1, DA, CO = shell(S, w, r, rwm, t, Rb, P1, P2, R0h)     # the FP64 evaluation
            k = KAPPA[S]
            qa2, qa1, qa0, qb1, qb0, qe0, qco = (Fr(v) for v in shell_constants(S, w, r))
            # exact: the same constants and FP64 site terms in rational arithmetic
            ta, Rba, P1a, P2a, R0a = Fr(t), Fr(Rb), Fr(P1), Fr(P2), Fr(R0h)
            WB1x = qb1 * ta + qb0 * Rba
            WA0x = Fr(qa2 * P2 + (qa1 * P1 + qa0 * R0h))      # the FP64 WA0 that both paths use
            DAx = k * WB1x - qe0 * ta
            COx = qco * Fr(rwm)
            bx = Fr(pair_b(cx, cy, Fr(U1), Fr(V1)))
            qx = WB1x + COx * bx * bx
            wex = WA0x + bx * bx * (k * qx + DAx)
            bf = pair_b(cx, cy, U1, V1)
            qf = WB1 + CO * bf * bf
            wef = WA0 + bf * bf * (k * qf + DA)
            Gp, Gm = fixed_G(coarse, fine, S, (t, Rb, P1, P2, R0h), w, r, U, V, cx, cy, rwm)
            for sgn, gfx in ((1, Gp), (-1, Gm)):
                exact = wex + sgn * bx * qx
                worst_fx = max(worst_fx, abs(from_fixed(gfx, fine[S]) - float(exact)) / abs(float(exact)))
                worst_fp = max(worst_fp, abs((wef + sgn * bf * qf) - float(exact)) / abs(float(exact)))
    print(f"|u| <= {urange}, T in {Trange}: fixed point {worst_fx:.2e}, FP64 {worst_fp:.2e}")
    assert worst_fx <= max(worst_fp, 2.3e-16)
