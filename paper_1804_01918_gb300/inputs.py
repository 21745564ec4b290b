"""Seeded synthetic inputs for the D2Q37 time step: Rayleigh-Taylor-shaped initial fields.

This module is the only code shared by the CUDA path and the oracle. It produces macroscopic
fields (density, velocity, temperature) on the host and holds none of the lattice-Boltzmann
arithmetic: no velocity set, no equilibrium, no collision. Both sides turn these fields into
populations with their own equilibrium.

The paper runs the D2Q37 code on Rayleigh-Taylor / convective-turbulence problems (Sec. 3) on
lattices of 1024x8192 to 4608x12288 sites (Table 1, Fig. 4 caption) but prints neither an
initial condition nor a dataset, so the recipe below is a stated reading:

* walls at the bottom (below row 0) and top (above row Ly-1), periodic in x;
* a heavy, cold fluid above a light, hot one: T_top = 2/(1+R), T_bottom = 2R/(1+R), where R is the
  temperature ratio, so the mean temperature is 1;
* the interface y_i(x) = Ly/2 + Ly * sum_{k=1..8} a_k cos(2 pi k x / Lx + phi_k), with a_k >= 0
  drawn from the seed and scaled so that sum a_k = amplitude, and phi_k uniform in [0, 2 pi);
* T(x, y) = 1 + (T_bottom - T_top)/2 * tanh((y_i(x) - y) / width), width = 2 sites;
* u = 0;
* rho(x, y) = exp(-g (y - y_i(x)) / T(x, y)) / T(x, y): locally isothermal hydrostatic balance
  with pressure p = rho T = 1 on the interface;
* gravity g = 0.1 * T_top / Ly pointing to -y (weak stratification, g Ly / T <= 0.1).

Random numbers come from numpy's PCG64 generator seeded with ``seed``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

N_MODES = 8


@dataclass(frozen=True)
class RTFields:
    """Initial macroscopic fields, each float64 C-contiguous with shape (Ly, Lx) (x fastest)."""

    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    T_top: float
    T_bottom: float
    gy: float  # gravity along y (negative: pointing down)


def wall_temperatures(R: float) -> tuple[float, float]:
    """(T_top, T_bottom) for temperature ratio R = T_bottom / T_top with mean temperature 1."""
    if not R > 0:
        raise ValueError("temperature ratio must be positive")
    return 2.0 / (1.0 + R), 2.0 * R / (1.0 + R)


def atwood_to_ratio(A: float) -> float:
    """Temperature ratio R = (1 + A) / (1 - A) for Atwood number A in (0, 1)."""
    if not 0.0 < A < 1.0:
        raise ValueError("Atwood number must lie in (0, 1)")
    return (1.0 + A) / (1.0 - A)


def rayleigh_taylor(Lx: int, Ly: int, R: float = 2.0, seed: int = 0,
                    amplitude: float = 1e-3, width: float = 2.0,
                    g_factor: float = 0.1) -> RTFields:
    """Seeded Rayleigh-Taylor initial fields on an Lx x Ly lattice (see module docstring)."""
    if Lx < 1 or Ly < 1:
        raise ValueError("lattice sizes must be positive")
    T_top, T_bottom = wall_temperatures(R)
    g = g_factor * T_top / Ly
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.random(N_MODES)
    a = a * (amplitude / a.sum())
    phi = rng.random(N_MODES) * (2.0 * np.pi)
    x = np.arange(Lx, dtype=np.float64)
    y = np.arange(Ly, dtype=np.float64)
    k = np.arange(1, N_MODES + 1, dtype=np.float64)
    yi = Ly / 2.0 + Ly * np.sum(a[:, None] * np.cos(2.0 * np.pi * k[:, None] * x[None, :] / Lx
                                                     + phi[:, None]), axis=0)
    T = 1.0 + 0.5 * (T_bottom - T_top) * np.tanh((yi[None, :] - y[:, None]) / width)
    rho = np.exp(-g * (y[:, None] - yi[None, :]) / T) / T
    zero = np.zeros((Ly, Lx), dtype=np.float64)
    return RTFields(rho=np.ascontiguousarray(rho), ux=zero.copy(), uy=zero.copy(),
                    T=np.ascontiguousarray(T), T_top=T_top, T_bottom=T_bottom, gy=-g)


def random_state(Lx: int, Ly: int, seed: int = 0, du: float = 0.05, dT: float = 0.2,
                 drho: float = 0.2) -> RTFields:
    """Seeded, spatially uncorrelated random fields (rho, u, T) for stress tests of the step.

    rho in [1 - drho, 1 + drho], each velocity component in [-du, du], T in [1 - dT, 1 + dT].
    Walls take temperatures 1 - dT/2 (top) and 1 + dT/2 (bottom); gravity is zero.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (Ly, Lx)
    rho = 1.0 + drho * (2.0 * rng.random(shape) - 1.0)
    ux = du * (2.0 * rng.random(shape) - 1.0)
    uy = du * (2.0 * rng.random(shape) - 1.0)
    T = 1.0 + dT * (2.0 * rng.random(shape) - 1.0)
    return RTFields(rho=rho, ux=ux, uy=uy, T=T, T_top=1.0 - dT / 2, T_bottom=1.0 + dT / 2, gy=0.0)


def tau_min_stable(A: float) -> float:
    """Smallest relaxation time drawn for a member of Atwood number A.

    The cold side of a member sits at T_top = 1 - A. The BGK D2Q37 step is linearly unstable far
    below the reference temperature at small tau: in a periodic box a 1e-3 perturbation of a
    uniform state grows to overflow at (T, tau) = (0.5, 0.6), (0.5, 0.65), (0.55, 0.6) and
    (0.6, 0.6), and decays at (0.5, 0.7), (0.55, 0.65), (0.6, 0.65) and at every T >= 0.65 for
    tau >= 0.6 (800 steps each on the oracle). This bound keeps a margin above that boundary:
    0.6 up to A = 0.3, then rising linearly to 0.75 at A = 0.5."""
    return 0.6 if A <= 0.3 else 0.6 + 0.75 * (A - 0.3)


def ensemble_members(n: int, seed: int = 0, lx_min: int = 128, lx_max: int = 1024,
                     lx_multiple: int = 32) -> list[dict]:
    """Seed-drawn descriptors of an ensemble of independent Rayleigh-Taylor lattices.

    Lx is uniform over the multiples of ``lx_multiple`` in [lx_min, lx_max], Ly = 4 Lx, the Atwood
    number is uniform in [0.05, 0.5] and the relaxation time uniform in [tau_min_stable(A), 1.2]
    (i.e. [0.6, 1.2] except where the member's cold side would make the step unstable). Each
    member also gets its own field seed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    choices = np.arange(lx_min, lx_max + 1, lx_multiple)
    out = []
    for m in range(n):
        Lx = int(choices[rng.integers(0, len(choices))])
        A = float(0.05 + 0.45 * rng.random())
        lo = tau_min_stable(A)
        tau = float(lo + (1.2 - lo) * rng.random())
        out.append({"Lx": Lx, "Ly": 4 * Lx, "atwood": A, "R": atwood_to_ratio(A), "tau": tau,
                    "seed": int(rng.integers(0, 2**31 - 1))})
    return out


def _splitmix64(state: int) -> tuple[int, int]:
    """One step of SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): (new state, output)."""
    mask = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & mask
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return state, z ^ (z >> 31)


def rayleigh_taylor_splitmix(Lx: int, Ly: int, R: float = 2.0, seed: int = 0) -> RTFields:
    """The Rayleigh-Taylor recipe above with its eight amplitudes and eight phases drawn, in that
    order, from SplitMix64 seeded with ``seed`` (u = (next >> 11) 2^-53) instead of PCG64: the
    generator the C library's lb_rt_fields / lb_init_rt implement from the same published
    definition. Arithmetic in the same order as there, so the two agree up to the last-place
    rounding of cos, tanh and exp."""
    if Lx < 1 or Ly < 1:
        raise ValueError("lattice sizes must be positive")
    T_top, T_bottom = wall_temperatures(R)
    g = 0.1 * T_top / Ly
    s = seed & ((1 << 64) - 1)
    a, phi = [], []
    total = 0.0
    for _ in range(N_MODES):
        s, z = _splitmix64(s)
        a.append((z >> 11) * 2.0**-53)
        total = total + a[-1]
    scale = 1e-3 / total
    a = [v * scale for v in a]
    two_pi = 6.283185307179586476925286766559
    for _ in range(N_MODES):
        s, z = _splitmix64(s)
        phi.append((z >> 11) * 2.0**-53 * two_pi)
    x = np.arange(Lx, dtype=np.float64)
    acc = np.zeros(Lx)
    for k in range(N_MODES):
        acc = acc + a[k] * np.cos(((two_pi * (k + 1)) * x) / Lx + phi[k])
    yi = Ly / 2.0 + Ly * acc
    y = np.arange(Ly, dtype=np.float64)[:, None]
    T = 1.0 + (0.5 * (T_bottom - T_top)) * np.tanh((yi[None, :] - y) / 2.0)
    rho = np.exp((-g * (y - yi[None, :])) / T) / T
    zero = np.zeros((Ly, Lx), dtype=np.float64)
    return RTFields(rho=np.ascontiguousarray(rho), ux=zero.copy(), uy=zero.copy(),
                    T=np.ascontiguousarray(T), T_top=T_top, T_bottom=T_bottom, gy=-g)


# ---- seeded network parameters for the learned collide's tests --------------------------------
# Packed like the library's network (W1[128][37] b1[128] W2[128][128] b2[128] W3[37][128] b3[37]);
# plain random numbers, no lattice-Boltzmann arithmetic.
MLP_SIZES = [(128, 37), (128,), (128, 128), (128,), (37, 128), (37,)]
MLP_FAN_IN = [37, 37, 128, 128, 128, 128]


def mlp_params(seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """float32 parameters, each uniform in +-scale / sqrt(fan_in) (PCG64 seeded with ``seed``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.uniform(-1.0, 1.0, shape) * (scale / np.sqrt(fan))
             for shape, fan in zip(MLP_SIZES, MLP_FAN_IN)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def mlp_norm(unit, seed: int = 0, mu_x: float = 0.02, sd_x: float = 0.05, mu_t: float = 1e-6,
             sd_t: float = 1e-5) -> np.ndarray:
    """float32 normalisation [4][37] (input mean and standard deviation, target mean and standard
    deviation), each entry the given level times unit[i] times a seeded factor in [0.5, 1.5);
    ``unit`` (37 values, in the network's population order) sets each population's scale."""
    rng = np.random.Generator(np.random.PCG64(seed))
    unit = np.asarray(unit, dtype=np.float64)
    levels = np.array([mu_x, sd_x, mu_t, sd_t])[:, None]
    return (levels * unit[None, :] * (0.5 + rng.random((4, 37)))).astype(np.float32)
