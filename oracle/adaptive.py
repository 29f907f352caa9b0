"""Adaptive time step (Sec. 4.7: the paper uses fixed steps and names CFL or
physics-based dynamic time stepping as the way to open its adjustable-accuracy
chemistry) -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Reading: before each step the step size is dt_max 2^-j with the smallest
j >= 0 for which it satisfies every active bound (and never below the
largest such power not under dt_min), from the field that pushes the
particles and the electron density of the last deposit:

* drift CFL: mu |E|max dt <= cfl h;
* diffusion: 2 D dt <= (cfl h)^2;
* dielectric relaxation (explicit coupling only): dt <= c_drt eps0 / sigma_max,
  sigma_max = q_e mu n_max (Eq. conductivity), n_max the largest CIC density;
* ionization (c_ion > 0): dt <= c_ion / k_ion(|E|max), k_ion = alpha(E) mu E,
  which grows with |E|.

Steps of a power-of-two fraction make the choice depend only on which side
of each bound the candidate falls, so two implementations whose fields agree
to rounding choose the same step (unless a bound sits within rounding of a
power of two).
"""
from __future__ import annotations

import math

import numpy as np

from .poisson import EPS0, Q_E


def field_max(E) -> float:
    """Largest |E| over the cells, |E| = sqrt((Ex^2 + Ey^2) + Ez^2)."""
    ex, ey, ez = (np.asarray(e, np.float64).ravel() for e in E)
    return float(np.max(np.sqrt((ex * ex + ey * ey) + ez * ez)))


def bounds(phys: dict, Emax: float, ne_max: int, cfl: float, c_drt: float, c_ion: float, explicit: bool) -> dict:
    """The active bounds on dt (inf where a bound does not apply)."""
    n = int(phys["n"])
    h = (phys["hi"][0] - phys["lo"][0]) / n
    mu, D = float(phys["mu"]), float(phys["D"])
    s = int(phys.get("frac_bits", 10))
    inf = math.inf
    out = {"drift": inf, "diffusion": inf, "relaxation": inf, "ionization": inf}
    if cfl > 0.0 and mu * Emax > 0.0:
        out["drift"] = cfl * h / (mu * Emax)
    if cfl > 0.0 and D > 0.0:
        out["diffusion"] = (cfl * h) * (cfl * h) / (2.0 * D)
    if explicit and c_drt > 0.0 and ne_max > 0:
        dV = (h * h) * h
        nmax = float(ne_max) * 2.0 ** (-3 * s) / dV
        out["relaxation"] = c_drt * EPS0 / (Q_E * mu * nmax)
    if c_ion > 0.0 and Emax > 0.0:
        k = float(phys["alpha_A"]) * math.exp(-float(phys["alpha_B"]) / Emax) * (mu * Emax)
        if k > 0.0:
            out["ionization"] = c_ion / k
    return out


def choose_dt(phys: dict, E, ne_fix, dt_max: float, dt_min: float, cfl: float, c_drt: float = 0.0,
              c_ion: float = 0.0, explicit: bool = True) -> float:
    """dt_max 2^-j, j the smallest with the candidate under every bound, no
    finer than the largest power of two fraction not under dt_min."""
    b = min(bounds(phys, field_max(E), int(np.max(ne_fix)) if np.size(ne_fix) else 0, cfl, c_drt, c_ion,
                   explicit).values())
    j = 0
    while j < 62 and math.ldexp(dt_max, -j) > b and math.ldexp(dt_max, -(j + 1)) >= dt_min:
        j += 1
    return math.ldexp(dt_max, -j)
