"""Pins of the oracle's adaptive step size (reading of Sec. 4.7's dynamic
time stepping): the chosen step satisfies every bound and is the largest
power-of-two fraction of dt_max that does (or the floor dt_min), its drift
over one step stays within cfl cells for a field known in closed form, and
finer steps follow stronger fields and denser plasma."""
import math

import numpy as np

from oracle import adaptive
from paper_2307_01797_gb300 import synth


def _uniform_E(ph, Ez):
    n = ph["n"]
    z = np.zeros((n, n, n))
    return (z, z, np.full((n, n, n), -Ez))


def test_drift_cfl_is_satisfied_and_tight():
    ph = synth.physics_small(32)
    h = (ph["hi"][0] - ph["lo"][0]) / ph["n"]
    for Ez in (1e5, 1.5e6, 7.3e6, 3e8):
        E = _uniform_E(ph, Ez)
        dt = adaptive.choose_dt(ph, E, np.zeros(ph["n"] ** 3, np.int64), dt_max=1e-9, dt_min=1e-16, cfl=0.5)
        drift = ph["mu"] * Ez * dt
        assert drift <= 0.5 * h
        assert dt == 1e-9 or ph["mu"] * Ez * 2 * dt > 0.5 * h or 2 * 0.1 * 2 * dt > (0.5 * h) ** 2
        assert math.log2(1e-9 / dt) == int(math.log2(1e-9 / dt))


def test_relaxation_bound_only_for_explicit_coupling():
    ph = synth.physics_small(16)
    E = _uniform_E(ph, 1e5)
    h = (ph["hi"][0] - ph["lo"][0]) / ph["n"]
    ne = np.zeros(16 ** 3, np.int64)
    N = int(1e19 * h ** 3)
    ne[7] = N << 30                           # about 1e19 m^-3 in one cell (fixed point, s = 10)
    sig = 1.602176634e-19 * ph["mu"] * (N / h ** 3)
    tau = 8.8541878128e-12 / sig              # dielectric relaxation time, ~2.6e-10 s
    dt_e = adaptive.choose_dt(ph, E, ne, 1e-9, 1e-16, cfl=0.5, c_drt=1.0, explicit=True)
    dt_s = adaptive.choose_dt(ph, E, ne, 1e-9, 1e-16, cfl=0.5, c_drt=1.0, explicit=False)
    assert dt_e <= tau * 1.0001 < 2 * dt_e
    assert dt_s > dt_e


def test_ionization_bound_and_monotone_in_field():
    ph = synth.physics_small(16)
    ne = np.zeros(16 ** 3, np.int64)
    prev = math.inf
    for Ez in (3e6, 5e6, 1e7, 3e7):
        dt = adaptive.choose_dt(ph, _uniform_E(ph, Ez), ne, 1e-9, 1e-16, cfl=10.0, c_ion=0.2)
        k = ph["alpha_A"] * math.exp(-ph["alpha_B"] / Ez) * ph["mu"] * Ez
        assert k * dt <= 0.2
        assert dt <= prev
        prev = dt


def test_floor_at_dt_min():
    ph = synth.physics_small(16)
    dt = adaptive.choose_dt(ph, _uniform_E(ph, 1e12), np.zeros(16 ** 3, np.int64), 1e-9, 1e-12, cfl=0.5)
    assert 1e-12 <= dt < 2e-12 and math.log2(1e-9 / dt) == int(math.log2(1e-9 / dt))
