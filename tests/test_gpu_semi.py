"""The semi-implicit coupling on the GPU (Sec. 4.3, Sec. 4.7) through the C ABI.

Whole steps of the step mode ITOKMC_SEMI_IMPLICIT against the oracle's
semi-implicit step: each step the GPU's field (its variable-coefficient
multigrid) must be within the field tolerance of the oracle's direct sparse
solve, and the oracle's step fed with the GPU's field must give the GPU's
particles, ion counts and firings bit for bit (the field is the only
quantity the two sides compute differently).  A high-contrast case
(sigma dt / eps0 above 20, the regime the scheme exists for) checks the
coarsening of the coefficients and the cycle count."""
import numpy as np
import pytest

import oracle
from oracle import semi_implicit as si
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, mixed_state, oracle_state, small_phys

pytestmark = pytest.mark.gpu

E_TOL = 1e-5


def _semi_handle(ph, st, ions, seed0, cap):
    cfg = itokmc.make_config(ph, cap, seed0=seed0, coupling=itokmc.SEMI_IMPLICIT)
    H = itokmc.Handle(cfg)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    if ions is not None:
        H.itokmc_set_ions(*ions)
    H.itokmc_solve_field()
    return H


def _neutral_ions(ph, st, seed):
    """Quasi-neutral start: a positive ion for every electron of a cell (NGP),
    plus random background counts, so that the space-charge field stays
    moderate (an electrons-only seed of 1e19 m^-3 makes fields near 1e8 V/m
    whose avalanche overflows 32-bit weights within a step)."""
    rnd = synth.random_ions(ph, seed=seed)
    return rnd[0] + synth.cell_counts(ph, st).astype(np.int64), rnd[1]


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_semi_implicit_steps_against_oracle_chain():
    ph = small_phys(16, dt=1e-11, photon_ratio=0.06)
    st = mixed_state(ph, seed=71, peak=1e19, n_random=800)
    ions = _neutral_ions(ph, st, 72)
    seed0 = 13
    H = _semi_handle(ph, st, ions, seed0, 400000)
    S = oracle_state(ph, st, seed0, *ions)
    for k in range(3):
        p = oracle.make_params(ph, seed=seed0, step=k)
        exact = si.transport(p, ph, S)["E"]
        H.itokmc_step(1)
        Eg = H.itokmc_read_densities(itokmc.E).reshape(3, -1)
        assert _maxrel(Eg, np.stack([e.ravel() for e in exact])) <= E_TOL
        S, info = si.step(p, ph, S, E=tuple(Eg))
        assert_particles_equal(H.itokmc_read_particles(), S)
        assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), S["Npos"])
        assert np.array_equal(H.itokmc_read_densities(itokmc.NNEG), S["Nneg"])
        f = H.itokmc_read_densities(itokmc.FIRINGS)
        assert np.array_equal(f[0], info["n_ion"]) and np.array_equal(f[1], info["n_att"])
        assert H.itokmc_get_stats()["mg_rel_residual"] <= 1e-10
    H.close()


def test_semi_implicit_high_contrast_field():
    """sigma dt / eps0 > 20 in the blob: the field within tolerance of the
    direct solve and convergence well inside mg_max_cycles."""
    ph = small_phys(32, dt=7e-10)
    st = mixed_state(ph, seed=81, peak=2e20, sigma=1.2e-3, n_random=300)
    ions = _neutral_ions(ph, st, 82)
    seed0 = 4
    H = _semi_handle(ph, st, ions, seed0, 4 * len(st["w"]) + 100000)
    S = oracle_state(ph, st, seed0, *ions)
    p = oracle.make_params(ph, seed=seed0, step=0)
    ref = si.transport(p, ph, S)
    cmax = float(np.max(si.coefficient(ref["sigma"], ph["dt"])))
    assert cmax > 20.0, cmax
    cycles, rel = H.itokmc_transport_semi_implicit()
    assert rel <= 1e-10 and 0 < cycles < 40, (cycles, rel)
    Eg = H.itokmc_read_densities(itokmc.E).reshape(3, -1)
    assert _maxrel(Eg, np.stack([e.ravel() for e in ref["E"]])) <= E_TOL
    H.close()


def test_semi_implicit_steps_deterministic():
    ph = small_phys(16, dt=1e-11, photon_ratio=0.06)
    st = mixed_state(ph, seed=75, peak=1e19, n_random=500)
    ions = _neutral_ions(ph, st, 76)
    out = []
    for _ in range(2):
        H = _semi_handle(ph, st, ions, 3, 300000)
        H.itokmc_step(3)
        out.append((H.itokmc_read_particles(), H.itokmc_read_densities(itokmc.PHI)))
        H.close()
    assert_particles_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
