"""The adaptive step size on the GPU against the oracle's controller (reading
of Sec. 4.7's dynamic time stepping): whole explicit steps fed the oracle's
field each step, the same power-of-two step sizes chosen from the same field
and the same last deposit, and the particles and ion counts bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import adaptive, poisson
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, mixed_state, oracle_state, small_phys

pytestmark = pytest.mark.gpu


def test_adaptive_steps_match_oracle_chain():
    ph = small_phys(16, dt=1e-10, photon_ratio=0.06)
    st = mixed_state(ph, seed=91, peak=8e18, n_random=500)
    rnd = synth.random_ions(ph, seed=92)
    ions = (rnd[0] + synth.cell_counts(ph, st).astype(np.int64) // 2, rnd[1])
    seed0 = 17
    knobs = dict(dt_min=1e-14, cfl=0.5, drt_factor=0.1, ion_factor=0.02)
    cfg = itokmc.make_config(ph, 400000, seed0=seed0, dt_adapt=1, **knobs)
    H = itokmc.Handle(cfg)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_ions(*ions)
    H.itokmc_solve_field()
    S = oracle_state(ph, st, seed0, *ions)
    p0 = oracle.make_params(ph, seed=seed0)
    ne, _ = oracle.deposit(p0, S["x"], S["y"], S["z"], S["w"], S["cell"])
    _, E = poisson.solve(oracle.rho_fixed(p0, ne, S["Npos"], S["Nneg"]), ph)
    dts = []
    for k in range(4):
        dt = adaptive.choose_dt(ph, E, ne, 1e-10, knobs["dt_min"], knobs["cfl"], knobs["drt_factor"],
                                knobs["ion_factor"], explicit=True)
        dts.append(dt)
        H.itokmc_set_field(*E)
        H.itokmc_step(1)
        assert H.itokmc_get_stats()["dt_last"] == dt
        S, info = oracle.step(oracle.make_params(dict(ph, dt=dt), seed=seed0, step=k), S, E)
        assert_particles_equal(H.itokmc_read_particles(), S)
        assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), S["Npos"])
        ne = info["ne_fix"]
        _, E = poisson.solve(info["rho_fixed"], ph)
    # the controller acted: steps below dt_max
    assert max(dts) < 1e-10
    H.close()


def test_fixed_step_reported():
    ph = small_phys(16, dt=3e-12)
    H = itokmc.Handle(itokmc.make_config(ph, 1000, seed0=1))
    assert H.itokmc_get_stats()["dt_last"] == 3e-12
    H.close()
