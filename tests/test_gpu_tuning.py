"""The autotuner (itokmc_autotune): it must pick a converging smoother pair
and a deposit window, leave the state as it found it (potential, field, the
last deposit), and later steps must still match a handle that never tuned,
up to the field tolerance."""
import numpy as np
import pytest

from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import gpu_handle, mixed_state, small_phys

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [itokmc.FP64, itokmc.MIXED])
def test_autotune_restores_state_and_keeps_results(precision):
    ph = small_phys(32, dt=5e-12, photon_ratio=0.06)
    st = mixed_state(ph, seed=51, peak=2e18)
    ions = synth.random_ions(ph, seed=52, mean=300)
    hs = []
    for _ in range(2):
        H = gpu_handle(ph, 8 * len(st["w"]) + 100000, seed0=5, precision=precision)
        H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
        H.itokmc_set_ions(*ions)
        H.itokmc_solve_field()
        hs.append(H)
    phi0 = hs[0].itokmc_read_densities(itokmc.PHI).copy()
    E0 = hs[0].itokmc_read_densities(itokmc.E).copy()
    t = hs[0].itokmc_autotune()
    assert 1 <= t["mg_nu1"] <= 3 and 1 <= t["mg_nu2"] <= 3
    assert len(t["tried"]) == 9 and t["ms_field"] > 0 and t["cycles"] >= 0
    assert any(ms >= 0 for _, ms in t["tried"])
    assert np.array_equal(hs[0].itokmc_read_densities(itokmc.PHI), phi0)
    assert np.array_equal(hs[0].itokmc_read_densities(itokmc.E), E0)
    # the deposit window: every candidate timed (the tuner checks that all
    # give the same densities), the chosen one among them, the last deposit
    # restored
    assert [w for w, _ in t["dep_tried"]] == [0, 256, 512, 1024, 2048]
    assert all(ms > 0 for _, ms in t["dep_tried"]) and t["dep_win"] in (0, 256, 512, 1024, 2048)
    for which in (itokmc.NE_FIX, itokmc.XE):
        assert np.array_equal(hs[0].itokmc_read_densities(which), hs[1].itokmc_read_densities(which))
    for H in hs:
        H.itokmc_step(2)
    # the particle path before the next solve is identical; the field differs
    # only within the solver tolerance
    a, b = (H.itokmc_read_densities(itokmc.E).ravel() for H in hs)
    assert np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(b))
    for H in hs:
        H.close()
