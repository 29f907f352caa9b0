"""Steps replayed from captured CUDA graphs (config.graph_step): one launch
per step, the particle count and step counter read on the device, the field
solved with a fixed cycle count and checked after the step.  Fed the same
field before every step, a graph-replayed run must equal the host-driven run
bit for bit (particles, densities, ion counts, firings) and its solved field
must agree within the field tolerance; ensemble members replayed in one
graph must equal the oracle's single runs.
"""
import numpy as np
import pytest

import oracle
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, mixed_state, oracle_state, small_phys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    itokmc.lib()


def _pair(ph, st, precision, species=None, R=1, real=None):
    out = []
    for graph in (0, 1):
        cfg = itokmc.make_config(ph, 4 * len(st["w"]) + 200000, seed0=9, precision=precision, realizations=R,
                                 graph_step=graph)
        H = itokmc.Handle(cfg)
        if species is None:
            H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"], real)
        else:
            H.itokmc_set_particles_species(st["x"], st["y"], st["z"], st["w"], species, real)
        H.itokmc_solve_field()
        out.append(H)
    return out


@pytest.mark.parametrize("case", ["fp64", "mixed", "mobile"])
def test_graph_steps_equal_host_steps(case):
    """Six steps with the field given before each: after the first
    (host-driven) step the graph handle replays every step (several cached
    graphs: the swapped buffers cycle); particles, X_e, ion counts and
    firings equal the host-driven handle's bit for bit, the solved field
    within 1e-5."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    species = None
    if case == "mobile":
        ph = synth.with_mobile_ions(ph, mu_ion=2e-2)
        ph["mobile_ions"] = True
        e = mixed_state(ph, seed=3, peak=5e18, n_random=500)
        ions = synth.ion_particles(ph, seed=4, mean=3000, frac=0.3)
        st = {k: np.concatenate([e[k], e[k], ions[k]]) for k in ("x", "y", "z", "w")}
        species = np.concatenate([np.zeros(len(e["w"]), np.int32), np.ones(len(e["w"]), np.int32),
                                  np.full(len(ions["w"]), 2, np.int32)])
    else:
        st = mixed_state(ph, seed=3, peak=5e18, n_random=500)
    prec = itokmc.MIXED if case == "mixed" else itokmc.FP64
    A, B = _pair(ph, st, prec, species)
    for k in range(6):
        E = synth.random_field(ph, seed=20 + k, amp=2e6, base=4e6)
        for H in (A, B):
            H.itokmc_set_field(*E)
            H.itokmc_step(1)
        ga, gb = A.itokmc_read_particles(), B.itokmc_read_particles()
        assert_particles_equal(gb, ga)
        for f in ("cell", "species"):
            assert np.array_equal(ga[f], gb[f])
        for which in (itokmc.XE, itokmc.NPOS, itokmc.NNEG, itokmc.FIRINGS):
            assert np.array_equal(A.itokmc_read_densities(which), B.itokmc_read_densities(which))
        Ea, Eb = A.itokmc_read_densities(itokmc.E), B.itokmc_read_densities(itokmc.E)
        assert np.max(np.abs(Ea - Eb)) <= 1e-5 * np.max(np.abs(Ea))
    assert A.itokmc_get_stats()["graph_steps"] == 0
    assert B.itokmc_get_stats()["graph_steps"] == 5
    A.close()
    B.close()


def test_graph_ensemble_members_equal_single_runs():
    """R = 3 realizations with uneven particle counts replayed from graphs:
    member r equals the oracle's single run with key seed0 + r, step by
    step, for four steps with the field given before each."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    R, seed0 = 3, 40
    states = [mixed_state(ph, seed=50 + r, peak=10 ** (18 + r * 0.5), n_random=200 * (r + 1)) for r in range(R)]
    E = synth.random_field(ph, seed=2, amp=2e6, base=4e6)
    cat = {k: np.concatenate([s[k] for s in states]) for k in ("x", "y", "z", "w")}
    real = np.concatenate([np.full(len(s["w"]), r, np.int32) for r, s in enumerate(states)])
    H = itokmc.Handle(itokmc.make_config(ph, 400000, seed0=seed0, realizations=R, graph_step=1))
    H.itokmc_set_particles(cat["x"], cat["y"], cat["z"], cat["w"], real)
    H.itokmc_solve_field()
    S = [oracle_state(ph, states[r], seed0 + r) for r in range(R)]
    for k in range(4):
        H.itokmc_set_field(*[np.tile(np.ravel(e), R) for e in E])
        H.itokmc_step(1)
        G = H.itokmc_read_particles()
        for r in range(R):
            S[r], _ = oracle.step(oracle.make_params(ph, seed=seed0 + r, step=k), S[r], E)
            sel = G["realization"] == r
            assert_particles_equal({f: v[sel] for f, v in G.items()}, S[r])
    assert H.itokmc_get_stats()["graph_steps"] == 3
    H.close()


def test_graph_not_used_with_an_adaptive_step():
    """The adaptive step size changes the kernels' constants every step: such
    runs stay host-driven."""
    ph = small_phys(16, dt=5e-12)
    st = mixed_state(ph, seed=3, n_random=500)
    H = itokmc.Handle(itokmc.make_config(ph, 200000, seed0=1, graph_step=1, dt_adapt=1, dt_min=1e-14, cfl=0.5))
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_solve_field()
    H.itokmc_step(4)
    assert H.itokmc_get_stats()["graph_steps"] == 0
    H.close()
