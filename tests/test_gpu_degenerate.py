"""GPU parity on the degenerate and extreme inputs of the method, bit for bit
against the FP64 oracle through the C ABI:

* the largest weight a particle holds (2^32 - 1) alone in a cell: split
  hierarchically into ppc particles (Sec. 4.6), node weights beyond 32 bits
  in the merge's sort, the KMC on 4e9 electrons in a cell (Poisson means
  far beyond 10: the PTRS path), its CIC density just inside the int64
  fixed-point range (2^62 in units of 2^-3s); two such particles in one
  cell leave that range and are reported as ERR_OVERFLOW;
* a cell holding 5000 particles (the merge's global work area, far beyond
  the shared-memory tiers);
* particles exactly on cell faces and on the lower walls of the box, and
  particles of weight 1 (nodes of weight 1 are never split);
* an ensemble with an empty member beside two populated ones (Sec. 4:
  independent realizations; the empty one stays empty and its field is
  the applied one).
"""
import numpy as np
import pytest

import oracle
from oracle import poisson
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, mixed_state, oracle_state, small_phys

pytestmark = pytest.mark.gpu

WMAX = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    itokmc.lib()


def _extreme_state(ph, seed):
    rng = np.random.default_rng(seed)
    n = ph["n"]
    lo = ph["lo"][0]
    h = (ph["hi"][0] - lo) / n
    cols = {k: [] for k in ("x", "y", "z", "w")}

    def add(cell, m, w, frac=None):
        if frac is None:
            frac = rng.uniform(0.02, 0.98, (3, m))
        for a, key in enumerate(("x", "y", "z")):
            cols[key].append(lo + (cell[a] + frac[a]) * h)
        cols["w"].append(np.broadcast_to(np.asarray(w, np.uint32), (m,)).copy())

    add((1, 1, 5), 1, WMAX)                                   # one maximal particle
    add((5, 2, 5), 5, 800_000_000)                            # five heavy ones
    add((3, 5, 4), 5000, rng.integers(1, 1 << 20, 5000))      # the global merge tier
    add((6, 6, 2), 40, 1)                                     # weight 1 only
    # exactly on faces: offsets 0 in one, two or three axes
    fr = rng.uniform(0.1, 0.9, (3, 24))
    fr[0, :8] = 0.0
    fr[1, 8:16] = 0.0
    fr[:, 16:] = 0.0
    add((2, 3, 3), 24, rng.integers(1, 100, 24), frac=fr)
    # on the lower walls of the box (x = lo, y = lo, z = lo)
    fw = rng.uniform(0.1, 0.9, (3, 12))
    fw[0, :4] = 0.0
    fw[1, 4:8] = 0.0
    fw[2, 8:] = 0.0
    cw = [(0, 4, 4)] * 4 + [(4, 0, 4)] * 4 + [(4, 4, 0)] * 4
    for i in range(12):
        add(cw[i], 1, rng.integers(1, 1000), frac=fw[:, i:i + 1])
    return {k: np.concatenate(v) for k, v in cols.items()}


def test_extreme_weights_long_lists_and_faces_bit_exact():
    ph = small_phys(8, dt=1e-13, ppc=32, photon_ratio=0.06)
    st = _extreme_state(ph, seed=5)
    E = synth.random_field(ph, seed=3, amp=2e6, base=4.5e6)
    seed0, step = 3, 2
    S = oracle_state(ph, st, seed0)
    p = oracle.make_params(ph, seed=seed0, step=step)
    new, info = oracle.step(p, S, E)
    # the extremes are reached: Poisson means in the PTRS range (the
    # ionizations of the maximal cells), node weights beyond 2^32, the
    # 5000-element list
    assert info["n_ion"].max() > 10_000
    H = itokmc.Handle(itokmc.make_config(ph, 100_000, seed0=seed0))
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_field(*E)
    for _ in range(step):
        H.itokmc_advance_counter()
    G0 = H.itokmc_read_particles()
    assert np.array_equal(G0["cell"], S["cell"]) and np.array_equal(G0["w"], S["w"])
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    assert_particles_equal(H.itokmc_read_particles(), info["sorted"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NE_FIX), info["ne_fix"])
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    for r, key in enumerate(("n_ion", "n_att", "n_ph")):
        assert np.array_equal(F[r], info[key]), key
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    G = H.itokmc_read_particles()
    assert_particles_equal(G, new)
    assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), new["Npos"])
    s = H.itokmc_get_stats()
    assert s["merge_max_list"] >= 5000
    # a maximal particle alone in its cell became ppc particles whose weights
    # differ by at most one (Sec. 4.6)
    c0 = int(G0["cell"][np.nonzero(G0["w"] == WMAX)[0][0]])
    w0 = G["w"][G["cell"] == c0].astype(np.int64)
    if len(w0) == ph["ppc"]:
        assert w0.max() - w0.min() <= 1
    H.close()


def test_density_beyond_fixed_point_range_is_reported():
    """Two particles of weight 2^32 - 1 in one cell put 2^63 - 2^31 units of
    2^-30 electrons on a node, beyond the 2^62 the space charge admits: the
    transport stage reports ERR_OVERFLOW instead of a wrapped density."""
    ph = small_phys(8, dt=1e-13)
    L, h = ph["hi"][0], (ph["hi"][0] - ph["lo"][0]) / 8
    c = ph["lo"][0] + 4.5 * h
    H = itokmc.Handle(itokmc.make_config(ph, 1000, seed0=1))
    H.itokmc_set_particles(np.array([c, c]), np.array([c, c]), np.array([c, c]), np.array([WMAX, WMAX], np.uint32))
    H.itokmc_set_field(*synth.uniform_field(ph, -1.0e6))
    with pytest.raises(itokmc.ItokmcError) as e:
        H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    assert e.value.code == -5
    H.close()


def test_ensemble_with_an_empty_member():
    """R = 3 with member 1 empty: members 0 and 2 equal the oracle's single
    runs step by step, member 1 stays empty with zero densities and the
    applied field."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    R, seed0 = 3, 60
    states = [mixed_state(ph, seed=70 + r, peak=3e18, n_random=300) for r in (0, 2)]
    cat = {k: np.concatenate([states[0][k], states[1][k]]) for k in ("x", "y", "z", "w")}
    real = np.concatenate([np.zeros(len(states[0]["w"]), np.int32), np.full(len(states[1]["w"]), 2, np.int32)])
    H = itokmc.Handle(itokmc.make_config(ph, 400_000, seed0=seed0, realizations=R))
    H.itokmc_set_particles(cat["x"], cat["y"], cat["z"], cat["w"], real)
    E = synth.random_field(ph, seed=4, amp=2e6, base=4e6)
    H.itokmc_set_field(*[np.tile(np.ravel(e), R) for e in E])
    S = {r: oracle_state(ph, states[i], seed0 + r) for i, r in enumerate((0, 2))}
    n3 = ph["n"] ** 3
    for k in range(3):
        H.itokmc_step(1)
        G = H.itokmc_read_particles()
        assert not np.any(G["realization"] == 1)
        for r in (0, 2):
            S[r], _ = oracle.step(oracle.make_params(ph, seed=seed0 + r, step=k), S[r], E)
            sel = G["realization"] == r
            assert_particles_equal({f: v[sel] for f, v in G.items()}, S[r])
        for which in (itokmc.NE_FIX, itokmc.XE, itokmc.FIRINGS):
            assert not np.any(H.itokmc_read_densities(which, realization=1))
        # the empty member's own solve: no charge, the applied field alone
        phi_o, E_o = poisson.solve(np.zeros(n3, np.int64), ph)
        E1 = H.itokmc_read_densities(itokmc.E, realization=1)
        assert np.max(np.abs(E1[2] - E_o[2].ravel())) <= 1e-5 * np.max(np.abs(E_o[2]))
        H.itokmc_set_field(*[np.tile(np.ravel(e), R) for e in E])
    H.close()
