"""The oracle's OpenMP build (the all-core CPU baseline) computes the same
values as its plain build: the pragmas only spread independent particle and
cell iterations over threads (each draws from its own Philox stream) and
make the integer density sums atomic."""
import numpy as np

from paper_2307_01797_gb300 import synth


def test_openmp_build_matches_plain(oracle_mod):
    ph = synth.physics_small(32)
    ph["photon_ratio"] = 0.06
    st = synth.blob_state(ph, seed=4, sigma=1.5e-3, peak=3e18, zfrac=0.6)
    E = synth.random_field(ph, seed=5, amp=2e6, base=4e6)
    out = []
    try:
        for omp in (False, True):
            oracle_mod.use_openmp(omp, threads=4)
            p = oracle_mod.make_params(ph, seed=3, step=2)
            S = oracle_mod.canonical(p, st)
            xo, yo, zo, c = oracle_mod.push(p, S["x"], S["y"], S["z"], E)
            perm = oracle_mod.sort_by_cell(c, ph["n"] ** 3)
            ne, Xe = oracle_mod.deposit(p, xo[perm], yo[perm], zo[perm], S["w"][perm], c[perm])
            f = oracle_mod.kmc(p, Xe, E)
            out.append((xo, yo, zo, c, ne, Xe, f))
    finally:
        oracle_mod.use_openmp(False)
    for a, b in zip(out[0], out[1]):
        if isinstance(a, tuple):
            assert all(np.array_equal(u, v) for u, v in zip(a, b))
        else:
            assert np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))
