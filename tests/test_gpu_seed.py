"""Device seeding of the initial electrons (itokmc_seed_blobs and
itokmc_init with blobs) against the oracle's seeding: the same Philox draws
give the same per-cell Poisson counts, weights and cells, and in the FP64
form the same positions bit for bit; the mixed form's offsets agree with the
FP64 positions to FP32 rounding."""
import numpy as np
import pytest

import oracle
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, gpu_handle, small_phys

pytestmark = pytest.mark.gpu

BLOBS = [dict(center=(0.005, 0.005, 0.008), sigma=5e-4, peak=1e18),
         dict(center=(0.0031, 0.0062, 0.004), sigma=3e-4, peak=4e19)]


def _oracle_realization(ph, blobs, seed0, r, step=0):
    p = oracle.make_params(ph, seed=seed0 + r, step=step)
    st, counts = oracle.seed_blobs(p, blobs, real=r)
    return st, counts


@pytest.mark.parametrize("n", [32, 64])
def test_seed_fp64_bit_exact(n):
    ph = small_phys(n)
    st, counts = _oracle_realization(ph, BLOBS, 7, 0)
    H = gpu_handle(ph, 2 * len(st["w"]) + 1000, seed0=7)
    H.itokmc_seed_blobs(BLOBS, itokmc.SEED_NEUTRAL)
    G = H.itokmc_read_particles()
    assert_particles_equal(G, st)
    assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), counts)
    H.close()


def test_seed_ensemble_blob_per_realization():
    ph = small_phys(32)
    blobs = BLOBS + [dict(center=(0.002, 0.002, 0.002), sigma=4e-4, peak=2e19, realization=1)]
    R = 3
    H = gpu_handle(ph, 400000, seed0=11, realizations=R)
    H.itokmc_seed_blobs(blobs)
    G = H.itokmc_read_particles()
    for r in range(R):
        st, counts = _oracle_realization(ph, blobs, 11, r)
        sel = G["realization"] == r
        assert_particles_equal({k: np.asarray(G[k])[sel] for k in ("x", "y", "z", "w", "cell")}, st)
    assert np.all(H.itokmc_read_densities(itokmc.NPOS, realization=-1) == 0)
    H.close()


def test_seed_mixed_form_offsets():
    ph = small_phys(32)
    st, counts = _oracle_realization(ph, BLOBS, 3, 0)
    H = gpu_handle(ph, 2 * len(st["w"]) + 1000, seed0=3, precision=itokmc.MIXED)
    H.itokmc_seed_blobs(BLOBS)
    G = H.itokmc_read_particles()
    assert np.array_equal(G["w"], st["w"]) and np.array_equal(G["cell"], st["cell"])
    h = synth.cell_size(ph)
    for k in ("x", "y", "z"):
        assert np.max(np.abs(G[k] - st[k])) / h <= 2.0 ** -23
    H.close()


def test_init_with_blobs_seeds_and_solves():
    """itokmc_init with blobs in the configuration: the particles of
    itokmc_seed_blobs, and the initial field of that charge already solved."""
    ph = small_phys(32)
    st, counts = _oracle_realization(ph, BLOBS, 5, 0)
    arr = itokmc.blob_array(BLOBS)
    cfg = itokmc.make_config(ph, 2 * len(st["w"]) + 1000, seed0=5)
    cfg.blobs = itokmc.ctypes.cast(arr, itokmc.ctypes.c_void_p)
    cfg.n_blobs = len(BLOBS)
    cfg.seed_flags = itokmc.SEED_NEUTRAL
    H = itokmc.Handle(cfg)
    assert_particles_equal(H.itokmc_read_particles(), st)
    E = H.itokmc_read_densities(itokmc.E)
    assert H.itokmc_get_stats()["mg_rel_residual"] <= 1e-10
    # neutral seed: the charge is the CIC spread of the electrons against
    # their NGP ions, so the field differs from the applied one
    assert np.max(np.abs(E[2] + ph["E0"])) > 0
    H.itokmc_step(1)
    H.close()


def test_seed_rejects_bad_blobs():
    ph = small_phys(16)
    H = gpu_handle(ph, 1000, seed0=1)
    for bad in (dict(center=(0.005, 0.005, 0.005), sigma=0.0, peak=1e18),
                dict(center=(0.005, 0.005, 0.005), sigma=1e-3, peak=-1.0),
                dict(center=(0.005, 0.005, 0.005), sigma=1e-3, peak=1e18, realization=-2)):
        with pytest.raises(itokmc.ItokmcError) as e:
            H.itokmc_seed_blobs([bad])
        assert e.value.code == -1
    with pytest.raises(itokmc.ItokmcError) as e:
        H.itokmc_seed_blobs([dict(center=(0.005, 0.005, 0.005), sigma=1e-3, peak=1e22)])
    assert e.value.code in (-4, -5)
    H.close()
