"""0-D KMC ensembles on the GPU (itokmc_kmc0d, Sec. 3.2.4) against the
oracle: independent single-cell realizations, bit-exact trajectories in the
FP64 form; the FP32 form's ensemble mean against the FP64 one within its
sampling error (common random numbers make the two close realization by
realization)."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_01797_gb300 import itokmc, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("E,X0,dt", [(2.0e6, 30, 1e-12), (3.6e6, 7, 5e-12), (5e6, 400, 1e-12), (8e6, 50000, 2e-12)])
def test_kmc0d_fp64_bit_exact(E, X0, dt):
    ph = synth.physics_small(8)
    ph["dt"] = dt
    ph["photon_ratio"] = 0.06
    M, K = 3000, 40
    ref = oracle.kmc0d(oracle.make_params(ph, seed=21), E, X0, M, K)
    cfg = itokmc.make_config(ph, 1, seed0=21)
    got = itokmc.itokmc_kmc0d(cfg, E, X0, M, K)
    assert np.array_equal(got, ref)


def test_kmc0d_mixed_mean_within_sampling_error():
    ph = synth.physics_small(8)
    M, K, E, X0 = 20000, 60, 5e6, 300
    a = itokmc.itokmc_kmc0d(itokmc.make_config(ph, 1, seed0=3), E, X0, M, K)
    b = itokmc.itokmc_kmc0d(itokmc.make_config(ph, 1, seed0=3, precision=itokmc.MIXED), E, X0, M, K)
    sd = a[:, -1].std()
    assert abs(a[:, -1].mean() - b[:, -1].mean()) < 5 * sd / math.sqrt(M)
    # common random numbers: most realizations end within a few electrons
    assert np.median(np.abs(a[:, -1] - b[:, -1])) <= 2


def test_kmc0d_rejects_bad_arguments():
    ph = synth.physics_small(8)
    cfg = itokmc.make_config(ph, 1)
    for args in ((5e6, -1, 10, 5), (5e6, 10, 0, 5), (-1.0, 10, 10, 5)):
        with pytest.raises(itokmc.ItokmcError) as e:
            itokmc.itokmc_kmc0d(cfg, *args)
        assert e.value.code == -1
