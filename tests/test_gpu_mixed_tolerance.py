"""The mixed form's stated tolerance over whole runs.

Per realization the FP32 form decorrelates from the FP64 form once an FP32
propensity changes a draw, so its tolerance beyond the first steps is
statistical: for the small-blob physics on its 64^3 grid, 16 realizations
(Philox keys 1..16) stepped in both forms from the same state, the
ensemble means must agree after k steps (k <= 50) within

  * 1e-6 relative in the electron count,
  * 5e-5 k relative L2 in the electron density (ne_fix),
  * 1e-6 k relative L2 in the field,

about twice the differences measured on one GB300 (2.4e-5 k and 2.6e-7 k at
k = 50).  Checked here for 20 steps."""
import numpy as np
import pytest

from paper_2307_01797_gb300 import itokmc, synth

pytestmark = pytest.mark.gpu


def test_mixed_ensemble_means_within_stated_tolerance():
    R, K = 16, 20
    ph = synth.physics_small(64)
    st = synth.blob_state(ph, seed=1, sigma=5e-4, peak=1e18, zfrac=0.8)
    N0 = len(st["w"])
    n3 = ph["n"] ** 3
    rep = {k: np.tile(np.asarray(st[k]), R) for k in ("x", "y", "z", "w")}
    real = np.repeat(np.arange(R, dtype=np.int32), N0)
    hs = {}
    for name, form in (("fp64", itokmc.FP64), ("mixed", itokmc.MIXED)):
        H = itokmc.Handle(itokmc.make_config(ph, 8 * R * N0 + 1_000_000, realizations=R, seed0=1, precision=form))
        H.itokmc_set_particles(rep["x"], rep["y"], rep["z"], rep["w"], real)
        H.itokmc_solve_field()
        hs[name] = H
    for k in range(1, K + 1):
        for H in hs.values():
            H.itokmc_step(1)
        ne = {m: H.itokmc_read_densities(itokmc.NE_FIX, realization=-1).reshape(R, n3).astype(np.float64)
              for m, H in hs.items()}
        tot = {m: v.sum(axis=1).mean() for m, v in ne.items()}
        assert abs(tot["mixed"] - tot["fp64"]) <= 1e-6 * tot["fp64"], k
        a, b = ne["mixed"].mean(axis=0), ne["fp64"].mean(axis=0)
        assert np.linalg.norm(a - b) <= 5e-5 * k * np.linalg.norm(b), (k, np.linalg.norm(a - b) / np.linalg.norm(b))
        Ea = hs["mixed"].itokmc_read_densities(itokmc.E, realization=-1).reshape(3, R, n3).mean(axis=1)
        Eb = hs["fp64"].itokmc_read_densities(itokmc.E, realization=-1).reshape(3, R, n3).mean(axis=1)
        assert np.linalg.norm(Ea - Eb) <= 1e-6 * k * np.linalg.norm(Eb), k
    for H in hs.values():
        H.close()
