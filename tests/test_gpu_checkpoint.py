"""Checkpoint and resume through the C ABI (itokmc_save / itokmc_load).

A run of four steps and a run of two steps, a checkpoint, a fresh handle
that loads it and two more steps must end in the same state byte for byte:
particles (positions, weights, cells, order), ion counts, potential and
field.  The checkpoint's own contract is checked too: a handle of another
configuration refuses it, a foreign file is refused, and loading restores
the step counter and the smoother counts."""
import os

import numpy as np
import pytest

from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, gpu_handle, mixed_state, small_phys

pytestmark = pytest.mark.gpu


def _state(H):
    G = H.itokmc_read_particles()
    return G, {w: H.itokmc_read_densities(w, realization=-1)
               for w in (itokmc.NPOS, itokmc.NNEG, itokmc.PHI, itokmc.E, itokmc.NE_FIX)}


def _setup(ph, precision, R):
    sts = [mixed_state(ph, seed=60 + r, peak=2e18) for r in range(R)]
    x = np.concatenate([s["x"] for s in sts]); y = np.concatenate([s["y"] for s in sts])
    z = np.concatenate([s["z"] for s in sts]); w = np.concatenate([s["w"] for s in sts])
    real = np.concatenate([np.full(len(s["w"]), r, np.int32) for r, s in enumerate(sts)]) if R > 1 else None
    ions = synth.random_ions(ph, seed=61, mean=200)
    H = gpu_handle(ph, 10 * len(w) + 200000, seed0=5, precision=precision, realizations=R)
    H.itokmc_set_particles(x, y, z, w, real)
    H.itokmc_set_ions(np.tile(ions[0], R), np.tile(ions[1], R))
    H.itokmc_solve_field()
    return H


@pytest.mark.parametrize("precision,R", [(itokmc.FP64, 1), (itokmc.MIXED, 1), (itokmc.FP64, 3), (itokmc.MIXED, 3)])
def test_resume_from_checkpoint_is_bit_identical(tmp_path, precision, R):
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    A = _setup(ph, precision, R)
    A.itokmc_step(4)
    ref_p, ref_d = _state(A)
    A.close()

    B = _setup(ph, precision, R)
    B.itokmc_step(2)
    path = os.path.join(tmp_path, "run.ckpt")
    B.itokmc_save(path)
    B.close()

    C = gpu_handle(ph, 12 * len(ref_p["w"]) + 200000, seed0=5, precision=precision, realizations=R)
    C.itokmc_load(path)
    assert C.itokmc_get_stats()["step"] == 2
    C.itokmc_step(2)
    got_p, got_d = _state(C)
    C.close()
    assert_particles_equal(got_p, ref_p)
    for k in ref_d:
        assert np.array_equal(np.asarray(got_d[k]).view(np.uint8), np.asarray(ref_d[k]).view(np.uint8)), k


def test_checkpoint_refuses_another_configuration(tmp_path):
    ph = small_phys(16, dt=5e-12)
    A = _setup(ph, itokmc.FP64, 1)
    A.itokmc_step(1)
    path = os.path.join(tmp_path, "a.ckpt")
    A.itokmc_save(path)
    A.close()
    other = small_phys(16, dt=6e-12)
    B = gpu_handle(other, 200000, seed0=5)
    with pytest.raises(itokmc.ItokmcError) as e:
        B.itokmc_load(path)
    assert e.value.code == -1 and "dt" in str(e.value)
    junk = os.path.join(tmp_path, "junk.ckpt")
    with open(junk, "wb") as f:
        f.write(b"not a checkpoint" * 8)
    with pytest.raises(itokmc.ItokmcError) as e:
        B.itokmc_load(junk)
    assert e.value.code == -1
    B.close()
