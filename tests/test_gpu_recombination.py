"""GPU parity of electron-ion and ion-ion recombination (Sec. 5.1, the air
chemistry table: propensities k_ep X_e X_+ and k_np X_+ X_-, k = beta / dV)
in the per-cell KMC: firings of all five reactions, ion counts and the
particles after products, photons and merge, bit for bit against the FP64
oracle in the FP64 form; the FP32 form against the same oracle within the
counting noise, with exact charge bookkeeping.
"""
import numpy as np
import pytest

import oracle
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, gpu_handle, mixed_state, oracle_state, small_phys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    itokmc.lib()


def _case(name):
    """(physics, particles, field, (N+, N-)) of a named case:
    air_x1e3 -- the air coefficients x 1e3, eps = 0.01 (substeps, attachment
      feeding the negative ions that then recombine), quasi-neutral ions;
    air_x1e5 -- x 1e5, eps = inf: most electrons of the dense cells recombine
      within the step (leaps rejected and halved);
    ion_only -- k_ep dt = 0.02 and k_np dt = 0.05 per pair, a blob of
      electrons and a few ions of both signs on half the cells: ion-ion
      recombination in cells without electrons, critical and SSA regimes."""
    if name == "ion_only":
        ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
        dV = synth.cell_size(ph) ** 3
        ph["beta_ep"] = 0.02 / ph["dt"] * dV
        ph["beta_np"] = 0.05 / ph["dt"] * dV
        st = synth.blob_state(ph, seed=7, sigma=1.0e-3, peak=3e17, zfrac=0.5)
        rng = np.random.default_rng(8)
        n3 = ph["n"] ** 3
        mask = rng.random(n3) < 0.5
        ions = (np.where(mask, rng.poisson(6, n3), 0).astype(np.int64),
                np.where(mask, rng.poisson(4, n3), 0).astype(np.int64))
    else:
        scale, eps = (1e3, 0.01) if name == "air_x1e3" else (1e5, float("inf"))
        ph = synth.with_recombination(small_phys(16, dt=5e-12, photon_ratio=0.06, eps=eps))
        ph["beta_ep"] *= scale
        ph["beta_np"] *= scale
        st = mixed_state(ph, seed=3, peak=2e19, n_random=800)
        S = oracle.canonical(oracle.make_params(ph, seed=1), st)
        cnt = np.bincount(S["cell"], weights=S["w"].astype(np.float64), minlength=ph["n"] ** 3).astype(np.int64)
        Np, Nn = synth.random_ions(ph, seed=4, mean=40.0, frac=0.4)
        ions = (cnt + Np, Nn)
    E = synth.random_field(ph, seed=9, amp=3e6, base=4.5e6)
    return ph, st, E, ions


def _handle(ph, st, E, ions, seed0, step, precision=itokmc.FP64):
    H = gpu_handle(ph, len(st["w"]) * 4 + 100000, seed0=seed0, precision=precision)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_field(*E)
    H.itokmc_set_ions(*ions)
    for _ in range(step):
        H.itokmc_advance_counter()
    return H


@pytest.mark.parametrize("name", ["air_x1e3", "air_x1e5", "ion_only"])
def test_recombination_stages_bit_exact(name):
    """Transport, then the KMC: the five firing counts per cell bit for bit;
    then products, photons and merge: N+, N- and the particles bit for bit;
    the step's statistics count the recombinations."""
    ph, st, E, ions = _case(name)
    seed0, step = 5, 2
    S = oracle_state(ph, st, seed0, *ions)
    new_state, info = oracle.step(oracle.make_params(ph, seed=seed0, step=step), S, E)
    assert info["n_ep"].sum() > 1000 and info["n_np"].sum() > 100
    if name == "ion_only":
        assert np.count_nonzero((info["Xe"] == 0) & (info["n_np"] > 0)) > 50
    H = _handle(ph, st, E, ions, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    assert_particles_equal(H.itokmc_read_particles(), info["sorted"])
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    assert F.shape[0] == 5
    for r, key in enumerate(("n_ion", "n_att", "n_ph", "n_ep", "n_np")):
        bad = np.flatnonzero(F[r] != info[key])
        assert bad.size == 0, (key, bad[:5], F[r][bad[:5]], info[key][bad[:5]])
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), new_state["Npos"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NNEG), new_state["Nneg"])
    assert_particles_equal(H.itokmc_read_particles(), new_state)
    s = H.itokmc_get_stats()
    assert s["recombinations_ep"] == int(info["n_ep"].sum())
    assert s["recombinations_np"] == int(info["n_np"].sum())
    H.close()


def test_recombination_off_leaves_the_network_first_order():
    """beta = 0: the recombination blocks of the firings stay zero, ion-only
    cells do not run, and the other firings are those of the oracle's
    first-order network."""
    ph, st, E, ions = _case("ion_only")
    ph = dict(ph, beta_ep=0.0, beta_np=0.0)
    seed0, step = 5, 2
    _, info = oracle.step(oracle.make_params(ph, seed=seed0, step=step), oracle_state(ph, st, seed0, *ions), E)
    H = _handle(ph, st, E, ions, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    assert not F[3].any() and not F[4].any()
    assert np.array_equal(F[0], info["n_ion"]) and np.array_equal(F[1], info["n_att"])
    assert np.array_equal(F[2], info["n_ph"])
    H.close()


def test_recombination_mixed_form_within_counting_noise():
    """The FP32 form of the same stages (air_x1e3): the total firings of each
    recombination within five Poisson standard deviations plus 0.1 % of the
    oracle's FP64 totals, and the charge bookkeeping exact --
    sum(N+ - N-) - sum(w) changes only by the electrons absorbed at the
    faces, counts stay non-negative."""
    ph, st, E, ions = _case("air_x1e3")
    seed0, step = 5, 2
    _, info = oracle.step(oracle.make_params(ph, seed=seed0, step=step), oracle_state(ph, st, seed0, *ions), E)
    H = _handle(ph, st, E, ions, seed0, step, precision=itokmc.MIXED)
    q0 = int(ions[0].sum() - ions[1].sum()) - int(np.asarray(st["w"], np.int64).sum())
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    out = H.itokmc_get_stats()["outflow_weight"]
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    for r, key in ((3, "n_ep"), (4, "n_np")):
        ref = float(info[key].sum())
        assert abs(float(F[r].sum()) - ref) <= 5 * np.sqrt(ref) + 1e-3 * ref, (key, F[r].sum(), ref)
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    Np = H.itokmc_read_densities(itokmc.NPOS)
    Nn = H.itokmc_read_densities(itokmc.NNEG)
    G = H.itokmc_read_particles()
    assert np.all(Np >= 0) and np.all(Nn >= 0)
    q1 = int(Np.sum() - Nn.sum()) - int(np.asarray(G["w"], np.int64).sum())
    assert q1 - q0 == out, (q1 - q0, out)
    H.close()


def test_checkpoint_binds_the_recombination_coefficients(tmp_path):
    """A checkpoint written with recombination on resumes bit for bit under
    the same coefficients and is refused under others."""
    ph, st, E, ions = _case("air_x1e3")
    seed0 = 5
    H = _handle(ph, st, E, ions, seed0, 0)
    H.itokmc_step()
    path = str(tmp_path / "rec.ckpt")
    H.itokmc_save(path)
    H.itokmc_step()
    ref = H.itokmc_read_densities(itokmc.FIRINGS)
    H.close()
    H2 = gpu_handle(ph, len(st["w"]) * 4 + 100000, seed0=seed0)
    H2.itokmc_load(path)
    H2.itokmc_step()
    assert np.array_equal(H2.itokmc_read_densities(itokmc.FIRINGS), ref)
    assert ref[3].sum() > 0
    H2.close()
    H3 = gpu_handle(dict(ph, beta_np=ph["beta_np"] * 2), len(st["w"]) * 4 + 100000, seed0=seed0)
    with pytest.raises(itokmc.ItokmcError):
        H3.itokmc_load(path)
    H3.close()
