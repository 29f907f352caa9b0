"""GPU parity of the mobile ions: positive and negative ions as Ito
particles (Sec. 4.3, Eq. particle_kernel with V = sgn(Z_s) mu_s E), stacked
as particle blocks beside the electrons, against the oracle's three-species
step (``oracle.step_mobile``): every species' particles, the firings, the
ion counts and the space charge bit for bit in the FP64 form; charge
bookkeeping over whole steps; paired seeding; checkpoints; rejections.
"""
import numpy as np
import pytest

import oracle
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, small_phys

pytestmark = pytest.mark.gpu

SPECIES = ("e", "pos", "neg")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    itokmc.lib()


def _phys(n=16, recomb=False, **kw):
    ph = synth.with_mobile_ions(small_phys(n, dt=5e-12, photon_ratio=0.06), mu_ion=2e-2)
    ph["mobile_ions"] = True
    if recomb:
        ph = synth.with_recombination(ph)
        ph["beta_ep"] *= 1e3
        ph["beta_np"] *= 1e3
    ph.update(kw)
    return ph


def _state(ph, seed=3):
    """Oracle-canonical species: a Gaussian electron blob, a positive ion at
    every electron particle plus scattered ions, scattered negative ions."""
    p = oracle.make_params(ph, seed=1)
    e = oracle.canonical(p, synth.blob_state(ph, seed=seed, sigma=1.2e-3, peak=5e18, zfrac=0.5))
    bg = synth.ion_particles(ph, seed=seed + 1, mean=4000, frac=0.3)
    pos = oracle.canonical(p, {k: np.concatenate([e[k], bg[k]]) for k in ("x", "y", "z", "w")})
    neg = oracle.canonical(p, synth.ion_particles(ph, seed=seed + 2, mean=3000, frac=0.3))
    return {"e": e, "pos": pos, "neg": neg}


def _handle(ph, S, E, seed0, step, precision=itokmc.FP64):
    n = sum(len(S[k]["w"]) for k in SPECIES)
    cfg = itokmc.make_config(ph, 4 * n + 100000, seed0=seed0, precision=precision)
    H = itokmc.Handle(cfg)
    cat = {f: np.concatenate([S[k][f] for k in SPECIES]) for f in ("x", "y", "z", "w")}
    sp = np.concatenate([np.full(len(S[k]["w"]), i, np.int32) for i, k in enumerate(SPECIES)])
    H.itokmc_set_particles_species(cat["x"], cat["y"], cat["z"], cat["w"], sp)
    if E is not None:
        H.itokmc_set_field(*E)
    for _ in range(step):
        H.itokmc_advance_counter()
    return H


def _split(G):
    return {k: {f: G[f][G["species"] == i] for f in ("x", "y", "z", "w", "cell")} for i, k in enumerate(SPECIES)}


@pytest.mark.parametrize("recomb", [False, True])
def test_mobile_ion_stages_bit_exact(recomb):
    """Transport of all three species (sorted particles of each block), the
    KMC on the NGP counts of the three blocks (firings, ion counts), the
    space charge from the CIC densities, then products, photo-ions, losses
    and the merge of every block: bit for bit against the oracle."""
    ph = _phys(16, recomb)
    S = _state(ph)
    E = synth.random_field(ph, seed=9, amp=3e6, base=4.5e6)
    seed0, step = 5, 2
    new, info = oracle.step_mobile(oracle.make_params(ph, seed=seed0, step=step), S, E)
    assert info["n_ion"].sum() > 0 and info["n_ph"].sum() > 0
    if recomb:
        assert info["n_ep"].sum() > 0 and info["n_np"].sum() > 0
    H = _handle(ph, S, E, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    T = _split(H.itokmc_read_particles())
    for k in SPECIES:
        assert_particles_equal(T[k], info["sorted"][k])
        assert np.array_equal(T[k]["cell"], info["sorted"][k]["cell"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.XE), info["counts"]["e"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), info["counts"]["pos"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NNEG), info["counts"]["neg"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.RHO), info["rho_fixed"])
    s = H.itokmc_get_stats()
    assert (s["outflow_weight"], s["outflow_ion_pos"], s["outflow_ion_neg"]) == \
        (info["outflow"]["e"], info["outflow"]["pos"], info["outflow"]["neg"])
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    for r, key in enumerate(("n_ion", "n_att", "n_ph", "n_ep", "n_np")):
        assert np.array_equal(F[r], info[key]), key
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    out = _split(H.itokmc_read_particles())
    for k in SPECIES:
        assert_particles_equal(out[k], new[k])
        assert np.array_equal(out[k]["cell"], new[k]["cell"])
    H.close()


def test_mobile_ion_whole_steps_keep_charge():
    """Whole steps (field solved from the charge of all three species):
    W+ - W- - We changes by the absorbed weights only, each species stays
    positive, ions move in opposite directions along the field."""
    ph = _phys(16, recomb=True)
    S = _state(ph)
    H = _handle(ph, S, None, 7, 0)
    H.itokmc_solve_field()

    def books():
        G = _split(H.itokmc_read_particles())
        return {k: int(np.asarray(G[k]["w"], np.int64).sum()) for k in SPECIES}, G
    W0, G0 = books()
    for _ in range(3):
        H.itokmc_step(1)
        W1, G1 = books()
        s = H.itokmc_get_stats()
        q0 = W0["pos"] - W0["neg"] - W0["e"]
        q1 = W1["pos"] - W1["neg"] - W1["e"]
        assert q1 - q0 == s["outflow_weight"] + s["outflow_ion_neg"] - s["outflow_ion_pos"]
        assert s["ionizations"] > 0 and s["recombinations_ep"] > 0
        for k in SPECIES:
            assert np.all(G1[k]["w"] > 0)
        W0 = W1
    H.close()


@pytest.mark.parametrize("precision", [itokmc.FP64, itokmc.MIXED])
def test_mobile_ion_seed_pairs(precision):
    """Seeding with electron-ion pairs puts a positive ion at every seed
    electron's position and weight (no negative ions); without pairs only
    electrons."""
    ph = _phys(16)
    cfg = itokmc.make_config(ph, 2_000_000, seed0=3, precision=precision)
    H = itokmc.Handle(cfg)
    blobs = [dict(center=(0.005, 0.005, 0.005), sigma=1e-3, peak=3e18)]
    H.itokmc_seed_blobs(blobs, flags=itokmc.SEED_NEUTRAL)
    G = _split(H.itokmc_read_particles())
    assert len(G["e"]["w"]) > 1000 and len(G["neg"]["w"]) == 0
    for f in ("x", "y", "z", "w", "cell"):
        assert np.array_equal(G["e"][f], G["pos"][f]), f
    H.itokmc_seed_blobs(blobs, flags=0)
    G = _split(H.itokmc_read_particles())
    assert len(G["pos"]["w"]) == 0 and len(G["e"]["w"]) > 1000
    H.close()


def test_mobile_ion_checkpoint_resumes_bit_for_bit(tmp_path):
    """Two steps, save, two more; a fresh handle that loads the file and runs
    the same two steps ends with the same particles of every species."""
    ph = _phys(16, recomb=True)
    S = _state(ph)
    H = _handle(ph, S, None, 11, 0)
    H.itokmc_solve_field()
    H.itokmc_step(2)
    path = str(tmp_path / "mobile.ckpt")
    H.itokmc_save(path)
    H.itokmc_step(2)
    ref = H.itokmc_read_particles()
    n = len(ref["w"])
    H.close()
    H2 = itokmc.Handle(itokmc.make_config(ph, 4 * n + 100000, seed0=11))
    H2.itokmc_load(path)
    H2.itokmc_step(2)
    got = H2.itokmc_read_particles()
    for f in ("x", "y", "z", "w", "cell", "species"):
        assert np.array_equal(got[f], ref[f]), f
    H2.close()


def test_mobile_ion_rejections():
    """Ion counts cannot be set when the ions are particles; ion species need
    mobile ions; mobile ions need the explicit coupling."""
    ph = _phys(8)
    H = itokmc.Handle(itokmc.make_config(ph, 10000, seed0=1))
    n3 = ph["n"] ** 3
    with pytest.raises(itokmc.ItokmcError):
        H.itokmc_set_ions(np.zeros(n3, np.int64), np.zeros(n3, np.int64))
    H.close()
    ph0 = dict(ph, mobile_ions=False)
    H = itokmc.Handle(itokmc.make_config(ph0, 10000, seed0=1))
    c = 0.5 * (ph["lo"][0] + ph["hi"][0])
    with pytest.raises(itokmc.ItokmcError):
        H.itokmc_set_particles_species([c], [c], [c], [5], [1])
    H.close()
    with pytest.raises(itokmc.ItokmcError):
        itokmc.Handle(itokmc.make_config(ph, 10000, seed0=1, coupling=itokmc.SEMI_IMPLICIT))
