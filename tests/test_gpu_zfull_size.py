"""Parity at full size: the 256^3 streamer workload that the bench times
(7.1e7 particles of the synthetic four-channel discharge tree, ppc 32,
photoionization on, dt 5 ps), built by the bench's own recipe and run in the
bench's launch configuration (the same capacity, seed and autotuned tiles,
host-driven ``itokmc_step``).

FP64 form (plain and with the recombination reactions): one full step
against the oracle's step fed the same field, bit for bit on every output
the step leaves (sorted particles after the merge, the deposited densities,
X_e, the space charge, the firings of all cells, the ion counts, the
outflow), and the field the step solves within 1e-5 of the exact solve of
the same charge.  The oracle runs whole (push, deposit
and KMC on all host cores through its OpenMP build, the rest single
threaded), so nothing is sampled.

Mixed form: the transport stage against the FP64 oracle within the stated
tolerance of the FP32 push (positions within 1e-5 cell for all but 0.2% of
the particles, densities within 1e-3), exact charge and weight bookkeeping
over the whole step, at most ppc particles per cell, and its field within
1e-5 of the exact solve of its own charge.

The largest grid, 512^3 (the discharge-tree configuration: 4 cm, 1.8 MV/m,
ppc 64, four Gaussian seeds sampled by ``itokmc_init``): in the FP64 form the
seeded particles, the charge, and one full step bit for bit against the
oracle fed the same field; in the mixed form (the tree study's) the same
checks at the stated tolerances.  The exact solve is too slow on the host at
this size, so the field is checked by what holds at any size: the discrete
equation's residual (recomputed on the host from the GPU's potential)
within the solver's tolerance and E the centred difference of that
potential.
"""
import types

import numpy as np
import pytest

import oracle
from oracle import poisson
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, oracle_state

pytestmark = pytest.mark.gpu

E_TOL = 1e-5
SEED0 = 1                  # the bench's key for rank 0


@pytest.fixture(scope="module")
def workload():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    itokmc.lib()
    import bench
    args = types.SimpleNamespace(n=256, particles=1e8, cap_factor=4.0)
    ph, st, ions = bench.workload(args)
    oracle.use_openmp(True)
    S = oracle_state(ph, st, SEED0, *ions)
    yield ph, st, ions, S, int(len(st["w"]) * args.cap_factor) + 20_000_000
    oracle.use_openmp(False)


def _handle(ph, st, ions, cap, precision):
    H = itokmc.Handle(itokmc.make_config(ph, cap, seed0=SEED0, precision=precision))
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_ions(*ions)
    H.itokmc_solve_field()
    H.itokmc_autotune()
    return H


def _field_err(H, phi_o, E_o):
    phi_g = H.itokmc_read_densities(itokmc.PHI)
    E_g = H.itokmc_read_densities(itokmc.E)
    ephi = np.max(np.abs(phi_g - phi_o.ravel())) / np.max(np.abs(phi_o))
    eE = max(np.max(np.abs(E_g[a] - E_o[a].ravel())) for a in range(3)) / max(np.max(np.abs(e)) for e in E_o)
    return ephi, eE


def _align_by_cell(cg, ct, n3):
    """Indices (into two cell-sorted lists) of the particles of the cells
    that hold the same number of particles in both, paired in list order."""
    ng, nt = np.bincount(cg, minlength=n3), np.bincount(ct, minlength=n3)
    sg = np.concatenate([[0], np.cumsum(ng)])
    st = np.concatenate([[0], np.cumsum(nt)])
    ig = np.nonzero((ng == nt)[cg])[0]
    c = cg[ig]
    return ig, ig - sg[c] + st[c]


@pytest.mark.parametrize("recombination", [False, True])
def test_full_size_fp64_step_bit_exact(workload, recombination):
    """One FP64 step of the bench workload, plain and with the air
    recombination coefficients (the bench's --recombination: five reactions,
    second-order propensities)."""
    ph, st, ions, S, cap = workload
    if recombination:
        # negative ions as well (an eighth of the positive ones) so that both
        # recombination reactions fire in the first step
        ph = synth.with_recombination(ph)
        ions = (ions[0], np.asarray(ions[0], np.int64) // 8)
        S = dict(S, Nneg=ions[1].copy())
    n3 = ph["n"] ** 3
    p = oracle.make_params(ph, seed=SEED0, step=0)
    H = _handle(ph, st, ions, cap, itokmc.FP64)
    ne0, _ = oracle.deposit(p, S["x"], S["y"], S["z"], S["w"], S["cell"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.RHO), oracle.rho_fixed(p, ne0, S["Npos"], S["Nneg"]))
    # the step pushes with the field solved at set-up; the oracle takes the
    # same doubles
    Eg = H.itokmc_read_densities(itokmc.E)
    E = (Eg[0].copy(), Eg[1].copy(), Eg[2].copy())
    H.itokmc_step(1)
    new, info = oracle.step(p, S, E)
    assert info["n_ion"].sum() > 0 and info["n_ph"].sum() > 0 and len(info["new_particles"][0]) > 0
    if recombination:
        assert info["n_ep"].sum() > 0 and info["n_np"].sum() > 0
    for which, ref in ((itokmc.NE_FIX, info["ne_fix"]), (itokmc.XE, info["Xe"]), (itokmc.RHO, info["rho_fixed"])):
        assert np.array_equal(H.itokmc_read_densities(which), ref), which
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    for r, key in enumerate(("n_ion", "n_att", "n_ph", "n_ep", "n_np")):
        assert np.array_equal(F[r], info[key]), key
    assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), new["Npos"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NNEG), new["Nneg"])
    assert H.itokmc_get_stats()["outflow_weight"] == info["outflow"]
    G = H.itokmc_read_particles()
    assert_particles_equal(G, new)
    assert np.bincount(G["cell"], minlength=n3).max() <= ph["ppc"]
    del G
    phi_o, E_o = poisson.solve(info["rho_fixed"], ph)
    ephi, eE = _field_err(H, phi_o, E_o)
    assert ephi < E_TOL and eE < E_TOL, (ephi, eE)
    H.close()


def test_full_size_mixed_step_within_tolerance(workload):
    ph, st, ions, S, cap = workload
    n3, s = ph["n"] ** 3, ph["frac_bits"]
    h = synth.cell_size(ph)
    p = oracle.make_params(ph, seed=SEED0, step=0)
    H = _handle(ph, st, ions, cap, itokmc.MIXED)
    Eg = H.itokmc_read_densities(itokmc.E)
    # the FP64 oracle's transport with the mixed handle's own field
    xo, yo, zo, cell = oracle.push(p, S["x"], S["y"], S["z"], (Eg[0], Eg[1], Eg[2]))
    perm = oracle.sort_by_cell(cell, n3)
    T = dict(x=xo[perm], y=yo[perm], z=zo[perm], w=S["w"][perm].copy(), cell=cell[perm])
    del xo, yo, zo
    ne, Xe = oracle.deposit(p, T["x"], T["y"], T["z"], T["w"], T["cell"])
    W0 = int(S["w"].astype(np.int64).sum())
    Q0 = int(np.sum(S["Npos"]) - np.sum(S["Nneg"])) - W0
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    out = H.itokmc_get_stats()["outflow_weight"]
    G = H.itokmc_read_particles()
    W = int(G["w"].astype(np.int64).sum())
    assert W == W0 - out
    neg = H.itokmc_read_densities(itokmc.NE_FIX)
    # the total, W 2^3s, exceeds int64 at this size: summed in two digits
    assert int((neg >> (3 * s)).sum()) * (1 << (3 * s)) + int((neg & ((1 << (3 * s)) - 1)).sum()) == W << (3 * s)
    assert int(H.itokmc_read_densities(itokmc.XE).sum()) == W
    assert abs(len(G["w"]) - len(T["w"])) <= 16
    # particle by particle: a particle whose cell differs between the forms
    # (FP32 rounding at a face) shifts every later particle of the sorted
    # list, so the lists are aligned cell by cell (both keep the input order
    # within a cell); the particles of cells whose populations differ count
    # as mismatched, like those further than 1e-5 cell from the oracle
    ig, it = _align_by_cell(G["cell"], T["cell"], n3)
    d = np.abs(G["x"][ig] - T["x"][it])
    d = np.maximum(d, np.abs(G["y"][ig] - T["y"][it]))
    d = np.maximum(d, np.abs(G["z"][ig] - T["z"][it])) / h
    bad = (len(G["w"]) - len(ig)) + int(np.count_nonzero((d > 1e-5) | (G["w"][ig] != T["w"][it])))
    assert bad / len(G["w"]) < 2e-3, bad / len(G["w"])
    del G, T, ig, it, d
    rel = np.linalg.norm((neg - ne).astype(np.float64)) / np.linalg.norm(ne.astype(np.float64))
    assert rel < 1e-3, rel
    assert np.abs(H.itokmc_read_densities(itokmc.XE) - Xe).sum() <= 1e-3 * Xe.sum()
    rho = H.itokmc_read_densities(itokmc.RHO)
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    H.itokmc_run_stage(itokmc.STAGE_FIELD)
    G = H.itokmc_read_particles()
    Np, Nn = H.itokmc_read_densities(itokmc.NPOS), H.itokmc_read_densities(itokmc.NNEG)
    # every created electron comes with a positive ion, every attachment
    # turns one into a negative ion, absorbed photons make pairs: the net
    # charge changes only by what left through the electrodes
    assert int(Np.sum() - Nn.sum()) - int(G["w"].astype(np.int64).sum()) == Q0 + out
    assert np.bincount(G["cell"], minlength=n3).max() <= ph["ppc"]
    del G
    phi_o, E_o = poisson.solve(rho, ph)
    ephi, eE = _field_err(H, phi_o, E_o)
    assert ephi < E_TOL and eE < E_TOL, (ephi, eE)
    H.close()


def _tree_512(precision):
    """The discharge-tree configuration as the bench's tree study builds it:
    the handle seeded and solved by itokmc_init, then autotuned."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ph = synth.physics_tree(512)
    L = ph["hi"][0] - ph["lo"][0]
    blobs = [dict(center=(L / 2 + sx * 5e-3, L / 2 + sy * 5e-3, 0.9 * L), sigma=3e-4, peak=5e18)
             for sx in (-1, 1) for sy in (-1, 1)]
    cfg = itokmc.make_config(ph, 100_000_000, seed0=SEED0, precision=precision)
    arr = itokmc.blob_array(blobs)
    cfg.blobs = itokmc.ctypes.cast(arr, itokmc.ctypes.c_void_p)
    cfg.n_blobs = len(blobs)
    H = itokmc.Handle(cfg)
    H.itokmc_autotune()
    h = L / ph["n"]
    phi_top = ph["E0"] * (ph["hi"][2] - ph["lo"][2])
    return ph, blobs, H, h, phi_top


def test_tree_512_fp64_seed_and_step_bit_exact():
    oracle.use_openmp(True)
    try:
        ph, blobs, H, h, phi_top = _tree_512(itokmc.FP64)
        n, n3 = ph["n"], ph["n"] ** 3
        p = oracle.make_params(ph, seed=SEED0, step=0)
        seeded, _ = oracle.seed_blobs(p, blobs, real=0)
        assert len(seeded["w"]) > 5_000_000
        assert_particles_equal(H.itokmc_read_particles(), seeded)
        S = dict(seeded, Npos=np.zeros(n3, np.int64), Nneg=np.zeros(n3, np.int64))
        ne0, _ = oracle.deposit(p, S["x"], S["y"], S["z"], S["w"], S["cell"])
        rho0 = oracle.rho_fixed(p, ne0, S["Npos"], S["Nneg"])
        del ne0
        assert np.array_equal(H.itokmc_read_densities(itokmc.RHO), rho0)
        _check_field_512(H, rho0, n, h, ph["frac_bits"], phi_top, ph.get("mg_rtol", 1e-10))
        del rho0
        Eg = H.itokmc_read_densities(itokmc.E)
        E = (Eg[0].copy(), Eg[1].copy(), Eg[2].copy())
        del Eg
        H.itokmc_step(1)
        new, info = oracle.step(p, S, E)
        del E, S
        assert info["n_ion"].sum() > 0 and info["n_ph"].sum() > 0
        for which, key in ((itokmc.NE_FIX, "ne_fix"), (itokmc.XE, "Xe"), (itokmc.RHO, "rho_fixed")):
            assert np.array_equal(H.itokmc_read_densities(which), info[key]), key
        F = H.itokmc_read_densities(itokmc.FIRINGS)
        for r, key in enumerate(("n_ion", "n_att", "n_ph")):
            assert np.array_equal(F[r], info[key]), key
        del F
        assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), new["Npos"])
        assert np.array_equal(H.itokmc_read_densities(itokmc.NNEG), new["Nneg"])
        assert_particles_equal(H.itokmc_read_particles(), new)
        _check_field_512(H, info["rho_fixed"], n, h, ph["frac_bits"], phi_top, ph.get("mg_rtol", 1e-10))
        H.close()
    finally:
        oracle.use_openmp(False)


def test_tree_512_mixed_seed_and_step_within_tolerance():
    """The tree study's own form (FP32 particles, fixed-point potential with
    FP32 V-cycles): the seeded offsets within FP32 rounding of the oracle's
    positions, the charge exact, the field by residual and gradient, the
    transport within the FP32 push's stated tolerance of the FP64 oracle,
    exact charge books over a whole step and at most ppc per cell."""
    oracle.use_openmp(True)
    try:
        ph, blobs, H, h, phi_top = _tree_512(itokmc.MIXED)
        n, n3, s = ph["n"], ph["n"] ** 3, ph["frac_bits"]
        p = oracle.make_params(ph, seed=SEED0, step=0)
        seeded, _ = oracle.seed_blobs(p, blobs, real=0)
        G0 = H.itokmc_read_particles()
        assert np.array_equal(G0["w"], seeded["w"]) and np.array_equal(G0["cell"], seeded["cell"])
        for k in ("x", "y", "z"):
            assert np.max(np.abs(G0[k] - seeded[k])) / h <= 2.0 ** -23
        del G0
        ne0, _ = oracle.deposit(p, seeded["x"], seeded["y"], seeded["z"], seeded["w"], seeded["cell"])
        ne_g = H.itokmc_read_densities(itokmc.NE_FIX)
        W0 = int(seeded["w"].astype(np.int64).sum())
        # the total W0 2^3s is near the int64 range: summed in two digits
        assert int((ne_g >> (3 * s)).sum()) * (1 << (3 * s)) + int((ne_g & ((1 << (3 * s)) - 1)).sum()) == W0 << (3 * s)
        assert np.linalg.norm((ne_g - ne0).astype(np.float64)) / np.linalg.norm(ne0.astype(np.float64)) < 1e-3
        del ne0, ne_g
        # the mixed form's E is the FP32 difference of the fixed-point
        # potential (three roundings of 2^-24 at most)
        _check_field_512(H, H.itokmc_read_densities(itokmc.RHO), n, h, s, phi_top, ph.get("mg_rtol", 1e-10), 4e-7)
        Eg = H.itokmc_read_densities(itokmc.E)
        xo, yo, zo, cell = oracle.push(p, seeded["x"], seeded["y"], seeded["z"], (Eg[0], Eg[1], Eg[2]))
        del Eg
        perm = oracle.sort_by_cell(cell, n3)
        T = dict(x=xo[perm], y=yo[perm], z=zo[perm], w=seeded["w"][perm].copy(), cell=cell[perm])
        del xo, yo, zo, cell, perm
        H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
        out = H.itokmc_get_stats()["outflow_weight"]
        G = H.itokmc_read_particles()
        assert int(G["w"].astype(np.int64).sum()) == W0 - out
        ig, it = _align_by_cell(G["cell"], T["cell"], n3)
        d = np.abs(G["x"][ig] - T["x"][it])
        d = np.maximum(d, np.abs(G["y"][ig] - T["y"][it]))
        d = np.maximum(d, np.abs(G["z"][ig] - T["z"][it])) / h
        bad = (len(G["w"]) - len(ig)) + int(np.count_nonzero((d > 1e-5) | (G["w"][ig] != T["w"][it])))
        assert bad / len(G["w"]) < 2e-3, bad / len(G["w"])
        del G, T, ig, it, d
        rho = H.itokmc_read_densities(itokmc.RHO)
        H.itokmc_run_stage(itokmc.STAGE_KMC)
        H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
        H.itokmc_run_stage(itokmc.STAGE_FIELD)
        G = H.itokmc_read_particles()
        Np, Nn = H.itokmc_read_densities(itokmc.NPOS), H.itokmc_read_densities(itokmc.NNEG)
        assert int(Np.sum() - Nn.sum()) - int(G["w"].astype(np.int64).sum()) == -W0 + out
        assert np.bincount(G["cell"], minlength=n3).max() <= ph["ppc"]
        del G, Np, Nn
        _check_field_512(H, rho, n, h, s, phi_top, ph.get("mg_rtol", 1e-10), 4e-7)
        H.close()
    finally:
        oracle.use_openmp(False)


def _check_field_512(H, rho_fixed, n, h, frac_bits, phi_top, rtol, e_tol=1e-12):
    """The GPU's potential satisfies the discrete field equation to the
    solver's tolerance (residual recomputed in FP64 on the host; the margin
    covers the host's own rounding, about 1e-14 of the norm of b here), and
    its E is the centred difference of that potential (to FP64 rounding, or
    e_tol where E is evaluated in FP32)."""
    phi = H.itokmc_read_densities(itokmc.PHI).reshape(n, n, n)
    # b holds the electrode potential folded into the top layer; the
    # operator below applies it through the ghost values, so it is compared
    # with -rho/eps0 alone
    b = poisson.rhs(rho_fixed, n, h, frac_bits, phi_top)
    bnorm = np.linalg.norm(b)
    b[n - 1] += 2.0 * phi_top / (h * h)
    r = poisson.apply_operator(phi, h, phi_top) - b
    rel = np.linalg.norm(r) / bnorm
    del r, b
    assert rel <= 1.5 * rtol, rel
    Eo = poisson.efield(phi, h, phi_top)
    Eg = H.itokmc_read_densities(itokmc.E)
    emax = max(np.max(np.abs(e)) for e in Eo)
    for a in range(3):
        assert np.max(np.abs(Eg[a] - Eo[a].ravel())) <= e_tol * emax, a
