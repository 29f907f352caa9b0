"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.  Integer outputs (sort order, weights, cells,
deposited densities, reaction counts, ion counts) and the FP64 positions are
compared bit for bit; the field within a relative 1e-5 (max norm).
"""
import numpy as np
import pytest

import oracle
from oracle import poisson
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import assert_particles_equal, gpu_handle, mixed_state, oracle_state, small_phys

pytestmark = pytest.mark.gpu

E_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    itokmc.lib()


def _setup(ph, st, E, ions, seed0, step=0, cap=None):
    H = gpu_handle(ph, cap or (len(st["w"]) * 4 + 100000), seed0=seed0)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_field(*E)
    if ions is not None:
        H.itokmc_set_ions(*ions)
    for _ in range(step):
        H.itokmc_advance_counter()
    return H


def _transport_oracle(ph, S, E, seed0, step):
    p = oracle.make_params(ph, seed=seed0, step=step)
    n3 = ph["n"] ** 3
    xo, yo, zo, cell = oracle.push(p, S["x"], S["y"], S["z"], E)
    perm = oracle.sort_by_cell(cell, n3)
    T = dict(x=xo[perm], y=yo[perm], z=zo[perm], w=S["w"][perm].copy(), cell=cell[perm])
    ne, Xe = oracle.deposit(p, T["x"], T["y"], T["z"], T["w"], T["cell"])
    rho = oracle.rho_fixed(p, ne, S["Npos"], S["Nneg"])
    out = int(S["w"][cell < 0].astype(np.int64).sum())
    return T, ne, Xe, rho, out


@pytest.mark.parametrize("dt,n,step", [(1e-12, 32, 0), (2e-9, 16, 3), (5e-8, 16, 7)])
def test_transport_bit_exact(dt, n, step):
    """a1-a4: push, stable sort, int64 CIC deposit, X_e and rho; dt from the
    paper-like 1 ps to a stress case where a third of the particles change
    cell and some leave through the faces."""
    ph = small_phys(n, dt=dt)
    st = mixed_state(ph, seed=11 + n)
    E = synth.random_field(ph, seed=5, amp=4e6)
    ions = synth.random_ions(ph, seed=6)
    seed0 = 77
    S = oracle_state(ph, st, seed0, *ions)
    T, ne, Xe, rho, out = _transport_oracle(ph, S, E, seed0, step)
    H = _setup(ph, st, E, ions, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    G = H.itokmc_read_particles()
    assert_particles_equal(G, T)
    assert np.array_equal(H.itokmc_read_densities(itokmc.NE_FIX), ne)
    assert np.array_equal(H.itokmc_read_densities(itokmc.XE), Xe)
    assert np.array_equal(H.itokmc_read_densities(itokmc.RHO), rho)
    stats = H.itokmc_get_stats()
    assert stats["outflow_weight"] == out
    if dt >= 2e-9:
        assert stats["n_movers"] > len(T["w"]) // 20


def test_kmc_and_particles_bit_exact():
    """a6-a9 after a transport stage: reaction counts per cell, ion counts,
    loss removal, products, photoionization and merge/split, bit for bit."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    st = mixed_state(ph, seed=3, peak=2e19, n_random=800)
    E = synth.random_field(ph, seed=9, amp=3e6, base=4.5e6)
    ions = synth.random_ions(ph, seed=4)
    seed0, step = 5, 2
    S = oracle_state(ph, st, seed0, *ions)
    p = oracle.make_params(ph, seed=seed0, step=step)
    new_state, info = oracle.step(p, S, E)
    H = _setup(ph, st, E, ions, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    assert_particles_equal(H.itokmc_read_particles(), info["sorted"])
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    assert np.array_equal(F[0], info["n_ion"])
    assert np.array_equal(F[1], info["n_att"])
    assert np.array_equal(F[2], info["n_ph"])
    assert info["n_ion"].sum() > 1000 and info["n_att"].sum() > 100 and info["n_ph"].sum() > 10
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), new_state["Npos"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NNEG), new_state["Nneg"])
    G = H.itokmc_read_particles()
    assert_particles_equal(G, new_state)
    assert np.bincount(G["cell"], minlength=16 ** 3).max() <= ph["ppc"]
    st_ = H.itokmc_get_stats()
    assert st_["photons_absorbed_weight"] + st_["photons_lost_weight"] == int(info["n_ph"].sum())


def test_kmc_stage_rerun_starts_its_cell_lists_afresh():
    """The KMC stage run four times on one transported state: every run lists
    the active cells from zero (the lists hold at most one entry per cell per
    run), gives the oracle's firings, and adds its ions once; the statistics
    of the particles stage count one run's reactions."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    st = mixed_state(ph, seed=3, peak=2e19, n_random=800)
    E = synth.random_field(ph, seed=9, amp=3e6, base=4.5e6)
    ions = synth.random_ions(ph, seed=4)
    seed0, step = 5, 2
    S = oracle_state(ph, st, seed0, *ions)
    _, info = oracle.step(oracle.make_params(ph, seed=seed0, step=step), S, E)
    H = _setup(ph, st, E, ions, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    Np0 = H.itokmc_read_densities(itokmc.NPOS)
    Nn0 = H.itokmc_read_densities(itokmc.NNEG)
    runs = 4
    for _ in range(runs):
        H.itokmc_run_stage(itokmc.STAGE_KMC)
        F = H.itokmc_read_densities(itokmc.FIRINGS)
        assert np.array_equal(F[0], info["n_ion"]) and np.array_equal(F[1], info["n_att"])
        assert np.array_equal(F[2], info["n_ph"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), Np0 + runs * info["n_ion"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NNEG), Nn0 + runs * info["n_att"])
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    s = H.itokmc_get_stats()
    assert s["ionizations"] == int(info["n_ion"].sum()) and s["attachments"] == int(info["n_att"].sum())
    H.close()


def test_stages_out_of_order_are_refused():
    """The KMC before any transport, the particles stage without a KMC after
    the last transport, and a KMC after the particles stage are refused on
    the host (ERR_ARG, nothing launched); the handle stays usable and the
    stages in order then run."""
    ph = small_phys(16, dt=5e-12)
    st = mixed_state(ph, seed=3, n_random=500)
    H = _setup(ph, st, synth.random_field(ph, seed=9, amp=3e6), synth.random_ions(ph, seed=4), 5)
    with pytest.raises(itokmc.ItokmcError, match="stage order"):
        H.itokmc_run_stage(itokmc.STAGE_KMC)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    with pytest.raises(itokmc.ItokmcError, match="stage order"):
        H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    with pytest.raises(itokmc.ItokmcError, match="stage order"):
        H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    with pytest.raises(itokmc.ItokmcError, match="stage order"):
        H.itokmc_run_stage(itokmc.STAGE_KMC)
    H.itokmc_run_stage(itokmc.STAGE_FIELD)
    H.itokmc_advance_counter()
    H.itokmc_step(1)
    assert H.itokmc_get_stats()["n_particles"] > 0
    H.close()


@pytest.mark.parametrize("dt", [5e-12, 5e-11])
def test_semi_implicit_transport_against_oracle(dt):
    """The semi-implicit transport stage (Sec. 4.3, Sec. 4.7 steps 1-5): the
    field of the variable-coefficient solve within the field tolerance of the
    oracle's direct solve; with that field, the diffusive and advective
    substeps, the sort and the deposit bit for bit like the oracle's."""
    from oracle import semi_implicit as si
    ph = small_phys(16, dt=dt)
    st = mixed_state(ph, seed=21, peak=2e19, n_random=1500)
    E0 = synth.random_field(ph, seed=5, amp=4e6)
    ions = synth.random_ions(ph, seed=6)
    seed0, step = 33, 2
    S = oracle_state(ph, st, seed0, *ions)
    p = oracle.make_params(ph, seed=seed0, step=step)
    ref = si.transport(p, ph, S)
    H = _setup(ph, st, E0, ions, seed0, step)
    cycles, rel = H.itokmc_transport_semi_implicit()
    assert 0 < cycles < 40 and rel <= 1e-10
    Eg = H.itokmc_read_densities(itokmc.E).reshape(3, -1)
    Eo = np.stack([e.ravel() for e in ref["E"]])
    assert np.max(np.abs(Eg - Eo)) <= E_TOL * np.max(np.abs(Eo))
    assert np.max(si.coefficient(ref["sigma"], dt)) > 1.0
    r = si.transport(p, ph, S, E=tuple(Eg))
    perm = oracle.sort_by_cell(r["cell"], ph["n"] ** 3)
    T = dict(x=r["xo"][perm], y=r["yo"][perm], z=r["zo"][perm], w=S["w"][perm].copy(), cell=r["cell"][perm])
    assert_particles_equal(H.itokmc_read_particles(), T)
    ne, Xe = oracle.deposit(p, T["x"], T["y"], T["z"], T["w"], T["cell"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.NE_FIX), ne)
    assert np.array_equal(H.itokmc_read_densities(itokmc.XE), Xe)
    H.close()


def test_kmc_finite_eps_bit_exact():
    """The Cao step bound for a finite eps (substeps of bounded relative
    change) in the FP64 KMC kernel: firings per cell bit for bit against the
    oracle, in a case where the bound splits the step (the firings differ
    from those of eps = inf)."""
    ph = small_phys(16, dt=5e-11, photon_ratio=0.06, eps=0.01)
    st = mixed_state(ph, seed=13, peak=2e19, n_random=800)
    E = synth.random_field(ph, seed=9, amp=3e6, base=4.5e6)
    ions = synth.random_ions(ph, seed=4)
    seed0, step = 5, 1
    S = oracle_state(ph, st, seed0, *ions)
    _, info = oracle.step(oracle.make_params(ph, seed=seed0, step=step), S, E)
    ph_inf = dict(ph, eps=float("inf"))
    _, info_inf = oracle.step(oracle.make_params(ph_inf, seed=seed0, step=step),
                              oracle_state(ph_inf, st, seed0, *ions), E)
    assert not np.array_equal(info["n_ion"], info_inf["n_ion"])
    H = _setup(ph, st, E, ions, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    F = H.itokmc_read_densities(itokmc.FIRINGS)
    assert np.array_equal(F[0], info["n_ion"])
    assert np.array_equal(F[1], info["n_att"])
    assert np.array_equal(F[2], info["n_ph"])
    H.close()


@pytest.mark.parametrize("ppc", [8, 32])
def test_merge_tiers_bit_exact(ppc):
    """Cells whose merge lists fall in each tier of the merge kernel (list plus
    leaves up to 96 and 256 elements in shared memory, longer ones in the
    global work area), some with equal coordinates: the whole particles stage
    bit for bit against the oracle."""
    ph = small_phys(8, dt=1e-13, ppc=ppc, photon_ratio=0.0)
    rng = np.random.default_rng(17 + ppc)
    h = (ph["hi"][0] - ph["lo"][0]) / ph["n"]
    cols = {k: [] for k in ("x", "y", "z", "w")}
    for (i, j, k), m in [((1, 1, 1), 30), ((2, 5, 6), 20), ((5, 1, 2), 50), ((0, 6, 1), 70), ((4, 4, 4), 90),
                         ((3, 4, 5), 150), ((6, 2, 3), 400)]:
        X = [ph["lo"][0] + (c + rng.uniform(0.05, 0.95, m)) * h for c in (i, j, k)]
        X[0][: m // 8] = X[0][0]            # equal x: the stable order decides
        X[2][m // 8: m // 4] = X[2][m // 8]
        for key, v in zip(("x", "y", "z"), X):
            cols[key].append(v)
        cols["w"].append(rng.integers(1, 5000, m).astype(np.uint32))
    st = {k: np.concatenate(v) for k, v in cols.items()}
    E = synth.random_field(ph, seed=11, amp=3e6, base=4.5e6)
    seed0, step = 7, 1
    S = oracle_state(ph, st, seed0)
    p = oracle.make_params(ph, seed=seed0, step=step)
    new_state, info = oracle.step(p, S, E)
    H = _setup(ph, st, E, None, seed0, step)
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    H.itokmc_run_stage(itokmc.STAGE_KMC)
    H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
    assert_particles_equal(H.itokmc_read_particles(), new_state)
    st_ = H.itokmc_get_stats()
    assert st_["merge_max_list"] >= 400 and st_["merge_cells"] >= 4
    H.close()


def _field_err(phi_g, E_g, phi_o, E_o):
    ephi = np.max(np.abs(phi_g - phi_o.ravel())) / np.max(np.abs(phi_o))
    Eo = np.stack([e.ravel() for e in E_o])
    eE = np.max(np.abs(E_g - Eo)) / np.max(np.abs(Eo))
    return ephi, eE


@pytest.mark.parametrize("precision", [itokmc.FP64, itokmc.MIXED])
def test_field_solve_matches_exact_solution(precision):
    """a5: multigrid phi and E against the exact separable solve of the same
    discrete system, relative 1e-5 in the max norm (FP64 and FP32-in-FP64-IR)."""
    ph = small_phys(32)
    st = mixed_state(ph, seed=21, peak=5e19)
    ions = synth.random_ions(ph, seed=22, mean=2000)
    cfg = itokmc.make_config(ph, len(st["w"]) + 10, seed0=1, field_precision=precision)
    H = itokmc.Handle(cfg)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_ions(*ions)
    H.itokmc_solve_field()
    p = oracle.make_params(ph, seed=1)
    S = oracle_state(ph, st, 1, *ions)
    ne, _ = oracle.deposit(p, S["x"], S["y"], S["z"], S["w"], S["cell"])
    rho = oracle.rho_fixed(p, ne, S["Npos"], S["Nneg"])
    assert np.array_equal(H.itokmc_read_densities(itokmc.RHO), rho)
    phi_o, E_o = poisson.solve(rho, ph)
    ephi, eE = _field_err(H.itokmc_read_densities(itokmc.PHI), H.itokmc_read_densities(itokmc.E), phi_o, E_o)
    assert ephi < E_TOL and eE < E_TOL, (ephi, eE)
    s = H.itokmc_get_stats()
    assert s["mg_rel_residual"] <= 1e-10


def test_full_steps_match_oracle_chain():
    """Three full steps through itokmc_step against the oracle's step chained
    with its exact field solve: particles bit-exact while the fields agree to
    rounding; the field within 1e-5 after each step."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    st = mixed_state(ph, seed=31, peak=1e19, n_random=500)
    seed0 = 9
    H = gpu_handle(ph, 200000, seed0=seed0)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_solve_field()
    p0 = oracle.make_params(ph, seed=seed0)
    S = oracle_state(ph, st, seed0)
    ne, _ = oracle.deposit(p0, S["x"], S["y"], S["z"], S["w"], S["cell"])
    phi, E = poisson.solve(oracle.rho_fixed(p0, ne, S["Npos"], S["Nneg"]), ph)
    # feed the oracle's field to both sides so that the step itself is compared
    H.itokmc_set_field(*E)
    for k in range(3):
        p = oracle.make_params(ph, seed=seed0, step=k)
        S, info = oracle.step(p, S, E)
        H.itokmc_step(1)
        assert_particles_equal(H.itokmc_read_particles(), S)
        assert np.array_equal(H.itokmc_read_densities(itokmc.NPOS), S["Npos"])
        phi, E = poisson.solve(info["rho_fixed"], ph)
        ephi, eE = _field_err(H.itokmc_read_densities(itokmc.PHI), H.itokmc_read_densities(itokmc.E), phi, E)
        assert ephi < E_TOL and eE < E_TOL
        H.itokmc_set_field(*E)


def test_ensemble_members_equal_single_runs():
    """R realizations in one handle: member r equals a single run with key
    seed0 + r (uneven particle counts per member)."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    R, seed0 = 3, 40
    states = [mixed_state(ph, seed=50 + r, peak=10 ** (18 + r * 0.5), n_random=200 * (r + 1)) for r in range(R)]
    E = synth.random_field(ph, seed=2, amp=2e6, base=4e6)
    x = np.concatenate([s["x"] for s in states]); y = np.concatenate([s["y"] for s in states])
    z = np.concatenate([s["z"] for s in states]); w = np.concatenate([s["w"] for s in states])
    real = np.concatenate([np.full(len(s["w"]), r, np.int32) for r, s in enumerate(states)])
    H = gpu_handle(ph, 400000, seed0=seed0, realizations=R)
    H.itokmc_set_particles(x, y, z, w, real)
    H.itokmc_set_field(*[np.tile(np.ravel(e), R) for e in E])
    for k in range(2):
        H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
        H.itokmc_run_stage(itokmc.STAGE_KMC)
        H.itokmc_run_stage(itokmc.STAGE_PARTICLES)
        H.itokmc_advance_counter()
    G = H.itokmc_read_particles()
    for r in range(R):
        S = oracle_state(ph, states[r], seed0 + r)
        for k in range(2):
            S, _ = oracle.step(oracle.make_params(ph, seed=seed0 + r, step=k), S, E)
        sel = G["realization"] == r
        assert_particles_equal({k: v[sel] for k, v in G.items()}, S)


def test_deterministic_rerun():
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    st = mixed_state(ph, seed=8, peak=3e16)
    out = []
    for _ in range(2):
        H = gpu_handle(ph, 100000, seed0=3)
        H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
        H.itokmc_solve_field()
        H.itokmc_step(3)
        G = H.itokmc_read_particles()
        out.append((G, H.itokmc_read_densities(itokmc.PHI)))
        H.close()
    assert_particles_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_edge_cases():
    ph = small_phys(8, dt=1e-12)
    # empty state steps cleanly
    H = gpu_handle(ph, 1000)
    H.itokmc_set_particles(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0, np.uint32))
    H.itokmc_solve_field()
    H.itokmc_step(2)
    assert H.itokmc_num_particles() == 0
    # one particle, weight 1
    L = ph["hi"][0]
    H.itokmc_set_particles(np.array([L / 2]), np.array([L / 2]), np.array([L / 2]), np.array([1], np.uint32))
    H.itokmc_step(1)
    assert H.itokmc_num_particles() in (0, 1, 2)
    # every particle leaves through the top electrode in one step
    ph2 = small_phys(8, dt=1e-8, D=0.0)
    H2 = gpu_handle(ph2, 1000)
    z = np.full(100, L - 1e-5)
    H2.itokmc_set_particles(np.full(100, L / 2), np.full(100, L / 2), z, np.full(100, 3, np.uint32))
    H2.itokmc_set_field(*synth.uniform_field(ph2, -1.5e6))
    H2.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    assert H2.itokmc_num_particles() == 0 and H2.itokmc_get_stats()["outflow_weight"] == 300
    # invalid input and capacity are reported, not crashed on
    with pytest.raises(itokmc.ItokmcError) as e:
        H2.itokmc_set_particles(np.array([2 * L]), np.array([0.0]), np.array([0.0]), np.array([1], np.uint32))
    assert e.value.code == -1
    with pytest.raises(itokmc.ItokmcError) as e:
        H2.itokmc_set_particles(np.zeros(2000) + L / 2, np.zeros(2000) + L / 2, np.zeros(2000) + L / 2,
                                np.ones(2000, np.uint32))
    assert e.value.code == -4


@pytest.mark.parametrize("precision", [itokmc.FP64, itokmc.MIXED])
def test_runaway_charge_reports_overflow(precision):
    """A cell whose ion surplus leaves the fixed-point range of rho (2^(62-3s)
    elementary charges, s = 10) is reported as ERR_OVERFLOW before any field
    is computed from it; the handle stays usable once the state is valid."""
    ph = small_phys(8, dt=1e-12)
    H = gpu_handle(ph, 1000, precision=precision)
    L = ph["hi"][0]
    H.itokmc_set_particles(np.array([L / 2]), np.array([L / 2]), np.array([L / 2]), np.array([1], np.uint32))
    n3 = ph["n"] ** 3
    npos = np.zeros(n3, np.int64)
    npos[n3 // 2] = 1 << 33
    H.itokmc_set_ions(npos, np.zeros(n3, np.int64))
    with pytest.raises(itokmc.ItokmcError) as e:
        H.itokmc_solve_field()
    assert e.value.code == -5
    npos[n3 // 2] = (1 << 32) - 1          # the largest surplus the guard admits
    H.itokmc_set_ions(npos, np.zeros(n3, np.int64))
    H.itokmc_solve_field()
    H.itokmc_set_ions(np.zeros(n3, np.int64), np.zeros(n3, np.int64))
    H.itokmc_solve_field()
    H.itokmc_step(1)
    H.close()


# ---------------------------------------------------------------- mixed form
def _mixed_handle(ph, st, E, ions, seed0, cap):
    H = gpu_handle(ph, cap, seed0=seed0, precision=itokmc.MIXED)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    if E is not None:
        H.itokmc_set_field(*E)
    if ions is not None:
        H.itokmc_set_ions(*ions)
    return H


def test_mixed_transport_against_fp64_oracle():
    """FP32 positions/push with common random numbers: positions within
    1e-5 cell of the FP64 oracle for all but a few particles whose cell
    membership flips at a face; exact charge conservation of the int64
    deposit; densities within 1e-3 (relative L2)."""
    ph = small_phys(32, dt=2e-10)
    st = mixed_state(ph, seed=17)
    E = synth.random_field(ph, seed=5, amp=4e6)
    ions = synth.random_ions(ph, seed=6)
    seed0 = 12
    S = oracle_state(ph, st, seed0, *ions)
    T, ne, Xe, rho, out = _transport_oracle(ph, S, E, seed0, 0)
    H = _mixed_handle(ph, st, E, ions, seed0, 4 * len(st["w"]))
    # the upload itself rounds positions to FP32 offsets: same cells, same order
    G0 = H.itokmc_read_particles()
    assert np.array_equal(G0["cell"], S["cell"]) and np.array_equal(G0["w"], S["w"])
    H.itokmc_run_stage(itokmc.STAGE_TRANSPORT)
    G = H.itokmc_read_particles()
    assert abs(len(G["w"]) - len(T["w"])) <= 2
    h = synth.cell_size(ph)
    W = int(G["w"].astype(np.int64).sum())
    neg = H.itokmc_read_densities(itokmc.NE_FIX)
    assert sum(int(v) for v in neg) == W << (3 * ph["frac_bits"])
    if len(G["w"]) == len(T["w"]):
        d = np.max(np.abs(np.stack([G["x"] - T["x"], G["y"] - T["y"], G["z"] - T["z"]])), axis=0) / h
        assert (d > 1e-5).mean() < 2e-3, (d > 1e-5).mean()
    rel = np.linalg.norm((neg - ne).astype(np.float64)) / np.linalg.norm(ne.astype(np.float64))
    assert rel < 1e-3, rel
    assert np.abs(H.itokmc_read_densities(itokmc.XE) - Xe).sum() <= 0.001 * Xe.sum()


def test_mixed_steps_against_fp64_oracle_chain():
    """Three full steps of the mixed form (FP32 particles, FP32 V-cycles in
    FP64 refinement) against the FP64 oracle chain: electron density and E
    within the stated tolerance, charge conservation exact."""
    ph = small_phys(16, dt=5e-12, photon_ratio=0.06)
    st = mixed_state(ph, seed=31, peak=1e19, n_random=500)
    seed0 = 9
    p0 = oracle.make_params(ph, seed=seed0)
    S = oracle_state(ph, st, seed0)
    ne, _ = oracle.deposit(p0, S["x"], S["y"], S["z"], S["w"], S["cell"])
    phi, E = poisson.solve(oracle.rho_fixed(p0, ne, S["Npos"], S["Nneg"]), ph)
    H = _mixed_handle(ph, st, E, None, seed0, 200000)
    Q0 = -int(st["w"].astype(np.int64).sum())
    out = 0
    for k in range(3):
        S, info = oracle.step(oracle.make_params(ph, seed=seed0, step=k), S, E)
        phi, E = poisson.solve(info["rho_fixed"], ph)
        H.itokmc_step(1)
        out += H.itokmc_get_stats()["outflow_weight"]
        neg = H.itokmc_read_densities(itokmc.NE_FIX).astype(np.float64)
        rel = np.linalg.norm(neg - info["ne_fix"]) / np.linalg.norm(info["ne_fix"].astype(np.float64))
        assert rel < 2e-2, (k, rel)
        Eg = H.itokmc_read_densities(itokmc.E)
        Eo = np.stack([e.ravel() for e in E])
        # FP32 rounding flips a few discrete decisions (a photon's absorption
        # cell, a particle's cell) so the charge differs locally after a few
        # steps: E agrees to 1e-3 in L2 and 1e-2 in the max norm
        assert np.linalg.norm(Eg - Eo) / np.linalg.norm(Eo) < 1e-3
        assert np.max(np.abs(Eg - Eo)) / np.max(np.abs(Eo)) < 1e-2
        G = H.itokmc_read_particles()
        Np, Nn = H.itokmc_read_densities(itokmc.NPOS), H.itokmc_read_densities(itokmc.NNEG)
        assert int(Np.sum() - Nn.sum()) - int(G["w"].astype(np.int64).sum()) == Q0 + out
        assert np.bincount(G["cell"], minlength=16 ** 3).max() <= ph["ppc"]
