"""Pins of the oracle's semi-implicit field coupling (Sec. 4.3, Sec. 4.7).

Each test checks ``oracle/semi_implicit.py`` and the C functions it calls
against an independent fact: the constant-coefficient solve it must reduce
to, a matrix-free flux sum written out cell by cell, the explicit push it
must equal when one of the two transport terms vanishes, and the property
the scheme exists for (no dielectric-relaxation runaway).  CPU only.
"""
import numpy as np
import pytest

from paper_2307_01797_gb300 import synth


def _phys(n, **kw):
    ph = synth.physics_small(n)
    ph.update(kw)
    return ph


def test_constant_coefficient_reduces_to_poisson(oracle_mod):
    """c = 1 is the system of the explicit field solve; a constant c scales
    the charge: div(c grad phi) = -rho/eps0 is lap(phi) = -(rho/c)/eps0 with
    the same electrode potentials."""
    from oracle import poisson, semi_implicit as si
    n = 8
    ph = _phys(n)
    rho = np.random.default_rng(1).integers(-10 ** 12, 10 ** 12, n ** 3)
    phi0, E0 = poisson.solve(rho, ph)
    phi1, E1 = si.solve(rho, np.ones((n, n, n)), ph)
    assert np.max(np.abs(phi1 - phi0)) <= 1e-12 * np.max(np.abs(phi0))
    Emax = max(np.max(np.abs(e)) for e in E0)
    for a, b in zip(E1, E0):
        assert np.max(np.abs(a - b)) <= 1e-11 * Emax
    c0 = 3.7
    phi2, _ = si.solve(rho, np.full((n, n, n), c0), ph)
    phi3, _ = poisson.solve(np.asarray(rho, np.float64) / c0, ph)
    assert np.max(np.abs(phi2 - phi3)) <= 1e-12 * np.max(np.abs(phi3))


def _flux_sum(phi, c, h, phi_top):
    """div(c grad phi) cell by cell from the six face fluxes: interior face
    coefficient (c_a + c_b)/2; a boundary face takes the cell's own c with
    the ghost values of the field problem (sides: ghost = phi; z = lo:
    ghost = -phi; z = hi: ghost = 2 phi_top - phi)."""
    n = phi.shape[0]
    out = np.zeros_like(phi)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                s = 0.0
                for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    kk, jj, ii = k + dk, j + dj, i + di
                    if 0 <= kk < n and 0 <= jj < n and 0 <= ii < n:
                        cf = 0.5 * (c[k, j, i] + c[kk, jj, ii])
                        g = phi[kk, jj, ii]
                    else:
                        cf = c[k, j, i]
                        if kk < 0:
                            g = -phi[k, j, i]
                        elif kk >= n:
                            g = 2.0 * phi_top - phi[k, j, i]
                        else:
                            g = phi[k, j, i]
                    s += cf * (g - phi[k, j, i])
                out[k, j, i] = s / (h * h)
    return out


def test_variable_coefficient_operator_and_solution(oracle_mod):
    """The sparse operator equals the face-flux sum written out for random
    coefficients, and the solve satisfies div(c grad phi) = -rho/eps0 with
    the electrode potentials to rounding."""
    from oracle import poisson, semi_implicit as si
    n = 4
    ph = _phys(n)
    h = (ph["hi"][0] - ph["lo"][0]) / n
    phi_top = ph["E0"] * (ph["hi"][2] - ph["lo"][2])
    rng = np.random.default_rng(2)
    c = rng.uniform(1.0, 30.0, (n, n, n))
    phi = rng.normal(size=(n, n, n)) * 100.0
    A = si.assemble(c, h)
    got = (A @ phi.ravel()).reshape(n, n, n)
    got[n - 1] += 2.0 * c[n - 1] * phi_top / (h * h)
    ref = _flux_sum(phi, c, h, phi_top)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    rho = rng.integers(-10 ** 12, 10 ** 12, n ** 3)
    phs, _ = si.solve(rho, c, ph)
    b = poisson.rhs(rho, n, h, 10, 0.0)
    res = _flux_sum(phs, c, h, phi_top) - b
    # rounding relative to the size of the flux terms (the electrode
    # potential makes them far larger than the charge term)
    scale = np.max(c) * max(np.max(np.abs(phs)), phi_top) / (h * h)
    assert np.max(np.abs(res)) <= 1e-12 * scale


def _state(oracle_mod, ph, seed, per_cell=8, w=500_000_000, block=(5, 11)):
    """Electrons spread uniformly over a block of cells, ions equal to the
    electrons of each cell (a neutral plasma up to the CIC spreading)."""
    n = ph["n"]
    h = (ph["hi"][0] - ph["lo"][0]) / n
    rng = np.random.default_rng(seed)
    cols = {k: [] for k in "xyz"}
    r = range(*block)
    for k in r:
        for j in r:
            for i in r:
                for key, c in zip("xyz", (i, j, k)):
                    cols[key].append((c + rng.uniform(0.0, 1.0, per_cell)) * h)
    st = {k: np.concatenate(v) for k, v in cols.items()}
    st["w"] = np.full(len(st["x"]), w, np.uint32)
    p = oracle_mod.make_params(ph, seed=seed)
    S = oracle_mod.canonical(p, st)
    _, Xe = oracle_mod.deposit(p, S["x"], S["y"], S["z"], S["w"], S["cell"])
    S["Npos"] = Xe.copy()
    S["Nneg"] = np.zeros(n ** 3, np.int64)
    return S


@pytest.mark.parametrize("which", ["diffusion", "drift"])
def test_one_transport_term_reduces_to_the_explicit_push(oracle_mod, which):
    """Without drift (mu = 0) the two substeps are the explicit push (same
    normals); without diffusion (D = 0) they are the explicit push in the
    new field evaluated at the start-of-step positions."""
    from oracle import semi_implicit as si
    kw = {"mu": 0.0} if which == "diffusion" else {"D": 0.0}
    ph = _phys(16, dt=5e-12, **kw)
    S = _state(oracle_mod, ph, seed=4, per_cell=3, w=1000)
    p = oracle_mod.make_params(ph, seed=4, step=3)
    r = si.transport(p, ph, S)
    E = r["E"] if which == "drift" else synth.random_field(ph, seed=5, amp=3e6, base=4.5e6)
    xo, yo, zo, cell = oracle_mod.push(p, S["x"], S["y"], S["z"], E)
    for a, b in ((r["xo"], xo), (r["yo"], yo), (r["zo"], zo)):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    assert np.array_equal(r["cell"], cell)
    if which == "diffusion":
        assert np.all(r["sigma"] == 0.0)
    else:
        assert np.array_equal(r["xd"], S["x"])


def test_semi_implicit_step_has_no_dielectric_relaxation_limit(oracle_mod):
    """Sec. 4.3: the explicit push is stable only for dt below the dielectric
    relaxation time eps0/sigma; the semi-implicit step is not limited.  A
    plasma block at sigma dt / eps0 ~ 23 with a positive charge added to one
    cell: the explicit push overshoots (the charge norm grows several fold in
    one step), the semi-implicit step relaxes it in every step and keeps every
    particle in the box."""
    from oracle import poisson, semi_implicit as si
    n = 16
    ph = _phys(n, dt=3e-9, D=0.0, E0=0.0)
    S0 = _state(oracle_mod, ph, seed=3)
    S0["Npos"][(8 * n + 8) * n + 8] += 1_000_000_000

    def run(mode, steps):
        S = dict(S0)
        norms, counts = [], []
        for k in range(steps):
            p = oracle_mod.make_params(ph, seed=3, step=k)
            ne, _ = oracle_mod.deposit(p, S["x"], S["y"], S["z"], S["w"], S["cell"])
            rho = oracle_mod.rho_fixed(p, ne, S["Npos"], S["Nneg"])
            norms.append(np.sqrt(np.sum(rho.astype(np.float64) ** 2)))
            counts.append(len(S["x"]))
            if mode == "explicit":
                _, E = poisson.solve(rho, ph)
                xo, yo, zo, cell = oracle_mod.push(p, S["x"], S["y"], S["z"], E)
            else:
                r = si.transport(p, ph, S)
                if k == 0:
                    assert np.max(si.coefficient(r["sigma"], ph["dt"])) > 20.0
                xo, yo, zo, cell = r["xo"], r["yo"], r["zo"], r["cell"]
            perm = oracle_mod.sort_by_cell(cell, n ** 3)
            S = dict(x=xo[perm], y=yo[perm], z=zo[perm], w=S["w"][perm], cell=cell[perm],
                     Npos=S["Npos"], Nneg=S["Nneg"])
        return norms, counts

    ne_, ce = run("explicit", 2)
    ns, cs = run("semi", 5)
    assert ne_[1] > 3.0 * ne_[0]
    assert all(b < a for a, b in zip(ns, ns[1:])) and ns[-1] < 0.8 * ns[0]
    assert cs[-1] == cs[0]


def test_velocity_is_taken_at_the_start_of_step_position(oracle_mod):
    """Eq. Vk1: with drift and diffusion the advective displacement X' - X+
    is -mu E^{k+1}(X^k) dt, the field at the position before the diffusive
    advance (it differs measurably from the field at X+)."""
    from oracle import semi_implicit as si
    ph = _phys(16, dt=5e-12)
    S = _state(oracle_mod, ph, seed=6, per_cell=3, w=1000)
    S["Npos"] = S["Npos"] + np.random.default_rng(7).integers(0, 5000, ph["n"] ** 3)
    p = oracle_mod.make_params(ph, seed=6, step=2)
    r = si.transport(p, ph, S)
    ph0 = dict(ph, D=0.0)
    p0 = oracle_mod.make_params(ph0, seed=6, step=2)
    at_xk = oracle_mod.push(p0, S["x"], S["y"], S["z"], r["E"])[2] - S["z"]
    at_xd = oracle_mod.push(p0, r["xd"], r["yd"], r["zd"], r["E"])[2] - r["zd"]
    got = r["zo"] - r["zd"]
    tol = 4 * np.finfo(np.float64).eps * np.max(np.abs(S["z"]))
    assert np.max(np.abs(got - at_xk)) <= tol
    assert np.max(np.abs(got - at_xd)) > 100 * tol


def test_semi_implicit_full_step_conserves_charge(oracle_mod):
    """Whole semi-implicit steps (transport, KMC, products, photons,
    merge/split): the net charge sum(N+ - N-) - sum(w) changes only by the
    electrons absorbed at the faces (a lost photon creates nothing), every
    count stays non-negative and every cell ends with at most ppc
    particles."""
    from oracle import semi_implicit as si
    ph = _phys(16, dt=5e-12, photon_ratio=0.06)
    st = synth.blob_state(ph, seed=3, sigma=1.2e-3, peak=5e18, zfrac=0.5)
    p = oracle_mod.make_params(ph, seed=8, step=0)
    S = oracle_mod.canonical(p, st)
    n3 = ph["n"] ** 3
    S["Npos"] = np.zeros(n3, np.int64)
    S["Nneg"] = np.zeros(n3, np.int64)
    q0 = int(S["Npos"].sum() - S["Nneg"].sum()) - int(S["w"].astype(np.int64).sum())
    for k in range(2):
        p = oracle_mod.make_params(ph, seed=8, step=k)
        S, info = si.step(p, ph, S)
        q1 = int(S["Npos"].sum() - S["Nneg"].sum()) - int(S["w"].astype(np.int64).sum())
        assert q1 - q0 == info["outflow"], (q1 - q0, info["outflow"])
        q0 = q1
        assert np.all(S["Npos"] >= 0) and np.all(S["Nneg"] >= 0) and np.all(S["w"] > 0)
        assert np.bincount(S["cell"], minlength=n3).max() <= ph["ppc"]
        assert info["n_ion"].sum() > 0
