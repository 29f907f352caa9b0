"""Pins of the oracle's mobile ions: the ions as Ito particles (Sec. 4.3,
Eq. particle_kernel with V = sgn(Z_s) mu_s E, Eq. Vk1), pushed, sorted,
deposited and merged like the electrons, coupled to the KMC through their
NGP counts and to the field through their CIC charge.

References independent of the oracle's arithmetic: the law of the Ito
update in a uniform field (mean displacement sgn(Z) mu E dt, variance
2 D dt per axis, independent species), the immobile limit (ions at rest at
the cell centres deposit as integer counts), and the exact bookkeeping of
charge and of each species' weight through whole steps.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2307_01797_gb300 import synth


def _phys(n=16, **kw):
    ph = synth.with_mobile_ions(synth.physics_small(n))
    ph.update(kw)
    return ph


def _uniform_field(ph, E):
    n3 = ph["n"] ** 3
    return tuple(np.full(n3, float(e)) for e in E)


def test_species_zero_is_the_electron_push(oracle_mod):
    """The species push with species 0 is ``push`` itself, bit for bit."""
    ph = _phys(16)
    st = synth.random_particles(ph, 3000, seed=3, wmax=100)
    E = synth.random_field(ph, seed=4, amp=3e6, base=2e6)
    p = oracle_mod.make_params(ph, seed=9, step=4)
    a = oracle_mod.push(p, st["x"], st["y"], st["z"], E)
    b = oracle_mod.push_species(p, 0, st["x"], st["y"], st["z"], E)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("species,sign", [(1, +1.0), (2, -1.0)])
def test_ion_displacement_law_in_a_uniform_field(oracle_mod, species, sign):
    """20 000 ions at the box centre in a uniform field E: the displacement
    per axis has mean sgn(Z) mu_ion E_a dt (within 5 standard errors, the
    drift is ~30 of them) and variance 2 D_ion dt (chi-square, 1e-4 level);
    the axes are uncorrelated."""
    E = (3.0e6, -2.0e6, 4.5e6)
    ph = _phys(16, dt=2e-10, mu_ion=2e-3)
    p = oracle_mod.make_params(ph, seed=5, step=3)
    m = 20000
    c = 0.5 * (ph["lo"][0] + ph["hi"][0])
    x = np.full(m, c) + np.linspace(-1e-5, 1e-5, m)
    y = np.full(m, c)
    z = np.full(m, c)
    xo, yo, zo, cell = oracle_mod.push_species(p, species, x, y, z, _uniform_field(ph, E))
    assert np.all(cell >= 0)
    D = np.stack([xo - x, yo - y, zo - z], axis=1)
    var = 2.0 * ph["D_ion"] * ph["dt"]
    for a in range(3):
        mean = sign * ph["mu_ion"] * E[a] * ph["dt"]
        se = np.sqrt(var / m)
        assert abs(D[:, a].mean() - mean) <= 5 * se, (a, D[:, a].mean(), mean, se)
        assert abs(mean) > 20 * se
        s2 = ((D[:, a] - mean) ** 2).sum() / var
        assert stats.chi2.ppf(1e-4, m) < s2 < stats.chi2.ppf(1 - 1e-4, m)
    corr = np.corrcoef(D.T - np.array([[sign * ph["mu_ion"] * e * ph["dt"]] for e in E]))
    assert np.max(np.abs(corr - np.eye(3))) < 0.04


def test_species_draw_independent_normals(oracle_mod):
    """The same particle index in the two ion species (and the electrons)
    draws from different streams: displacements in zero field are
    uncorrelated across species."""
    ph = _phys(16, dt=2e-10, mu=0.0)
    p = oracle_mod.make_params(ph, seed=5, step=1)
    m = 20000
    c = np.full(m, 0.5 * (ph["lo"][0] + ph["hi"][0]))
    E0 = _uniform_field(ph, (0.0, 0.0, 0.0))
    d = [oracle_mod.push_species(p, s, c, c, c, E0)[0] - c for s in range(3)]
    for i in range(3):
        for j in range(i + 1, 3):
            assert abs(np.corrcoef(d[i], d[j])[0, 1]) < 0.04


def test_immobile_ions_at_cell_centres_deposit_as_counts(oracle_mod):
    """mu_ion = D_ion = 0: ion particles keep their positions bit for bit;
    one ion particle of weight N at each cell centre deposits exactly
    2^3s N into its own cell, so the charge n+ - n- equals the count model's
    2^3s (N+ - N-)."""
    ph = _phys(12, mu_ion=0.0, D_ion=0.0)
    p = oracle_mod.make_params(ph, seed=2, step=0)
    n = ph["n"]
    rng = np.random.default_rng(3)
    cells = np.flatnonzero(rng.random(n ** 3) < 0.5)
    h = synth.cell_size(ph)
    ijk = np.stack([cells % n, (cells // n) % n, cells // (n * n)], axis=1)
    X = [ph["lo"][a] + (ijk[:, a] + 0.5) * h for a in range(3)]
    w = rng.integers(1, 10 ** 6, len(cells)).astype(np.uint32)
    E = synth.random_field(ph, seed=4, amp=3e6)
    for sp in (1, 2):
        xo, yo, zo, cell = oracle_mod.push_species(p, sp, X[0], X[1], X[2], E)
        assert np.array_equal(xo, X[0]) and np.array_equal(yo, X[1]) and np.array_equal(zo, X[2])
        assert np.array_equal(cell, cells)
    ne, cnt = oracle_mod.deposit(p, X[0], X[1], X[2], w, cells)
    N = np.zeros(n ** 3, np.int64)
    N[cells] = w
    assert np.array_equal(cnt, N)
    assert np.array_equal(ne, N << (3 * ph["frac_bits"]))


def _mobile_state(oracle_mod, ph, seed=3, interior=False, sigma=1.2e-3):
    """Electrons: a Gaussian blob; positive ions: one per electron particle at
    its position (pairs) plus scattered ions; negative ions scattered (with
    ``interior`` only in cells two or more cells from every face)."""
    p = oracle_mod.make_params(ph, seed=1)
    e = oracle_mod.canonical(p, synth.blob_state(ph, seed=seed, sigma=sigma, peak=5e18, zfrac=0.5))
    cells = None
    if interior:
        n = ph["n"]
        c = np.arange(n ** 3)
        ijk = np.stack([c % n, (c // n) % n, c // (n * n)])
        c = c[np.all((ijk >= 2) & (ijk <= n - 3), axis=0)]
        cells = c[np.random.default_rng(seed).random(len(c)) < 0.3]
    bg = synth.ion_particles(ph, seed=seed + 1, mean=4000, frac=0.3, cells=cells)
    pos = oracle_mod.canonical(p, {k: np.concatenate([e[k], bg[k]]) for k in ("x", "y", "z", "w")})
    neg = oracle_mod.canonical(p, synth.ion_particles(ph, seed=seed + 2, mean=3000, frac=0.3, cells=cells))
    return {"e": e, "pos": pos, "neg": neg}


def _W(S):
    return int(np.asarray(S["w"], np.int64).sum())


@pytest.mark.parametrize("recomb", [False, True])
def test_mobile_steps_keep_charge_and_species_books(oracle_mod, recomb):
    """Whole steps with mobile ions (explicit coupling, photons on; with and
    without the air recombination coefficients): the net charge
    W+ - W- - We changes only by the weights that left the box (electrons
    and negative ions raise it, positive ions lower it); each ion species
    changes by exactly its KMC balance (positive: n_ion - n_ep - n_np plus
    the absorbed photons; negative: n_att - n_np) minus its outflow; weights
    stay positive and every cell holds at most ppc particles per species."""
    ph = _phys(16, dt=5e-12, photon_ratio=0.06, mu_ion=2e-2)
    if recomb:
        ph = synth.with_recombination(ph)
        ph["beta_ep"] *= 1e3
        ph["beta_np"] *= 1e3
    S = _mobile_state(oracle_mod, ph)
    E = synth.random_field(ph, seed=3, amp=2e6, base=4e6)
    n3 = ph["n"] ** 3
    for k in range(2):
        p = oracle_mod.make_params(ph, seed=8, step=k)
        W0 = {s: _W(S[s]) for s in ("e", "pos", "neg")}
        S, info = oracle_mod.step_mobile(p, S, E)
        W1 = {s: _W(S[s]) for s in ("e", "pos", "neg")}
        out = info["outflow"]
        q0 = W0["pos"] - W0["neg"] - W0["e"]
        q1 = W1["pos"] - W1["neg"] - W1["e"]
        assert q1 - q0 == out["e"] + out["neg"] - out["pos"]
        absorbed = int(info["n_ph"].sum()) - info["lost_photon"]
        assert W1["pos"] - W0["pos"] == int((info["n_ion"] - info["n_ep"] - info["n_np"]).sum()) + absorbed - out["pos"]
        assert W1["neg"] - W0["neg"] == int((info["n_att"] - info["n_np"]).sum()) - out["neg"]
        for s in ("e", "pos", "neg"):
            assert np.all(S[s]["w"] > 0)
            assert np.bincount(S[s]["cell"], minlength=n3).max() <= ph["ppc"]
        assert info["n_ion"].sum() > 0 and absorbed > 0
        if recomb:
            assert info["n_ep"].sum() > 0 and info["n_np"].sum() > 0
        # the charge the field sees: CIC densities of the three species
        assert np.array_equal(info["rho_fixed"], info["fix"]["pos"] - info["fix"]["neg"] - info["fix"]["e"])


def test_ions_move_by_the_drift_over_steps(oracle_mod):
    """With a large ion mobility the positive and negative ion clouds move in
    opposite directions along E over a few steps, by mu_ion E dt per step in
    the mean (weight-averaged centroid, to within the diffusion spread and
    the merge's centroid-preserving reshuffle)."""
    E0 = 4e6
    ph = _phys(16, dt=5e-11, photon_ratio=0.0, mu_ion=0.2, eta=0.0, alpha_A=0.0)
    S = _mobile_state(oracle_mod, ph, interior=True, sigma=5e-4)
    E = _uniform_field(ph, (0.0, 0.0, -E0))

    def zc(T):
        w = np.asarray(T["w"], np.float64)
        return float((w * T["z"]).sum() / w.sum())
    z0 = {s: zc(S[s]) for s in ("pos", "neg")}
    steps = 3
    for k in range(steps):
        S, info = oracle_mod.step_mobile(oracle_mod.make_params(ph, seed=8, step=k), S, E)
        assert info["outflow"]["pos"] == 0 and info["outflow"]["neg"] == 0
    dz = steps * ph["mu_ion"] * E0 * ph["dt"]
    assert abs((zc(S["pos"]) - z0["pos"]) - (-dz)) < 0.05 * dz
    assert abs((zc(S["neg"]) - z0["neg"]) - dz) < 0.05 * dz
