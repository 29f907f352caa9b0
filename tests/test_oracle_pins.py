"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against an independent fact -- a published
known-answer vector, a closed form, an invariant, a textbook special case or a
brute-force enumeration -- never against a retyped copy of its own formula.
All run on the CPU (no GPU marker).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from paper_2307_01797_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ RNG
def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle_mod.philox(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_uniforms_open_interval_and_uniform(oracle_mod):
    u = oracle_mod.uniform_draws(1, 7, 3, oracle_mod.TAG_PUSH, 0, 200000)
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # streams with different counters are uncorrelated
    v = oracle_mod.uniform_draws(1, 8, 3, oracle_mod.TAG_PUSH, 0, 200000)
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.02
    w = oracle_mod.uniform_draws(2, 7, 3, oracle_mod.TAG_PUSH, 0, 200000)
    assert abs(np.corrcoef(u, w)[0, 1]) < 0.02


# ------------------------------------------------------------------ math
def _ulp_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.spacing(np.maximum(np.abs(b), 1e-300))


def test_log_accuracy(oracle_mod):
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.random(20000), 10.0 ** rng.uniform(-300, 300, 20000),
                         1.0 + rng.uniform(-1e-6, 1e-6, 2000), [2.0 ** -53, 1.0 - 2.0 ** -53, 5e-324]])
    got = np.array([oracle_mod.log(x) for x in xs])
    ref = np.log(xs)
    err = _ulp_err(got, ref)
    assert err.max() <= 2.0, err.max()
    assert oracle_mod.log(1.0) == 0.0


def test_exp_accuracy(oracle_mod):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(-745, 709, 20000), rng.uniform(-1, 1, 5000), [0.0, -1e-300]])
    got = np.array([oracle_mod.exp(x) for x in xs])
    ref = np.exp(xs)
    normal = ref > 2.3e-308
    assert _ulp_err(got[normal], ref[normal]).max() <= 2.0
    assert np.all(np.abs(got[~normal] - ref[~normal]) <= 2 * 5e-324)
    assert oracle_mod.exp(-800.0) == 0.0


def test_sincos2pi_accuracy(oracle_mod):
    rng = np.random.default_rng(2)
    us = np.concatenate([rng.random(20000), [0.125, 0.25, 0.5, 0.75, 2.0 ** -53]])
    sc = np.array([oracle_mod.sincos2pi(u) for u in us])
    # reference in extended precision: 2 pi u is not exact in double
    pi_ld = np.longdouble("3.14159265358979323846264338327950288")
    ang = 2 * pi_ld * us.astype(np.longdouble) if np.finfo(np.longdouble).eps < 1e-17 else None
    if ang is None:
        pytest.skip("no extended precision long double on this host")
    ref_s = np.sin(ang).astype(np.float64)
    ref_c = np.cos(ang).astype(np.float64)
    for got, ref in ((sc[:, 0], ref_s), (sc[:, 1], ref_c)):
        err = np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), 0.5))
        assert err.max() <= 2.0, err.max()
    assert np.allclose(sc[:, 0] ** 2 + sc[:, 1] ** 2, 1.0, atol=1e-15)
    assert sc[-2][0] == -1.0 and sc[-3][1] == -1.0  # u = 3/4 and u = 1/2 exactly


# ------------------------------------------------------------------ Poisson
@pytest.mark.parametrize("mu", [0.3, 2.5, 9.99, 10.0, 37.5, 1.0e3, 2.0e6])
def test_poisson_sampler_law(oracle_mod, mu):
    n = 40000
    k = oracle_mod.poisson_draws(5, 11, 0, oracle_mod.TAG_KMC, 0, mu, n)
    assert k.min() >= 0
    m, v = k.mean(), k.var()
    assert abs(m - mu) < 5 * math.sqrt(mu / n)
    assert abs(v - mu) < 6 * mu * math.sqrt(2.0 / n) + 5 * math.sqrt(mu / n)
    # chi-square against the Poisson pmf on the central bins
    lo, hi = stats.poisson.ppf(1e-4, mu), stats.poisson.ppf(1 - 1e-4, mu)
    if mu > 100:  # bin widths of about a tenth of a standard deviation
        edges = np.linspace(lo, hi + 1, 60).round()
    else:
        edges = np.arange(lo, hi + 2)
    edges = np.unique(edges)
    obs, _ = np.histogram(k, bins=edges)
    cdf = stats.poisson.cdf(edges - 1, mu)
    exp_ = n * np.diff(cdf)
    keep = exp_ > 20
    chi2 = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
    dof = keep.sum() - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)


def test_poisson_zero_mean(oracle_mod):
    assert np.all(oracle_mod.poisson_draws(1, 0, 0, oracle_mod.TAG_KMC, 0, 0.0, 10) == 0)


# ------------------------------------------------------------------ push
def _phys_small(n=16, **kw):
    ph = synth.physics_small(n)
    ph.update(kw)
    return ph


def test_ziggurat_normals_follow_the_standard_normal(oracle_mod):
    """The push normals (ziggurat method, Marsaglia & Tsang 2000) are N(0, 1):
    Kolmogorov-Smirnov against the normal CDF, the first four moments, and the
    probability of the tail beyond the base strip r and beyond 4."""
    from scipy import stats
    x = oracle_mod.normal_draws(11, 5, 2, 2, 0, 400000)
    assert stats.kstest(x, "norm").pvalue > 1e-3
    n = len(x)
    assert abs(x.mean()) < 5 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.skew(x)) < 5 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(x)) < 5 * math.sqrt(24.0 / n)
    for t in (3.442619855899, 4.0):
        p = 2 * stats.norm.sf(t)
        assert abs((np.abs(x) > t).mean() - p) < 5 * math.sqrt(p / n)
    # symmetric sign and independent successive draws
    assert abs((x > 0).mean() - 0.5) < 5 * 0.5 / math.sqrt(n)
    assert abs(np.corrcoef(x[:-1], x[1:])[0, 1]) < 5 / math.sqrt(n)


def test_push_free_cloud_moments(oracle_mod):
    """Eq. ensemble_averages: <dX> = v dt, <|dX - v dt|^2> = 2 D d dt, with
    v = -mu E for electrons (Eq. Vk1, sgn = -1).  Uniform E = -E0 z."""
    ph = _phys_small(16)
    p = oracle_mod.make_params(ph, seed=3)
    N = 200000
    L = ph["hi"][0]
    x = np.full(N, 0.5 * L + 1e-6); y = np.full(N, 0.5 * L - 2e-6); z = np.full(N, 0.5 * L + 3e-6)
    E = synth.uniform_field(ph, -ph["E0"])
    xo, yo, zo, cell = oracle_mod.push(p, x, y, z, E)
    assert np.all(cell >= 0)
    d = np.stack([xo - x, yo - y, zo - z])
    v = np.array([0.0, 0.0, ph["mu"] * ph["E0"]])
    sd = math.sqrt(2 * ph["D"] * ph["dt"])
    for a in range(3):
        assert abs(d[a].mean() - v[a] * ph["dt"]) < 5 * sd / math.sqrt(N)
        var = ((d[a] - v[a] * ph["dt"]) ** 2).mean()
        assert abs(var / sd ** 2 - 1.0) < 5 * math.sqrt(2.0 / N)
    tot = ((d - (v * ph["dt"])[:, None]) ** 2).sum(0).mean()
    assert abs(tot / (2 * ph["D"] * 3 * ph["dt"]) - 1.0) < 5 * math.sqrt(2.0 / (3 * N))
    # independent normals across axes
    assert abs(np.corrcoef(d[0], d[1])[0, 1]) < 0.02
    assert abs(np.corrcoef(d[1], d[2])[0, 1]) < 0.02


def test_push_interpolates_linear_field_exactly(oracle_mod):
    """Trilinear interpolation reproduces any field linear in x, y, z at
    interior points; with D = 0 the push is x' = x - mu E(x) dt."""
    ph = _phys_small(16, D=0.0, dt=1e-9)
    p = oracle_mod.make_params(ph, seed=1)
    n = ph["n"]
    h = synth.cell_size(ph)
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    coef = np.array([[1e5, 2e7, -3e7, 5e6], [-2e5, 1e6, 4e7, -2e7], [3e5, -5e6, 2e6, 3e7]])
    E = tuple(coef[a, 0] + coef[a, 1] * X + coef[a, 2] * Y + coef[a, 3] * Z for a in range(3))
    st = synth.random_particles(ph, 5000, seed=4, margin=0.6)
    xo, yo, zo, cell = oracle_mod.push(p, st["x"], st["y"], st["z"], E)
    P = np.stack([st["x"], st["y"], st["z"]])
    Ep = coef[:, :1] + coef[:, 1:] @ P
    expect = P - ph["mu"] * Ep * ph["dt"]
    got = np.stack([xo, yo, zo])
    assert np.max(np.abs(got - expect)) < 1e-15


def test_push_boundary_clamp_is_constant_extrapolation(oracle_mod):
    """In the half cell next to a wall the stencil folds onto the wall cell."""
    ph = _phys_small(8, D=0.0, dt=1e-10)
    p = oracle_mod.make_params(ph, seed=1)
    n = ph["n"]
    h = synth.cell_size(ph)
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    Ex = 1e6 * (1.0 + X / h)
    E = (Ex, np.zeros_like(Ex), np.zeros_like(Ex))
    x = np.array([0.1 * h, 0.3 * h, (n - 0.2) * h]); y = np.full(3, 3.5 * h); z = np.full(3, 3.5 * h)
    xo, _, _, _ = oracle_mod.push(p, x, y, z, E)
    Eb = np.array([1e6 * 1.5, 1e6 * 1.5, 1e6 * (1 + n - 0.5)])
    assert np.allclose(xo - x, -ph["mu"] * Eb * ph["dt"], rtol=1e-14, atol=0)


def test_push_removal_at_faces(oracle_mod):
    ph = _phys_small(8, D=0.0, dt=1e-9)
    p = oracle_mod.make_params(ph, seed=1)
    L = ph["hi"][0]
    h = synth.cell_size(ph)
    # E large enough to move 0.2 mm in one step: particles near z=L leave
    Ez = -0.2e-3 / (ph["mu"] * ph["dt"])
    E = synth.uniform_field(ph, Ez)
    z = np.array([L - 0.1e-3, L - 0.3e-3, 0.5 * L])
    x = np.full(3, 0.5 * L); y = np.full(3, 0.5 * L)
    xo, yo, zo, cell = oracle_mod.push(p, x, y, z, E)
    assert cell[0] == -1 and cell[1] >= 0 and cell[2] >= 0
    k = int((zo[1] / h))
    assert cell[1] // (8 * 8) == k


# ------------------------------------------------------------------ sort
def test_sort_is_stable_permutation(oracle_mod):
    rng = np.random.default_rng(3)
    cell = rng.integers(-1, 50, size=10000)
    perm = oracle_mod.sort_by_cell(cell, 50)
    ref = np.argsort(np.where(cell < 0, 10 ** 9, cell), kind="stable")[: (cell >= 0).sum()]
    assert np.array_equal(perm, ref)


# ------------------------------------------------------------------ deposit
def test_deposit_centre_and_corner(oracle_mod):
    ph = _phys_small(8)
    p = oracle_mod.make_params(ph, seed=1)
    h = synth.cell_size(ph)
    s = ph["frac_bits"]
    # particle at the centre of cell (3,4,5): all weight in that cell
    x = np.array([3.5 * h]); y = np.array([4.5 * h]); z = np.array([5.5 * h])
    w = np.array([7], dtype=np.uint32)
    cell = np.array([(5 * 8 + 4) * 8 + 3])
    ne, Xe = oracle_mod.deposit(p, x, y, z, w, cell)
    assert ne[cell[0]] == 7 << (3 * s) and ne.sum() == 7 << (3 * s)
    assert Xe[cell[0]] == 7 and Xe.sum() == 7
    # particle on the corner shared by cells (3..4, 4..5, 5..6): 1/8 each
    x = np.array([4.0 * h]); y = np.array([5.0 * h]); z = np.array([6.0 * h])
    ne, _ = oracle_mod.deposit(p, x, y, z, w, np.array([(6 * 8 + 5) * 8 + 4]))
    nz = np.nonzero(ne)[0]
    assert len(nz) == 8 and np.all(ne[nz] == 7 << (3 * s - 3))
    ks, js, is_ = nz // 64, (nz // 8) % 8, nz % 8
    assert set(is_) == {3, 4} and set(js) == {4, 5} and set(ks) == {5, 6}


def test_deposit_conserves_and_has_correct_first_moment(oracle_mod):
    """Sum = 2^3s sum w exactly; the deposited charge's centroid per particle
    equals the particle position to within the 2^-s quantisation (a CIC
    property that fails for swapped weights or axes)."""
    ph = _phys_small(16)
    p = oracle_mod.make_params(ph, seed=1)
    n = ph["n"]
    s = ph["frac_bits"]
    h = synth.cell_size(ph)
    st = synth.random_particles(ph, 3000, seed=9, margin=0.6)
    ix = np.floor(st["x"] / h).astype(np.int64); iy = np.floor(st["y"] / h).astype(np.int64)
    iz = np.floor(st["z"] / h).astype(np.int64)
    cell = (iz * n + iy) * n + ix
    ne, Xe = oracle_mod.deposit(p, st["x"], st["y"], st["z"], st["w"], cell)
    W = int(st["w"].astype(np.int64).sum())
    assert int(ne.sum()) == W << (3 * s)
    assert int(Xe.sum()) == W
    for q in range(0, 3000, 97):
        one = {k: st[k][q:q + 1] for k in st}
        ne1, _ = oracle_mod.deposit(p, one["x"], one["y"], one["z"], one["w"], cell[q:q + 1])
        idx = np.nonzero(ne1)[0]
        cen = np.stack([(idx % n + 0.5) * h, ((idx // n) % n + 0.5) * h, (idx // (n * n) + 0.5) * h])
        m = (cen * ne1[idx]).sum(1) / ne1[idx].sum()
        assert np.max(np.abs(m - np.array([one["x"][0], one["y"][0], one["z"][0]]))) <= h * 2.0 ** -s


# ------------------------------------------------------------------ KMC
def test_kmc_leap_mean_and_variance_discrete_closed_form(oracle_mod):
    """X0 = 1e6, no critical reactions, eps = inf: every step is one leap
    over dt, so E X_k = X0 (1 + (ka - ke) dt)^k (the discrete growth of
    Sec. 2, W^k = (1 + alpha v dt)^k), Var via v' = a^2 v + b m."""
    ph = _phys_small(8, dt=1e-12)
    ka, ke = 3.0e10, 1.0e10
    X0, K, R = 10 ** 6, 4, 3000
    finals = np.zeros(R)
    for r in range(R):
        X = X0
        for k in range(K):
            p = oracle_mod.make_params(ph, seed=11, step=k)
            X, fired = oracle_mod.kmc_single(p, X, ka, ke, 0.0, index=r)
            assert X >= 0
        finals[r] = X
    a = 1 + (ka - ke) * ph["dt"]
    b = (ka + ke) * ph["dt"]
    m, v = float(X0), 0.0
    for _ in range(K):
        v = a * a * v + b * m
        m = a * m
    assert abs(finals.mean() - m) < 5 * math.sqrt(v / R)
    assert abs(finals.var() / v - 1.0) < 5 * math.sqrt(2.0 / R)


def test_kmc_finite_eps_follows_the_yule_process(oracle_mod):
    """Finite eps (Sec. 3.2.3 step 4, the Cao step bound): a pure birth
    process over lambda dt = 1 is split into substeps of relative change
    ~eps, so the final count approaches the exact Yule law, mean X0 e and
    variance X0 e (e - 1), to a bias of order eps; one eps = inf leap has mean
    X0 (1 + lambda dt) = 2 X0 instead."""
    ph = _phys_small(8, dt=1e-12)
    lam = 1.0 / ph["dt"]
    X0, R = 2000, 400

    def finals(eps):
        p = oracle_mod.make_params(dict(ph, eps=eps), seed=21, step=0)
        return np.array([oracle_mod.kmc_single(p, X0, lam, 0.0, 0.0, index=r)[0] for r in range(R)],
                        dtype=np.float64)

    mean_y, var_y = X0 * math.e, X0 * math.e * (math.e - 1.0)
    f = finals(0.03)
    se = math.sqrt(var_y / R)
    assert 0.95 * mean_y < f.mean() < mean_y + 5 * se
    assert abs(f.var() / var_y - 1.0) < 0.25
    g = finals(float("inf"))
    assert abs(g.mean() - 2 * X0) < 5 * math.sqrt(2 * X0 / R) + 1


def test_kmc_birth_death_small_numbers_kendall(oracle_mod):
    """From one electron with A dt << 1 the hybrid runs the exact SSA/critical
    branches: mean and extinction probability of a linear birth-death process
    (Kendall 1948): E X = e^{lt}, P0 = m(e^{lt}-1)/(b e^{lt} - m), l = b - m."""
    ph = _phys_small(8, dt=2e-12)
    bi, de = 2.0e10, 1.0e10
    K, R = 50, 8000
    finals = np.zeros(R, dtype=np.int64)
    for r in range(R):
        X = 1
        for k in range(K):
            if X == 0:
                break
            p = oracle_mod.make_params(ph, seed=5, step=k)
            X, _ = oracle_mod.kmc_single(p, X, bi, de, 0.0, index=r)
        finals[r] = X
    t = K * ph["dt"]
    lam = bi - de
    e = math.exp(lam * t)
    p0 = de * (e - 1) / (bi * e - de)
    var = (bi + de) / lam * e * (e - 1)
    assert abs(finals.mean() - e) < 5 * math.sqrt(var / R)
    assert abs((finals == 0).mean() - p0) < 5 * math.sqrt(p0 * (1 - p0) / R)


def test_kmc_non_negative_and_conserving(oracle_mod):
    ph = _phys_small(8, dt=5e-11)
    rng = np.random.default_rng(4)
    for r in range(3000):
        X0 = int(rng.integers(1, 40))
        p = oracle_mod.make_params(ph, seed=2, step=r)
        X, fired = oracle_mod.kmc_single(p, X0, 1e9, 3e11, 2e9, index=r)
        assert X >= 0
        assert X == X0 + fired[0] - fired[1]
        assert fired.min() >= 0


def test_kmc_rre_limit(oracle_mod):
    """Large X, small dt: the mean follows the RRE X0 exp((ka-ke) t) (Eq. rre)."""
    ph = _phys_small(8, dt=1e-13)
    ka, ke = 5e10, 1e10
    X0, K, R = 10 ** 7, 20, 200
    vals = []
    for r in range(R):
        X = X0
        for k in range(K):
            X, _ = oracle_mod.kmc_single(oracle_mod.make_params(ph, seed=9, step=k), X, ka, ke, 0.0, r)
        vals.append(X)
    rre = X0 * math.exp((ka - ke) * K * ph["dt"])
    assert abs(np.mean(vals) / rre - 1.0) < 2e-3


# ------------------------------------------------------------------ products / photons
def _one_cell_state(ph, cell_ijk, weights, seed=0):
    n = ph["n"]
    h = synth.cell_size(ph)
    rng = np.random.default_rng(seed)
    i, j, k = cell_ijk
    m = len(weights)
    x = (i + rng.random(m)) * h; y = (j + rng.random(m)) * h; z = (k + rng.random(m)) * h
    c = np.full(m, (k * n + j) * n + i, dtype=np.int64)
    return x, y, z, np.asarray(weights, dtype=np.uint32), c


def test_products_weight_rule_and_paper_mean_weight(oracle_mod):
    gold = json.load(open(os.path.join(GOLD, "paper_values.json")))
    ph = _phys_small(8)
    n = ph["n"]
    h = synth.cell_size(ph)
    p = oracle_mod.make_params(ph, seed=4, step=2)
    x, y, z, w, c = _one_cell_state(ph, (2, 3, 4), [10])
    nc = n ** 3
    Xe = np.zeros(nc, np.int64); Xe[c[0]] = 10
    for dN, m_exp in [(1000, 64), (10, 10), (64, 64), (65, 64)]:
        ion = np.zeros(nc, np.int64); ion[c[0]] = dN
        zero = np.zeros(nc, np.int64)
        Np, Nn = np.zeros(nc, np.int64), np.zeros(nc, np.int64)
        new, lost = oracle_mod.products_photons(p, x, y, z, w.copy(), c, Xe, (ion, zero, zero), Np, Nn)
        nx, ny, nz, nw, ncell = new
        assert len(nw) == m_exp
        assert int(nw.astype(np.int64).sum()) == dN
        assert nw[0] == dN // m_exp + dN % m_exp and np.all(nw[1:] == dN // m_exp)
        assert np.all(ncell == c[0]) and Np[c[0]] == dN and Nn.sum() == 0
        for arr, lo_ in ((nx, 2 * h), (ny, 3 * h), (nz, 4 * h)):
            assert np.all(arr >= lo_) and np.all(arr <= lo_ + h)
    g = gold["mean_weight_streamer_head"]
    N = round(g["n_e"] * g["dx"] ** 3)
    assert abs((N / g["ppc"]) / g["w"] - 1.0) < g["rel_tol"]
    assert N // g["ppc"] in (15, 16)
    g2 = gold["mean_weight_sprite"]
    assert abs(g2["n_e"] * g2["dx"] ** 3 / g2["ppc"] / g2["w"] - 1.0) < g2["rel_tol"]


def test_loss_removal_exact_and_unbiased(oracle_mod):
    ph = _phys_small(8)
    n = ph["n"]
    nc = n ** 3
    weights = np.array([5, 100, 1, 37, 12, 1, 60], dtype=np.uint32)
    W = int(weights.sum())
    L = 70
    x, y, z, _, c = _one_cell_state(ph, (1, 1, 1), weights)
    Xe = np.zeros(nc, np.int64); Xe[c[0]] = W
    att = np.zeros(nc, np.int64); att[c[0]] = L
    zero = np.zeros(nc, np.int64)
    acc = np.zeros(len(weights))
    R = 3000
    for r in range(R):
        p = oracle_mod.make_params(ph, seed=100 + r, step=0)
        w = weights.copy()
        Np, Nn = np.zeros(nc, np.int64), np.zeros(nc, np.int64)
        new, _ = oracle_mod.products_photons(p, x, y, z, w, c, Xe, (zero, att, zero), Np, Nn)
        assert len(new[3]) == 0
        loss = weights.astype(np.int64) - w.astype(np.int64)
        assert loss.sum() == L and np.all(loss >= 0) and np.all(loss <= weights)
        assert Nn[c[0]] == L
        acc += loss
    expect = weights * L / W
    sd = np.sqrt(np.maximum(expect * (1 - expect / np.maximum(weights, 1)), 1e-3) / R) + 0.02
    assert np.all(np.abs(acc / R - expect) < 6 * sd)


def test_photon_sampler_laws(oracle_mod):
    gold = json.load(open(os.path.join(GOLD, "paper_values.json")))["zheleznyak_kappa"]
    ph = _phys_small(8, kappa_lo=gold["K1"], kappa_hi=gold["K2"], photon_ratio=0.06)
    m = 40000
    Y0s, ks, rs, ds = [], [], [], []
    for step in range(m // 64):
        p = oracle_mod.make_params(ph, seed=3, step=step)
        Y0, k, r, d = oracle_mod.photon_samples(p, 2, 5, 6, 64)
        Y0s.append(Y0); ks.append(k); rs.append(r); ds.append(d)
    Y0 = np.concatenate(Y0s); k = np.concatenate(ks); r = np.concatenate(rs); d = np.concatenate(ds)
    K1, K2 = gold["K1"], gold["K2"]
    t = (np.log(k) - math.log(K1)) / math.log(K2 / K1)
    assert stats.kstest(t, "uniform").pvalue > 1e-4
    assert k.min() >= K1 and k.max() <= K2
    Er = (1 / K1 - 1 / K2) / math.log(K2 / K1)
    assert abs(r.mean() / Er - 1) < 0.03
    # r | kappa is exponential: kappa r ~ Exp(1)
    assert stats.kstest(k * r, "expon").pvalue > 1e-4
    assert np.allclose((d ** 2).sum(1), 1.0, atol=1e-14)
    assert stats.kstest((d[:, 2] + 1) / 2, "uniform").pvalue > 1e-4
    phi = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-4
    assert np.all(np.abs(d.mean(0)) < 0.02)
    h = synth.cell_size(ph)
    for a, i in enumerate((2, 5, 6)):
        assert np.all(Y0[:, a] >= i * h) and np.all(Y0[:, a] <= (i + 1) * h)


def test_photoionization_charge_and_counts(oracle_mod):
    """Absorbed photons add e + M+ in the absorption cell; lost ones leave the
    box; total weight of emitted superphotons = number of photon events."""
    ph = _phys_small(16, photon_ratio=0.06)
    n = ph["n"]
    nc = n ** 3
    p = oracle_mod.make_params(ph, seed=8, step=1)
    x, y, z, w, c = _one_cell_state(ph, (8, 8, 8), [1000])
    Xe = np.zeros(nc, np.int64); Xe[c[0]] = 1000
    phot = np.zeros(nc, np.int64); phot[c[0]] = 5000
    zero = np.zeros(nc, np.int64)
    Np, Nn = np.zeros(nc, np.int64), np.zeros(nc, np.int64)
    new, lost = oracle_mod.products_photons(p, x, y, z, w, c, Xe, (zero, zero, phot), Np, Nn)
    nx, ny, nz, nw, ncell = new
    assert len(nw) <= 64
    assert int(nw.astype(np.int64).sum()) + lost == 5000
    assert int(Np.sum()) == int(nw.astype(np.int64).sum())
    for q in range(len(nw)):
        assert Np[ncell[q]] >= nw[q]
    h = synth.cell_size(ph)
    cc = ((nz // h).astype(np.int64) * n + (ny // h).astype(np.int64)) * n + (nx // h).astype(np.int64)
    assert np.array_equal(cc, ncell)


# ------------------------------------------------------------------ merge/split
def test_merge_paper_example(oracle_mod):
    """Sec. 4.6 / Fig. BVH: 1000 particles, w uniform on [1,100], -> 64 leaves
    whose weights differ by at most one; weight and first moment conserved."""
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["merge_example"]
    rng = np.random.default_rng(12)
    M = g["M"]
    x, y, z = rng.random(M), rng.random(M), rng.random(M)
    w = rng.integers(g["wmin"], g["wmax"] + 1, size=M).astype(np.uint64)
    ox, oy, oz, ow = oracle_mod.merge_list(x, y, z, w, g["ppc"])
    assert len(ow) == g["ppc"]
    assert int(ow.max()) - int(ow.min()) <= g["max_weight_spread"]
    assert int(ow.sum()) == int(w.sum())
    W = float(w.sum())
    for a, b in ((x, ox), (y, oy), (z, oz)):
        assert abs((w * a).sum() / W - (ow * b).sum() / W) < 1e-13
        assert b.min() >= a.min() and b.max() <= a.max()


def _bruteforce_split(X, w):
    """Eq. weight_median by enumeration: sorted order along the widest axis,
    smallest p' with sum_{<p'} + w_p' > sum_{>p'}; returns (W_left, W_right)."""
    ext = X.max(0) - X.min(0)
    ax = int(np.argmax(ext))
    order = np.argsort(X[:, ax], kind="stable")
    ws = w[order]
    W = int(ws.sum())
    for pp in range(len(ws)):
        left = int(ws[:pp].sum()); right = int(ws[pp + 1:].sum())
        if left + ws[pp] > right:
            break
    if ws[pp] == 1:
        return (left + 1, right) if left <= right else (left, right + 1)
    return (W + 1) // 2, W // 2


def test_merge_single_split_bruteforce(oracle_mod):
    rng = np.random.default_rng(5)
    for trial in range(400):
        M = int(rng.integers(1, 7))
        X = rng.random((M, 3))
        w = rng.integers(1, 6, size=M).astype(np.uint64)
        if w.sum() < 2:
            continue
        ox, oy, oz, ow = oracle_mod.merge_list(X[:, 0], X[:, 1], X[:, 2], w, 2)
        assert len(ow) == 2
        assert (int(ow[0]), int(ow[1])) == _bruteforce_split(X, w)


def test_merge_splits_heavy_particle_and_small_weights(oracle_mod):
    ox, oy, oz, ow = oracle_mod.merge_list([0.3], [0.4], [0.5], [1000], 64)
    assert len(ow) == 64 and ow.sum() == 1000 and ow.max() - ow.min() <= 1
    assert np.all(ox == 0.3) and np.all(oy == 0.4) and np.all(oz == 0.5)
    ox, oy, oz, ow = oracle_mod.merge_list([0.1, 0.2, 0.9], [0.1] * 3, [0.1] * 3, [2, 1, 2], 8)
    assert len(ow) == 5 and np.all(ow == 1)


# ------------------------------------------------------------------ Poisson (field)
def test_poisson_zero_charge_gives_linear_potential(oracle_mod):
    from oracle import poisson
    ph = _phys_small(16)
    n = ph["n"]
    phi, (Ex, Ey, Ez) = poisson.solve(np.zeros(n ** 3, np.int64), ph)
    h = synth.cell_size(ph)
    zc = (np.arange(n) + 0.5) * h
    assert np.allclose(phi, ph["E0"] * zc[:, None, None], rtol=0, atol=1e-9 * ph["E0"] * ph["hi"][2])
    assert np.allclose(Ez, -ph["E0"], rtol=1e-10)
    assert np.max(np.abs(Ex)) < 1e-6 * ph["E0"] and np.max(np.abs(Ey)) < 1e-6 * ph["E0"]


def test_poisson_manufactured_second_order(oracle_mod):
    from oracle import poisson
    L = 0.01
    A = 100.0
    errs = []
    for n in (16, 32):
        h = L / n
        c = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        exact = A * np.cos(np.pi * X / L) * np.cos(np.pi * Y / L) * np.sin(np.pi * Z / L)
        lap = -3 * (np.pi / L) ** 2 * exact
        phi = poisson.solve_b(lap, h)
        errs.append(np.max(np.abs(phi - exact)))
    order = math.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.3, errs


def test_poisson_residual_of_random_charge(oracle_mod):
    from oracle import poisson
    ph = _phys_small(16)
    n = ph["n"]
    h = synth.cell_size(ph)
    rng = np.random.default_rng(8)
    rho = rng.integers(-(1 << 40), 1 << 40, size=n ** 3)
    phi, _ = poisson.solve(rho, ph)
    top = ph["E0"] * ph["hi"][2]
    b = poisson.rhs(rho, n, h, ph["frac_bits"], top)
    # apply_operator includes the boundary values; compare with b without them
    b_no_bc = b.copy(); b_no_bc[n - 1] += 2.0 * top / (h * h)
    r = poisson.apply_operator(phi, h, top) - b_no_bc
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


# ------------------------------------------------------------------ whole step
def test_whole_step_invariants(oracle_mod):
    """Charge sum(N+ - N-) - sum(w) changes only by the outflow; every cell
    ends with at most ppc particles of balanced weight; no negative counts."""
    ph = _phys_small(16, photon_ratio=0.06, dt=5e-12)
    ph["ppc"] = 8
    st = synth.blob_state(ph, seed=2, sigma=1.2e-3, peak=5e18, zfrac=0.6)
    n = ph["n"]
    h = synth.cell_size(ph)
    ix = np.floor(st["x"] / h).astype(np.int64); iy = np.floor(st["y"] / h).astype(np.int64)
    iz = np.floor(st["z"] / h).astype(np.int64)
    st["cell"] = (iz * n + iy) * n + ix
    order = np.argsort(st["cell"], kind="stable")
    st = {k: v[order] for k, v in st.items()}
    st["Npos"] = np.zeros(n ** 3, np.int64); st["Nneg"] = np.zeros(n ** 3, np.int64)
    E = synth.random_field(ph, seed=3, amp=2e6, base=4e6)
    Q = int((st["Npos"] - st["Nneg"]).sum()) - int(st["w"].astype(np.int64).sum())
    out_cum = 0
    for k in range(3):
        p = oracle_mod.make_params(ph, seed=21, step=k)
        st, info = oracle_mod.step(p, st, E)
        out_cum += info["outflow"]
        Qk = int((st["Npos"] - st["Nneg"]).sum()) - int(st["w"].astype(np.int64).sum())
        assert Qk == Q + out_cum
        assert np.all(np.diff(st["cell"]) >= 0)
        cnt = np.bincount(st["cell"], minlength=n ** 3)
        assert cnt.max() <= ph["ppc"]
        assert st["Npos"].min() >= 0 and st["Nneg"].min() >= 0
        assert int(info["n_ion"].sum()) > 0
        # rho snapshot integrates to the charge before this step's chemistry
        # (summed as Python integers: the domain total exceeds int64)
        assert sum(int(v) for v in info["rho_fixed"]) == (Q + out_cum) << (3 * ph["frac_bits"])


def test_kmc_rates_breakdown_field(oracle_mod):
    """Ionization and attachment balance where alpha(|E|) = eta, i.e. at
    |E_b| = B / ln(A/eta) (the breakdown field of the 0-D comparison,
    Sec. 3.2.4), whatever the field's direction; at 2 E_b ionization
    outnumbers attachment by alpha/eta = (A/eta)^(1/2)."""
    ph = _phys_small(8, dt=1e-13)
    n = ph["n"]
    Eb = ph["alpha_B"] / math.log(ph["alpha_A"] / ph["eta"])
    p = oracle_mod.make_params(ph, seed=4, step=0)
    Xe = np.full(n ** 3, 10 ** 6, dtype=np.int64)
    for scale, ratio in ((1.0, 1.0), (2.0, math.sqrt(ph["alpha_A"] / ph["eta"]))):
        E = [np.zeros(n ** 3) for _ in range(3)]
        half = n ** 3 // 2
        E[0][:half] = scale * Eb            # field along x in one half ...
        E[2][half:] = -scale * Eb           # ... along -z in the other
        ion, att, ph_ = oracle_mod.kmc(p, Xe, E)[:3]
        for sl in (slice(0, half), slice(half, None)):
            a, b = ion[sl].sum(), att[sl].sum()
            assert abs(a / b - ratio) < 6 * ratio * math.sqrt(1 / a + 1 / b)
        assert ph_.sum() == 0


def test_kmc0d_ensemble_mean_follows_the_rate_equation(oracle_mod):
    """0-D ensembles (Sec. 3.2.4): with every reaction non-critical the
    tau-leap mean after K steps is X0 (1 + (k_ion - k_att) dt)^K exactly
    (the discrete rate equation), so the ensemble mean must lie within the
    sampling error of it; at a field below breakdown the count decays."""
    ph = synth.physics_small(8)
    p = oracle_mod.make_params(ph, seed=4)
    E = 5e6
    ve = ph["mu"] * E
    ka = ph["alpha_A"] * math.exp(-ph["alpha_B"] / E) * ve
    kb = ph["eta"] * ve
    K, X0 = 50, 2000
    X = oracle_mod.kmc0d(p, E, X0, 2000, K)
    mean = X0 * (1 + (ka - kb) * ph["dt"]) ** K
    assert abs(X[:, -1].mean() - mean) < 5 * X[:, -1].std() / math.sqrt(X.shape[0])
    assert np.all(X[:, 0] == X0)
    # below breakdown, A dt < 1: the exact SSA path, mean X0 exp((k_ion - k_att) t)
    E2 = 2e6
    ka2 = ph["alpha_A"] * math.exp(-ph["alpha_B"] / E2) * ph["mu"] * E2
    kb2 = ph["eta"] * ph["mu"] * E2
    Y = oracle_mod.kmc0d(p, E2, 200, 4000, 200)
    mean2 = 200 * math.exp((ka2 - kb2) * 200 * ph["dt"])
    assert mean2 < 200 and abs(Y[:, -1].mean() - mean2) < 5 * Y[:, -1].std() / math.sqrt(Y.shape[0])
