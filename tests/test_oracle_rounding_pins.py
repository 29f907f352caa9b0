"""Pins of the oracle's evaluation choices against their plain definitions.

The oracle fixes some roundings the paper leaves open: the grid quotient
(x - lo)/h is formed from the reciprocal of h with one fused correction, the
CIC interpolation accumulates by fused multiply-adds, and the PTRS acceptance
test of the tau-leap's Poisson draw (Sec. 3.2.3, Eq. tau_leaping) takes one
logarithm.  Each test below checks such a choice against the definition it
stands for, evaluated independently (exact rational arithmetic, IEEE
division, libm's log and lgamma, scipy's Poisson CDF), so that a mistake shared
by the oracle and the kernels (a wrong sign in the correction, a dropped
term) fails here even where the bit-exact GPU tests pass.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from paper_2307_01797_gb300 import synth

GRIDS = [
    # (lo, hi, n): the configs' boxes and cells, and boxes whose lo is not 0
    # and whose cell size is not a short binary fraction
    (0.0, 0.02, 256), (0.0, 0.01, 64), (0.0, 0.04, 512), (-0.013, 0.0071, 48), (0.0031, 0.0197, 40),
]


def _params(oracle_mod, lo, hi, n, s=10):
    ph = synth.physics_small(n)
    ph.update(lo=(lo, lo, lo), hi=(hi, hi, hi), frac_bits=s)
    return oracle_mod.make_params(ph, seed=1)


def _sweep(lo, hi, n, rng, per_face=4, random=20000):
    """Every cell face and every cell centre, each with its neighbours up to
    per_face ulps on both sides, the wall half-cells and random points, all
    inside [lo, hi)."""
    h = (hi - lo) / n
    pts = [lo + k * h for k in range(n + 1)] + [lo + (k + 0.5) * h for k in range(n)]
    out = []
    for p in pts:
        v = p
        for _ in range(per_face + 1):
            out.append(v)
            v = np.nextafter(v, np.inf)
        v = p
        for _ in range(per_face):
            v = np.nextafter(v, -np.inf)
            out.append(v)
    out += list(lo + rng.random(random) * (hi - lo))
    out += list(lo + rng.random(2000) * (0.5 * h))            # lower wall half-cell
    out += list(hi - rng.random(2000) * (0.5 * h))            # upper wall half-cell
    x = np.asarray(out, np.float64)
    return x[(x >= lo) & (x < hi)]


@pytest.mark.parametrize("lo,hi,n", GRIDS)
def test_grid_quotient_is_the_correctly_rounded_quotient(oracle_mod, lo, hi, n):
    """q = (x - lo)/h with the difference and the quotient each rounded once
    (IEEE division), and the cell floor(q), on every face and centre +- a few
    ulps: the reciprocal-plus-correction form must give the same double."""
    rng = np.random.default_rng(n)
    p = _params(oracle_mod, lo, hi, n)
    h = (hi - lo) / n
    for ax in range(3):
        x = _sweep(lo, hi, n, rng)
        g = oracle_mod.grid_axis(p, ax, x)
        plain = (x - lo) / h
        bad = np.flatnonzero(g["q"] != plain)
        assert bad.size == 0, (ax, x[bad[:5]], g["q"][bad[:5]], plain[bad[:5]])
        assert np.array_equal(g["cell"], np.clip(np.floor(plain), 0, n - 1).astype(np.int64))
    # numpy's quotient itself against exact rational arithmetic on a subset
    sub = x[:: max(1, len(x) // 3000)]
    for v in sub:
        d = v - lo
        assert (d / h) == float(Fraction(d) / Fraction(h))


@pytest.mark.parametrize("lo,hi,n", GRIDS)
@pytest.mark.parametrize("s", [10, 6])
def test_cic_fraction_and_fixed_point_weight_from_the_exact_quotient(oracle_mod, lo, hi, n, s):
    """From q: u = q - 1/2, i0 = floor(u), f = u - i0 and a = floor(f 2^s),
    taken in exact rational arithmetic.  Where q >= 1/2 the oracle's FP64 f
    and a must equal the exact ones; below 1/2 (the lower wall's first half
    cell) both CIC indices fold onto cell 0, so only the fold is checked."""
    rng = np.random.default_rng(100 + n)
    p = _params(oracle_mod, lo, hi, n, s)
    x = _sweep(lo, hi, n, rng, per_face=3, random=3000)
    g = oracle_mod.grid_axis(p, 2, x)
    for k in range(len(x)):
        q = Fraction(g["q"][k])
        u = q - Fraction(1, 2)
        i0 = math.floor(u)
        if q >= Fraction(1, 2):
            f = u - i0
            assert Fraction(g["f"][k]) == f, (x[k], g["f"][k], float(f))
            assert g["a"][k] == math.floor(f * 2 ** s)
            assert g["ia"][k] == min(max(i0, 0), n - 1) and g["ib"][k] == min(max(i0 + 1, 0), n - 1)
        else:
            assert i0 == -1 and g["ia"][k] == 0 and g["ib"][k] == 0
        assert 0 <= g["a"][k] < 2 ** s


def _exact_interp(F, n, q3):
    """Exact trilinear interpolation (rational arithmetic) of the cell-centred
    field F at grid quotients q3 = (qx, qy, qz), with the wall fold; returns
    (value, sum of |weight * F|)."""
    idx, wts = [], []
    for q in q3:
        u = Fraction(q) - Fraction(1, 2)
        i0 = math.floor(u)
        f = u - i0
        idx.append((min(max(i0, 0), n - 1), min(max(i0 + 1, 0), n - 1)))
        wts.append((1 - f, f))
    val, mag = Fraction(0), Fraction(0)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                w = wts[0][a] * wts[1][b] * wts[2][c]
                fv = Fraction(F[idx[2][c], idx[1][b], idx[0][a]])
                val += w * fv
                mag += abs(w * fv)
    return val, mag


@pytest.mark.parametrize("signed", [True, False])
def test_interpolation_sum_within_its_rounding_bound(oracle_mod, signed):
    """The fused-multiply-add interpolation (Sec. 4.2, W_cic) against the exact
    trilinear value: |oracle - exact| <= 12 u sum|w F| (two rounded weight
    products and eight accumulations, u = 2^-53); the plain unfused sum obeys
    the same bound.  For a positive field sum|w F| is the exact value itself,
    so the fused sum lies within 10 u |exact|, i.e. at most 5 ulps of it."""
    n, lo, hi = 16, 0.0, 0.01
    p = _params(oracle_mod, lo, hi, n)
    rng = np.random.default_rng(7 if signed else 8)
    F = rng.normal(0.0, 1e6, (n, n, n)) if signed else rng.uniform(1e5, 5e6, (n, n, n))
    m = 3000
    pts = lo + rng.random((m, 3)) * (hi - lo)
    pts[:200, 0] = lo + rng.random(200) * (hi - lo) / (2 * n)          # wall half-cells
    pts[200:400, 2] = hi - rng.random(200) * (hi - lo) / (2 * n)
    got = oracle_mod.interp_points(p, F, pts[:, 0], pts[:, 1], pts[:, 2])
    h = (hi - lo) / n
    q = (pts - lo) / h                                                   # pinned equal to the oracle's quotient
    u2 = 2.0 ** -53
    plain = np.empty(m)
    ulps = np.empty(m)
    for k in range(m):
        ex, mag = _exact_interp(F, n, q[k])
        bound = 12 * u2 * float(mag)
        assert abs(Fraction(got[k]) - ex) <= Fraction(bound), (k, got[k], float(ex), bound)
        ulps[k] = abs(float(Fraction(got[k]) - ex)) / np.spacing(abs(float(ex)))
        # plain evaluation: rounded products, then ordinary additions
        i0 = np.floor(q[k] - 0.5).astype(int)
        f = (q[k] - 0.5) - np.floor(q[k] - 0.5)
        acc = 0.0
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    w = ((f[0] if a else 1.0 - f[0]) * (f[1] if b else 1.0 - f[1])) * (f[2] if c else 1.0 - f[2])
                    ii = [min(max(i0[t] + (a, b, c)[t], 0), n - 1) for t in range(3)]
                    acc = acc + w * F[ii[2], ii[1], ii[0]]
        plain[k] = acc
        assert abs(Fraction(acc) - ex) <= Fraction(bound)
    if not signed:
        assert ulps.max() <= 5.0, ulps.max()


def _ptrs_three_logs(uniforms, mu, count):
    """PTRS (Hoermann 1993) with the acceptance test as printed there:
    log V + log(1/alpha) - log(a/us^2 + b) <= -mu + k log mu - log k!, with
    libm's log and lgamma.  Consumes the uniforms in order; returns the draws
    and the number of trials that reached the logarithmic test."""
    it = iter(uniforms)
    slam = math.sqrt(mu)
    loglam = math.log(mu)
    b = 0.931 + 2.53 * slam
    a = -0.059 + 0.02483 * b
    invalpha = 1.1239 + 1.1328 / (b - 3.4)
    vr = 0.9277 - 3.6224 / (b - 2.0)
    out, slow = [], 0
    while len(out) < count:
        U = next(it) - 0.5
        V = next(it)
        us = 0.5 - abs(U)
        k = math.floor(((2.0 * a / us) + b) * U + mu + 0.43)
        if us >= 0.07 and V <= vr:
            out.append(k)
            continue
        if k < 0 or (us < 0.013 and V > us):
            continue
        slow += 1
        if math.log(V) + math.log(invalpha) - math.log(a / (us * us) + b) <= -mu + k * loglam - math.lgamma(k + 1):
            out.append(k)
    return np.asarray(out, np.int64), slow


@pytest.mark.parametrize("mu", [10.0, 13.7, 40.0, 250.0, 3.3e3, 1e5, 2.5e6])
def test_ptrs_one_log_test_decides_as_hoermanns_three_logs(oracle_mod, mu):
    """Same uniforms, same accept/reject decisions: the oracle's one-log form
    of the slow test (and its Stirling log k!) against the literal form with
    libm, draw by draw."""
    n = 6000
    got = oracle_mod.poisson_draws(11, 5, 2, oracle_mod.TAG_KMC, 0, mu, n)
    # the oracle's PTRS uses two uniforms per trial from one stream; at most
    # a few trials per draw (acceptance above 0.9), so 4n pairs suffice
    u = oracle_mod.uniform_draws(11, 5, 2, oracle_mod.TAG_KMC, 0, 8 * n + 1000)
    ref, slow = _ptrs_three_logs(u, mu, n)
    assert slow > 50, slow                      # the logarithmic test was exercised
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mu", [0.05, 1.0, 4.2, 9.99])
def test_poisson_inversion_is_the_inverse_cdf(oracle_mod, mu):
    """Below mean 10 the draw is the smallest k with u <= F(k): scipy's
    Poisson quantile of the same uniform, except where u lies within
    rounding of a CDF step."""
    n = 20000
    got = oracle_mod.poisson_draws(3, 9, 1, oracle_mod.TAG_KMC, 0, mu, n)
    u = oracle_mod.uniform_draws(3, 9, 1, oracle_mod.TAG_KMC, 0, n)
    ref = stats.poisson.ppf(u, mu).astype(np.int64)
    diff = np.flatnonzero(got != ref)
    for k in diff:
        assert abs(u[k] - stats.poisson.cdf(min(got[k], ref[k]), mu)) < 1e-12
    assert diff.size <= 2
