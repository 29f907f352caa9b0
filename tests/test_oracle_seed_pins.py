"""Pins of the oracle's Gaussian seeding (initial electrons, Sec. 5.1).

The per-cell counts are Poisson draws of n(x_c) dV; the pins check what
that fixes independently of the oracle's own arithmetic: the count total
against the continuous integral of the blob, the standardized per-cell
deviations against the unit normal, the weight rule of Eq. w in every cell,
every particle inside its cell and uniform there, and the realization
selection of the blobs."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2307_01797_gb300 import synth


def _grid(ph):
    n = ph["n"]
    h = (ph["hi"][0] - ph["lo"][0]) / n
    c = ph["lo"][0] + (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return n, h, X.ravel(), Y.ravel(), Z.ravel()


def _mean_counts(ph, blobs):
    n, h, X, Y, Z = _grid(ph)
    dens = np.zeros(n ** 3)
    for b in blobs:
        cx, cy, cz = b["center"]
        dens += b["peak"] * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2 * b["sigma"] ** 2))
    return dens * h ** 3


@pytest.fixture(scope="module")
def seeded(oracle_mod):
    ph = synth.physics_small(64)
    blobs = [dict(center=(0.005, 0.005, 0.008), sigma=5e-4, peak=1e18),
             dict(center=(0.0031, 0.0062, 0.004), sigma=3e-4, peak=4e17)]
    p = oracle_mod.make_params(ph, seed=3)
    st, counts = oracle_mod.seed_blobs(p, blobs)
    return ph, blobs, st, counts


def test_seed_total_matches_the_blob_integral(seeded):
    """Sum of counts ~ Poisson(sum of means); the means themselves integrate
    to A (2 pi)^(3/2) s^3 per blob (blobs well inside the box)."""
    ph, blobs, st, counts = seeded
    mu = _mean_counts(ph, blobs)
    total = counts.sum()
    assert abs(total - mu.sum()) <= 5 * math.sqrt(mu.sum())
    integral = sum(b["peak"] * (2 * math.pi) ** 1.5 * b["sigma"] ** 3 for b in blobs)
    assert abs(mu.sum() / integral - 1) < 5e-3
    assert int(st["w"].astype(np.int64).sum()) == total


def test_seed_counts_are_poisson_per_cell(seeded):
    """Cells with a large mean: (N - mu)/sqrt(mu) is standard normal; cells
    with a tiny mean are almost always empty."""
    ph, blobs, st, counts = seeded
    mu = _mean_counts(ph, blobs)
    big = mu > 1e3
    zs = (counts[big] - mu[big]) / np.sqrt(mu[big])
    assert big.sum() > 2000
    assert stats.kstest(zs, "norm").pvalue > 1e-4
    tiny = (mu > 0) & (mu < 1e-6)
    assert counts[tiny].sum() <= 2


def test_seed_weight_rule_and_positions(seeded):
    """Per cell m = min(N, ppc) particles, weights N // m with the remainder
    on the first (Eq. w); every particle inside its cell, uniform there."""
    ph, blobs, st, counts = seeded
    n, h = ph["n"], (ph["hi"][0] - ph["lo"][0]) / ph["n"]
    ppc = ph["ppc"]
    cells, first, m = np.unique(st["cell"], return_index=True, return_counts=True)
    assert np.array_equal(np.flatnonzero(counts), cells)
    N = counts[cells]
    assert np.array_equal(m, np.minimum(N, ppc))
    wq, rem = N // m, N % m
    assert np.array_equal(st["w"][first].astype(np.int64), wq + rem)
    rest = np.ones(len(st["w"]), bool)
    rest[first] = False
    assert np.array_equal(st["w"][rest].astype(np.int64), np.repeat(wq, m)[rest])
    assert np.all(np.diff(st["cell"]) >= 0)
    frac = []
    for a, k in enumerate(("x", "y", "z")):
        q = (st[k] - ph["lo"][a]) / h
        idx = (st["cell"] // n ** a) % n
        assert np.array_equal(np.floor(q).astype(np.int64), idx)
        frac.append(q - idx)
    for f in frac:
        assert stats.kstest(f, "uniform").pvalue > 1e-4


def test_seed_blob_realization_selection(oracle_mod):
    """A blob tied to realization 1 seeds nothing in realization 0; a blob
    for every realization seeds both identically when the key is the same."""
    ph = synth.physics_small(16)
    b1 = [dict(center=(0.005, 0.005, 0.005), sigma=1e-3, peak=1e18, realization=1)]
    p = oracle_mod.make_params(ph, seed=9)
    st0, c0 = oracle_mod.seed_blobs(p, b1, real=0)
    st1, c1 = oracle_mod.seed_blobs(p, b1, real=1)
    assert len(st0["w"]) == 0 and c0.sum() == 0 and c1.sum() > 0
    ball = [dict(center=(0.005, 0.005, 0.005), sigma=1e-3, peak=1e18)]
    a, ca = oracle_mod.seed_blobs(p, ball, real=0)
    b, cb = oracle_mod.seed_blobs(p, ball, real=1)
    assert np.array_equal(ca, cb) and np.array_equal(a["x"], b["x"])
