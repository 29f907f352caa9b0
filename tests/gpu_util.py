"""Shared helpers of the GPU parity tests: build a library handle and the
oracle's state from the same seeded synthetic inputs."""
import numpy as np

import oracle
from paper_2307_01797_gb300 import itokmc, synth


def small_phys(n=32, **kw):
    ph = synth.physics_small(n)
    ph.update(kw)
    return ph


def mixed_state(ph, seed, n_random=3000, peak=3e18, sigma=None, zfrac=0.55):
    """A Gaussian blob (several particles per cell, up to ppc) plus particles
    scattered over the whole box, some within a cell of the faces."""
    L = ph["hi"][0] - ph["lo"][0]
    sig = sigma if sigma is not None else 0.08 * L
    blob = synth.blob_state(ph, seed=seed, sigma=sig, peak=peak, zfrac=zfrac)
    rnd = synth.random_particles(ph, n_random, seed=seed + 1000, wmax=5000)
    return {k: np.concatenate([blob[k], rnd[k]]) for k in ("x", "y", "z", "w")}


def gpu_handle(ph, cap, seed0=1, precision=itokmc.FP64, realizations=1, field_precision=-1):
    cfg = itokmc.make_config(ph, cap, realizations=realizations, seed0=seed0, precision=precision,
                             field_precision=field_precision)
    return itokmc.Handle(cfg)


def oracle_state(ph, st, seed, Npos=None, Nneg=None):
    p = oracle.make_params(ph, seed=seed)
    S = oracle.canonical(p, st)
    n3 = ph["n"] ** 3
    S["Npos"] = np.zeros(n3, np.int64) if Npos is None else np.asarray(Npos, np.int64).copy()
    S["Nneg"] = np.zeros(n3, np.int64) if Nneg is None else np.asarray(Nneg, np.int64).copy()
    return S


def assert_particles_equal(G, S):
    assert len(G["w"]) == len(S["w"]), (len(G["w"]), len(S["w"]))
    for k in ("x", "y", "z"):
        a, b = np.asarray(G[k]), np.asarray(S[k])
        bad = np.nonzero(a.view(np.uint64) != b.view(np.uint64))[0]
        assert bad.size == 0, f"{k}: {bad.size} differ, first {bad[:5]} gpu {a[bad[:3]]} oracle {b[bad[:3]]}"
    assert np.array_equal(G["w"], S["w"])
    assert np.array_equal(G["cell"], S["cell"])
