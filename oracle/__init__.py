"""FP64 CPU oracle of one Ito-KMC time step (arXiv 2307.01797).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA library.  The particle, KMC and photon steps
are plain C (``itokmc_oracle.c``, built without FMA contraction); the field
solve is numpy (``poisson.py``); the step composition is ``stages.py``; the
semi-implicit field coupling of Sec. 4.3 (variable-coefficient solve and the
diffusive/advective substeps) is ``semi_implicit.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "itokmc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

TAG_INIT, TAG_PUSH, TAG_KMC, TAG_PRODUCT, TAG_PHOTON = 1, 2, 3, 4, 5


_OMP_PATH = os.path.join(_HERE, "_build", "liboracle_omp.so")
_use_omp = False


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction, no fast-math), once
    plain and once with OpenMP (the same arithmetic spread over threads)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    for path, extra in ((_LIB_PATH, []), (_OMP_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", *extra,
                   "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, path)
    return _LIB_PATH


def use_openmp(on: bool = True, threads: int | None = None) -> None:
    """Route the oracle's calls to the OpenMP build (threads: OMP_NUM_THREADS,
    default every core this process may run on) or back to the plain one."""
    global _lib, _use_omp
    with _lock:
        if bool(on) != _use_omp:
            _lib = None
        _use_omp = bool(on)
        if on:
            os.environ["OMP_NUM_THREADS"] = str(threads or len(os.sched_getaffinity(0)))


class Params(ctypes.Structure):
    """Mirror of ``ora_params`` in itokmc_oracle.c."""
    _fields_ = [
        ("n", ctypes.c_int32), ("ppc", ctypes.c_int32), ("n_new", ctypes.c_int32),
        ("n_crit", ctypes.c_int32), ("n_ssa", ctypes.c_int32), ("frac_bits", ctypes.c_int32),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("dt", ctypes.c_double), ("mu", ctypes.c_double), ("D", ctypes.c_double),
        ("alpha_A", ctypes.c_double), ("alpha_B", ctypes.c_double), ("eta", ctypes.c_double),
        ("photon_ratio", ctypes.c_double), ("kappa_lo", ctypes.c_double), ("kappa_hi", ctypes.c_double),
        ("eps", ctypes.c_double), ("seed", ctypes.c_uint64), ("step", ctypes.c_uint32),
        ("pad", ctypes.c_uint32), ("beta_ep", ctypes.c_double), ("beta_np", ctypes.c_double),
        ("mu_ion", ctypes.c_double), ("D_ion", ctypes.c_double),
    ]


def make_params(phys: dict, seed: int, step: int = 0) -> Params:
    """Build oracle parameters from a physics dict (see the package's
    ``synth.physics_*`` helpers for the keys)."""
    p = Params()
    p.n = int(phys["n"])
    p.ppc = int(phys.get("ppc", 8))
    p.n_new = int(phys.get("n_new", 64))
    p.n_crit = int(phys.get("n_crit", 5))
    p.n_ssa = int(phys.get("n_ssa", 10))
    p.frac_bits = int(phys.get("frac_bits", 10))
    for a in range(3):
        p.lo[a] = float(phys["lo"][a])
        p.hi[a] = float(phys["hi"][a])
    p.dt = float(phys["dt"])
    p.mu = float(phys["mu"])
    p.D = float(phys["D"])
    p.alpha_A = float(phys["alpha_A"])
    p.alpha_B = float(phys["alpha_B"])
    p.eta = float(phys["eta"])
    p.photon_ratio = float(phys.get("photon_ratio", 0.0))
    p.kappa_lo = float(phys.get("kappa_lo", 520.0))
    p.kappa_hi = float(phys.get("kappa_hi", 3.0e4))
    p.eps = float(phys.get("eps", float("inf")))
    p.beta_ep = float(phys.get("beta_ep", 0.0))
    p.beta_np = float(phys.get("beta_np", 0.0))
    p.mu_ion = float(phys.get("mu_ion", 0.0))
    p.D_ion = float(phys.get("D_ion", 0.0))
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.step = int(step) & 0xFFFFFFFF
    return p


def _P(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_OMP_PATH if _use_omp else _LIB_PATH)
            d, i64, u32, u64, i32 = (ctypes.c_double, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_int32)
            pd, pi64, pu32, pu64 = (ctypes.POINTER(d), ctypes.POINTER(i64), ctypes.POINTER(u32),
                                    ctypes.POINTER(u64))
            pp = ctypes.POINTER(Params)
            L.ora_philox4x32_10.argtypes = [pu32, pu32, pu32]
            L.ora_log.argtypes = [d]; L.ora_log.restype = d
            L.ora_exp.argtypes = [d]; L.ora_exp.restype = d
            L.ora_sincos2pi.argtypes = [d, pd, pd]
            L.ora_poisson_draws.argtypes = [u64, u32, u32, u32, u32, d, i64, pi64]
            L.ora_uniform_draws.argtypes = [u64, u32, u32, u32, u32, i64, pd]
            L.ora_normal_draws.argtypes = [u64, u32, u32, u32, u32, i64, pd]
            L.ora_push.argtypes = [pp, i64, pd, pd, pd, pd, pd, pd, pd, pd, pd, pi64]
            L.ora_diffuse.argtypes = [pp, i64, pd, pd, pd, pd, pd, pd]
            L.ora_advect.argtypes = [pp, i64, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pd, pi64]
            L.ora_sort_by_cell.argtypes = [i64, i64, pi64, pi64]; L.ora_sort_by_cell.restype = i64
            L.ora_deposit.argtypes = [pp, i64, pd, pd, pd, pu32, pi64, pi64, pi64]
            L.ora_kmc.argtypes = [pp, pi64, pi64, pi64, pd, pd, pd, pi64, pi64, pi64, pi64, pi64]
            L.ora_kmc.restype = ctypes.c_int
            L.ora_kmc_single.argtypes = [pp, i64, d, d, d, u32, pi64]; L.ora_kmc_single.restype = i64
            L.ora_kmc_network.argtypes = [pp, pi64, pd, u32, pi64, pi64]; L.ora_kmc_network.restype = ctypes.c_int
            pi32 = ctypes.POINTER(ctypes.c_int32)
            L.ora_products_photons.argtypes = [pp, i64, pd, pd, pd, pu32, pi64, pi64, pi64, pi64, pi64,
                                               pi64, pi64, pi64, pi64, pd, pd, pd, pu32, pi64, i64, pi64,
                                               pi64, pi32, pi32]
            L.ora_push_species.argtypes = [pp, ctypes.c_int32, i64, pd, pd, pd, pd, pd, pd, pd, pd, pd, pi64]
            L.ora_push_species.restype = None
            L.ora_species_products.argtypes = [pp, ctypes.c_int32, pi64, pi64, pi64, pu32, pd, pd, pd, pu32, pi64,
                                               pi64, pi32, pi32, i64]
            L.ora_species_products.restype = i64
            L.ora_products_photons.restype = i64
            L.ora_merge.argtypes = [pp, pd, pd, pd, pu32, pi64, pd, pd, pd, pu32, pi64, i64]
            L.ora_merge.restype = i64
            L.ora_merge_list.argtypes = [i64, pd, pd, pd, pu64, i32, pd, pd, pd, pu64]
            L.ora_merge_list.restype = i64
            L.ora_photon_samples.argtypes = [pp, i32, i32, i32, i64, pd, pd, pd, pd]
            L.ora_cells.argtypes = [pp, i64, pd, pd, pd, pi64]
            L.ora_grid_axis.argtypes = [pp, i32, i64, pd, pd, pi64, pi64, pi64, pd, pi64]
            L.ora_interp_points.argtypes = [pp, pd, i64, pd, pd, pd, pd]
            pi32 = ctypes.POINTER(i32)
            L.ora_seed_blobs.argtypes = [pp, i32, pd, pd, pd, pi32, i32, pd, pd, pd, pu32, pi64, pi64, i64]
            L.ora_seed_blobs.restype = i64
            L.ora_kmc0d.argtypes = [pp, d, i64, i32, i32, pi64]
            L.ora_kmc0d.restype = ctypes.c_int
            _lib = L
    return _lib


# ---------------------------------------------------------------- primitives
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_P(c, ctypes.c_uint32), _P(k, ctypes.c_uint32), _P(out, ctypes.c_uint32))
    return out


def log(x: float) -> float:
    return lib().ora_log(float(x))


def exp(x: float) -> float:
    return lib().ora_exp(float(x))


def sincos2pi(u: float):
    s = ctypes.c_double()
    c = ctypes.c_double()
    lib().ora_sincos2pi(float(u), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def uniform_draws(seed, index, step, tag, sub, n):
    out = np.zeros(n, dtype=np.float64)
    lib().ora_uniform_draws(seed, index, step, tag, sub, n, _P(out, ctypes.c_double))
    return out


def normal_draws(seed, index, step, tag, sub, n):
    out = np.zeros(n, dtype=np.float64)
    lib().ora_normal_draws(seed, index, step, tag, sub, n, _P(out, ctypes.c_double))
    return out


def poisson_draws(seed, index, step, tag, sub, mu, n):
    out = np.zeros(n, dtype=np.int64)
    lib().ora_poisson_draws(seed, index, step, tag, sub, float(mu), n, _P(out, ctypes.c_int64))
    return out


def kmc_single(params: Params, X0: int, k_ion: float, k_att: float, k_ph: float, index: int):
    fired = np.zeros(3, dtype=np.int64)
    X = lib().ora_kmc_single(ctypes.byref(params), int(X0), float(k_ion), float(k_att), float(k_ph),
                             int(index), _P(fired, ctypes.c_int64))
    return int(X), fired


def kmc_network(params: Params, X0, kr, index: int):
    """One cell of the five-reaction network (Sec. 5.1): counts X0 = (X_e,
    X_+, X_-), frequencies kr = (k_alpha, k_eta, k_gamma, k_ep, k_np), stream
    (index, params.step, KMC).  Returns (X[3], fired[5])."""
    X0 = np.ascontiguousarray(X0, dtype=np.int64)
    kr = np.ascontiguousarray(kr, dtype=np.float64)
    assert X0.shape == (3,) and kr.shape == (5,)
    X = np.zeros(3, np.int64)
    fired = np.zeros(5, np.int64)
    if lib().ora_kmc_network(ctypes.byref(params), _P(X0, ctypes.c_int64), _P(kr, ctypes.c_double),
                             int(index), _P(X, ctypes.c_int64), _P(fired, ctypes.c_int64)) != 0:
        raise RuntimeError("kmc_network: iteration guard")
    return X, fired


def photon_samples(params: Params, i: int, j: int, k: int, m: int):
    """Photon draws of cell (i,j,k), slots 0..m-1: (Y0[m,3], kappa[m], r[m], dir[m,3])."""
    Y0 = np.zeros((m, 3)); kap = np.zeros(m); r = np.zeros(m); d = np.zeros((m, 3))
    lib().ora_photon_samples(ctypes.byref(params), i, j, k, m, _P(Y0, ctypes.c_double),
                             _P(kap, ctypes.c_double), _P(r, ctypes.c_double), _P(d, ctypes.c_double))
    return Y0, kap, r, d


def cells(params: Params, x, y, z):
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    out = np.empty(len(x), np.int64)
    lib().ora_cells(ctypes.byref(params), len(x), _P(x, ctypes.c_double), _P(y, ctypes.c_double),
                    _P(z, ctypes.c_double), _P(out, ctypes.c_int64))
    return out


def grid_axis(params: Params, ax: int, x):
    """Grid arithmetic of one axis at coordinates x: dict(q, cell, ia, ib, f, a)
    (quotient (x-lo)/h, cell, folded CIC indices, CIC fraction, fixed-point
    deposit weight floor(f 2^s))."""
    x = np.ascontiguousarray(x, np.float64)
    n = len(x)
    q = np.empty(n); f = np.empty(n)
    cell = np.empty(n, np.int64); ia = np.empty(n, np.int64); ib = np.empty(n, np.int64); a = np.empty(n, np.int64)
    lib().ora_grid_axis(ctypes.byref(params), int(ax), n, _P(x, ctypes.c_double), _P(q, ctypes.c_double),
                        _P(cell, ctypes.c_int64), _P(ia, ctypes.c_int64), _P(ib, ctypes.c_int64),
                        _P(f, ctypes.c_double), _P(a, ctypes.c_int64))
    return dict(q=q, cell=cell, ia=ia, ib=ib, f=f, a=a)


def interp_points(params: Params, F, x, y, z):
    """CIC interpolation of the cell-centred scalar field F (n^3, x fastest)
    at the points (x, y, z), as the push interpolates each component of E."""
    F = np.ascontiguousarray(F, np.float64).ravel()
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    out = np.empty(len(x))
    lib().ora_interp_points(ctypes.byref(params), _P(F, ctypes.c_double), len(x), _P(x, ctypes.c_double),
                            _P(y, ctypes.c_double), _P(z, ctypes.c_double), _P(out, ctypes.c_double))
    return out


def seed_blobs(params: Params, blobs, real: int = 0, cap: int = 50_000_000):
    """Initial electrons of one realization from Gaussian blobs, each blob a
    dict(center=(x, y, z), sigma, peak, realization=-1): dict(x, y, z, w,
    cell) in canonical order and counts (electrons per cell)."""
    nb = len(blobs)
    C = np.ascontiguousarray([b["center"] for b in blobs], np.float64).reshape(-1)
    S = np.ascontiguousarray([b["sigma"] for b in blobs], np.float64)
    A = np.ascontiguousarray([b["peak"] for b in blobs], np.float64)
    Rb = np.ascontiguousarray([b.get("realization", -1) for b in blobs], np.int32)
    n3 = params.n ** 3
    cap = int(min(cap, n3 * params.ppc))
    x = np.empty(cap); y = np.empty(cap); z = np.empty(cap)
    w = np.empty(cap, np.uint32); cell = np.empty(cap, np.int64); counts = np.zeros(n3, np.int64)
    np_ = lib().ora_seed_blobs(ctypes.byref(params), nb, _P(C, ctypes.c_double), _P(S, ctypes.c_double),
                               _P(A, ctypes.c_double), Rb.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(real),
                               _P(x, ctypes.c_double), _P(y, ctypes.c_double), _P(z, ctypes.c_double),
                               _P(w, ctypes.c_uint32), _P(cell, ctypes.c_int64), _P(counts, ctypes.c_int64), cap)
    if np_ < 0:
        raise RuntimeError("seed_blobs: " + ("capacity" if np_ == -1 else "weight overflow"))
    return dict(x=x[:np_], y=y[:np_], z=z[:np_], w=w[:np_], cell=cell[:np_]), counts


def kmc0d(params: Params, E_mag: float, X0: int, n_real: int, n_steps: int):
    """0-D KMC ensemble (Sec. 3.2.4): int64 (n_real, n_steps + 1) electron
    counts; realization m, step k draw from the stream (seed, m, k, KMC)."""
    X = np.zeros((int(n_real), int(n_steps) + 1), np.int64)
    st = lib().ora_kmc0d(ctypes.byref(params), float(E_mag), int(X0), int(n_real), int(n_steps),
                         _P(X, ctypes.c_int64))
    if st != 0:
        raise RuntimeError("kmc0d: iteration guard")
    return X


def canonical(params: Params, st: dict) -> dict:
    """Particles of ``st`` (x, y, z, w; any order) in canonical order (cell,
    input order) with their cells; particles outside the box are dropped."""
    c = cells(params, st["x"], st["y"], st["z"])
    perm = stages.sort_by_cell(c, params.n ** 3)
    return dict(x=np.asarray(st["x"], np.float64)[perm], y=np.asarray(st["y"], np.float64)[perm],
                z=np.asarray(st["z"], np.float64)[perm], w=np.asarray(st["w"], np.uint32)[perm], cell=c[perm])


def merge_list(x, y, z, w, T):
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64); w = np.ascontiguousarray(w, np.uint64)
    M = len(w)
    ox = np.zeros(T, np.float64); oy = np.zeros(T, np.float64); oz = np.zeros(T, np.float64)
    ow = np.zeros(T, np.uint64)
    n = lib().ora_merge_list(M, _P(x, ctypes.c_double), _P(y, ctypes.c_double), _P(z, ctypes.c_double),
                             _P(w, ctypes.c_uint64), int(T), _P(ox, ctypes.c_double),
                             _P(oy, ctypes.c_double), _P(oz, ctypes.c_double), _P(ow, ctypes.c_uint64))
    return ox[:n], oy[:n], oz[:n], ow[:n]


from . import stages  # noqa: E402  (stage wrappers and the step composition)
from .stages import (push, sort_by_cell, deposit, kmc, products_photons, merge, step, push_species,  # noqa: E402,F401
                     species_products, step_mobile,  # noqa: E402,F401
                     rho_fixed)
from .poisson import solve as solve_field  # noqa: E402,F401
