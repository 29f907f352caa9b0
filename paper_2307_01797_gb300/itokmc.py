"""Thin ctypes binding of libitokmc.so (the C ABI in ``include/itokmc.h``).

Argument marshalling only: every step of the Ito-KMC path runs in the CUDA
kernels of the library.  Function names mirror the C entry points.  Device
memory comes from PyTorch's caching allocator (through the allocator hooks of
``itokmc_config``) and the work runs on PyTorch's current CUDA stream.  There
is no CPU fallback: if the library is missing the import of ``lib()`` fails.
"""
from __future__ import annotations

import ctypes
import math
import os
import re
import threading

import numpy as np

from . import build as _build

ITOKMC_OK = 0
ERR_NAMES = {-1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_CAPACITY", -5: "ERR_OVERFLOW",
             -6: "ERR_NOCONV", -7: "ERR_TIMEOUT", -8: "ERR_POISONED", -9: "ERR_KMC", -10: "ERR_INTERNAL"}
FP64, MIXED = 0, 1
EXPLICIT, SEMI_IMPLICIT = 0, 1
HOST, DEVICE = 0, 1
NE_FIX, XE, NPOS, NNEG, PHI, E, RHO, FIRINGS = range(8)
STAGE_TRANSPORT, STAGE_KMC, STAGE_PARTICLES, STAGE_FIELD = range(4)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3), ("n_realizations", ctypes.c_int32),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("dt", ctypes.c_double), ("seed0", ctypes.c_uint64),
        ("mu", ctypes.c_double), ("D", ctypes.c_double),
        ("alpha_A", ctypes.c_double), ("alpha_B", ctypes.c_double), ("eta", ctypes.c_double),
        ("E0", ctypes.c_double), ("photon_ratio", ctypes.c_double),
        ("kappa_lo", ctypes.c_double), ("kappa_hi", ctypes.c_double), ("eps", ctypes.c_double),
        ("ppc", ctypes.c_int32), ("n_new", ctypes.c_int32), ("n_crit", ctypes.c_int32),
        ("n_ssa", ctypes.c_int32), ("frac_bits", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("mg_rtol", ctypes.c_double), ("mg_nu1", ctypes.c_int32), ("mg_nu2", ctypes.c_int32),
        ("mg_max_cycles", ctypes.c_int32), ("field_precision", ctypes.c_int32),
        ("particle_capacity", ctypes.c_int64), ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
        ("blobs", ctypes.c_void_p), ("n_blobs", ctypes.c_int32), ("seed_flags", ctypes.c_int32),
        ("coupling", ctypes.c_int32), ("dt_adapt", ctypes.c_int32), ("dt_min", ctypes.c_double),
        ("cfl", ctypes.c_double), ("drt_factor", ctypes.c_double), ("ion_factor", ctypes.c_double),
        ("beta_ep", ctypes.c_double), ("beta_np", ctypes.c_double),
        ("mobile_ions", ctypes.c_int32), ("pad_ions", ctypes.c_int32), ("mu_ion", ctypes.c_double),
        ("D_ion", ctypes.c_double), ("graph_step", ctypes.c_int32), ("pad_graph", ctypes.c_int32),
    ]


class SeedBlob(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 3), ("sigma", ctypes.c_double), ("peak", ctypes.c_double),
                ("realization", ctypes.c_int32), ("pad", ctypes.c_int32)]


SEED_NEUTRAL = 1


def blob_array(blobs):
    """A ctypes array of itokmc_seed_blob from dicts (center, sigma, peak,
    realization=-1)."""
    arr = (SeedBlob * max(1, len(blobs)))()
    for i, b in enumerate(blobs):
        for a in range(3):
            arr[i].center[a] = float(b["center"][a])
        arr[i].sigma = float(b["sigma"])
        arr[i].peak = float(b["peak"])
        arr[i].realization = int(b.get("realization", -1))
    return arr


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_particles", ctypes.c_int64), ("step", ctypes.c_int64), ("n_movers", ctypes.c_int64),
        ("outflow_weight", ctypes.c_int64), ("ionizations", ctypes.c_int64),
        ("attachments", ctypes.c_int64), ("photon_emissions", ctypes.c_int64),
        ("photons_absorbed_weight", ctypes.c_int64), ("photons_lost_weight", ctypes.c_int64),
        ("n_new_particles", ctypes.c_int64), ("mg_cycles", ctypes.c_int32), ("kmc_status", ctypes.c_int32),
        ("mg_rel_residual", ctypes.c_double), ("ms_transport", ctypes.c_double), ("ms_kmc", ctypes.c_double),
        ("ms_particles", ctypes.c_double), ("ms_field", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64), ("merge_cells", ctypes.c_int64), ("merge_elements", ctypes.c_int64),
        ("merge_elements_sq", ctypes.c_int64), ("merge_max_list", ctypes.c_int64), ("dt_last", ctypes.c_double),
        ("recombinations_ep", ctypes.c_int64), ("recombinations_np", ctypes.c_int64),
        ("outflow_ion_pos", ctypes.c_int64), ("outflow_ion_neg", ctypes.c_int64), ("graph_steps", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TUNE_CANDIDATES = 9
TUNE_DEPOSIT = 5


class Tuning(ctypes.Structure):
    _fields_ = [
        ("mg_nu1", ctypes.c_int32), ("mg_nu2", ctypes.c_int32), ("ms_field", ctypes.c_double),
        ("cycles", ctypes.c_int32), ("n_tried", ctypes.c_int32),
        ("nu_tried", (ctypes.c_int32 * 2) * TUNE_CANDIDATES), ("ms_tried", ctypes.c_double * TUNE_CANDIDATES),
        ("dep_win", ctypes.c_int32), ("n_dep_tried", ctypes.c_int32), ("dep_tried", ctypes.c_int32 * TUNE_DEPOSIT),
        ("ms_dep_tried", ctypes.c_double * TUNE_DEPOSIT),
    ]


class ItokmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None
HEADER = os.path.join(_build.ROOT, "include", "itokmc.h")


def header_functions():
    """Names of the functions declared in include/itokmc.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(itokmc_\w+)\s*\(", txt, re.M)))


def lib(build_if_missing: bool = True):
    """The loaded libitokmc.so (built in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libitokmc.so not built ({path}); run paper_2307_01797_gb300.build")
            L = ctypes.CDLL(path)
            i32, i64, u64, vp, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double
            H = ctypes.c_void_p
            sig = {
                "itokmc_config_defaults": ([ctypes.POINTER(Config)], ctypes.c_int),
                "itokmc_init": ([ctypes.POINTER(Config), ctypes.POINTER(H)], ctypes.c_int),
                "itokmc_destroy": ([H], ctypes.c_int),
                "itokmc_set_particles": ([H, vp, vp, vp, vp, vp, i64, i32], ctypes.c_int),
                "itokmc_set_particles_species": ([H, vp, vp, vp, vp, vp, vp, i64, i32], ctypes.c_int),
                "itokmc_read_particles": ([H, vp, vp, vp, vp, vp, vp, i64, ctypes.POINTER(i64), i32], ctypes.c_int),
                "itokmc_set_ions": ([H, vp, vp, i32], ctypes.c_int),
                "itokmc_set_field": ([H, vp, i32], ctypes.c_int),
                "itokmc_solve_field": ([H], ctypes.c_int),
                "itokmc_step": ([H, i32], ctypes.c_int),
                "itokmc_run_stage": ([H, i32], ctypes.c_int),
                "itokmc_advance_counter": ([H], ctypes.c_int),
                "itokmc_transport_semi_implicit": ([H, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)],
                                                   ctypes.c_int),
                "itokmc_autotune": ([H, ctypes.POINTER(Tuning)], ctypes.c_int),
                "itokmc_read_densities": ([H, i32, i32, vp, ctypes.c_size_t], ctypes.c_int),
                "itokmc_get_stats": ([H, ctypes.POINTER(Stats)], ctypes.c_int),
                "itokmc_num_particles": ([H, ctypes.POINTER(i64)], ctypes.c_int),
                "itokmc_last_error": ([H], ctypes.c_char_p),
                "itokmc_version": ([], ctypes.c_char_p),
                "itokmc_field_solve_noalloc": ([ctypes.POINTER(Config), vp, vp, vp, ctypes.POINTER(i32),
                                                ctypes.POINTER(d)], ctypes.c_int),
                "itokmc_probe_fp64_peak": ([vp, ctypes.POINTER(d), ctypes.POINTER(d)], ctypes.c_int),
                "itokmc_seed_blobs": ([H, ctypes.POINTER(SeedBlob), i32, i32], ctypes.c_int),
                "itokmc_kmc0d": ([ctypes.POINTER(Config), d, i64, i32, i32, vp, i32], ctypes.c_int),
                "itokmc_save": ([H, ctypes.c_char_p], ctypes.c_int),
                "itokmc_load": ([H, ctypes.c_char_p], ctypes.c_int),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def itokmc_kmc0d(cfg: Config, E_mag: float, X0: int, n_real: int, n_steps: int):
    """0-D KMC ensemble: int64 array (n_real, n_steps + 1) of electron counts."""
    X = np.empty((int(n_real), int(n_steps) + 1), np.int64)
    _check(lib().itokmc_kmc0d(ctypes.byref(cfg), float(E_mag), int(X0), int(n_real), int(n_steps), _ptr(X), HOST))
    return X


def itokmc_probe_fp64_peak(stream=None):
    """Measured FP64 FMA rate of the current device: (TFLOP/s, ms)."""
    t = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib().itokmc_probe_fp64_peak(stream, ctypes.byref(t), ctypes.byref(ms)), None)
    return t.value, ms.value


def itokmc_field_solve_noalloc(cfg: Config, rho, phi, E):
    """Field solve on caller device buffers (torch tensors) with no device
    allocation by the library: rho int64 n^3, phi float64 n^3 (initial guess
    in, potential out), E float64 3 n^3 (out).  Returns (cycles, rel)."""
    cyc = ctypes.c_int32()
    rel = ctypes.c_double()
    code = lib().itokmc_field_solve_noalloc(ctypes.byref(cfg), _ptr(rho), _ptr(phi), _ptr(E), ctypes.byref(cyc),
                                            ctypes.byref(rel))
    if code != ITOKMC_OK:
        raise ItokmcError(code, lib().itokmc_last_error(None).decode())
    return cyc.value, rel.value


# ------------------------------------------------------------------ allocator
class _TorchAllocator:
    """Device memory from torch's caching allocator, kept alive by pointer."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        except Exception:  # out of memory: the library reports ERR_OOM
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())   # torch tensor


def _check(code, h=None):
    if code != ITOKMC_OK:
        msg = lib().itokmc_last_error(h).decode()
        raise ItokmcError(code, msg)


def make_config(phys: dict, capacity: int, realizations: int = 1, seed0: int = 1,
                precision: int = FP64, field_precision: int = -1, stream=None, **overrides) -> Config:
    c = Config()
    _check(lib().itokmc_config_defaults(ctypes.byref(c)))
    n = int(phys["n"])
    c.n[0] = c.n[1] = c.n[2] = n
    c.n_realizations = int(realizations)
    for a in range(3):
        c.lo[a] = float(phys["lo"][a])
        c.hi[a] = float(phys["hi"][a])
    c.dt = float(phys["dt"])
    c.seed0 = int(seed0)
    for k in ("mu", "D", "alpha_A", "alpha_B", "eta", "E0", "photon_ratio", "kappa_lo", "kappa_hi",
              "beta_ep", "beta_np", "mu_ion", "D_ion"):
        setattr(c, k, float(phys.get(k, getattr(c, k))))
    c.mobile_ions = int(bool(phys.get("mobile_ions", False)))
    c.eps = float(phys.get("eps", math.inf))
    for k in ("ppc", "n_new", "n_crit", "n_ssa", "frac_bits"):
        if k in phys:
            setattr(c, k, int(phys[k]))
    c.mg_rtol = float(phys.get("mg_rtol", 1e-10))
    c.precision = int(precision)
    c.field_precision = int(field_precision)
    c.particle_capacity = int(capacity)
    if stream is not None:
        c.stream = ctypes.c_void_p(stream)
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


class Handle:
    """Owns one itokmc handle; every method is one C call plus marshalling."""

    def __init__(self, cfg: Config, torch_memory: bool = True):
        import torch
        self.torch = torch
        self._alloc = None
        if torch_memory:
            self._alloc = _TorchAllocator()
            cfg.alloc = self._alloc.alloc_cb
            cfg.free_fn = self._alloc.free_cb
        if not cfg.stream:
            cfg.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        self.cfg = cfg
        self.n = cfg.n[0]
        self.R = cfg.n_realizations
        h = ctypes.c_void_p()
        code = lib().itokmc_init(ctypes.byref(cfg), ctypes.byref(h))
        if code != ITOKMC_OK:
            raise ItokmcError(code, lib().itokmc_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().itokmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state
    def itokmc_set_particles(self, x, y, z, w, realization=None, mem=HOST):
        n = len(w)
        if mem == HOST:
            x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
            z = np.ascontiguousarray(z, np.float64); w = np.ascontiguousarray(w, np.uint32)
            if realization is not None:
                realization = np.ascontiguousarray(realization, np.int32)
        _check(lib().itokmc_set_particles(self.h, _ptr(x), _ptr(y), _ptr(z), _ptr(w), _ptr(realization), n, mem),
               self.h)

    def itokmc_set_particles_species(self, x, y, z, w, species, realization=None, mem=HOST):
        n = len(w)
        if mem == HOST:
            x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
            z = np.ascontiguousarray(z, np.float64); w = np.ascontiguousarray(w, np.uint32)
            species = np.ascontiguousarray(species, np.int32)
            if realization is not None:
                realization = np.ascontiguousarray(realization, np.int32)
        _check(lib().itokmc_set_particles_species(self.h, _ptr(x), _ptr(y), _ptr(z), _ptr(w), _ptr(realization),
                                                  _ptr(species), n, mem), self.h)

    def itokmc_read_particles(self):
        n = ctypes.c_int64()
        lib().itokmc_num_particles(self.h, ctypes.byref(n))
        N = n.value
        x, y, z = np.empty(N), np.empty(N), np.empty(N)
        w = np.empty(N, np.uint32)
        r = np.empty(N, np.int32)
        c = np.empty(N, np.int64)
        _check(lib().itokmc_read_particles(self.h, _ptr(x), _ptr(y), _ptr(z), _ptr(w), _ptr(r), _ptr(c), N,
                                           ctypes.byref(n), HOST), self.h)
        # the particle block b: species b // R, realization b % R
        return dict(x=x, y=y, z=z, w=w, realization=r % self.R, species=r // self.R, cell=c)

    def itokmc_set_ions(self, npos, nneg):
        npos = np.ascontiguousarray(npos, np.int64); nneg = np.ascontiguousarray(nneg, np.int64)
        _check(lib().itokmc_set_ions(self.h, _ptr(npos), _ptr(nneg), HOST), self.h)

    def itokmc_set_field(self, Ex, Ey, Ez):
        E = np.ascontiguousarray(np.concatenate([np.ravel(Ex), np.ravel(Ey), np.ravel(Ez)]), np.float64)
        _check(lib().itokmc_set_field(self.h, _ptr(E), HOST), self.h)

    def itokmc_solve_field(self):
        _check(lib().itokmc_solve_field(self.h), self.h)

    def itokmc_step(self, nsteps=1):
        _check(lib().itokmc_step(self.h, int(nsteps)), self.h)

    def itokmc_run_stage(self, stage):
        _check(lib().itokmc_run_stage(self.h, int(stage)), self.h)

    def itokmc_autotune(self):
        t = Tuning()
        _check(lib().itokmc_autotune(self.h, ctypes.byref(t)), self.h)
        return {"mg_nu1": t.mg_nu1, "mg_nu2": t.mg_nu2, "ms_field": t.ms_field, "cycles": t.cycles,
                "tried": [((t.nu_tried[k][0], t.nu_tried[k][1]), t.ms_tried[k]) for k in range(t.n_tried)],
                "dep_win": t.dep_win,
                "dep_tried": [(t.dep_tried[k], t.ms_dep_tried[k]) for k in range(t.n_dep_tried)]}

    def itokmc_advance_counter(self):
        _check(lib().itokmc_advance_counter(self.h), self.h)

    def itokmc_transport_semi_implicit(self):
        """The semi-implicit transport stage; returns (V-cycles, relative residual)."""
        cyc = ctypes.c_int32()
        rel = ctypes.c_double()
        _check(lib().itokmc_transport_semi_implicit(self.h, ctypes.byref(cyc), ctypes.byref(rel)), self.h)
        return cyc.value, rel.value

    def itokmc_read_densities(self, which, realization=0):
        cells = self.n ** 3 * (self.R if realization < 0 else 1)
        blocks = {E: 3, FIRINGS: 5}.get(which, 1)
        dt = np.float64 if which in (PHI, E) else np.int64
        out = np.empty(blocks * cells, dtype=dt)
        _check(lib().itokmc_read_densities(self.h, int(realization), int(which), _ptr(out), out.nbytes), self.h)
        return out.reshape(blocks, cells) if blocks > 1 else out

    def itokmc_seed_blobs(self, blobs, flags=0):
        arr = blob_array(blobs)
        _check(lib().itokmc_seed_blobs(self.h, arr, len(blobs), int(flags)), self.h)

    def itokmc_save(self, path):
        _check(lib().itokmc_save(self.h, os.fsencode(path)), self.h)

    def itokmc_load(self, path):
        _check(lib().itokmc_load(self.h, os.fsencode(path)), self.h)

    def itokmc_get_stats(self):
        st = Stats()
        _check(lib().itokmc_get_stats(self.h, ctypes.byref(st)), self.h)
        return st.as_dict()

    def itokmc_num_particles(self):
        n = ctypes.c_int64()
        _check(lib().itokmc_num_particles(self.h, ctypes.byref(n)), self.h)
        return n.value
