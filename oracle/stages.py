"""Stage wrappers and the full-step composition of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The arithmetic of every
stage is in ``itokmc_oracle.c``; this module marshals numpy arrays and chains the
stages in the order of one time step:

  push (a1+a2) -> stable sort by cell (a3) -> deposit ne_fix, X_e (a4)
  -> rho snapshot -> KMC (a6) -> products and photons (a7, a8)
  -> merge/split (a9)

with the field for the next step solved from the rho snapshot (a5,
``poisson.py``).  The order is the Godunov split of the paper's final algorithm
(Sec. 4.7: transport, then chemistry, then superparticle management) with the
explicit Euler-Maruyama push of Sec. 4.3.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Params, _P, lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def push(p: Params, x, y, z, E):
    """a1+a2.  E = (Ex, Ey, Ez) cell-centred arrays of n^3 (x fastest).
    Returns (xo, yo, zo, cell) with cell = -1 for removed particles."""
    x, y, z = _d(x), _d(y), _d(z)
    Ex, Ey, Ez = (_d(np.asarray(e).ravel()) for e in E)
    n = len(x)
    xo, yo, zo = np.empty(n), np.empty(n), np.empty(n)
    cell = np.empty(n, dtype=np.int64)
    lib().ora_push(ctypes.byref(p), n, _P(x, ctypes.c_double), _P(y, ctypes.c_double),
                   _P(z, ctypes.c_double), _P(Ex, ctypes.c_double), _P(Ey, ctypes.c_double),
                   _P(Ez, ctypes.c_double), _P(xo, ctypes.c_double), _P(yo, ctypes.c_double),
                   _P(zo, ctypes.c_double), _P(cell, ctypes.c_int64))
    return xo, yo, zo, cell


def sort_by_cell(cell, ncell: int):
    """a3.  Stable permutation by cell; removed (-1) dropped."""
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    perm = np.empty(len(cell), dtype=np.int64)
    k = lib().ora_sort_by_cell(len(cell), int(ncell), _P(cell, ctypes.c_int64), _P(perm, ctypes.c_int64))
    return perm[:k]


def deposit(p: Params, x, y, z, w, cell):
    """a4.  Returns (ne_fix, Xe), int64 arrays of n^3."""
    ncell = p.n ** 3
    x, y, z = _d(x), _d(y), _d(z)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    ne = np.zeros(ncell, dtype=np.int64)
    Xe = np.zeros(ncell, dtype=np.int64)
    lib().ora_deposit(ctypes.byref(p), len(x), _P(x, ctypes.c_double), _P(y, ctypes.c_double),
                      _P(z, ctypes.c_double), _P(w, ctypes.c_uint32), _P(cell, ctypes.c_int64),
                      _P(ne, ctypes.c_int64), _P(Xe, ctypes.c_int64))
    return ne, Xe


def kmc(p: Params, Xe, E, Npos=None, Nneg=None):
    """a6.  Returns the firings per cell (n_ion, n_att, n_ph, n_ep, n_np):
    ionization, attachment, photon emission, electron-ion and ion-ion
    recombination (the last two zero unless p.beta_ep / p.beta_np > 0, which
    need the ion counts Npos, Nneg at the start of the chemistry)."""
    ncell = p.n ** 3
    Xe = np.ascontiguousarray(Xe, dtype=np.int64)
    Ex, Ey, Ez = (_d(np.asarray(e).ravel()) for e in E)
    a, b, c, d, e = (np.zeros(ncell, dtype=np.int64) for _ in range(5))
    zero = np.zeros(ncell, dtype=np.int64)
    Np = np.ascontiguousarray(Npos if Npos is not None else zero, dtype=np.int64)
    Nn = np.ascontiguousarray(Nneg if Nneg is not None else zero, dtype=np.int64)
    st = lib().ora_kmc(ctypes.byref(p), _P(Xe, ctypes.c_int64), _P(Np, ctypes.c_int64), _P(Nn, ctypes.c_int64),
                       _P(Ex, ctypes.c_double), _P(Ey, ctypes.c_double), _P(Ez, ctypes.c_double),
                       _P(a, ctypes.c_int64), _P(b, ctypes.c_int64), _P(c, ctypes.c_int64),
                       _P(d, ctypes.c_int64), _P(e, ctypes.c_int64))
    if st != 0:
        raise RuntimeError("oracle KMC iteration guard hit")
    return a, b, c, d, e


def cell_start_of(cell, ncell):
    return np.searchsorted(cell, np.arange(ncell + 1), side="left").astype(np.int64)


def products_photons(p: Params, x, y, z, w, cell, Xe, fired, Npos, Nneg, with_meta=False):
    """a7 + a8.  w (uint32) is updated in place for losses; Npos/Nneg in place.
    Returns (new particle arrays (x, y, z, w, cell), lost photon weight), and
    with ``with_meta`` also (source cell, kind 0 product / 1 photoelectron,
    slot) of each new particle."""
    ncell = p.n ** 3
    cs = cell_start_of(cell, ncell)
    n_ion, n_att, n_ph = (np.ascontiguousarray(f, dtype=np.int64) for f in fired[:3])
    zero = np.zeros(ncell, dtype=np.int64)
    n_ep = np.ascontiguousarray(fired[3], dtype=np.int64) if len(fired) > 3 else zero
    n_np = np.ascontiguousarray(fired[4], dtype=np.int64) if len(fired) > 4 else zero
    cap = int(np.minimum(n_ion + n_ph, 2 * p.n_new).sum()) + 16
    nx, ny, nz = np.empty(cap), np.empty(cap), np.empty(cap)
    nw = np.empty(cap, dtype=np.uint32)
    nc = np.empty(cap, dtype=np.int64)
    src = np.empty(cap, dtype=np.int64)
    kind = np.empty(cap, dtype=np.int32)
    slot = np.empty(cap, dtype=np.int32)
    lost = ctypes.c_int64(0)
    x, y, z = _d(x), _d(y), _d(z)
    Xe = np.ascontiguousarray(Xe, dtype=np.int64)
    assert w.dtype == np.uint32 and w.flags.c_contiguous
    assert Npos.dtype == np.int64 and Nneg.dtype == np.int64
    k = lib().ora_products_photons(ctypes.byref(p), len(x), _P(x, ctypes.c_double), _P(y, ctypes.c_double),
                                   _P(z, ctypes.c_double), _P(w, ctypes.c_uint32), _P(cs, ctypes.c_int64),
                                   _P(Xe, ctypes.c_int64), _P(n_ion, ctypes.c_int64),
                                   _P(n_att, ctypes.c_int64), _P(n_ph, ctypes.c_int64),
                                   _P(n_ep, ctypes.c_int64), _P(n_np, ctypes.c_int64),
                                   _P(Npos, ctypes.c_int64), _P(Nneg, ctypes.c_int64),
                                   _P(nx, ctypes.c_double), _P(ny, ctypes.c_double), _P(nz, ctypes.c_double),
                                   _P(nw, ctypes.c_uint32), _P(nc, ctypes.c_int64), cap, ctypes.byref(lost),
                                   _P(src, ctypes.c_int64), _P(kind, ctypes.c_int32), _P(slot, ctypes.c_int32))
    if k < 0:
        raise RuntimeError(f"oracle products/photons failed ({k})")
    new = (nx[:k], ny[:k], nz[:k], nw[:k], nc[:k])
    if with_meta:
        return new, int(lost.value), (src[:k], kind[:k], slot[:k])
    return new, int(lost.value)


# ---------------------------------------------------------------- mobile ions
SPECIES = ("e", "pos", "neg")          # charge numbers -1, +1, -1


def push_species(p: Params, species: int, x, y, z, E):
    """a1+a2 for species 0 (electrons, V = -mu E), 1 (positive ions, V =
    +mu_ion E) or 2 (negative ions, V = -mu_ion E): Eq. ito_kernel with
    Eq. Vk1's sgn(Z_s).  Returns (xo, yo, zo, cell) as ``push``."""
    x, y, z = _d(x), _d(y), _d(z)
    Ex, Ey, Ez = (_d(np.asarray(e).ravel()) for e in E)
    n = len(x)
    xo, yo, zo = np.empty(n), np.empty(n), np.empty(n)
    cell = np.empty(n, dtype=np.int64)
    lib().ora_push_species(ctypes.byref(p), int(species), n, _P(x, ctypes.c_double), _P(y, ctypes.c_double),
                           _P(z, ctypes.c_double), _P(Ex, ctypes.c_double), _P(Ey, ctypes.c_double),
                           _P(Ez, ctypes.c_double), _P(xo, ctypes.c_double), _P(yo, ctypes.c_double),
                           _P(zo, ctypes.c_double), _P(cell, ctypes.c_int64))
    return xo, yo, zo, cell


def species_products(p: Params, species: int, cell, w, X, dN):
    """Gain (new particles) or loss (w updated in place) of ion species 1 or
    2 per cell.  Returns the new particles (x, y, z, w, cell) and their
    (source cell, kind, slot)."""
    ncell = p.n ** 3
    cs = cell_start_of(cell, ncell)
    dN = np.ascontiguousarray(dN, dtype=np.int64)
    X = np.ascontiguousarray(X, dtype=np.int64)
    assert w.dtype == np.uint32 and w.flags.c_contiguous
    cap = int(np.minimum(np.maximum(dN, 0), p.n_new).sum()) + 16
    nx, ny, nz = np.empty(cap), np.empty(cap), np.empty(cap)
    nw = np.empty(cap, dtype=np.uint32)
    nc = np.empty(cap, dtype=np.int64)
    src = np.empty(cap, dtype=np.int64)
    kind = np.empty(cap, dtype=np.int32)
    slot = np.empty(cap, dtype=np.int32)
    k = lib().ora_species_products(ctypes.byref(p), int(species), _P(cs, ctypes.c_int64), _P(X, ctypes.c_int64),
                                   _P(dN, ctypes.c_int64), _P(w, ctypes.c_uint32), _P(nx, ctypes.c_double),
                                   _P(ny, ctypes.c_double), _P(nz, ctypes.c_double), _P(nw, ctypes.c_uint32),
                                   _P(nc, ctypes.c_int64), _P(src, ctypes.c_int64), _P(kind, ctypes.c_int32),
                                   _P(slot, ctypes.c_int32), cap)
    if k < 0:
        raise RuntimeError(f"oracle ion products failed ({k})")
    return (nx[:k], ny[:k], nz[:k], nw[:k], nc[:k]), (src[:k], kind[:k], slot[:k])


def step_mobile(p: Params, state: dict, E):
    """One explicit step with the ions as Ito particles (the paper's
    all-particle model, Sec. 4.3 Eq. particle_kernel with sgn(Z_s); SURVEY
    row f2).  state: "e", "pos", "neg", each x, y, z (float64), w (uint32),
    cell (int64) in canonical order.  Every species is pushed (its own
    mobility, diffusion and stream tag), sorted and deposited; the space
    charge is the CIC densities' n+ - n- - ne (units q_e 2^-3s); the KMC
    reads the NGP counts of the three species; electrons gain products,
    losses and photoelectrons as in ``step``; each ion species gains or
    loses dN (positive ions n_ion - n_ep - n_np plus one ion per absorbed
    photon at its electron's position and weight, negative ions n_att -
    n_np); each species is merged with its new particles in (source cell,
    product before photo-ion, slot) order.  Returns (new_state, info)."""
    ncell = p.n ** 3
    srt, fix, cnt, outflow = {}, {}, {}, {}
    for sp, key in enumerate(SPECIES):
        S = state[key]
        w0 = np.asarray(S["w"], np.uint32)
        xo, yo, zo, cnew = push_species(p, sp, S["x"], S["y"], S["z"], E)
        outflow[key] = int(w0[cnew < 0].astype(np.int64).sum())
        perm = sort_by_cell(cnew, ncell)
        srt[key] = dict(x=xo[perm], y=yo[perm], z=zo[perm], w=w0[perm].copy(), cell=cnew[perm])
        T = srt[key]
        fix[key], cnt[key] = deposit(p, T["x"], T["y"], T["z"], T["w"], T["cell"])
    rho = fix["pos"] - fix["neg"] - fix["e"]
    sorted_state = {k: {f: v.copy() for f, v in srt[k].items()} for k in SPECIES}
    fired = kmc(p, cnt["e"], E, cnt["pos"], cnt["neg"])
    n_ion, n_att, n_ph, n_ep, n_np = fired
    T = srt["e"]
    dummy_p, dummy_n = np.zeros(ncell, np.int64), np.zeros(ncell, np.int64)
    new_e, lost, meta_e = products_photons(p, T["x"], T["y"], T["z"], T["w"], T["cell"], cnt["e"], fired,
                                           dummy_p, dummy_n, with_meta=True)
    new = {"e": (new_e, None)}
    for sp, key, dN in ((1, "pos", n_ion - n_ep - n_np), (2, "neg", n_att - n_np)):
        T = srt[key]
        nk, mk = species_products(p, sp, T["cell"], T["w"], cnt[key], dN)
        if sp == 1:
            ph = meta_e[1] == 1
            nk = tuple(np.concatenate([a, b[ph]]) for a, b in zip(nk, new_e))
            mk = tuple(np.concatenate([a, b[ph]]) for a, b in zip(mk, meta_e))
        order = np.lexsort((mk[2], mk[1], mk[0], nk[4]))
        new[key] = (tuple(a[order] for a in nk), None)
    out = {}
    for key in SPECIES:
        T = srt[key]
        nk = new[key][0]
        ax = np.concatenate([T["x"], nk[0]]); ay = np.concatenate([T["y"], nk[1]])
        az = np.concatenate([T["z"], nk[2]]); aw = np.concatenate([T["w"], nk[3]])
        ac = np.concatenate([T["cell"], nk[4]])
        order = np.argsort(ac, kind="stable")
        mx, my, mz, mw, mc = merge(p, ax[order], ay[order], az[order], aw[order], ac[order])
        out[key] = dict(x=mx, y=my, z=mz, w=mw, cell=mc)
    info = dict(sorted=sorted_state, fix=fix, counts=cnt, rho_fixed=rho, n_ion=n_ion, n_att=n_att, n_ph=n_ph,
                n_ep=n_ep, n_np=n_np, outflow=outflow, lost_photon=lost,
                weights_after_loss={k: srt[k]["w"] for k in SPECIES}, new_particles={k: new[k][0] for k in SPECIES})
    return out, info


def merge(p: Params, x, y, z, w, cell):
    """a9 on a list grouped by cell (canonical order).  Returns the merged
    particle arrays (x, y, z, w, cell)."""
    ncell = p.n ** 3
    cs = cell_start_of(cell, ncell)
    x, y, z = _d(x), _d(y), _d(z)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    W = np.zeros(ncell, np.int64)
    np.add.at(W, np.asarray(cell, np.int64), w.astype(np.int64))
    cap = int(np.minimum(W, p.ppc).sum()) + 1
    ox, oy, oz = np.empty(cap), np.empty(cap), np.empty(cap)
    ow = np.empty(cap, dtype=np.uint32)
    oc = np.empty(cap, dtype=np.int64)
    k = lib().ora_merge(ctypes.byref(p), _P(x, ctypes.c_double), _P(y, ctypes.c_double),
                        _P(z, ctypes.c_double), _P(w, ctypes.c_uint32), _P(cs, ctypes.c_int64),
                        _P(ox, ctypes.c_double), _P(oy, ctypes.c_double), _P(oz, ctypes.c_double),
                        _P(ow, ctypes.c_uint32), _P(oc, ctypes.c_int64), cap)
    if k < 0:
        raise RuntimeError(f"oracle merge failed ({k})")
    return ox[:k], oy[:k], oz[:k], ow[:k], oc[:k]


def rho_fixed(p: Params, ne_fix, Npos, Nneg):
    """Space charge per cell in units of q_e 2^-3s: 2^3s (N+ - N-) - ne_fix."""
    return (np.asarray(Npos, np.int64) - np.asarray(Nneg, np.int64)) * (1 << (3 * p.frac_bits)) - ne_fix


def step(p: Params, state: dict, E):
    """One full step (a1-a4, a6-a9) from ``state`` with field E = (Ex,Ey,Ez).

    state: x, y, z (float64), w (uint32), cell (int64), canonical order;
    Npos, Nneg (int64 n^3).  Returns (new_state, info) where info holds the
    intermediate results: sorted particles, ne_fix, Xe, rho_fixed (for the
    next field solve), firings, outflow and lost-photon weights."""
    xo, yo, zo, cnew = push(p, state["x"], state["y"], state["z"], E)
    return after_transport(p, state, xo, yo, zo, cnew, E)


def after_transport(p: Params, state: dict, xo, yo, zo, cnew, E):
    """The rest of a step once the particles of ``state`` have moved to
    (xo, yo, zo) in cells cnew (-1: left the box): the stable sort, the
    deposit and charge, KMC with the field E, products, photons and the
    merge/split.  Returns (new_state, info) as ``step``."""
    ncell = p.n ** 3
    w0 = np.asarray(state["w"], np.uint32)
    outflow = int(w0[cnew < 0].astype(np.int64).sum())
    perm = sort_by_cell(cnew, ncell)
    sx, sy, sz, sw, sc = xo[perm], yo[perm], zo[perm], w0[perm].copy(), cnew[perm]
    ne, Xe = deposit(p, sx, sy, sz, sw, sc)
    Npos = np.array(state["Npos"], dtype=np.int64, copy=True)
    Nneg = np.array(state["Nneg"], dtype=np.int64, copy=True)
    rho = rho_fixed(p, ne, Npos, Nneg)
    fired = kmc(p, Xe, E, Npos, Nneg)
    sorted_state = dict(x=sx.copy(), y=sy.copy(), z=sz.copy(), w=sw.copy(), cell=sc.copy())
    new, lost = products_photons(p, sx, sy, sz, sw, sc, Xe, fired, Npos, Nneg)
    ax = np.concatenate([sx, new[0]]); ay = np.concatenate([sy, new[1]])
    az = np.concatenate([sz, new[2]]); aw = np.concatenate([sw, new[3]])
    ac = np.concatenate([sc, new[4]])
    order = np.argsort(ac, kind="stable")
    mx, my, mz, mw, mc = merge(p, ax[order], ay[order], az[order], aw[order], ac[order])
    new_state = dict(x=mx, y=my, z=mz, w=mw, cell=mc, Npos=Npos, Nneg=Nneg)
    info = dict(sorted=sorted_state, ne_fix=ne, Xe=Xe, rho_fixed=rho, n_ion=fired[0], n_att=fired[1],
                n_ph=fired[2], n_ep=fired[3], n_np=fired[4], outflow=outflow, lost_photon=lost,
                weights_after_loss=sw, new_particles=new)
    return new_state, info
