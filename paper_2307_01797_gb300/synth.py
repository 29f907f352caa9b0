"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only builds parameter sets
and random initial states (particles, fields, ion counts) with numpy's PCG64
generator.  Both the CUDA library and the CPU oracle are fed from here.

Workload recipes (the paper's own inputs -- needle geometry, AMR grids,
BOLSIG+ transport data -- are not available, so these stand in):

* ``physics_small``: 64^3 over a 1 cm cube, 1.5 MV/m, mu=0.0211, D=0.1,
  alpha=4.3e5 exp(-1.9e7/|E|), eta=2e3, dt=1 ps, ppc=8, no photons; a Gaussian
  electron blob (sigma 0.5 mm, peak 1e18 m^-3, centre (L/2, L/2, 0.8L)).
* ``physics_streamer``: 256^3 over a 2 cm cube, 1.5 MV/m, dt=5 ps, ppc=32,
  photoionization on (k_gamma = 0.06 k_alpha, kappa log-uniform in
  [520, 3e4] 1/m); seed blob sigma 0.2 mm, peak 1e19 at z=0.9L.
* ``physics_ensemble_member``: 128^3 over a 1 cm cube, ppc=16, photons on.
* ``physics_tree``: 512^3 over a 4 cm cube, 1.8 MV/m, ppc=64, photons on.
* ``streamer_tree_state``: a developed discharge tree on a grid -- K channels
  (line segments from the anode side downwards, Gaussian radial profile of
  peak density n_ch and radius sigma_r) -- sampled to at most ppc particles
  per cell; sized so that the particle count reaches the target (about 1e8 on
  the 256^3 grid).
* ``uniform_slab_state``: N particles uniform in a z-slab (count-pinned sweep).
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------- parameters
def _base(n, L, E0, dt, ppc, photons):
    return dict(
        n=n, lo=(0.0, 0.0, 0.0), hi=(L, L, L), dt=dt, E0=E0,
        mu=0.0211, D=0.1, alpha_A=4.3e5, alpha_B=1.9e7, eta=2.0e3,
        photon_ratio=0.06 if photons else 0.0, kappa_lo=520.0, kappa_hi=3.0e4,
        ppc=ppc, n_new=64, n_crit=5, n_ssa=10, frac_bits=10, eps=float("inf"),
        mg_rtol=1e-10,
    )


def with_recombination(phys, T=300.0):
    """A copy of ``phys`` with the air recombination coefficients of Sec. 5.1:
    beta_ep = 1.138e-11 T_e^-0.7 m^3/s and beta_np = 2e-13 (300/T)^0.5 m^3/s,
    T the gas temperature in K.  The transport here has a constant mobility
    and diffusion coefficient, so the electron temperature is the one of the
    Einstein relation, k_B T_e = e D / mu (in K: T_e = (D / mu) e / k_B), and
    the coefficients are constants."""
    e_over_kB = 1.602176634e-19 / 1.380649e-23
    Te = (phys["D"] / phys["mu"]) * e_over_kB
    out = dict(phys)
    out["beta_ep"] = 1.138e-11 * Te ** -0.7
    out["beta_np"] = 2e-13 * (300.0 / T) ** 0.5
    return out


def with_mobile_ions(phys, mu_ion=2e-4, T=300.0):
    """A copy of ``phys`` with mobile ions (the ions as Ito particles, Sec.
    4.3 Eq. particle_kernel with sgn(Z_s)): ion mobility mu_ion in m^2/Vs
    (the paper gives none; 2e-4 is the order of N2+/O2- in air at 1 bar) and
    the ions' diffusion coefficient from the Einstein relation at the gas
    temperature T, D = mu k_B T / e."""
    out = dict(phys)
    out["mu_ion"] = float(mu_ion)
    out["D_ion"] = float(mu_ion) * (1.380649e-23 * T / 1.602176634e-19)
    return out


def ion_particles(phys, seed, n_per_cell=2, mean=40, frac=0.4, cells=None):
    """Ion superparticles (x, y, z, w, sorted by cell) on a random fraction of
    the cells: n_per_cell particles uniform in each chosen cell sharing a
    Poisson(mean) count (cells drawing 0 hold none)."""
    n = phys["n"]
    rng = np.random.Generator(np.random.PCG64(seed))
    if cells is None:
        cells = np.flatnonzero(rng.random(n ** 3) < frac)
    N = rng.poisson(mean, len(cells)).astype(np.int64)
    keep = N > 0
    cells, N = cells[keep], N[keep]
    m = np.minimum(N, n_per_cell)
    reps, w = _split_counts(N, m)
    c = cells[reps]
    h = cell_size(phys)
    lo = phys["lo"]
    ijk = np.stack([c % n, (c // n) % n, c // (n * n)], axis=1)
    X = [lo[a] + (ijk[:, a] + rng.random(len(c))) * h for a in range(3)]
    return dict(x=X[0], y=X[1], z=X[2], w=w.astype(np.uint32))


def ions_from_counts(phys, N, seed, per_cell=8):
    """Ion superparticles from per-cell counts N (int64 n^3): in each cell
    with N > 0, m = min(N, per_cell) particles uniform in the cell sharing N
    (near-equal integer weights).  Returns dict(x, y, z, w) sorted by cell."""
    n = phys["n"]
    N = np.asarray(N, np.int64)
    cells = np.flatnonzero(N > 0)
    m = np.minimum(N[cells], per_cell)
    reps, w = _split_counts(N[cells], m)
    c = cells[reps]
    rng = np.random.Generator(np.random.PCG64(seed))
    h = cell_size(phys)
    lo = phys["lo"]
    ijk = np.stack([c % n, (c // n) % n, c // (n * n)], axis=1)
    X = [lo[a] + (ijk[:, a] + rng.random(len(c))) * h for a in range(3)]
    return dict(x=X[0], y=X[1], z=X[2], w=w.astype(np.uint32))


def physics_small(n=64):
    """64^3, 1 cm, 1.5 MV/m, dt = 1 ps, ppc = 8, photons off."""
    return _base(n, 0.01, 1.5e6, 1e-12, 8, False)


def physics_streamer(n=256):
    """256^3, 2 cm, 1.5 MV/m, dt = 5 ps, ppc = 32, photons on."""
    return _base(n, 0.02, 1.5e6, 5e-12, 32, True)


def physics_ensemble_member(n=128):
    """128^3, 1 cm, 1.5 MV/m, dt = 5 ps, ppc = 16, photons on."""
    return _base(n, 0.01, 1.5e6, 5e-12, 16, True)


def physics_tree(n=512):
    """512^3, 4 cm, 1.8 MV/m, dt = 5 ps, ppc = 64, photons on."""
    return _base(n, 0.04, 1.8e6, 5e-12, 64, True)


def cell_size(phys):
    return (phys["hi"][0] - phys["lo"][0]) / phys["n"]


# --------------------------------------------------------------- particles
def _split_counts(N, m):
    """Split integer totals N (per cell) into m near-equal integer parts."""
    reps = np.repeat(np.arange(len(N)), m)
    first = np.repeat(np.cumsum(m) - m, m)
    slot = np.arange(reps.size) - first
    base = np.repeat(N // np.maximum(m, 1), m)
    extra = (slot < np.repeat(N % np.maximum(m, 1), m)).astype(np.int64)
    return reps, base + extra


def sample_density(phys, density_fn, seed, max_per_cell=None, cells=None):
    """Per cell: N_c ~ Poisson(n(x_c) dV), then min(ppc, N_c) particles
    uniform in the cell sharing N_c.  Returns dict(x, y, z, w) sorted by cell.
    ``density_fn(xc, yc, zc)`` gives n in m^-3 at cell centres."""
    n = phys["n"]
    h = cell_size(phys)
    lo = np.asarray(phys["lo"], dtype=np.float64)
    ppc = phys["ppc"] if max_per_cell is None else max_per_cell
    rng = np.random.Generator(np.random.PCG64(seed))
    if cells is None:
        cells = np.arange(n ** 3, dtype=np.int64)
    i = cells % n
    j = (cells // n) % n
    k = cells // (n * n)
    xc = lo[0] + (i + 0.5) * h
    yc = lo[1] + (j + 0.5) * h
    zc = lo[2] + (k + 0.5) * h
    lam = density_fn(xc, yc, zc) * h ** 3
    N = rng.poisson(lam).astype(np.int64)
    N = np.minimum(N, 2 ** 31)
    occ = N > 0
    cells, N, i, j, k = cells[occ], N[occ], i[occ], j[occ], k[occ]
    m = np.minimum(N, ppc)
    reps, w = _split_counts(N, m)
    u = rng.random((3, reps.size))
    u = np.clip(u, 1e-9, 1.0 - 1e-9)
    x = lo[0] + (i[reps] + u[0]) * h
    y = lo[1] + (j[reps] + u[1]) * h
    z = lo[2] + (k[reps] + u[2]) * h
    return dict(x=x, y=y, z=z, w=w.astype(np.uint32))


def gaussian_blobs(centers, sigma, peak):
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)

    def fn(x, y, z):
        out = np.zeros_like(x)
        for c in centers:
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            out += peak * np.exp(-r2 / (2.0 * sigma * sigma))
        return out
    return fn


def blob_state(phys, seed=1, sigma=5e-4, peak=1e18, zfrac=0.8, centers=None):
    """Gaussian electron seed (electrons only) sampled per cell."""
    L = phys["hi"][0] - phys["lo"][0]
    if centers is None:
        centers = [(phys["lo"][0] + L / 2, phys["lo"][1] + L / 2, phys["lo"][2] + zfrac * L)]
    n = phys["n"]
    h = cell_size(phys)
    # only cells within 7 sigma of a centre can hold a particle
    cen = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    lo = np.asarray(phys["lo"])
    sel = []
    for c in cen:
        rmin = np.floor((c - 7 * sigma - lo) / h).astype(int).clip(0, n - 1)
        rmax = np.floor((c + 7 * sigma - lo) / h).astype(int).clip(0, n - 1)
        ii, jj, kk = np.meshgrid(np.arange(rmin[0], rmax[0] + 1), np.arange(rmin[1], rmax[1] + 1),
                                 np.arange(rmin[2], rmax[2] + 1), indexing="ij")
        sel.append(((kk * n + jj) * n + ii).ravel())
    cells = np.unique(np.concatenate(sel)).astype(np.int64)
    return sample_density(phys, gaussian_blobs(centers, sigma, peak), seed, cells=cells)


def streamer_tree_geometry(phys, target_particles, seed=7, n_ch=1e19, sigma_r=5e-4, branches=4):
    """Channel segments of a synthetic discharge tree: ``branches`` line
    segments from the anode side (z = 0.9 L) downward and outward, their
    length chosen so that ~``target_particles`` superparticles fill them."""
    L = phys["hi"][0] - phys["lo"][0]
    h = cell_size(phys)
    lo = np.asarray(phys["lo"])
    ppc = phys["ppc"]
    r_occ = sigma_r * math.sqrt(2.0 * math.log(max(n_ch * h ** 3, 2.0)))
    cells_per_len = math.pi * (r_occ / h) ** 2
    # about 55% of the cells within r_occ reach ppc particles (Gaussian tail)
    length = min(0.85 * L, target_particles / (0.55 * ppc * branches * cells_per_len) * h)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    top = np.array([lo[0] + L / 2, lo[1] + L / 2, lo[2] + 0.9 * L])
    segs = []
    for b in range(branches):
        ang = 2 * math.pi * b / branches + rng.uniform(-0.3, 0.3)
        tilt = 0.25 if branches > 1 else 0.0
        d = np.array([tilt * math.cos(ang), tilt * math.sin(ang), -1.0])
        d /= np.linalg.norm(d)
        segs.append((top, top + length * d))
    return segs, r_occ


def streamer_tree_state(phys, target_particles, seed=7, n_ch=1e19, sigma_r=5e-4, branches=4):
    """A developed streamer tree: the channels of ``streamer_tree_geometry``
    with Gaussian radial profile n_ch exp(-r^2/2 sigma_r^2), sampled to at
    most ppc particles per cell."""
    n = phys["n"]
    h = cell_size(phys)
    lo = np.asarray(phys["lo"])
    segs, r_occ = streamer_tree_geometry(phys, target_particles, seed, n_ch, sigma_r, branches)

    def fn(x, y, z):
        out = np.zeros_like(x)
        P = np.stack([x, y, z], axis=-1)
        for a, bpt in segs:
            ab = bpt - a
            t = np.clip(((P - a) @ ab) / (ab @ ab), 0.0, 1.0)
            d2 = ((P - (a + t[:, None] * ab)) ** 2).sum(-1)
            out = np.maximum(out, n_ch * np.exp(-d2 / (2 * sigma_r * sigma_r)))
        return out

    # candidate cells: bounding boxes of the segments padded by r_occ
    sel = []
    for a, bpt in segs:
        mn = np.minimum(a, bpt) - 1.5 * r_occ
        mx = np.maximum(a, bpt) + 1.5 * r_occ
        rmin = np.floor((mn - lo) / h).astype(int).clip(0, n - 1)
        rmax = np.floor((mx - lo) / h).astype(int).clip(0, n - 1)
        ii, jj, kk = np.meshgrid(np.arange(rmin[0], rmax[0] + 1), np.arange(rmin[1], rmax[1] + 1),
                                 np.arange(rmin[2], rmax[2] + 1), indexing="ij")
        sel.append(((kk * n + jj) * n + ii).ravel())
    cells = np.unique(np.concatenate(sel)).astype(np.int64)
    out = {k: [] for k in ("x", "y", "z", "w")}
    for c0 in range(0, cells.size, 1 << 22):
        part = sample_density(phys, fn, seed + 17 * c0, cells=cells[c0:c0 + (1 << 22)])
        for k in out:
            out[k].append(part[k])
    return {k: np.concatenate(v) for k, v in out.items()}


def cell_counts(phys, st):
    """Electrons per cell of a particle state (NGP by floor of the position)."""
    n = phys["n"]
    h = cell_size(phys)
    lo = np.asarray(phys["lo"])
    ijk = [np.clip(np.floor((np.asarray(st[a]) - lo[q]) / h).astype(np.int64), 0, n - 1)
           for q, a in enumerate(("x", "y", "z"))]
    c = (ijk[2] * n + ijk[1]) * n + ijk[0]
    return np.bincount(c, weights=np.asarray(st["w"], np.float64), minlength=n ** 3)


def streamer_ions(phys, st, seed=8, head_density=3e18, target_particles=None, sigma_r=5e-4, branches=4):
    """Ion counts for a streamer-tree state: a quasi-neutral channel (N+ =
    electrons per cell) plus a net positive head charge (Gaussian ball of
    density ``head_density``) at each channel tip; N- = 0."""
    n = phys["n"]
    h = cell_size(phys)
    lo = np.asarray(phys["lo"])
    Np = np.rint(cell_counts(phys, st)).astype(np.int64)
    if target_particles is None:
        target_particles = len(st["w"])
    segs, _ = streamer_tree_geometry(phys, target_particles, seed - 1, sigma_r=sigma_r, branches=branches)
    c = lo[0] + (np.arange(n) + 0.5) * h
    rng = np.random.Generator(np.random.PCG64(seed))
    for _, tip in segs:
        r = int(math.ceil(4 * sigma_r / h))
        ic = np.clip(np.floor((tip - lo) / h).astype(int), r, n - 1 - r)
        sl = [slice(ic[q] - r, ic[q] + r + 1) for q in range(3)]
        Z, Y, X = np.meshgrid(c[sl[2]], c[sl[1]], c[sl[0]], indexing="ij")
        d2 = (X - tip[0]) ** 2 + (Y - tip[1]) ** 2 + (Z - tip[2]) ** 2
        add = rng.poisson(head_density * np.exp(-d2 / (2 * sigma_r ** 2)) * h ** 3)
        V = Np.reshape(n, n, n)
        V[sl[2], sl[1], sl[0]] += add
    return Np, np.zeros(n ** 3, np.int64)


def uniform_slab_state(phys, count, seed=1, z0=0.4, z1=0.6, weight=100):
    """``count`` particles uniform in the slab z in [z0 L, z1 L), weight w."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = phys["hi"][0] - phys["lo"][0]
    lo = np.asarray(phys["lo"])
    x = lo[0] + rng.random(count) * L
    y = lo[1] + rng.random(count) * L
    z = lo[2] + (z0 + (z1 - z0) * rng.random(count)) * L
    return dict(x=x, y=y, z=z, w=np.full(count, weight, dtype=np.uint32))


def random_particles(phys, count, seed, wmax=1000, margin=0.0):
    """Particles uniform over the domain (optionally inset by ``margin`` cells)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = cell_size(phys)
    lo = np.asarray(phys["lo"]) + margin * h
    hi = np.asarray(phys["hi"]) - margin * h
    P = lo[:, None] + rng.random((3, count)) * (hi - lo)[:, None]
    w = rng.integers(1, wmax + 1, size=count).astype(np.uint32)
    return dict(x=P[0], y=P[1], z=P[2], w=w)


# --------------------------------------------------------------- fields
def random_field(phys, seed, amp=3e6, base=None):
    """Cell-centred E = applied field (0, 0, -E0) plus smooth random modes of
    amplitude ``amp`` V/m.  Returns (Ex, Ey, Ez) as (n, n, n) [k, j, i]."""
    n = phys["n"]
    rng = np.random.Generator(np.random.PCG64(seed))
    h = cell_size(phys)
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    L = phys["hi"][0] - phys["lo"][0]
    E0 = phys["E0"] if base is None else base
    out = []
    for comp in range(3):
        f = np.zeros((n, n, n))
        for _ in range(3):
            kx, ky, kz = rng.integers(1, 4, size=3)
            ph = rng.random(3) * 2 * np.pi
            f += (amp / 3) * (np.sin(2 * np.pi * kx * X / L + ph[0]) * np.sin(2 * np.pi * ky * Y / L + ph[1])
                              * np.sin(2 * np.pi * kz * Z / L + ph[2]))
        if comp == 2:
            f -= E0
        out.append(f)
    return tuple(out)


def uniform_field(phys, Ez):
    n = phys["n"]
    z = np.zeros((n, n, n))
    return (z.copy(), z.copy(), np.full((n, n, n), float(Ez)))


def random_ions(phys, seed, mean=50.0, frac=0.3):
    """Random ion counts (N+, N-) on a fraction of the cells."""
    n = phys["n"]
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = rng.random(n ** 3) < frac
    Np = np.where(mask, rng.poisson(mean, n ** 3), 0).astype(np.int64)
    Nn = np.where(mask, rng.poisson(mean / 5, n ** 3), 0).astype(np.int64)
    return Np, Nn
