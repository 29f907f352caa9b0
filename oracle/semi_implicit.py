"""Semi-implicit field coupling (Sec. 4.3 and Sec. 4.7) -- oracle side, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's transport step removes the dielectric-relaxation limit of the
explicit Euler-Maruyama push by solving for the field of the end of the step
(Sec. 4.7, steps 1-5):

1. conductivity sigma^k = q_e mu n_e^k (Eq. conductivity; the electrons are
   the only mobile species here, so the sum over species has one term); n_e^k
   is the CIC density of the particles at X^k;
2. diffusive advance X+ = X^k + sqrt(2 D dt) N (Eq. Xdagger);
3. rho+ = rho(X+) and the variable-coefficient Poisson equation
   div[(1 + sigma^k dt / eps0) E^{k+1}] = rho+ / eps0 (Eq. poisson_simp),
   E = -grad(phi);
4. V = -mu E^{k+1}(X^k) (Eq. Vk1, the field interpolated at the position of
   the start of the step);
5. X^{k+1} = X+ + V dt (Eq. particle_kernel).

Discretisation (readings of Sec. 4.3, which states a finite-volume 7-point
operator solved by multigrid): cell-centred unknowns as in ``poisson.py``;
the coefficient of a face between two cells is the arithmetic mean of the
two cells' coefficients; at a boundary face the ghost cell takes the
boundary cell's coefficient, with the ghosts of ``poisson.py`` (Dirichlet
electrodes: ghost = 2 phi_b - phi_1; Neumann side faces: ghost = phi_1, no
flux).  With sigma = 0 the system is exactly the one of ``poisson.py``.
The linear system is solved directly (scipy's sparse LU): the exact discrete
solution up to rounding, not an iteration.
"""
from __future__ import annotations

import numpy as np

from .poisson import EPS0, Q_E, efield, rhs


def coefficient(sigma, dt: float) -> np.ndarray:
    """Cell coefficient 1 + sigma dt / eps0 (Eq. poisson_simp)."""
    return 1.0 + np.asarray(sigma, dtype=np.float64) * dt / EPS0


def conductivity(ne_fix, phys: dict) -> np.ndarray:
    """sigma = q_e mu n_e per cell (Eq. conductivity), n_e from the int64
    fixed-point CIC electron count (units of 2^-3s electrons per cell);
    shape (n, n, n) indexed [k, j, i]."""
    n = int(phys["n"])
    h = (phys["hi"][0] - phys["lo"][0]) / n
    s = int(phys.get("frac_bits", 10))
    ne = np.asarray(ne_fix, dtype=np.float64).reshape(n, n, n) * (2.0 ** (-3 * s)) / (h * h * h)
    return Q_E * float(phys["mu"]) * ne


def assemble(c: np.ndarray, h: float):
    """Sparse matrix of phi -> div(c grad phi) on the cell-centred grid
    (homogeneous part: the electrode potential enters the right-hand side),
    in CSR form, unknowns ordered as c.ravel() (x fastest)."""
    import scipy.sparse as sp

    n = c.shape[0]
    idx = np.arange(n ** 3).reshape(n, n, n)
    rows, cols, vals = [], [], []
    diag = np.zeros((n, n, n))
    # interior faces along each axis: coefficient (c_a + c_b) / 2
    for axis in range(3):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[axis] = slice(0, n - 1)
        b[axis] = slice(1, n)
        a, b = tuple(a), tuple(b)
        cf = 0.5 * (c[a] + c[b])
        ia, ib = idx[a].ravel(), idx[b].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [cf.ravel(), cf.ravel()]
        diag[a] -= cf
        diag[b] -= cf
    # Dirichlet faces at z = lo and z = hi (axis 0 of the [k, j, i] layout):
    # flux c_1 (ghost - phi_1) with ghost = 2 phi_b - phi_1
    diag[0] -= 2.0 * c[0]
    diag[n - 1] -= 2.0 * c[n - 1]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals) / (h * h), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n ** 3, n ** 3))
    return A.tocsr()


def solve(rho_fixed, c: np.ndarray, phys: dict):
    """div(c grad phi) = -rho/eps0 with the electrode potentials; returns
    (phi, (Ex, Ey, Ez)) as (n, n, n) arrays [k, j, i], E = -grad(phi) by the
    centred differences of ``poisson.py``."""
    import scipy.sparse.linalg as spla

    n = int(phys["n"])
    lo, hi = phys["lo"], phys["hi"]
    h = (hi[0] - lo[0]) / n
    phi_top = float(phys["E0"]) * (hi[2] - lo[2])
    c = np.asarray(c, dtype=np.float64).reshape(n, n, n)
    b = rhs(rho_fixed, n, h, int(phys.get("frac_bits", 10)), 0.0)
    b[n - 1] -= 2.0 * c[n - 1] * phi_top / (h * h)
    phi = spla.spsolve(assemble(c, h).tocsc(), b.ravel()).reshape(n, n, n)
    return phi, efield(phi, h, phi_top)


def transport(p, phys: dict, S: dict, E=None):
    """Sec. 4.7 steps 1-5 for the particles of S (canonical order: x, y, z,
    w, cell; Npos, Nneg per cell).  Returns a dict with the advected
    positions (xo, yo, zo), their cells (-1: left the box), the diffused
    positions (xd, yd, zd), sigma, rho+ and the new field (phi, E).  A given
    field E (Ex, Ey, Ez) replaces the solve in step 3 (phi is then None):
    the substeps can be checked on their own against a field from
    elsewhere."""
    from . import lib, _P
    from .stages import deposit, rho_fixed
    import ctypes

    x = np.ascontiguousarray(S["x"], np.float64)
    y = np.ascontiguousarray(S["y"], np.float64)
    z = np.ascontiguousarray(S["z"], np.float64)
    w = np.ascontiguousarray(S["w"], np.uint32)
    npart = len(x)
    pd = ctypes.c_double
    # 1. conductivity of the start of the step
    ne_k, _ = deposit(p, x, y, z, w, S["cell"])
    sigma = conductivity(ne_k, phys)
    # 2. diffusive advance
    xd, yd, zd = np.empty(npart), np.empty(npart), np.empty(npart)
    lib().ora_diffuse(ctypes.byref(p), npart, _P(x, pd), _P(y, pd), _P(z, pd), _P(xd, pd), _P(yd, pd),
                      _P(zd, pd))
    # 3. charge of the diffused particles (the folded stencil keeps every one
    # of them, also those diffused past a face; their X_e tally is not used)
    ne_d, _ = deposit(p, xd, yd, zd, w, np.zeros(npart, np.int64))
    rho_d = rho_fixed(p, ne_d, S["Npos"], S["Nneg"])
    if E is None:
        phi, E = solve(rho_d, coefficient(sigma, float(phys["dt"])), phys)
    else:
        phi = None
    # 4.-5. velocity from the new field at X^k, advective step from X+
    Ex, Ey, Ez = (np.ascontiguousarray(np.ravel(e), np.float64) for e in E)
    xo, yo, zo = np.empty(npart), np.empty(npart), np.empty(npart)
    cell = np.empty(npart, np.int64)
    lib().ora_advect(ctypes.byref(p), npart, _P(x, pd), _P(y, pd), _P(z, pd), _P(xd, pd), _P(yd, pd),
                     _P(zd, pd), _P(Ex, pd), _P(Ey, pd), _P(Ez, pd), _P(xo, pd), _P(yo, pd), _P(zo, pd),
                     _P(cell, ctypes.c_int64))
    return dict(xo=xo, yo=yo, zo=zo, cell=cell, xd=xd, yd=yd, zd=zd, sigma=sigma, rho=rho_d, phi=phi, E=E)


def step(p, phys: dict, S: dict, E=None):
    """One semi-implicit time step (Sec. 4.7): the transport of Sec. 4.7 steps
    1-5 (``transport``; a given field E replaces its solve), then the sort,
    the deposit, KMC in the field of the end of the step, products, photons
    and the merge/split, as the explicit step does after its push.  Returns
    (new_state, info); info also holds the transport's results under
    "transport"."""
    from .stages import after_transport
    T = transport(p, phys, S, E=E)
    new, info = after_transport(p, S, T["xo"], T["yo"], T["zo"], T["cell"], T["E"])
    info["transport"] = T
    return new, info
