"""Exact solve of the discrete field problem (a5) -- oracle side, numpy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Problem (Sec. 4, Eq. poisson; E = -grad phi): lap(phi) = -rho/eps0 on the
uniform cell-centred grid, discretised by finite volumes with the standard
second-order 7-point stencil (the 3D form of the paper's "standard stencil",
Sec. 4.3).  Boundary conditions: plane electrodes phi(z=lo)=0 and
phi(z=hi)=E0*(hi_z-lo_z) (Dirichlet, ghost = 2 phi_b - phi_1); homogeneous
Neumann on the side faces (ghost = phi_1), as in Sec. 5.1.

The discrete operator is separable: A = (T_x (x) I (x) I + I (x) T_y (x) I +
I (x) I (x) T_z) / h^2 with 1D tridiagonal T (Neumann rows end in -1, Dirichlet
rows in -3).  Each T is diagonalised numerically (numpy.linalg.eigh), the
right-hand side is transformed, divided by the eigenvalue sums and transformed
back: the exact solution of the linear system up to rounding.  This is the
definition of the discrete solution written out, not an iteration.

E at cell centres by centred differences with the same ghosts.
"""
from __future__ import annotations

import numpy as np

Q_E = 1.602176634e-19
EPS0 = 8.8541878128e-12


def tridiag(n: int, dirichlet: bool) -> np.ndarray:
    T = np.zeros((n, n))
    i = np.arange(n)
    T[i, i] = -2.0
    T[i[:-1], i[:-1] + 1] = 1.0
    T[i[1:], i[1:] - 1] = 1.0
    end = -3.0 if dirichlet else -1.0
    T[0, 0] = end
    T[n - 1, n - 1] = end
    return T


def rhs(rho_fixed, n: int, h: float, frac_bits: int, phi_top: float) -> np.ndarray:
    """b = -rho/eps0 with the Dirichlet boundary values folded in; shape (n,n,n)
    indexed [k, j, i] (z, y, x)."""
    dV = h * h * h
    rho = (np.asarray(rho_fixed, dtype=np.float64).reshape(n, n, n) * Q_E
           * (2.0 ** (-3 * frac_bits)) / dV)
    b = -rho / EPS0
    b[n - 1, :, :] -= 2.0 * phi_top / (h * h)
    return b


def apply_operator(phi: np.ndarray, h: float, phi_top: float) -> np.ndarray:
    """Matrix-free A(phi) including the boundary values (for residual checks)."""
    n = phi.shape[0]
    P = np.zeros((n + 2, n + 2, n + 2))
    P[1:-1, 1:-1, 1:-1] = phi
    P[1:-1, 1:-1, 0] = phi[:, :, 0]
    P[1:-1, 1:-1, -1] = phi[:, :, -1]
    P[1:-1, 0, 1:-1] = phi[:, 0, :]
    P[1:-1, -1, 1:-1] = phi[:, -1, :]
    P[0, 1:-1, 1:-1] = -phi[0]
    P[-1, 1:-1, 1:-1] = 2.0 * phi_top - phi[-1]
    c = P[1:-1, 1:-1, 1:-1]
    lap = (P[1:-1, 1:-1, 2:] + P[1:-1, 1:-1, :-2] + P[1:-1, 2:, 1:-1] + P[1:-1, :-2, 1:-1]
           + P[2:, 1:-1, 1:-1] + P[:-2, 1:-1, 1:-1] - 6.0 * c)
    return lap / (h * h)


def solve_b(b: np.ndarray, h: float) -> np.ndarray:
    n = b.shape[0]
    lx, Qx = np.linalg.eigh(tridiag(n, False))
    lz, Qz = np.linalg.eigh(tridiag(n, True))
    bh = np.einsum("ia,kji->kja", Qx, b)
    bh = np.einsum("jb,kja->kba", Qx, bh)
    bh = np.einsum("kc,kba->cba", Qz, bh)
    lam = (lz[:, None, None] + lx[None, :, None] + lx[None, None, :]) / (h * h)
    ph = bh / lam
    ph = np.einsum("kc,cba->kba", Qz, ph)
    ph = np.einsum("jb,kba->kja", Qx, ph)
    ph = np.einsum("ia,kja->kji", Qx, ph)
    return ph


def efield(phi: np.ndarray, h: float, phi_top: float):
    """E = -grad(phi) by centred differences, boundary ghosts as in the solve."""
    n = phi.shape[0]
    P = np.zeros((n + 2, n + 2, n + 2))
    P[1:-1, 1:-1, 1:-1] = phi
    P[1:-1, 1:-1, 0] = phi[:, :, 0]
    P[1:-1, 1:-1, -1] = phi[:, :, -1]
    P[1:-1, 0, 1:-1] = phi[:, 0, :]
    P[1:-1, -1, 1:-1] = phi[:, -1, :]
    P[0, 1:-1, 1:-1] = -phi[0]
    P[-1, 1:-1, 1:-1] = 2.0 * phi_top - phi[-1]
    Ex = (P[1:-1, 1:-1, :-2] - P[1:-1, 1:-1, 2:]) / (2.0 * h)
    Ey = (P[1:-1, :-2, 1:-1] - P[1:-1, 2:, 1:-1]) / (2.0 * h)
    Ez = (P[:-2, 1:-1, 1:-1] - P[2:, 1:-1, 1:-1]) / (2.0 * h)
    return Ex, Ey, Ez


def solve(rho_fixed, phys: dict):
    """Returns (phi, (Ex, Ey, Ez)) as (n,n,n) arrays [k,j,i]."""
    n = int(phys["n"])
    lo, hi = phys["lo"], phys["hi"]
    h = (hi[0] - lo[0]) / n
    phi_top = float(phys["E0"]) * (hi[2] - lo[2])
    b = rhs(rho_fixed, n, h, int(phys.get("frac_bits", 10)), phi_top)
    phi = solve_b(b, h)
    return phi, efield(phi, h, phi_top)
