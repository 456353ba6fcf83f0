"""DCT-II closed-form solve of the backward-Euler heat step on a full box with
constant K and zero-flux walls (TEST INFRASTRUCTURE ONLY).

On a box of nx x ny x nz cells with zero-flux walls, the 1D second-difference
operator with its wall rows (Sect. 3.2, Neumann with F = 0) has the
orthonormal DCT-II vectors v_k(i) = cos(pi k (i + 1/2) / n) as eigenvectors,
with eigenvalues 4 sin^2(pi k / (2 n)).  The level matrix of Eq. (Er_imp1)
for constant K is I + (dt K / dx^2)(L_x + L_y + L_z), so it is diagonal in the
tensor DCT-II basis.  This gives the exact discrete solution without any
iteration: an independent pin for both the assembly and the CG.
"""
from __future__ import annotations

import numpy as np


def dct2_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT-II matrix Q (rows = basis vectors): Q @ Q.T = I."""
    i = np.arange(n)
    k = np.arange(n)[:, None]
    Q = np.cos(np.pi * k * (i[None, :] + 0.5) / n)
    Q[0, :] *= np.sqrt(1.0 / n)
    Q[1:, :] *= np.sqrt(2.0 / n)
    return Q


def neumann_eigenvalues(n: int) -> np.ndarray:
    k = np.arange(n)
    return 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2


def solve_box(b_grid: np.ndarray, dt: float, dx: float, K: float) -> np.ndarray:
    """Solve (I + dt K/dx^2 (Lx + Ly + Lz)) x = b on a full box; b_grid is
    [nx, ny, nz] in lexicographic cell coordinates."""
    nx, ny, nz = b_grid.shape
    Qx, Qy, Qz = dct2_matrix(nx), dct2_matrix(ny), dct2_matrix(nz)
    bh = np.einsum("ai,bj,ck,ijk->abc", Qx, Qy, Qz, b_grid, optimize=True)
    c = dt * K / (dx * dx)
    lam = (1.0 + c * (neumann_eigenvalues(nx)[:, None, None]
                      + neumann_eigenvalues(ny)[None, :, None]
                      + neumann_eigenvalues(nz)[None, None, :]))
    xh = bh / lam
    return np.einsum("ai,bj,ck,abc->ijk", Qx, Qy, Qz, xh, optimize=True)


def solve_level_box(level, dt: float, K: float, b: np.ndarray) -> np.ndarray:
    """Same solve for a box level given in oct order: gathers b into the
    lexicographic grid, solves, scatters back to oct order."""
    xyz = level.cell_xyz()
    lo = xyz.min(axis=0)
    shape = tuple(xyz.max(axis=0) - lo + 1)
    if int(np.prod(shape)) != xyz.shape[0]:
        raise ValueError("not a full box")
    g = np.zeros(shape)
    q = xyz - lo
    g[q[:, 0], q[:, 1], q[:, 2]] = b
    x = solve_box(g, dt, level.dx, K)
    return x[q[:, 0], q[:, 1], q[:, 2]]
