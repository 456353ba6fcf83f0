"""Equilibrium test with a nonlinear diffusion coefficient (Sect. 4.2), on a
uniform grid (TEST INFRASTRUCTURE ONLY).

The set-up: E = 4 at x = 0 and E = 0.5 at x = 1 held by Dirichlet walls, a
step initial state, and a diffusion coefficient that is a power of E.  The
system relaxes to a steady state with a closed form, so the spatial accuracy
of the scheme shows without any time-discretisation error.

Readings:
  * the closed-form profile is E_ana(x) = [(E1^(a+1) - E0^(a+1)) x +
    E0^(a+1)]^(1/(a+1)) with a = 3/2 (the printed exponent 1/(n+1) read as
    1/(a+1)); it is the steady state of d/dx (K dE/dx) = 0 when K is
    proportional to E^a, so that law is used: K = K0 E^a;
  * K is evaluated at E^n and held over each backward-Euler step (one
    linear solve per step, as for the flux-limited coefficients);
  * the walls hold the boundary values in ghost cells one cell width away
    (relation REL_SAME), the ghost's K being K0 E_wall^a;
  * the L2 norm is the paper's: sqrt(sum_i [(E_i - E_ana(x_i)) dx_i]^2 / N_eff)
    over the cells of the one-dimensional profile, N_eff the number of cells
    at the finest resolution.

On an AMR hierarchy (the paper's adaptive-time-step runs) the same steps go
through the level driver (``oracle.driver``): fine levels first, each level
with the power-law coefficient from its own E^n, Dirichlet sides on every
level that touches them.

The oracle takes time steps until the steady state is reached: each step
assembles the level matrix with the lagged K and solves it with the oracle's
PCG.  The fixed point of the lagged steps is the discrete nonlinear steady
state whatever dt is.
"""
from __future__ import annotations

import numpy as np

from . import STOP_CERTIFIED, assemble, pcg

A_EXP = 1.5          # a in kappa_R = 1e10 E^a (Sect. 4.2)
E_LEFT, E_RIGHT = 4.0, 0.5


def analytic(x, E0=E_LEFT, E1=E_RIGHT, a=A_EXP):
    """Closed-form steady state (Sect. 4.2, reading above)."""
    x = np.asarray(x, dtype=np.float64)
    return ((E1 ** (a + 1) - E0 ** (a + 1)) * x + E0 ** (a + 1)) ** (1.0 / (a + 1))


def power_law_K(E, K0=1.0, a=A_EXP):
    """K = K0 E^a."""
    return K0 * np.asarray(E, dtype=np.float64) ** a


def relax(level, E_init, face_E, K0=1.0, a=A_EXP, dt=0.1, tol_step=1e-10, max_steps=2000, tol=5e-11):
    """Backward-Euler steps of dt with K lagged at E^n until the largest
    relative change of a step is below tol_step (the slowest mode decays by
    about 1 / (1 + dt K_min pi^2) per step, K_min = K0 E_right^a on a unit
    box).  Returns (E, steps, converged)."""
    E = np.array(E_init, dtype=np.float64, copy=True)
    face_K = power_law_K(face_E, K0, a)
    for step in range(1, max_steps + 1):
        S = assemble(level, dt, power_law_K(E, K0, a), E, face_K=face_K, face_E=face_E)
        x, info = pcg(S, E, tol=tol, stop_rule=STOP_CERTIFIED)
        if info["status"] != 0:
            raise RuntimeError(f"oracle PCG failed at step {step}: {info}")
        change = np.max(np.abs(x - E)) / np.max(np.abs(E))
        E = x
        if change < tol_step:
            return E, step, True
    return E, max_steps, False


def profile(level, E):
    """The one-dimensional profile: the cells of the y = z = 0 row, in x order
    (the column is uniform in y and z).  Returns (x index, E)."""
    xyz = level.cell_xyz()
    row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0)
    order = np.argsort(xyz[row, 0])
    return xyz[row, 0][order], np.asarray(E)[row][order]


def l2_error(level, E, n_eff=None):
    """The paper's L2 norm of the error against the closed form (uniform
    grid: dx_i = dx, N_eff = the number of cells in x unless given)."""
    ix, e = profile(level, E)
    dx = level.dx
    x = (ix + 0.5) * dx
    n_eff = len(ix) if n_eff is None else n_eff
    return float(np.sqrt(np.sum(((e - analytic(x)) * dx) ** 2) / n_eff))


def relax_amr(levels, E_init, walls, K0=1.0, a=A_EXP, dt=0.1, tol_step=1e-10, max_steps=2000, tol=5e-11):
    """Coarse steps of dt (the finer levels take their substeps, fine first)
    until the largest relative change of the leaf values over a coarse step
    is below tol_step.  walls: {side: E_wall}.  Returns (per-level E, steps,
    converged)."""
    from .driver import Hierarchy

    states = [(np.array(e, dtype=np.float64), power_law_K(e, K0, a)) for e in E_init]
    H = Hierarchy(levels, states, order="fine_first",
                  walls={side: (e, float(power_law_K(e, K0, a))) for side, e in walls.items()}, power_law=(K0, a))
    leaves = [lv.leaf_cells() for lv in levels]
    prev = [H.state(l)[leaves[l]] for l in range(len(levels))]
    for step in range(1, max_steps + 1):
        H.advance(0, dt, tol=tol)
        cur = [H.state(l)[leaves[l]] for l in range(len(levels))]
        scale = max(float(np.max(np.abs(c))) for c in cur)
        change = max(float(np.max(np.abs(c - p))) for c, p in zip(cur, prev)) / scale
        prev = cur
        if change < tol_step:
            return [H.state(l) for l in range(len(levels))], step, True
    return [H.state(l) for l in range(len(levels))], max_steps, False


def l2_error_amr(levels, E_levels, n_eff):
    """The paper's L2 norm over the leaf cells of the y = z = 0 row of every
    level, dx_i the cell's own width, N_eff the cells at the finest
    resolution."""
    tot = 0.0
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0) & lv.leaf_cells()
        x = (xyz[row, 0] + 0.5) * lv.dx
        tot += float(np.sum(((np.asarray(E)[row] - analytic(x)) * lv.dx) ** 2))
    return float(np.sqrt(tot / n_eff))
