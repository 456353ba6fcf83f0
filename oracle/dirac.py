"""Linear diffusion test (Sect. 4.1) with adaptive refinement, in 1D
(TEST INFRASTRUCTURE ONLY).

An energy pulse (E = 1 everywhere but one cell at x = 0.5 holding E0 / dx, a
Dirac of weight E0 = 1e5) diffuses with K = c / (3 rho kappa_R) = 1e10 (cgs,
rho kappa_R = 1) on a column with a base of 32 cells and up to three levels
of refinement; a cell is refined where the relative difference to a
neighbour, 2 |E_i - E_j| / (E_i + E_j), exceeds 25 %; every level takes half
the step of the next coarser one (coarse step 3.125e-15, fine levels first)
and the mesh follows the pulse: it is rebuilt from the criterion before every
coarse step.  The interface rows are Dirichlet (alpha = 1), Robin (alpha =
0.5) or Neumann with the stored fine-side flux (alpha = 0).

Readings: the box's walls are zero-flux instead of periodic (the pulse's
width at t = 2e-13, sqrt(2 K t) = 0.063, keeps it far from them, and a
closed box conserves energy as a periodic one does); a refined region is
the flagged cells plus one cell on each side, kept one cell inside its own
level (proper nesting and 2:1 balance); values move to the new mesh by
injection (new fine cells take their parent's value) and restriction
(removed fine cells leave the mean of their children), both of which keep
the total energy.  The analytic solution is 1 + E0 / sqrt(4 pi K t)
exp(-(x - x0)^2 / (4 K t)), x0 the centre of the Dirac cell.
"""
from __future__ import annotations

import numpy as np

import workloads as W

from .driver import Hierarchy

N0 = 32
L_MAX = 3
K_DIFF = 1e10
E0_WEIGHT = 1e5
DT0 = 3.125e-15
THRESHOLD = 0.25


def initial_profile(n_eff=N0 * 2 ** L_MAX, E0=E0_WEIGHT):
    """The initial state at the finest resolution: 1, and E0 / dx in the cell
    starting at x = 0.5.  Returns (values [n_eff], x0)."""
    dx = 1.0 / n_eff
    v = np.ones(n_eff)
    v[n_eff // 2] = E0 / dx
    return v, 0.5 + 0.5 * dx


def analytic(x, t, x0, E0=E0_WEIGHT, K=K_DIFF):
    return 1.0 + E0 / np.sqrt(4.0 * np.pi * K * t) * np.exp(-(np.asarray(x) - x0) ** 2 / (4.0 * K * t))


def _rows(levels, E_levels):
    """Per level: {x cell: value} of the cells of the y = z = 0 row."""
    out = []
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0)
        out.append(dict(zip(xyz[row, 0].tolist(), np.asarray(E)[row].tolist())))
    return out


def build_mesh(value, n0=N0, l_max=L_MAX, threshold=THRESHOLD):
    """Refined x cells per level from value(l, ix) (the state to follow).
    Returns (refined_x lists, {level: {ix: value}} of every cell of the new
    mesh)."""
    cells = {0: {ix: value(0, ix) for ix in range(n0)}}
    refined = []
    for l in range(l_max):
        cur = cells[l]
        flagged = set()
        for i, e in cur.items():
            for j in (i - 1, i + 1):
                if j in cur and 2.0 * abs(e - cur[j]) / (e + cur[j]) > threshold:
                    flagged.add(i)
        grown = {j for i in flagged for j in (i - 1, i, i + 1) if j in cur}
        n_l = n0 * 2 ** l
        keep = sorted(i for i in grown if all(k in cur or k < 0 or k >= n_l for k in (i - 1, i + 1)))
        if not keep:
            break
        refined.append(keep)
        cells[l + 1] = {2 * i + c: value(l + 1, 2 * i + c) for i in keep for c in (0, 1)}
    return refined, cells


def mesh_state(refined, cells, K=K_DIFF, n0=N0):
    """Levels and per-level (E, K) of a mesh whose row values are `cells`
    (the column is uniform in y and z)."""
    levels = W.column_hierarchy(n0, refined)
    states = []
    for l, lv in enumerate(levels):
        ix = lv.cell_xyz()[:, 0]
        E = np.array([cells[l][int(i)] for i in ix], dtype=np.float64)
        states.append((E, np.full(lv.n_cell, K)))
    return levels, states


def initial_mesh(profile, n0=N0, l_max=L_MAX):
    """Mesh and state of the initial profile (finest-resolution values):
    a cell of level l holds the mean of the profile over it."""
    n_eff = len(profile)

    def value(l, ix):
        w = n_eff // (n0 * 2 ** l)
        return float(np.mean(profile[ix * w:(ix + 1) * w]))

    return mesh_state(*build_mesh(value, n0, l_max))


def regrid(levels, E_levels, n0=N0, l_max=L_MAX):
    """New mesh from the current state (every level's row values, refined
    cells holding the restriction of their children): a cell present at its
    level keeps its value, a new cell takes its parent's (injection)."""
    rows = _rows(levels, E_levels)

    def value(l, ix):
        while l >= len(rows) or ix not in rows[l]:
            l, ix = l - 1, ix // 2
        return rows[l][ix]

    return mesh_state(*build_mesh(value, n0, l_max))


def leaf_energy(levels, E_levels):
    """Total energy of the leaf cells (1D: E dx over the row)."""
    tot = 0.0
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0) & lv.leaf_cells()
        tot += float(np.sum(np.asarray(E)[row])) * lv.dx
    return tot


def leaf_profile(levels, E_levels):
    """(x centres, dx, E) of the leaf cells of the row, in x order."""
    xs, dxs, es = [], [], []
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0) & lv.leaf_cells()
        xs.append((xyz[row, 0] + 0.5) * lv.dx)
        dxs.append(np.full(int(row.sum()), lv.dx))
        es.append(np.asarray(E)[row])
    x, dx, e = np.concatenate(xs), np.concatenate(dxs), np.concatenate(es)
    o = np.argsort(x)
    return x[o], dx[o], e[o]


def run(interface="dirichlet", alpha=1.0, n_steps=64, tol=5e-11):
    """The test: regrid, one coarse step, repeat.  Returns (levels, per-level
    E, energies after every step (index 0: the start), x0)."""
    profile, x0 = initial_profile()
    levels, states = initial_mesh(profile)
    energies = [leaf_energy(levels, [e for e, _ in states])]
    for step in range(n_steps):
        if step > 0:
            levels, states = regrid(levels, E_levels)
        H = Hierarchy(levels, states, order="fine_first", interface=interface, alpha=alpha)
        H.advance(0, DT0, tol=tol)
        E_levels = [H.state(l) for l in range(len(levels))]
        energies.append(leaf_energy(levels, E_levels))
    return levels, E_levels, np.array(energies), x0
