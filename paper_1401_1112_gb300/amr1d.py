"""Adaptive mesh for one-dimensional runs on the library's hierarchy: the
linear diffusion (Dirac) test of Sect. 4.1.

A column over [0, 1] (uniform in y and z) with a base of 32 cells and up to
three levels; before every coarse step the mesh is rebuilt where the relative
difference of a cell to a neighbour, 2 |E_i - E_j| / (E_i + E_j), exceeds
25 % (a refined region: the flagged cells and one more on each side, kept one
cell inside its level).  The state moves to the new mesh by injection (a new
fine cell takes its parent's value) and restriction (a removed fine region
leaves the mean of its children in the parent), so the total energy does
not change.  Each coarse step is one ``ats_level_advance`` of the base level
(fine levels first, every level half the step of the next coarser one).
"""
from __future__ import annotations

import numpy as np

from . import ats as A

BASE_CELLS = 32
MAX_LEVEL = 3
K_PULSE = 1e10      # c / (3 rho kappa_R), rho kappa_R = 1, c = 3e10 (cgs)
PULSE_WEIGHT = 1e5  # E0 = E_centre dx
COARSE_DT = 3.125e-15
CRITERION = 0.25


def _row_values(levels, E_levels):
    rows = []
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        sel = (xyz[:, 1] == 0) & (xyz[:, 2] == 0)
        rows.append({int(i): float(v) for i, v in zip(xyz[sel, 0], np.asarray(E)[sel])})
    return rows


def _mesh(cell_value):
    """Refined x cells per level, and the row values of every level's cells."""
    per_level = [{ix: cell_value(0, ix) for ix in range(BASE_CELLS)}]
    refined = []
    for l in range(MAX_LEVEL):
        vals = per_level[l]
        n_l = BASE_CELLS << l
        marks = set()
        for i, e in vals.items():
            if any(j in vals and 2.0 * abs(e - vals[j]) / (e + vals[j]) > CRITERION for j in (i - 1, i + 1)):
                marks.update(k for k in (i - 1, i, i + 1) if k in vals)
        nested = [i for i in sorted(marks)
                  if (i == 0 or i - 1 in vals) and (i == n_l - 1 or i + 1 in vals)]
        if not nested:
            break
        refined.append(nested)
        per_level.append({c: cell_value(l + 1, c) for i in nested for c in (2 * i, 2 * i + 1)})
    return refined, per_level


class ColumnLevel:
    """One level of the column: octs in x-major order, the leaf mask of the
    refined x cells, no face descriptors (the hierarchy derives them)."""

    def __init__(self, l, refined_here):
        across = 1 << l  # octs across y and z at level l
        self.dx = 1.0 / (BASE_CELLS << l)
        self._l = l
        self.oct_xyz = None
        self.leaf = None
        self.face_cell = np.zeros(0, np.int32)
        self.face_dir = self.face_kind = self.face_rel = np.zeros(0, np.int8)
        self.face_alpha = np.zeros(0)
        self._across = across
        self._refined = set(refined_here)

    def set_octs(self, x_octs):
        a = self._across
        xyz = [(x, y, z) for x in x_octs for y in range(a) for z in range(a)]
        self.oct_xyz = np.array(xyz, dtype=np.int32).reshape(-1, 3)
        leaf = np.full(len(xyz), 0xFF, dtype=np.uint8)
        for o, (x, _, _) in enumerate(xyz):
            for c in range(8):
                if 2 * x + (c & 1) in self._refined:
                    leaf[o] &= np.uint8(~(1 << c) & 0xFF)
        self.leaf = leaf

    @property
    def n_oct(self):
        return int(self.oct_xyz.shape[0])

    @property
    def n_cell(self):
        return 8 * self.n_oct

    def cell_xyz(self):
        c = np.arange(8)
        bits = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
        return (2 * self.oct_xyz.astype(np.int64)[:, None, :] + bits[None, :, :]).reshape(-1, 3)

    def leaf_cells(self):
        return ((self.leaf[:, None] >> np.arange(8)[None, :]) & 1).astype(bool).reshape(-1)


def _levels_and_state(refined, per_level):
    levels = []
    x_octs = list(range(BASE_CELLS // 2))
    for l in range(len(refined) + 1):
        lv = ColumnLevel(l, refined[l] if l < len(refined) else [])
        lv.set_octs(x_octs)
        levels.append(lv)
        if l < len(refined):
            x_octs = list(refined[l])  # a refined level-l x cell is a level-(l+1) x oct
    E = [np.array([per_level[l][int(i)] for i in lv.cell_xyz()[:, 0]], dtype=np.float64)
         for l, lv in enumerate(levels)]
    return levels, E


def pulse_mesh():
    """Mesh and state of the initial pulse (finest-resolution profile: 1, and
    PULSE_WEIGHT / dx in the cell starting at x = 0.5; a coarser cell holds
    the mean over it).  Returns (levels, E per level, centre of the pulse)."""
    n_f = BASE_CELLS << MAX_LEVEL
    prof = np.ones(n_f)
    prof[n_f // 2] = PULSE_WEIGHT * n_f

    def value(l, ix):
        w = n_f // (BASE_CELLS << l)
        return float(prof[ix * w:(ix + 1) * w].mean())

    levels, E = _levels_and_state(*_mesh(value))
    return levels, E, (n_f // 2 + 0.5) / n_f


def remesh(levels, E_levels):
    """The new mesh of the current state (row values; refined cells hold the
    restriction of their children)."""
    rows = _row_values(levels, E_levels)

    def value(l, ix):
        while l >= len(rows) or ix not in rows[l]:
            l, ix = l - 1, ix >> 1
        return rows[l][ix]

    return _levels_and_state(*_mesh(value))


def energy(levels, E_levels):
    """Sum of E dx over the leaf cells of the row."""
    tot = 0.0
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        sel = (xyz[:, 1] == 0) & (xyz[:, 2] == 0) & lv.leaf_cells()
        tot += float(np.asarray(E)[sel].sum()) * lv.dx
    return tot


def pulse_solution(x, t, x0):
    """1 + E0 / sqrt(4 pi K t) exp(-(x - x0)^2 / (4 K t))."""
    return 1.0 + PULSE_WEIGHT / np.sqrt(4.0 * np.pi * K_PULSE * t) * np.exp(-(np.asarray(x) - x0) ** 2 /
                                                                           (4.0 * K_PULSE * t))


def leaf_row(levels, E_levels):
    """(x, dx, E) of the row's leaf cells in x order."""
    parts = []
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        sel = (xyz[:, 1] == 0) & (xyz[:, 2] == 0) & lv.leaf_cells()
        parts.append(np.stack([(xyz[sel, 0] + 0.5) * lv.dx, np.full(int(sel.sum()), lv.dx),
                               np.asarray(E)[sel]], axis=1))
    rows = np.concatenate(parts)
    rows = rows[np.argsort(rows[:, 0])]
    return rows[:, 0], rows[:, 1], rows[:, 2]


def run_pulse(ctx, kind=A.ATS_FACE_DIRICHLET, alpha=1.0, n_steps=64, precision=A.ATS_PREC_MIXED, tol=5e-11,
              use_graph=2):
    """The test through the library: remesh, one coarse step, repeat.
    Returns (levels, E per level, energy after every step (index 0: start),
    pulse centre, seconds per coarse step including the remesh)."""
    import time

    levels, E, x0 = pulse_mesh()
    energies = [energy(levels, E)]
    t0 = time.perf_counter()
    for step in range(n_steps):
        if step:
            levels, E = remesh(levels, E)
        H = A.Hierarchy(ctx, levels, A.ATS_ORDER_FINE_FIRST)
        try:
            H.set_interface(kind, alpha)
            for l, e in enumerate(E):
                H.set_state(l, e, np.full(len(e), K_PULSE))
            code, st = H.advance(0, COARSE_DT, tol=tol, stop_rule=A.ATS_STOP_CERTIFIED, precision=precision,
                                 use_graph=use_graph)
            if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                raise RuntimeError(f"pulse coarse step {step} failed: {code} {st}")
            E = [H.state(l) for l in range(len(levels))]
        finally:
            H.close()
        energies.append(energy(levels, E))
    return levels, E, np.array(energies), x0, (time.perf_counter() - t0) / max(1, n_steps)
