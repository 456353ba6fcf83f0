"""Adaptive time stepping over an AMR hierarchy, level by level (TEST
INFRASTRUCTURE ONLY).

Sect. 2.2: a level advances with its own time step dt^l = dt^{l+1}_1 +
dt^{l+1}_2, finer levels first.  Sect. 3.3.1: a leaf of level l next to a
coarser leaf takes a Dirichlet value, the coarse energy held at E^n over the
two fine steps, with the coefficient C^{l->l-1} = 2/3 A^l.  Sect. 3.3.2: a
leaf next to a refined cell takes the restriction of that cell -- the mean of
its oct of children after their update -- with C^{l->l+1} = A^l, Dirichlet.
Each level is assembled and solved on its own (oracle.assemble + oracle.pcg).

This file derives the interface faces of every level directly from the cell
coordinates with Python dictionaries; it shares nothing with the library.

The "coarse first" order (the two-level workload's reading) solves the
coarse level first and gives the fine substeps the coarse value linear in
time, E_c^n + (k/2)(E_c^{n+1} - E_c^n) at the end of fine substep k.
"""
from __future__ import annotations

import numpy as np

from . import DIRICHLET, REL_COARSER, REL_FINER, STOP_CERTIFIED, assemble, pcg
from . import fld as fldmod

AX = (0, 0, 1, 1, 2, 2)
SG = (-1, 1, -1, 1, -1, 1)


class _Level:
    def __init__(self, desc):
        self.desc = desc
        self.cell_of = {}   # level cell coordinate -> cell index
        self.is_leaf = {}
        leaf = desc.leaf
        for o, (x, y, z) in enumerate(desc.oct_xyz.tolist()):
            for c in range(8):
                p = (2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1))
                self.cell_of[p] = 8 * o + c
                self.is_leaf[8 * o + c] = True if leaf is None else bool((int(leaf[o]) >> c) & 1)
        self.coord = {v: k for k, v in self.cell_of.items()}


class Hierarchy:
    def __init__(self, levels, states, order="fine_first", fld=None):
        """states: per level (E, K).  fld: None, or (per-level rho, per-level T,
        k0) for the radiation-matter mode (K, s, src from the gas state before
        every level solve, T updated after it)."""
        self.L = [_Level(d) for d in levels]
        self.E = [np.array(e, dtype=np.float64) for e, _ in states]
        self.K = [np.array(k, dtype=np.float64) for _, k in states]
        self.fld = None
        if fld is not None:
            rho, T, k0 = fld
            self.fld = ([np.array(r, dtype=np.float64) for r in rho], [np.array(t, dtype=np.float64) for t in T], k0)
            for l, d in enumerate(levels):
                leaf = d.leaf_cells()
                K0, _, _ = fldmod.coefficients(d, self.fld[0][l], self.fld[1][l], self.E[l], 1.0, k0)
                self.K[l][leaf] = K0[leaf]
        self.E_prev = [e.copy() for e in self.E]
        self.order = order
        self.faces = [self._faces(l) for l in range(len(levels))]
        self.iterations = 0

    def _faces(self, l):
        """(cell, dir, rel, src) of every interface face of level l."""
        lev = self.L[l]
        out = []
        for cell in range(8 * len(lev.desc.oct_xyz)):
            if not lev.is_leaf[cell]:
                continue
            p = lev.coord[cell]
            for d in range(6):
                q = list(p)
                q[AX[d]] += SG[d]
                q = tuple(q)
                j = lev.cell_of.get(q)
                if j is not None:
                    if not lev.is_leaf[j]:
                        out.append((cell, d, REL_FINER, j))
                    continue
                if l == 0:
                    continue
                qc = tuple(v // 2 for v in q)   # Python floor division
                jc = self.L[l - 1].cell_of.get(qc)
                if jc is not None:
                    assert self.L[l - 1].is_leaf[jc]
                    out.append((cell, d, REL_COARSER, jc))
        return out

    def restrict(self, l):
        """Refined cells of level l take the mean of their children (E and K)."""
        if l + 1 >= len(self.L):
            return
        fine = self.L[l + 1]
        for o, (x, y, z) in enumerate(fine.desc.oct_xyz.tolist()):
            R = self.L[l].cell_of[(x, y, z)]
            self.E[l][R] = np.mean(self.E[l + 1][8 * o: 8 * o + 8])
            self.K[l][R] = np.mean(self.K[l + 1][8 * o: 8 * o + 8])

    def solve_level(self, l, dt, theta, tol):
        self.restrict(l)
        desc = self.L[l].desc
        s_shift = src = None
        if self.fld is not None:
            leaf = desc.leaf_cells()
            Kf, s_shift, src = fldmod.coefficients(desc, self.fld[0][l], self.fld[1][l], self.E[l], dt, self.fld[2])
            self.K[l][leaf] = Kf[leaf]
            s_shift = np.where(leaf, s_shift, 0.0)
            src = np.where(leaf, src, 0.0)
        f = self.faces[l]
        fcell = np.array([a for a, _, _, _ in f], dtype=np.int32)
        fdir = np.array([b for _, b, _, _ in f], dtype=np.int8)
        frel = np.array([c for _, _, c, _ in f], dtype=np.int8)
        fE = np.zeros(len(f))
        fK = np.zeros(len(f))
        for k, (_, _, rel, j) in enumerate(f):
            if rel == REL_FINER:
                fE[k] = self.E[l][j]
                fK[k] = self.K[l][j]
            else:
                if self.order == "fine_first":
                    fE[k] = self.E[l - 1][j]       # coarse held at E^n
                else:
                    e0, e1 = self.E_prev[l - 1][j], self.E[l - 1][j]
                    fE[k] = e0 + theta * (e1 - e0)
                fK[k] = self.K[l - 1][j]

        class D:
            pass

        lv = D()
        lv.oct_xyz, lv.leaf, lv.dx = desc.oct_xyz, desc.leaf, desc.dx
        lv.face_cell, lv.face_dir, lv.face_rel = fcell, fdir, frel
        lv.face_kind = np.full(len(f), DIRICHLET, dtype=np.int8)
        lv.face_alpha = np.ones(len(f))
        self.E_prev[l] = self.E[l].copy()
        S = assemble(lv, dt, self.K[l], self.E[l], s=s_shift, src=src, face_K=fK, face_E=fE)
        x, info = pcg(S, self.E[l], tol=tol, stop_rule=STOP_CERTIFIED)
        assert info["status"] == 0, info
        self.iterations += info["iterations"]
        self.E[l] = x
        if self.fld is not None:
            leaf = desc.leaf_cells()
            Tn = fldmod.update_temperature(self.fld[0][l], self.fld[1][l], x, dt, self.fld[2])
            self.fld[1][l] = np.where(leaf, Tn, self.fld[1][l])

    def advance(self, l, dt, tol=5e-11, theta=1.0):
        fine = l + 1 < len(self.L)
        if self.order == "fine_first":
            if fine:
                self.advance(l + 1, dt / 2, tol)
                self.advance(l + 1, dt / 2, tol)
            self.solve_level(l, dt, 0.0, tol)
        else:
            self.solve_level(l, dt, theta, tol)
            if fine:
                self.advance(l + 1, dt / 2, tol, theta=0.5)
                self.advance(l + 1, dt / 2, tol, theta=1.0)
                self.restrict(l)

    def state(self, l):
        for k in range(len(self.L) - 2, l - 1, -1):
            self.restrict(k)
        return self.E[l].copy()
