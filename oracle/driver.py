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

Energy-conserving interfaces (Sect. 3.3.1 - 3.3.2, fine first only): at the
end of every fine update the energy that crossed each fine-to-coarse face is
stored (its time integral over the fine steps, which is the Delta t-weighted
mean flux of Eq. mean_flux times the coarse step).  The coarse level's
coarse-to-fine faces then take either the Dirichlet row (the restriction,
as above), the Neumann row with that stored energy as the imposed flux F
(energy conserved exactly), or the Robin row with weight alpha between the
two.  In the units of the level system (energy per unit cell volume over the
step, the reading of the Neumann sign), a fine face f next to coarse cell c
moves C_f (E_f^{k} - E_c) V_f / V_c = C_f (E_f^k - E_c) / 8 into c during
fine step k, with C_f = (2/3) dt_f/(2 dx_f^2) (K_f + K_c).

Domain sides: zero flux, or Dirichlet with a ghost value E_w and ghost
coefficient K_w one cell width of the level away (the leaves of every level
on that side).  Power-law coefficient (the equilibrium test of Sect. 4.2):
K = K0 E^a on the leaves from E^n before every level solve.
"""
from __future__ import annotations

import numpy as np

from . import DIRICHLET, NEUMANN, REL_COARSER, REL_FINER, REL_SAME, ROBIN, STOP_CERTIFIED, assemble, pcg
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
    def __init__(self, levels, states, order="fine_first", fld=None, interface="dirichlet", alpha=1.0, walls=None,
                 power_law=None):
        """states: per level (E, K).  fld: None, or (per-level rho, per-level T,
        k0) for the radiation-matter mode (K, s, src from the gas state before
        every level solve, T updated after it).  interface: the row of the
        coarse-to-fine faces, "dirichlet", "neumann" (stored flux) or "robin"
        (weight alpha on the Dirichlet part).  walls: None (zero-flux domain)
        or {side: (E_w, K_w)} for the Dirichlet sides (0..5 = -x, +x, -y, +y,
        -z, +z).  power_law: None or (K0, a)."""
        if interface not in ("dirichlet", "neumann", "robin"):
            raise ValueError(interface)
        if interface != "dirichlet" and order != "fine_first":
            raise ValueError("stored interface fluxes need the fine-first order")
        self.interface = interface
        self.walls = dict(walls or {})
        self.power_law = power_law
        self.alpha = {"dirichlet": 1.0, "neumann": 0.0, "robin": float(alpha)}[interface]
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
        # stored interface energy per coarse-to-fine face of each level (energy
        # per unit volume of the coarse cell), and where each fine-to-coarse
        # face of the level below sends its energy
        self.store = [np.zeros(len(f)) for f in self.faces]
        self.send = []
        for l in range(len(levels)):
            if l == 0:
                self.send.append({})
                continue
            index = {(cell, d): k for k, (cell, d, rel, _) in enumerate(self.faces[l - 1]) if rel == REL_FINER}
            self.send.append({k: index[(jc, d ^ 1)] for k, (_, d, rel, jc) in enumerate(self.faces[l])
                              if rel == REL_COARSER})
        # per level solve: (level, energy its leaves gained through their
        # coarse-to-fine faces, stored fine-side energy the solve consumed)
        self.audit = []

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
                    if d in self.walls:
                        out.append((cell, d, REL_SAME, d))
                    continue
                qc = tuple(v // 2 for v in q)   # Python floor division
                jc = self.L[l - 1].cell_of.get(qc)
                if jc is not None:
                    assert self.L[l - 1].is_leaf[jc]
                    out.append((cell, d, REL_COARSER, jc))
                    continue
                # no cell beyond the face at any coarser level: the domain side
                r, inside = qc, False
                for k in range(l - 2, -1, -1):
                    r = tuple(v // 2 for v in r)
                    inside = inside or r in self.L[k].cell_of
                assert not inside, "2:1 balance violated"
                if d in self.walls:
                    out.append((cell, d, REL_SAME, d))
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
        if self.power_law is not None:
            leaf = desc.leaf_cells()
            K0, a = self.power_law
            self.K[l][leaf] = K0 * self.E[l][leaf] ** a
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
            elif rel == REL_SAME:
                fE[k], fK[k] = self.walls[j]
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
        fF = np.zeros(len(f))
        if self.interface != "dirichlet":
            fine_side = frel == REL_FINER
            lv.face_kind[fine_side] = NEUMANN if self.interface == "neumann" else ROBIN
            lv.face_alpha[fine_side] = self.alpha
            fF[fine_side] = self.store[l][fine_side]
        self.E_prev[l] = self.E[l].copy()
        S = assemble(lv, dt, self.K[l], self.E[l], s=s_shift, src=src, face_K=fK, face_E=fE, face_F=fF)
        x, info = pcg(S, self.E[l], tol=tol, stop_rule=STOP_CERTIFIED)
        assert info["status"] == 0, info
        self.iterations += info["iterations"]
        self.E[l] = x
        # energy (per unit coarse volume) this level's coarse-to-fine faces gave
        # its leaves, by the face rows of Sect. 3.2: Dirichlet alpha C (E_nb - x),
        # Neumann / Robin (1 - alpha) F on top
        h = dt / (2.0 * desc.dx * desc.dx)
        gained = 0.0
        for k, (cell, _, rel, _) in enumerate(f):
            if rel != REL_FINER:
                continue
            C = h * (self.K[l][cell] + fK[k])
            gained += self.alpha * C * (fE[k] - x[cell]) + (1.0 - self.alpha) * fF[k]
        consumed = float(np.sum(self.store[l])) * desc.dx ** 3
        self.audit.append((l, gained * desc.dx ** 3, consumed))
        self.store[l][:] = 0.0
        # energy this level's fine-to-coarse faces took from the coarser cells
        for k, kc in self.send[l].items():
            cell = f[k][0]
            C = (2.0 / 3.0) * h * (self.K[l][cell] + fK[k])
            self.store[l - 1][kc] += C * (x[cell] - fE[k]) / 8.0
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

    def energy(self):
        """Total energy: E times the cell volume over the leaf cells of every
        level."""
        tot = 0.0
        for lev, E in zip(self.L, self.E):
            leaf = lev.desc.leaf_cells()
            tot += float(np.sum(E[leaf])) * lev.desc.dx ** 3
        return tot

    def state(self, l):
        for k in range(len(self.L) - 2, l - 1, -1):
            self.restrict(k)
        return self.E[l].copy()
