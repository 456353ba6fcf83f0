"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the method: it only lays out octs, draws
random fields, and lists which cell faces carry an interface / wall condition
and with which parameters.  Coefficients, right-hand sides and solves are
computed independently by the library (``paper_1401_1112_gb300``) and by the
oracle (``oracle``).

Geometry conventions (shared by both sides, stated in the C header too):
  * an oct is 2x2x2 cells; oct ``o`` has integer coordinates ``oct_xyz[o]``;
  * its cell ``c = ix + 2 iy + 4 iz`` has level coordinates
    ``2*oct_xyz[o] + (ix, iy, iz)`` and global index ``8 o + c``;
  * face directions: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z;
  * ``leaf[o]`` bit ``c`` set = cell is a leaf (an unknown of the level);
  * faces without a same-level leaf neighbour may carry a descriptor
    (kind, relation, alpha) and per-step values (K_nb, E_nb, F); a face with
    no descriptor is a zero-flux wall.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

DIRICHLET, NEUMANN, ROBIN = 0, 1, 2
REL_SAME, REL_COARSER, REL_FINER = 0, 1, 2
_AX = np.array([0, 0, 1, 1, 2, 2])
_SG = np.array([-1, 1, -1, 1, -1, 1])


@dataclasses.dataclass
class LevelDesc:
    oct_xyz: np.ndarray            # int32 [n_oct, 3]
    leaf: Optional[np.ndarray]     # uint8 [n_oct] or None (all leaves)
    dx: float
    face_cell: np.ndarray          # int32 [n_face]
    face_dir: np.ndarray           # int8  [n_face]
    face_kind: np.ndarray          # int8  [n_face]
    face_rel: np.ndarray           # int8  [n_face]
    face_alpha: np.ndarray         # float64 [n_face]

    @property
    def n_oct(self) -> int:
        return int(self.oct_xyz.shape[0])

    @property
    def n_cell(self) -> int:
        return 8 * self.n_oct

    @property
    def n_face(self) -> int:
        return int(self.face_cell.shape[0])

    def cell_xyz(self) -> np.ndarray:
        """int64 [N, 3] level coordinates of every cell."""
        c = np.arange(8)
        bits = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
        return (2 * self.oct_xyz.astype(np.int64)[:, None, :] + bits[None, :, :]).reshape(-1, 3)

    def leaf_cells(self) -> np.ndarray:
        """bool [N] leaf flag per cell."""
        if self.leaf is None:
            return np.ones(self.n_cell, dtype=bool)
        return ((self.leaf[:, None].astype(np.int64) >> np.arange(8)[None, :]) & 1).reshape(-1).astype(bool)


@dataclasses.dataclass
class Step:
    """Per-step values for one level solve."""

    dt: float
    K: np.ndarray
    E: np.ndarray
    face_K: Optional[np.ndarray] = None
    face_E: Optional[np.ndarray] = None
    face_F: Optional[np.ndarray] = None
    s: Optional[np.ndarray] = None
    src: Optional[np.ndarray] = None


def morton3(x, y, z, bits: int = 21) -> np.ndarray:
    """Interleave the bits of non-negative integer coordinates (x lowest)."""
    x = np.asarray(x, dtype=np.uint64)
    y = np.asarray(y, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    key = np.zeros(x.shape, dtype=np.uint64)
    for b in range(bits):
        bb = np.uint64(b)
        key |= ((x >> bb) & np.uint64(1)) << np.uint64(3 * b)
        key |= ((y >> bb) & np.uint64(1)) << np.uint64(3 * b + 1)
        key |= ((z >> bb) & np.uint64(1)) << np.uint64(3 * b + 2)
    return key


def morton_sort(oct_xyz: np.ndarray) -> np.ndarray:
    """Return the permutation that puts octs in Morton order."""
    m = oct_xyz.min(axis=0) if len(oct_xyz) else np.zeros(3, dtype=np.int64)
    sh = oct_xyz.astype(np.int64) - m
    return np.argsort(morton3(sh[:, 0], sh[:, 1], sh[:, 2]), kind="stable")


def _cell_index_map(level_oct_xyz: np.ndarray, leaf_cells: np.ndarray):
    """dict-free lookup: returns a function mapping cell coords -> (index, is_leaf)."""
    cx = level_oct_xyz.astype(np.int64)
    lo = cx.min(axis=0) * 2 - 2
    hi = cx.max(axis=0) * 2 + 4
    shape = hi - lo
    grid = np.full(tuple(shape), -1, dtype=np.int64)
    c = np.arange(8)
    bits = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
    cells = (2 * cx[:, None, :] + bits[None]).reshape(-1, 3) - lo
    grid[cells[:, 0], cells[:, 1], cells[:, 2]] = np.arange(cells.shape[0])

    def find(xyz):
        q = xyz - lo
        inside = np.all((q >= 0) & (q < shape), axis=1)
        out = np.full(xyz.shape[0], -1, dtype=np.int64)
        qi = q[inside]
        out[inside] = grid[qi[:, 0], qi[:, 1], qi[:, 2]]
        leafy = np.zeros(xyz.shape[0], dtype=bool)
        ok = out >= 0
        leafy[ok] = leaf_cells[out[ok]]
        return out, leafy

    return find


def ghost_faces(oct_xyz: np.ndarray, leaf: Optional[np.ndarray]):
    """All (cell, dir) of leaf cells whose neighbour is not a same-level leaf.

    Returns (cell int64[n], dir int64[n], nb_cell int64[n]) where nb_cell is the
    level index of the neighbouring (refined) cell, or -1 if no oct is there.
    Sorted by (cell, dir)."""
    lv = LevelDesc(oct_xyz, leaf, 1.0, *(np.zeros(0),) * 5)
    lc = lv.leaf_cells()
    xyz = lv.cell_xyz()
    find = _cell_index_map(oct_xyz, lc)
    cells, dirs, nbs = [], [], []
    for d in range(6):
        n = xyz.copy()
        n[:, _AX[d]] += _SG[d]
        idx, leafy = find(n)
        sel = lc & ~leafy
        cells.append(np.nonzero(sel)[0])
        dirs.append(np.full(int(sel.sum()), d))
        nbs.append(idx[sel])
    cell = np.concatenate(cells)
    dr = np.concatenate(dirs)
    nb = np.concatenate(nbs)
    order = np.lexsort((dr, cell))
    return cell[order], dr[order], nb[order]


def box_octs(nox: int, noy: int, noz: int, origin=(0, 0, 0)) -> np.ndarray:
    """Oct coordinates of a full nox x noy x noz oct box, Morton ordered."""
    g = np.stack(np.meshgrid(np.arange(nox), np.arange(noy), np.arange(noz), indexing="ij"), -1)
    xyz = g.reshape(-1, 3).astype(np.int32) + np.asarray(origin, dtype=np.int32)
    return xyz[morton_sort(xyz)]


def box_wall_faces(oct_xyz: np.ndarray, nox: int, noy: int, noz: int):
    """The faces of a full box of octs (all cells leaves) that lie on its
    walls, as ``ghost_faces`` lists them (cell int64[n], dir int64[n], sorted
    by (cell, dir)), found from the cell coordinates instead of a search."""
    ext = (2 * nox, 2 * noy, 2 * noz)
    o = oct_xyz.astype(np.int64)
    cells, dirs = [], []
    for c in range(8):
        bit = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
        for d in range(6):
            a, side = d >> 1, d & 1
            coord = 2 * o[:, a] + bit[a]
            on = np.nonzero(coord == (ext[a] - 1 if side else 0))[0]
            cells.append(8 * on + c)
            dirs.append(np.full(on.size, d, dtype=np.int64))
    cell = np.concatenate(cells)
    dr = np.concatenate(dirs)
    order = np.lexsort((dr, cell))
    return cell[order], dr[order]


def box_level(nox, noy, noz, dx, walls=None) -> LevelDesc:
    """A single-level box of octs.  ``walls`` is None (all zero-flux) or a list
    of 6 (kind, alpha) tuples or None per direction (None = zero-flux wall);
    every boundary cell face of a wall with a tuple gets a descriptor with
    relation REL_SAME."""
    xyz = box_octs(nox, noy, noz)
    lv = LevelDesc(xyz, None, float(dx), *(np.zeros(0, dtype=t) for t in (np.int32, np.int8, np.int8, np.int8, np.float64)))
    if walls is None:
        return lv
    cell, dr = box_wall_faces(xyz, nox, noy, noz)
    keep = np.array([walls[d] is not None for d in dr], dtype=bool)
    cell, dr = cell[keep], dr[keep]
    kind = np.array([walls[d][0] for d in dr], dtype=np.int8)
    alpha = np.array([walls[d][1] for d in dr], dtype=np.float64)
    lv.face_cell = cell.astype(np.int32)
    lv.face_dir = dr.astype(np.int8)
    lv.face_kind = kind
    lv.face_rel = np.zeros(len(cell), dtype=np.int8)
    lv.face_alpha = alpha
    return lv


def cell_centres(level: LevelDesc, origin) -> np.ndarray:
    """Physical cell centres [N, 3] for a level of spacing dx whose cell (0,0,0)
    starts at ``origin``."""
    return np.asarray(origin, dtype=np.float64)[None, :] + (level.cell_xyz() + 0.5) * level.dx


def gaussian(xyz: np.ndarray, sigma: float = 0.05, floor: float = 1e-3) -> np.ndarray:
    r2 = (xyz ** 2).sum(axis=1)
    return np.exp(-r2 / (2.0 * sigma * sigma)) + floor


# ---------------------------------------------------------------------------
# The five workload configurations: sizes and recipes
# ---------------------------------------------------------------------------

def equilibrium_column(n: int, E_left: float = 4.0, E_right: float = 0.5):
    """The equilibrium test's set-up (Sect. 4.2) on a uniform grid of n cells
    in x over [0, 1] (n even): a column of n/2 octs, one oct thick in y and z
    with zero-flux walls there (the problem stays one-dimensional);
    Dirichlet walls at x = 0 and x = 1 holding E_left / E_right in the ghost
    cells (relation REL_SAME: ghost centre one cell width away); the initial
    state is the step E_left for x < 0.5, E_right above.  Returns (level,
    E_init, face_E per wall descriptor, x of every cell centre)."""
    assert n % 2 == 0 and n >= 2
    lv = box_level(n // 2, 1, 1, 1.0 / n, walls=[(DIRICHLET, 1.0), (DIRICHLET, 1.0), None, None, None, None])
    x = (lv.cell_xyz()[:, 0] + 0.5) / n
    E = np.where(x < 0.5, E_left, E_right).astype(np.float64)
    face_E = np.where(lv.face_dir == 0, E_left, E_right).astype(np.float64)
    return lv, E, face_E, x


def column_hierarchy(n0: int, refined_x):
    """A one-dimensional AMR column over [0, 1]: the base level has n0 cells
    in x (n0 even) and one oct in y and z; refined_x[l] lists the level-l x
    cells to refine (every cell of those x slices, so the column stays
    uniform in y and z; level l has 2^(l+1) cells across y and z).  Returns
    the LevelDesc list (no face descriptors)."""
    assert n0 % 2 == 0
    base = np.stack(np.meshgrid(np.arange(n0 // 2), [0], [0], indexing="ij"), -1).reshape(-1, 3)
    refined = []
    for l, xs in enumerate(refined_x):
        m = 2 ** (l + 1)
        yz = np.stack(np.meshgrid(np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 2)
        cells = [np.column_stack([np.full(len(yz), int(ix)), yz]) for ix in sorted(set(int(v) for v in xs))]
        refined.append(np.concatenate(cells).astype(np.int64) if cells else np.zeros((0, 3), np.int64))
    return hierarchy_from_refined(base.astype(np.int32), refined, 1.0 / n0)


def equilibrium_amr(l_max: int, n0: int = 8):
    """The equilibrium test's AMR set-up on a static mesh: base n0 cells over
    [0, 1]; level l + 1 refines the right half of level l's x range
    ([1 - 2^-(l+1), 1]: the steep end of the steady profile), up to l_max.
    Dirichlet sides -x (E = 4) and +x (E = 0.5); step initial state.
    Returns (levels, per-level E_init, walls {side: E})."""
    refined_x = []
    for l in range(l_max):
        n_l = n0 * 2 ** l                    # level-l cells across the whole domain
        refined_x.append(list(range(n_l - n0 // 2, n_l)))
    levels = column_hierarchy(n0, refined_x)
    E = []
    for lv in levels:
        x = (lv.cell_xyz()[:, 0] + 0.5) * lv.dx
        E.append(np.where(x < 0.5, 4.0, 0.5).astype(np.float64))
    return levels, E, {0: 4.0, 1: 0.5}


def dirac_column(E0: float = 1e5, K: float = 1e10):
    """The linear diffusion test's set-up (Sect. 4.1) on a static mesh: a
    column over [0, 1] with a base of 32 cells and three levels of refinement
    nested around the centre (level 1 on [0.25, 0.75], level 2 on
    [0.3125, 0.6875], level 3 on [0.375, 0.625]: effective resolution 256);
    E = 1 everywhere except the finest cells of the slice starting at
    x = 0.5, which hold E0 / dx (a Dirac of weight E0); K = c / (3 rho
    kappa_R) with rho kappa_R = 1 and c = 3e10 (cgs); coarse step 3.125e-15,
    64 coarse steps to t = 2e-13.  Returns (levels, per-level (E, K), dt0,
    n_steps, x0 = centre of the Dirac cell)."""
    levels = column_hierarchy(32, [list(range(8, 24)), list(range(20, 44)), list(range(48, 80))])
    states = []
    dx3 = levels[-1].dx
    for l, lv in enumerate(levels):
        E = np.ones(lv.n_cell)
        if l == len(levels) - 1:
            E[lv.cell_xyz()[:, 0] == 128] = E0 / dx3
        states.append((E, np.full(lv.n_cell, K)))
    return levels, states, 3.125e-15, 64, 0.5 + 0.5 * dx3


def gaussian_32cube(n: int = 32, K: float = 1.0, cfl: float = 10.0):
    """Single-level uniform n^3 box on [-1/2, 1/2]^3, constant K, one backward-
    Euler step of dt = cfl * dx^2 / (2K), Gaussian (sigma 0.05) + 1e-3 floor,
    zero-flux walls."""
    dx = 1.0 / n
    lv = box_level(n // 2, n // 2, n // 2, dx)
    xyz = cell_centres(lv, (-0.5, -0.5, -0.5))
    E = gaussian(xyz)
    Kc = np.full(lv.n_cell, K)
    dt = cfl * dx * dx / (2.0 * K)
    return lv, Step(dt=dt, K=Kc, E=E)


def _near_cubic(o: int):
    a = max(1, int(round(o ** (1.0 / 3.0))))
    b = max(1, int(round(math.sqrt(o / a))))
    c = max(1, int(round(o / (a * b))))
    return a, b, c


def random_box_solve(rng: np.random.Generator, n_oct_target: float, dt_lo=1e-3, dt_hi=1e2,
                     robin=False, neumann_flux=False):
    """One batched-workload solve: a near-cubic oct box, K = exp(N(0,1)) per
    cell, E ~ U(0.5, 1.5), dt log-uniform in [dt_lo, dt_hi] x dx^2/(2 K_med)
    (K_med = 1), each wall zero-flux Neumann or Dirichlet (E_nb ~ U(0, 2));
    with ``robin`` each wall is Dirichlet / Neumann / Robin (1/3 each,
    alpha ~ U(0,1)) and Neumann / Robin walls carry a flux F."""
    a, b, c = _near_cubic(int(round(n_oct_target)))
    dx = 1.0 / (2 * max(a, b, c))
    walls, wall_E, wall_F = [], [], []
    for d in range(6):
        if robin:
            k = int(rng.integers(0, 3))
            al = float(rng.uniform(0.0, 1.0)) if k == ROBIN else (1.0 if k == DIRICHLET else 0.0)
            walls.append((k, al))
        else:
            k = DIRICHLET if rng.uniform() < 0.5 else NEUMANN
            walls.append((k, 1.0) if k == DIRICHLET else None)
        wall_E.append(float(rng.uniform(0.0, 2.0)))
        wall_F.append(float(rng.uniform(-0.05, 0.05)) if (robin or neumann_flux) else 0.0)
    lv = box_level(a, b, c, dx, walls)
    K = np.exp(rng.standard_normal(lv.n_cell))
    E = rng.uniform(0.5, 1.5, lv.n_cell)
    f = math.exp(rng.uniform(math.log(dt_lo), math.log(dt_hi)))
    dt = f * dx * dx / 2.0
    fd = lv.face_dir.astype(np.int64)
    face_E = np.array(wall_E)[fd] if lv.n_face else np.zeros(0)
    face_F = np.array(wall_F)[fd] if lv.n_face else np.zeros(0)
    return lv, Step(dt=dt, K=K, E=E, face_E=face_E, face_F=face_F)


def ragged_batch(n_solves: int = 512, seed: int = 1404, lo_oct: int = 64, hi_oct: int = 32768):
    """Batched level solves: oct counts log-uniform in [lo_oct, hi_oct]
    (8^3 .. 64^3 cells), ragged near-cubic boxes, per-solve dt log-uniform in
    1e-3..1e2 x explicit CFL, K log-normal (sigma 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_solves):
        o = math.exp(rng.uniform(math.log(lo_oct), math.log(hi_oct)))
        out.append(random_box_solve(rng, o))
    return out


def served_requests(n_req: int = 2000, seed: int = 1405, lo_cells: int = 16 ** 3, hi_cells: int = 256 ** 3,
                     rate: float = 1.0):
    """Served request stream: Poisson arrival times (rate per second), cells
    log-uniform in [lo_cells, hi_cells], Dirichlet / Neumann / Robin walls,
    tol 1e-6 or 1e-10 (50/50).  Returns a list of dicts with the arrival time,
    tolerance and a zero-argument builder of (level, step) so large requests
    are only materialised when used."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(n_req):
        t += float(rng.exponential(1.0 / rate))
        cells = math.exp(rng.uniform(math.log(lo_cells), math.log(hi_cells)))
        tol = 1e-6 if rng.uniform() < 0.5 else 1e-10
        sub_seed = int(rng.integers(0, 2 ** 62))
        reqs.append({"id": i, "t": t, "tol": tol, "octs": cells / 8.0, "seed": sub_seed})
    return reqs


def build_request(req):
    rng = np.random.default_rng(req["seed"])
    return random_box_solve(rng, req["octs"], robin=True)


def random_amr_level(seed: int, n_box: int = 3, refine_frac: float = 0.2, dx: float = 0.1,
                     kinds=(DIRICHLET, NEUMANN, ROBIN), box_hi: int = 4):
    """A small irregular level for parity tests: a union of random oct boxes
    (corners in [0, box_hi)^3, extents in [1, box_hi) octs per axis), some
    leaf cells refined (non-leaf), and a descriptor of random kind / relation /
    alpha on every face without a same-level leaf neighbour, except a random
    subset left as zero-flux walls.  Per-step values are random."""
    rng = np.random.default_rng(seed)
    pts = []
    for _ in range(n_box):
        lo = rng.integers(0, box_hi, 3)
        ext = rng.integers(1, box_hi, 3)
        g = np.stack(np.meshgrid(*[np.arange(lo[k], lo[k] + ext[k]) for k in range(3)], indexing="ij"), -1)
        pts.append(g.reshape(-1, 3))
    xyz = np.unique(np.concatenate(pts), axis=0).astype(np.int32)
    xyz = xyz[morton_sort(xyz)]
    n_oct = xyz.shape[0]
    leaf = np.full(n_oct, 0xFF, dtype=np.uint8)
    for o in range(n_oct):
        for c in range(8):
            if rng.uniform() < refine_frac / 4:
                leaf[o] &= np.uint8(~(1 << c) & 0xFF)
    # keep at least one leaf
    if not np.any(leaf):
        leaf[0] = 1
    cell, dr, nb = ghost_faces(xyz, leaf)
    keep = rng.uniform(size=len(cell)) < 0.85
    cell, dr, nb = cell[keep], dr[keep], nb[keep]
    kind = rng.choice(np.array(kinds, dtype=np.int8), size=len(cell))
    rel = np.where(nb >= 0, REL_FINER, np.where(rng.uniform(size=len(cell)) < 0.5, REL_COARSER, REL_SAME)).astype(np.int8)
    alpha = np.where(kind == DIRICHLET, 1.0, np.where(kind == NEUMANN, 0.0, rng.uniform(0, 1, len(cell))))
    lv = LevelDesc(xyz, leaf, dx, cell.astype(np.int32), dr.astype(np.int8), kind, rel, alpha.astype(np.float64))
    N = lv.n_cell
    K = np.exp(rng.standard_normal(N))
    E = rng.uniform(0.5, 1.5, N)
    nf = lv.n_face
    step = Step(
        dt=float(rng.uniform(0.5, 20.0)) * dx * dx / 2.0,
        K=K,
        E=E,
        face_K=np.exp(rng.standard_normal(nf)),
        face_E=rng.uniform(0.0, 2.0, nf),
        face_F=rng.uniform(-0.1, 0.1, nf),
    )
    return lv, step


def split_round_robin(n_units: int, world: int, rank: int) -> List[int]:
    """Units owned by ``rank`` when independent solves are sharded over ranks."""
    return list(range(rank, n_units, world))


# ---------------------------------------------------------------------------
# AMR hierarchies (levels of octs; level l+1 octs = refined cells of level l)
# ---------------------------------------------------------------------------

def _cells_of_octs(oct_xyz: np.ndarray) -> np.ndarray:
    c = np.arange(8)
    bits = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
    return (2 * oct_xyz.astype(np.int64)[:, None, :] + bits[None]).reshape(-1, 3)


def hierarchy_from_refined(base_octs: np.ndarray, refined_per_level, dx0: float):
    """Levels from the base oct list and, per level l, the set of refined
    cells (int64 [m, 3] level-l cell coordinates).  Returns a list of
    LevelDesc (Morton-ordered octs, leaf masks, no face descriptors)."""
    levels = []
    octs = base_octs[morton_sort(base_octs)].astype(np.int32)
    for l in range(len(refined_per_level) + 1):
        ref = refined_per_level[l] if l < len(refined_per_level) else np.zeros((0, 3), np.int64)
        cells = _cells_of_octs(octs)
        if len(ref):
            refset = set(map(tuple, np.asarray(ref, dtype=np.int64)))
            is_ref = np.array([tuple(c) in refset for c in cells], dtype=bool)
        else:
            is_ref = np.zeros(len(cells), dtype=bool)
        leaf = np.zeros(len(octs), dtype=np.uint8)
        for c in range(8):
            leaf |= ((~is_ref.reshape(-1, 8)[:, c]).astype(np.uint8) << np.uint8(c))
        empty = np.zeros(0)
        levels.append(LevelDesc(octs, leaf, dx0 / 2 ** l, empty.astype(np.int32), empty.astype(np.int8),
                                empty.astype(np.int8), empty.astype(np.int8), empty.astype(np.float64)))
        if len(ref):
            nxt = np.asarray(ref, dtype=np.int64).astype(np.int32)
            octs = nxt[morton_sort(nxt)]
    return levels


def balance_refinement(existing_cells: np.ndarray, want: np.ndarray, domain_cells: int) -> np.ndarray:
    """Keep only the wanted refined cells whose face neighbours inside the
    domain all exist at this level (so every fine-to-coarse face meets a
    leaf one level down: 2:1 balance).  Coordinates are level cell coords;
    the domain is [0, domain_cells)^3 at this level."""
    have = set(map(tuple, existing_cells.tolist()))
    keep = []
    for c in want.tolist():
        ok = True
        for a in range(3):
            for s in (-1, 1):
                q = list(c)
                q[a] += s
                if 0 <= q[a] < domain_cells and tuple(q) not in have:
                    ok = False
        if ok:
            keep.append(c)
    return np.array(keep, dtype=np.int64).reshape(-1, 3)


def two_level_gaussian_64cube(n0: int = 64, K: float = 1.0, cfl: float = 10.0, sigma: float = 0.05):
    """Two-level heat test: base n0^3 on [-1/2, 1/2]^3, level 1 (2x) covering
    the central 1/8 of the volume ([-1/4, 1/4]^3), constant K, Gaussian pulse
    at the origin; dt_coarse = cfl dx0^2 / (2K), fine substeps dt/2.  Returns
    (levels, per-level (E, K), dt_coarse)."""
    dx0 = 1.0 / n0
    base = box_octs(n0 // 2, n0 // 2, n0 // 2)
    q0, q1 = n0 // 4, 3 * n0 // 4
    g = np.stack(np.meshgrid(*[np.arange(q0, q1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    levels = hierarchy_from_refined(base, [g], dx0)
    states = []
    for lv in levels:
        xyz = cell_centres(lv, (-0.5, -0.5, -0.5))
        states.append((gaussian(xyz, sigma=sigma), np.full(lv.n_cell, K)))
    return levels, states, cfl * dx0 * dx0 / (2.0 * K)


def random_hierarchy(seed: int, n0: int = 8, n_levels: int = 3, frac: float = 0.35):
    """Small random 2:1-balanced hierarchy for parity tests: base n0^3 cells,
    each further level refines a random blob (ball around a random centre) of
    the previous one.  K log-normal, E random."""
    rng = np.random.default_rng(seed)
    dx0 = 1.0 / n0
    base = box_octs(n0 // 2, n0 // 2, n0 // 2)
    refined = []
    octs = base.astype(np.int64)
    for l in range(n_levels - 1):
        cells = _cells_of_octs(octs)
        nl = n0 * 2 ** l
        centre = rng.uniform(0.3, 0.7, 3) * nl
        r = np.linalg.norm(cells + 0.5 - centre, axis=1)
        want = cells[r < np.quantile(r, frac)]
        ref = balance_refinement(cells, want, nl)
        if len(ref) == 0:
            break
        refined.append(ref)
        octs = ref
    levels = hierarchy_from_refined(base, refined, dx0)
    states = []
    for lv in levels:
        states.append((rng.uniform(0.5, 1.5, lv.n_cell), np.exp(rng.standard_normal(lv.n_cell))))
    return levels, states, float(rng.uniform(2.0, 20.0)) * dx0 * dx0 / 2.0


def _trilinear(field: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of a cell-centred field on [-1/2, 1/2]^3
    (n^3 cells) at points pts [m, 3], clamped at the walls."""
    n = field.shape[0]
    u = (pts + 0.5) * n - 0.5
    i0 = np.clip(np.floor(u).astype(np.int64), 0, n - 1)
    i1 = np.clip(i0 + 1, 0, n - 1)
    f = np.clip(u - i0, 0.0, 1.0)
    out = np.zeros(len(pts))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                ix = i1[:, 0] if dx else i0[:, 0]
                iy = i1[:, 1] if dy else i0[:, 1]
                iz = i1[:, 2] if dz else i0[:, 2]
                w = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
                out += w * field[ix, iy, iz]
    return out


def radiation_matter_amr(n0: int = 128, n_levels: int = 4, sigma_ln: float = 1.5, r0: float = 0.05,
                         seed: int = 1403, cfl: float = 30.0):
    """FLD radiation-matter workload on an AMR grid: base n0^3 on
    [-1/2, 1/2]^3; density = trilinear interpolation of a seeded log-normal
    base field (sigma_ln, mean 1) times a central core 1/(1+(r/r0)^2); a cell
    of level l < n_levels-1 is refined where density > 4^(l+1) x the base
    mean, then eroded to keep 2:1 balance.  T0 = 1; E0 = a_R T0^4 (1 + 10
    exp(-r^2/(2 0.05^2))); k0 makes the median base-cell optical depth
    rho kappa_R dx0 = 1.  Returns (levels, per-level (E, rho, T), k0, cfl) -- the
    time step is set from the base-level K by the caller (cfl x explicit)."""
    rng = np.random.default_rng(seed)
    dx0 = 1.0 / n0
    lnrho = sigma_ln * rng.standard_normal((n0, n0, n0))
    base_field = np.exp(lnrho)
    base_field /= base_field.mean()
    base = box_octs(n0 // 2, n0 // 2, n0 // 2)

    def density(lv_cells, dx):
        xyz = -0.5 + (lv_cells + 0.5) * dx
        r2 = (xyz ** 2).sum(1)
        return _trilinear(base_field, xyz) / (1.0 + r2 / (r0 * r0))

    base_cells = _cells_of_octs(base)
    rho_mean = density(base_cells, dx0).mean()
    refined = []
    octs = base.astype(np.int64)
    for l in range(n_levels - 1):
        cells = _cells_of_octs(octs)
        dx = dx0 / 2 ** l
        rho = density(cells, dx)
        want = cells[rho > 4.0 ** (l + 1) * rho_mean]
        ref = balance_refinement(cells, want, n0 * 2 ** l)
        if len(ref) == 0:
            break
        refined.append(ref)
        octs = ref
    levels = hierarchy_from_refined(base, refined, dx0)
    states = []
    for lv in levels:
        cells = lv.cell_xyz()
        rho = density(cells, lv.dx)
        xyz = cell_centres(lv, (-0.5, -0.5, -0.5))
        E = 1.0 + 10.0 * np.exp(-(xyz ** 2).sum(1) / (2 * 0.05 ** 2))
        states.append((E, rho, np.ones(lv.n_cell)))
    rho0 = states[0][1]
    k0 = 1.0 / (np.median(rho0 * rho0) * dx0)
    return levels, states, k0, cfl
