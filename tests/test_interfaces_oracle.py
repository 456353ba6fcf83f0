"""Energy-conserving interfaces in the oracle (Sect. 3.3.1 - 3.3.2): pins that
do not depend on the implementation.

* Neumann coarse-to-fine rows fed by the stored fine-side flux conserve the
  total energy of a closed box (zero-flux walls, no source) exactly, up to
  the solve tolerance (Sect. 3.3.2; the alpha = 0 case of the diffusion test).
* With Dirichlet rows the energy changes by exactly the interface mismatch:
  in a closed box, the total change equals the sum over the coarse solves of
  the energy their coarse-to-fine faces delivered minus the fine-side energy
  stored for them; Robin rows change it by alpha times that Dirichlet-type
  mismatch ((1 - alpha) of the energy is conserved).
* Sect. 3.3.5: the flux-conserving (Neumann) rows can drive a level's energy
  negative; the Dirichlet rows cannot.  With Dirichlet rows and no source
  every level matrix is an M-matrix whose rows sum to 1 plus the Dirichlet
  weights, so the solution obeys the discrete maximum principle: it stays
  between the least and the greatest of E^n and the ghost values.
* In a 1D column with constant K the change equals the paper's two-level
  mismatch expression (Sect. 3.3.2, with the fine-to-coarse flux
  (E_1 - E_c) + (E_2 - E_c), and the oct mean of the fine cells where the
  paper assumes a uniform oct).
"""
import numpy as np
import pytest

import workloads as W
from oracle import driver

TOL = 1e-13


@pytest.mark.parametrize("seed", [3, 8])
def test_neumann_interfaces_conserve_energy(seed):
    levels, states, dt = W.random_hierarchy(seed, n0=8, n_levels=3)
    H = driver.Hierarchy(levels, states, order="fine_first", interface="neumann")
    e0 = H.energy()
    H.advance(0, dt, tol=TOL)
    e1 = H.energy()
    assert abs(e1 - e0) <= 1e-11 * abs(e0), (e0, e1)
    for _, gained, consumed in H.audit:
        assert abs(gained - consumed) <= 1e-13 * abs(e0) + 1e-15


@pytest.mark.parametrize("interface,alpha", [("dirichlet", 1.0), ("robin", 0.5), ("robin", 0.2)])
def test_energy_changes_by_the_interface_mismatch(interface, alpha):
    levels, states, dt = W.random_hierarchy(5, n0=8, n_levels=3)
    H = driver.Hierarchy(levels, states, order="fine_first", interface=interface, alpha=alpha)
    e0 = H.energy()
    H.advance(0, dt, tol=TOL)
    de = H.energy() - e0
    mismatch = sum(g - c for _, g, c in H.audit)
    assert abs(de) > 1e-9 * abs(e0)  # the test case does not conserve
    assert abs(de - mismatch) <= 1e-11 * abs(e0), (de, mismatch)


def test_robin_conserves_one_minus_alpha_of_the_mismatch():
    """Two levels, one coarse step: the measured energy change equals alpha
    times (the Dirichlet flux of the coarse-to-fine faces, recomputed here
    from the final state: restricted E and K of the refined cells, the coarse
    solution, minus the stored fine-side energy)."""
    levels, states, dt = W.random_hierarchy(5, n0=8, n_levels=2)
    for alpha in (0.25, 0.75):
        H = driver.Hierarchy(levels, states, order="fine_first", interface="robin", alpha=alpha)
        e0 = H.energy()
        H.advance(0, dt, tol=TOL)
        de = H.energy() - e0
        (_, _, consumed), = [a for a in H.audit if a[0] == 0]
        dx = levels[0].dx
        h = dt / (2.0 * dx * dx)
        dirichlet = 0.0
        for cell, _, rel, R in H.faces[0]:
            if rel == driver.REL_FINER:
                dirichlet += h * (H.K[0][cell] + H.K[0][R]) * (H.E[0][R] - H.E[0][cell]) * dx ** 3
        assert abs(de - alpha * (dirichlet - consumed)) <= 1e-11 * abs(e0), (de, dirichlet, consumed)


def test_column_matches_the_papers_mismatch_expression():
    nx = 4
    dx0 = 1.0 / (2 * nx)
    base = np.array([[x, 0, 0] for x in range(nx)], dtype=np.int64)
    ref = np.array([[x, y, z] for x in range(nx, 2 * nx) for y in (0, 1) for z in (0, 1)], dtype=np.int64)
    levels = W.hierarchy_from_refined(base, [ref], dx0)
    K = 1.3
    rng = np.random.default_rng(11)
    states = []
    for lv in levels:
        # E depends on x only
        xyz = lv.oct_xyz.astype(np.int64)
        cx = (2 * xyz[:, 0:1] + (np.arange(8)[None, :] & 1)).reshape(-1)
        prof = 1.0 + rng.uniform(0.0, 2.0, int(cx.max()) + 1)
        states.append((prof[cx], np.full(lv.n_cell, K)))
    dt = 3.0 * dx0 * dx0
    H = driver.Hierarchy(levels, states, order="fine_first", interface="dirichlet")
    e0 = H.energy()
    fine, coarse = levels[1], levels[0]
    dxf = fine.dx
    # the fine cells at the interface: x cell coordinate 2 nx (level 1); the
    # coarse interface cell: x cell coordinate nx - 1 (level 0)
    def column(l, xc):
        xyz = levels[l].oct_xyz.astype(np.int64)
        cx = (2 * xyz[:, 0:1] + (np.arange(8)[None, :] & 1)).reshape(-1)
        return np.nonzero(cx == xc)[0]

    fi, fi2, ci = column(1, 2 * nx), column(1, 2 * nx + 1), column(0, nx - 1)
    Ec_n = float(H.E[0][ci[0]])
    H.advance(1, dt / 2, tol=TOL)
    E1 = float(H.E[1][fi[0]])
    H.advance(1, dt / 2, tol=TOL)
    E2 = float(H.E[1][fi[0]])
    ER = 0.5 * (E2 + float(H.E[1][fi2[0]]))  # mean of the oct next to the interface
    H.solve_level(0, dt, 0.0, TOL)
    Ec_1 = float(H.E[0][ci[0]])
    # all cells of a column share the value (the problem is 1D)
    assert np.ptp(H.E[1][fi]) <= 1e-12 * abs(E2) and np.ptp(H.E[0][ci]) <= 1e-12 * abs(Ec_1)
    F_f = 0.5 * K / (1.5 * dxf) * ((E1 - Ec_n) + (E2 - Ec_n))  # fine -> coarse, mean over the two steps
    F_c = K / (2.0 * dxf) * (Ec_1 - ER)                      # coarse -> fine
    area = (2 * dx0) ** 2                                     # the column's cross-section
    expected = -area * dt * (F_f + F_c)
    de = H.energy() - e0
    assert abs(de) > 1e-8 * e0
    assert abs(de - expected) <= 1e-11 * abs(e0), (de, expected)


@pytest.mark.parametrize("seed", [1, 5])
def test_dirichlet_rows_keep_the_maximum_principle_neumann_rows_do_not(seed):
    levels, states, dt = W.random_hierarchy(seed, n0=8, n_levels=3)
    lo = min(float(e.min()) for e, _ in states)
    hi = max(float(e.max()) for e, _ in states)
    mins = {}
    for interface in ("dirichlet", "neumann"):
        H = driver.Hierarchy(levels, [(e.copy(), k.copy()) for e, k in states], order="fine_first",
                             interface=interface)
        mn, mx = np.inf, -np.inf
        for _ in range(2):
            H.advance(0, dt, tol=TOL)
            for l, lv in enumerate(levels):
                leaf = H.state(l)[lv.leaf_cells()]
                mn, mx = min(mn, float(leaf.min())), max(mx, float(leaf.max()))
        mins[interface] = mn
        if interface == "dirichlet":
            assert lo - 1e-10 <= mn and mx <= hi + 1e-10, (lo, hi, mn, mx)
    assert mins["neumann"] < 0.0, mins

