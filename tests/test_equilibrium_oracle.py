"""Equilibrium test with a nonlinear diffusion coefficient (Sect. 4.2) on
uniform grids: pins of the oracle's steady states that do not depend on the
implementation.

* The closed-form profile holds the wall values and carries a constant flux
  K(E) dE/dx (it is the steady state of the law K = K0 E^a).
* The relaxed state is the discrete equilibrium: every face flux, the two
  wall faces (ghost value one cell width away) included, is the same.
* The relaxed state does not depend on the time step (it is the fixed point
  of the lagged steps).
* Against the closed form, the paper's L2 norm falls by close to 4 per
  halving of dx (the paper: close to second order on uniform grids).
"""
import numpy as np
import pytest

import workloads as W
from oracle import equilibrium as Q

RESOLUTIONS = (8, 16, 32, 64, 128)


@pytest.fixture(scope="module")
def relaxed():
    out = {}
    for n in RESOLUTIONS:
        lv, E, fE, _ = W.equilibrium_column(n)
        Es, steps, ok = Q.relax(lv, E, fE)
        assert ok, (n, steps)
        out[n] = (lv, Es, fE)
    return out


def test_closed_form_holds_the_walls_and_a_constant_flux():
    a = Q.A_EXP
    assert Q.analytic(0.0) == pytest.approx(Q.E_LEFT, rel=1e-15)
    assert Q.analytic(1.0) == pytest.approx(Q.E_RIGHT, rel=1e-15)
    x = np.linspace(0.05, 0.95, 37)
    h = 2e-4
    # fourth-order central difference of the closed form
    d = (-Q.analytic(x + 2 * h) + 8 * Q.analytic(x + h) - 8 * Q.analytic(x - h) + Q.analytic(x - 2 * h)) / (12 * h)
    flux = Q.power_law_K(Q.analytic(x), 1.0, a) * d
    assert np.max(np.abs(flux - flux[0])) <= 1e-8 * abs(flux[0])
    assert flux[0] < 0.0  # energy flows from the hot wall at x = 0


def test_relaxed_state_is_the_discrete_equilibrium(relaxed):
    lv, E, fE = relaxed[32]
    xyz = lv.cell_xyz()
    for ix in range(32):  # uniform in y and z
        col = E[xyz[:, 0] == ix]
        assert np.max(col) - np.min(col) <= 1e-12 * np.max(col)
    _, e = Q.profile(lv, E)
    dx = lv.dx
    K = Q.power_law_K(e)
    inner = 0.5 * (K[1:] + K[:-1]) * (e[1:] - e[:-1]) / dx
    left = 0.5 * (K[0] + Q.power_law_K(Q.E_LEFT)) * (e[0] - Q.E_LEFT) / dx
    right = 0.5 * (K[-1] + Q.power_law_K(Q.E_RIGHT)) * (Q.E_RIGHT - e[-1]) / dx
    flux = np.concatenate([[left], inner, [right]])
    assert np.max(np.abs(flux - flux.mean())) <= 1e-7 * abs(flux.mean())


def test_relaxed_state_does_not_depend_on_the_step(relaxed):
    lv, E, fE = relaxed[16]
    _, E0, _, _ = W.equilibrium_column(16)
    E_big, _, ok = Q.relax(lv, E0, fE, dt=2.0)
    assert ok
    assert np.max(np.abs(E_big - E)) <= 1e-8 * np.max(E)


def test_uniform_grids_converge_at_close_to_second_order(relaxed):
    l2 = [Q.l2_error(relaxed[n][0], relaxed[n][1]) for n in RESOLUTIONS]
    ratios = [l2[i] / l2[i + 1] for i in range(len(l2) - 1)]
    assert all(3.0 <= r <= 4.5 for r in ratios), ratios
    assert ratios[-1] >= 3.5, ratios


def test_walled_hierarchy_holds_the_exact_linear_steady_state():
    """Constant K (a = 0), Dirichlet sides on a three-level column refined in
    its interior: the linear profile through the two ghost values (at
    x = -dx0/2 and 1 + dx0/2) is reproduced exactly by every level's rows
    (fine-to-coarse ghosts, restrictions and walls are all exact for a
    linear function), so the relaxed state equals it on every leaf."""
    levels = W.column_hierarchy(8, [[3, 4], [7, 8]])
    E0, E1 = 3.0, 1.0
    E_init = [np.full(lv.n_cell, 2.0) for lv in levels]
    Es, steps, ok = Q.relax_amr(levels, E_init, {0: E0, 1: E1}, K0=1.0, a=0.0)
    assert ok, steps
    dx0 = levels[0].dx
    for lv, E in zip(levels, Es):
        x = (lv.cell_xyz()[:, 0] + 0.5) * lv.dx
        lin = E0 + (E1 - E0) * (x + 0.5 * dx0) / (1.0 + dx0)
        leaf = lv.leaf_cells()
        assert np.max(np.abs(E[leaf] - lin[leaf])) <= 1e-9


def test_single_level_hierarchy_matches_the_uniform_relaxation(relaxed):
    levels, E_init, walls = W.equilibrium_amr(0)
    Es, _, ok = Q.relax_amr(levels, E_init, walls)
    assert ok
    lv, E, _ = relaxed[8]
    assert np.max(np.abs(Es[0] - E)) <= 1e-9 * np.max(E)


def test_adaptive_levels_lower_the_error():
    """The paper's adaptive-time-step runs of this test (static mesh refined
    toward the steep end): each added level lowers the L2 norm; the error of
    the coarse region, which the refinement does not touch, keeps it from
    falling as fast as on uniform grids (the paper: first order at best with
    more than two levels)."""
    l2 = []
    for l_max in range(4):
        levels, E_init, walls = W.equilibrium_amr(l_max)
        Es, steps, ok = Q.relax_amr(levels, E_init, walls)
        assert ok, (l_max, steps)
        l2.append(Q.l2_error_amr(levels, Es, 8 * 2 ** l_max))
    ratios = [l2[i] / l2[i + 1] for i in range(len(l2) - 1)]
    assert all(1.2 <= r <= 4.0 for r in ratios), ratios
