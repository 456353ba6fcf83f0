"""Linear diffusion (Dirac) test of Sect. 4.1 with adaptive refinement: pins
of the oracle's runs that do not depend on the implementation.

* Moving the state to a new mesh (injection into new fine cells,
  restriction out of removed ones) keeps the total energy.
* The mesh refines every cell the 25 % criterion flags, up to the finest
  level, and the Dirac sits on the finest level.
* With the stored-flux Neumann rows (alpha = 0) the closed box keeps its
  energy (to the solve tolerance); the Dirichlet rows (alpha = 1) do not, and
  the Robin rows (alpha = 0.5) change it by about half as much -- the
  ordering the paper reports.
* The profile follows the analytic spreading of the pulse to a few percent
  in its core.
"""
import numpy as np
import pytest

from oracle import dirac as D

STEPS = 8


@pytest.fixture(scope="module")
def runs():
    return {name: D.run(iface, alpha, n_steps=STEPS)
            for name, iface, alpha in (("dirichlet", "dirichlet", 1.0), ("robin", "robin", 0.5),
                                       ("neumann", "neumann", 0.0))}


def test_initial_mesh_puts_the_dirac_on_the_finest_level():
    profile, x0 = D.initial_profile()
    levels, states = D.initial_mesh(profile)
    assert len(levels) == D.L_MAX + 1
    x, dx, e = D.leaf_profile(levels, [s[0] for s in states])
    k = int(np.argmax(e))
    assert dx[k] == pytest.approx(1.0 / (D.N0 * 2 ** D.L_MAX))
    assert x[k] == pytest.approx(x0)
    assert D.leaf_energy(levels, [s[0] for s in states]) == pytest.approx(float(np.sum(profile)) / len(profile),
                                                                         rel=1e-14)


def test_regrid_keeps_the_energy_and_refines_flagged_cells(runs):
    levels, E, _, _ = runs["dirichlet"]
    before = D.leaf_energy(levels, E)
    new_levels, states = D.regrid(levels, E)
    assert D.leaf_energy(new_levels, [s[0] for s in states]) == pytest.approx(before, rel=1e-13)
    # every flagged cell of a level below the finest is refined, unless it sits
    # on its level's edge (proper nesting)
    for l in range(len(new_levels) - 1):
        lv = new_levels[l]
        xyz = lv.cell_xyz()
        row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0)
        vals = dict(zip(xyz[row, 0].tolist(), states[l][0][row].tolist()))
        leaf = dict(zip(xyz[row, 0].tolist(), lv.leaf_cells()[row].tolist()))
        for i, e in vals.items():
            inner = (i - 1 in vals or i == 0) and (i + 1 in vals or i + 1 == D.N0 * 2 ** l)
            flagged = any(j in vals and 2 * abs(e - vals[j]) / (e + vals[j]) > D.THRESHOLD for j in (i - 1, i + 1))
            if flagged and inner:
                assert not leaf[i], (l, i)


def test_energy_by_interface_row(runs):
    rel = {k: v[2] / v[2][0] - 1.0 for k, v in runs.items()}
    assert np.max(np.abs(rel["neumann"])) <= 1e-9
    assert rel["dirichlet"][-1] > 1e-3
    assert 0.4 <= rel["robin"][-1] / rel["dirichlet"][-1] <= 0.6


def test_profile_follows_the_analytic_spreading(runs):
    t = STEPS * D.DT0
    for name, (levels, E, _, x0) in runs.items():
        x, dx, e = D.leaf_profile(levels, E)
        ref = D.analytic(x, t, x0)
        core = np.abs(x - x0) < 2.0 * np.sqrt(2.0 * D.K_DIFF * t)
        assert np.max(np.abs(e[core] - ref[core]) / ref[core]) <= 0.05, name
