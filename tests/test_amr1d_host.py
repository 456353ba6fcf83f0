"""Host side of the library's linear-diffusion (Dirac) driver against the
oracle's independent version (CPU): the initial mesh and state, a remesh of
an evolved state and the leaf-row readout agree exactly, the energies to
round-off (cells compared by their level coordinates: the two order their
octs differently)."""
import numpy as np
import pytest

from oracle import dirac as D
from paper_1401_1112_gb300 import amr1d as A


def _cells(lv, E):
    """{(x, y, z): (leaf, value)} of a level."""
    xyz = lv.cell_xyz()
    leaf = lv.leaf_cells()
    return {tuple(map(int, p)): (bool(f), float(v)) for p, f, v in zip(xyz, leaf, np.asarray(E))}


def _same_mesh(lib_levels, lib_E, ora_levels, ora_E):
    assert len(lib_levels) == len(ora_levels)
    for lv, lo, e, eo in zip(lib_levels, ora_levels, lib_E, ora_E):
        assert lv.dx == lo.dx and lv.n_oct == lo.n_oct
        assert _cells(lv, e) == _cells(lo, eo)


def test_initial_mesh_matches_the_oracle():
    levels, E, x0 = A.pulse_mesh()
    profile, x0_ref = D.initial_profile()
    ora_levels, states = D.initial_mesh(profile)
    ora_E = [s[0] for s in states]
    assert x0 == x0_ref and len(levels) == D.L_MAX + 1
    _same_mesh(levels, E, ora_levels, ora_E)
    assert A.energy(levels, E) == pytest.approx(D.leaf_energy(ora_levels, ora_E), rel=1e-14)
    for a, b in zip(A.leaf_row(levels, E), D.leaf_profile(ora_levels, ora_E)):
        np.testing.assert_array_equal(a, b)


def test_remesh_of_an_evolved_state_matches_the_oracle():
    ora_levels, ora_E, _, _ = D.run("dirichlet", 1.0, n_steps=2)  # an evolved state
    lib_levels, lib_E = A.remesh(ora_levels, ora_E)
    new_levels, states = D.regrid(ora_levels, ora_E)
    new_E = [s[0] for s in states]
    _same_mesh(lib_levels, lib_E, new_levels, new_E)
    assert A.energy(lib_levels, lib_E) == pytest.approx(D.leaf_energy(new_levels, new_E), rel=1e-14)
