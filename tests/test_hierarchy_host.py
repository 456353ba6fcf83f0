"""Host-side checks of the hierarchy topology (no GPU): the interface faces
the library derives for each level equal the ones the oracle's driver
derives independently, and 2:1 violations are rejected."""
import numpy as np
import pytest

import workloads as W
from oracle import driver


@pytest.fixture(scope="module")
def ats():
    from paper_1401_1112_gb300 import ats as A
    from paper_1401_1112_gb300 import build

    build.build()
    return A


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_faces_match_oracle_driver(ats, seed):
    levels, states, _ = W.random_hierarchy(seed, n0=8, n_levels=3)
    H = driver.Hierarchy(levels, states)
    for l in range(len(levels)):
        cell, dr, rel, src = ats.ats_hierarchy_plan_faces(levels, l)
        mine = sorted(zip(cell.tolist(), dr.tolist(), rel.tolist(), src.tolist()))
        theirs = sorted(H.faces[l])
        assert mine == theirs


def test_two_level_faces(ats):
    levels, states, _ = W.two_level_gaussian_64cube(n0=16)
    H = driver.Hierarchy(levels, states)
    for l in range(2):
        cell, dr, rel, src = ats.ats_hierarchy_plan_faces(levels, l)
        assert sorted(zip(cell.tolist(), dr.tolist(), rel.tolist(), src.tolist())) == sorted(H.faces[l])
    # the refined block is 8^3 coarse cells: 6 * 8^2 coarse-to-fine faces and
    # 6 * (16^2) fine-to-coarse faces
    c0 = ats.ats_hierarchy_plan_faces(levels, 0)
    c1 = ats.ats_hierarchy_plan_faces(levels, 1)
    assert len(c0[0]) == 6 * 64 and np.all(c0[2] == ats.ATS_REL_FINER)
    assert len(c1[0]) == 6 * 256 and np.all(c1[2] == ats.ATS_REL_COARSER)


def test_unbalanced_rejected(ats):
    levels, _, _ = W.two_level_gaussian_64cube(n0=16)
    # refine one more level at a corner of level 1 that touches level 0 directly
    fine = levels[1]
    corner = fine.oct_xyz.min(axis=0).astype(np.int64) * 2
    ref = np.array([corner], dtype=np.int64)
    lv = W.hierarchy_from_refined(levels[0].oct_xyz, [np.array(
        [tuple(c) for c in levels[1].oct_xyz.tolist()], dtype=np.int64), ref], levels[0].dx)
    with pytest.raises(ats.AtsError, match="2:1"):
        ats.ats_hierarchy_plan_faces(lv, 2)


@pytest.mark.parametrize("sides", [{0: 1.0, 1: 2.0}, {2: 1.0, 5: 3.0}, {0: 1.0, 1: 1.0, 2: 1.0, 3: 1.0, 4: 1.0, 5: 1.0}])
def test_domain_side_faces_match_oracle_driver(ats, sides):
    """Dirichlet domain sides: every leaf of every level on such a side gets a
    face (relation REL_SAME, src = the side), as the oracle's driver derives
    them independently; the zero-flux sides get none."""
    levels = W.column_hierarchy(8, [[5, 6, 7], [12, 13, 14, 15]])   # refinement reaching the +x side
    states = [(np.ones(lv.n_cell), np.ones(lv.n_cell)) for lv in levels]
    walls = {s: (e, 1.0) for s, e in sides.items()}
    H = driver.Hierarchy(levels, states, walls=walls)
    for l in range(len(levels)):
        cell, dr, rel, src = ats.ats_hierarchy_plan_faces(levels, l, walls=walls)
        mine = sorted(zip(cell.tolist(), dr.tolist(), rel.tolist(), src.tolist()))
        assert mine == sorted(H.faces[l]), l
        wall = rel == ats.ATS_REL_SAME
        assert set(dr[wall].tolist()) <= set(sides)
        assert np.all(src[wall] == dr[wall])
    # a +x side face on the finest level (the refinement reaches it)
    cell, dr, rel, _ = ats.ats_hierarchy_plan_faces(levels, 2, walls=walls)
    assert (1 in sides) == bool(np.any((rel == ats.ATS_REL_SAME) & (dr == 1)))
