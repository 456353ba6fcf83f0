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
    levels, states, _ = W.config2(n0=16)
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
    levels, _, _ = W.config2(n0=16)
    # refine one more level at a corner of level 1 that touches level 0 directly
    fine = levels[1]
    corner = fine.oct_xyz.min(axis=0).astype(np.int64) * 2
    ref = np.array([corner], dtype=np.int64)
    lv = W.hierarchy_from_refined(levels[0].oct_xyz, [np.array(
        [tuple(c) for c in levels[1].oct_xyz.tolist()], dtype=np.int64), ref], levels[0].dx)
    with pytest.raises(ats.AtsError, match="2:1"):
        ats.ats_hierarchy_plan_faces(lv, 2)
