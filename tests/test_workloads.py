"""The seeded input generators follow the stated recipes (CPU): the same
seed gives the same arrays, and the sizes, ranges and boundary mixes are the
ones the benchmark line and the parity tests describe."""
import numpy as np
import pytest

import workloads as W


def _same(a, b):
    (la, sa), (lb, sb) = a, b
    np.testing.assert_array_equal(la.oct_xyz, lb.oct_xyz)
    np.testing.assert_array_equal(la.face_kind, lb.face_kind)
    assert sa.dt == sb.dt
    for f in ("K", "E", "face_E", "face_F"):
        np.testing.assert_array_equal(getattr(sa, f), getattr(sb, f))


def test_ragged_batch_is_seeded():
    a, b = W.ragged_batch(n_solves=8), W.ragged_batch(n_solves=8)
    for x, y in zip(a, b):
        _same(x, y)
    c = W.ragged_batch(n_solves=8, seed=1405)
    assert any(x[0].n_oct != z[0].n_oct for x, z in zip(a, c))


@pytest.fixture(scope="module")
def batch():
    return W.ragged_batch()


def test_ragged_batch_recipe(batch):
    """512 solves of 64..32 768 octs (21 087 200 cells in all), near-cubic
    boxes, K > 0 log-normal, E in [0.5, 1.5], dt in [1e-3, 1e2] x dx^2 / 2,
    each wall zero-flux or Dirichlet with E_nb in [0, 2]."""
    assert len(batch) == 512
    assert sum(lv.n_cell for lv, _ in batch) == 21087200
    octs = np.array([lv.n_oct for lv, _ in batch])
    assert octs.min() >= 64 and octs.max() <= 32768
    ratio = np.array([st.dt / (lv.dx ** 2 / 2) for lv, st in batch])
    assert ratio.min() >= 1e-3 * (1 - 1e-12) and ratio.max() <= 1e2 * (1 + 1e-12)
    assert np.log10(ratio).std() > 1.0  # spread over the five decades
    kinds = set()
    for lv, st in batch:
        assert np.all(st.K > 0) and st.E.min() >= 0.5 and st.E.max() <= 1.5
        ext = lv.oct_xyz.max(axis=0) - lv.oct_xyz.min(axis=0) + 1
        assert int(np.prod(ext)) == lv.n_oct and ext.max() <= 2 * ext.min() + 1
        kinds |= set(np.unique(lv.face_kind).tolist())
        if lv.n_face:
            assert st.face_E.min() >= 0.0 and st.face_E.max() <= 2.0
            assert np.all(st.face_F == 0.0)
    assert kinds == {W.DIRICHLET}  # zero-flux walls carry no descriptor
    logK = np.log(np.concatenate([st.K for _, st in batch[:16]]))
    assert abs(logK.mean()) < 0.01 and abs(logK.std() - 1.0) < 0.01


def test_gaussian_32cube_recipe():
    lv, st = W.gaussian_32cube()
    assert lv.n_cell == 32 ** 3 and lv.n_face == 0 and lv.dx == 1.0 / 32
    assert st.dt == pytest.approx(10.0 * lv.dx ** 2 / 2.0, rel=1e-15)
    assert np.all(st.K == 1.0)
    assert st.E.min() >= 1e-3 and st.E.max() <= 1.0 + 1e-3


def test_served_requests_recipe():
    reqs = W.served_requests()
    assert len(reqs) == 2000
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    cells = np.array([8 * r["octs"] for r in reqs])
    assert cells.min() >= 16 ** 3 * (1 - 1e-12) and cells.max() <= 256 ** 3 * (1 + 1e-12)
    tols = [r["tol"] for r in reqs]
    assert set(tols) == {1e-6, 1e-10} and 0.45 < tols.count(1e-6) / len(tols) < 0.55


def test_box_wall_faces_equal_the_general_search():
    """The analytic wall faces of a box equal the general ghost-face search
    (same faces, same (cell, dir) order)."""
    for dims in ((1, 1, 1), (3, 5, 7), (9, 2, 4), (8, 8, 8)):
        xyz = W.box_octs(*dims)
        c1, d1, _ = W.ghost_faces(xyz, None)
        c2, d2 = W.box_wall_faces(xyz, *dims)
        np.testing.assert_array_equal(c1, c2)
        np.testing.assert_array_equal(d1, d2)
