"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test fails for a plausible mistake somewhere in the oracle: a wrong
face-coefficient scale or mean (golden hand values, second-moment identity),
a wrong sign of the Neumann flux (conservation with F != 0), a dropped alpha
in the Robin row (golden), a wrong 2/3 factor (golden), an asymmetric
off-diagonal (exact symmetry), a CG bug (DCT closed form, dense Cholesky).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import dense, spectral

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "one_oct_cases.json")


def _one_oct(kind, rel, alpha):
    return W.LevelDesc(
        np.zeros((1, 3), np.int32), None, 0.5,
        np.array([0, 2, 4, 6], np.int32), np.zeros(4, np.int8),
        np.full(4, kind, np.int8), np.full(4, rel, np.int8), np.full(4, alpha),
    )


def test_golden_one_oct_interface_rows():
    """Hand-derived exact values for the Dirichlet (2/3 factor), Neumann,
    Robin and face-mean rows (Sect. 3.1-3.2)."""
    cases = json.load(open(GOLDEN))
    for case in cases["cases"]:
        lv = _one_oct(case["kind"], case["rel"], case["alpha"])
        S = oracle.assemble(
            lv, 0.25, np.ones(8), np.ones(8),
            face_K=np.full(4, case["face_K"]), face_E=np.full(4, case["face_E"]),
            face_F=np.full(4, case["face_F"]),
        )
        x, info = oracle.pcg(S, np.ones(8), tol=1e-15, stop_rule=oracle.STOP_CERTIFIED)
        a = case["a"][0] / case["a"][1]
        c = case["c"][0] / case["c"][1]
        expect = np.array([a if (k & 1) == 0 else c for k in range(8)])
        np.testing.assert_allclose(x, expect, rtol=1e-13, err_msg=case["name"])
    im = cases["interior_mean_case"]
    lv = W.LevelDesc(np.zeros((1, 3), np.int32), None, 0.5, *(np.zeros(0, t) for t in (np.int32, np.int8, np.int8, np.int8, np.float64)))
    K = np.array([1.0 if (k & 1) == 0 else 3.0 for k in range(8)])
    E = np.array([1.0 if (k & 1) == 0 else 0.0 for k in range(8)])
    S = oracle.assemble(lv, 0.25, K, E)
    x, _ = oracle.pcg(S, E, tol=1e-15, stop_rule=oracle.STOP_CERTIFIED)
    expect = np.array([im["a"][0] / im["a"][1] if (k & 1) == 0 else im["c"][0] / im["c"][1] for k in range(8)])
    np.testing.assert_allclose(x, expect, rtol=1e-13)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_matrix_symmetric_and_spd(seed):
    """The level matrix is D + dt L with L a weighted graph Laplacian plus
    non-negative interface diagonal terms: exactly symmetric, lambda_min >= 1."""
    lv, st = W.random_amr_level(seed)
    S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    A = S.to_scipy()
    assert (A != A.T).nnz == 0  # bitwise symmetric
    Al, _, _ = dense.leaf_block(S)
    if Al.shape[0] <= 600:
        lam = np.linalg.eigvalsh(Al)
        assert lam.min() >= 1.0 - 1e-12


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_conservation_zero_flux_and_neumann_sign(seed):
    """With only Neumann faces every column of dt L sums to zero, so
    sum(x) = sum(b) = sum(E^n) + sum(F): energy is conserved exactly and an
    imposed flux F > 0 adds energy (reading of the Neumann sign)."""
    lv, st = W.random_amr_level(seed, kinds=(W.NEUMANN,))
    S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    x, info = oracle.pcg(S, st.E, tol=1e-13, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0
    leaf = lv.leaf_cells()
    total_in = st.E[leaf].sum() + st.face_F.sum()
    assert abs(x[leaf].sum() - total_in) <= 1e-12 * abs(total_in)
    # column sums of the leaf block are exactly 1 (the identity part)
    Al, _, _ = dense.leaf_block(S)
    np.testing.assert_allclose(Al.sum(axis=0), 1.0, atol=1e-12)


def test_robin_limits_equal_dirichlet_and_neumann():
    """Robin with alpha = 1 is the Dirichlet row, alpha = 0 the Neumann row."""
    lv, st = W.random_amr_level(21, kinds=(W.ROBIN,))
    fk = dict(face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    for alpha, kind in ((1.0, W.DIRICHLET), (0.0, W.NEUMANN)):
        lr = W.LevelDesc(lv.oct_xyz, lv.leaf, lv.dx, lv.face_cell, lv.face_dir, lv.face_kind, lv.face_rel, np.full(lv.n_face, alpha))
        lk = W.LevelDesc(lv.oct_xyz, lv.leaf, lv.dx, lv.face_cell, lv.face_dir, np.full(lv.n_face, kind, np.int8), lv.face_rel, lv.face_alpha)
        Sr = oracle.assemble(lr, st.dt, st.K, st.E, **fk)
        Sk = oracle.assemble(lk, st.dt, st.K, st.E, **fk)
        np.testing.assert_allclose(Sr.b, Sk.b, rtol=1e-15, atol=1e-15)
        np.testing.assert_allclose(Sr.val, Sk.val, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("dims", [(16, 16, 16), (3, 5, 2), (1, 1, 7)])
def test_dct_closed_form(dims):
    """Constant K, zero-flux walls: the DCT-II diagonalisation is the exact
    discrete solution (config-1 case is 32^3 at dt = 10 dx^2 / 2K)."""
    n = 32
    dx = 1.0 / n
    lv = W.box_level(*dims, dx)
    xyz = W.cell_centres(lv, (-0.5, -0.5, -0.5))
    E = W.gaussian(xyz)
    K = 1.7
    dt = 10 * dx * dx / (2 * K)
    S = oracle.assemble(lv, dt, np.full(lv.n_cell, K), E)
    x, info = oracle.pcg(S, E, tol=1e-14, stop_rule=oracle.STOP_CERTIFIED)
    xd = spectral.solve_level_box(lv, dt, K, S.b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


@pytest.mark.parametrize("seed", [31, 32, 33, 34])
def test_dense_cholesky(seed):
    """Tiny levels with every face type: own Cholesky, numpy's solver and the
    oracle's CG agree."""
    lv, st = W.random_amr_level(seed)
    S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    Al, bl, idx = dense.leaf_block(S)
    if Al.shape[0] > 400:
        pytest.skip("level too large for the dense check")
    xc = dense.cholesky_solve(Al, bl)
    xn = np.linalg.solve(Al, bl)
    assert np.linalg.norm(xc - xn) <= 1e-13 * np.linalg.norm(xn)
    x, info = oracle.pcg(S, st.E, tol=1e-13, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0
    assert np.linalg.norm(x[idx] - xn) <= 2e-13 * np.linalg.norm(xn)
    # non-leaf cells keep their initial value
    nl = ~lv.leaf_cells()
    np.testing.assert_array_equal(x[nl], st.E[nl])


def test_second_moment_identity():
    """Backward Euler on the discrete heat operator grows the second moment by
    exactly 2 K dt M0 per dimension (summation by parts), the continuum
    result; with a pulse far from the walls the identity holds to ~1e-10."""
    lv, st = W.gaussian_32cube(n=32, cfl=0.25)
    xyz = W.cell_centres(lv, (-0.5, -0.5, -0.5))
    r2 = (xyz ** 2).sum(1)
    c = 1e-3
    S = oracle.assemble(lv, st.dt, st.K, st.E)
    x, _ = oracle.pcg(S, st.E, tol=1e-14, stop_rule=oracle.STOP_CERTIFIED)
    ratio = ((r2 * (x - c)).sum() - (r2 * (st.E - c)).sum()) / (6 * st.dt * (x - c).sum())
    assert abs(ratio - 1.0) < 1e-9


def test_analytic_gaussian_first_order_in_time():
    """Loose pin against the analytic Gaussian (sigma_t^2 = sigma_0^2 + 2Kt):
    errors of a few percent, falling about linearly with dt (backward Euler
    is first order, Sect. 3.3.5)."""
    n = 32
    dx = 1.0 / n
    lv = W.box_level(n // 2, n // 2, n // 2, dx)
    xyz = W.cell_centres(lv, (-0.5, -0.5, -0.5))
    r2 = (xyz ** 2).sum(1)
    s0 = 0.1
    T = 4 * dx * dx
    errs = []
    for cfl in (8.0, 2.0):
        dt = cfl * dx * dx / 2
        x = W.gaussian(xyz, sigma=s0, floor=0.0)
        for _ in range(int(round(T / dt))):
            S = oracle.assemble(lv, dt, np.ones(lv.n_cell), x)
            x, _ = oracle.pcg(S, x, tol=1e-12, stop_rule=oracle.STOP_CERTIFIED)
        s2 = s0 ** 2 + 2 * T
        ana = (s0 ** 2 / s2) ** 1.5 * np.exp(-r2 / (2 * s2))
        errs.append(np.linalg.norm(x - ana) / np.linalg.norm(ana))
    assert errs[0] < 0.2 and errs[1] < 0.06
    assert errs[0] / errs[1] > 2.5  # ~first order over a 4x dt reduction


def test_stopping_rules():
    """Sect. 3.3.4: the L2 rule stops at ||r||/||r0|| < eps; the paper rule
    also needs the max relative change below eps; the certified rule bounds
    the true residual by tol ||x||."""
    lv, st = W.random_amr_level(41)
    S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    x1, i1 = oracle.pcg(S, st.E, tol=1e-6, stop_rule=oracle.STOP_RESIDUAL)
    assert i1["status"] == 0 and i1["residual"] / i1["r0"] < 2e-6
    x2, i2 = oracle.pcg(S, st.E, tol=1e-6, stop_rule=oracle.STOP_PAPER)
    assert i2["max_change"] < 1e-6 and i2["iterations"] >= i1["iterations"]
    x3, i3 = oracle.pcg(S, st.E, tol=1e-11, stop_rule=oracle.STOP_CERTIFIED)
    assert i3["residual"] <= 1e-11 * i3["x_norm"]


def test_invalid_descriptions_rejected():
    lv, st = W.random_amr_level(51)
    bad = W.LevelDesc(lv.oct_xyz, lv.leaf, lv.dx, np.concatenate([lv.face_cell, lv.face_cell[:1]]),
                      np.concatenate([lv.face_dir, lv.face_dir[:1]]), np.concatenate([lv.face_kind, lv.face_kind[:1]]),
                      np.concatenate([lv.face_rel, lv.face_rel[:1]]), np.concatenate([lv.face_alpha, lv.face_alpha[:1]]))
    with pytest.raises(ValueError):
        oracle.assemble(bad, st.dt, st.K, st.E)
