"""Crank-Nicolson step of the oracle (the second-order integrator named in
Sect. 3.3.5): pins that do not depend on the implementation.

* Constant K, zero-flux box: the step is diagonal in the DCT-II basis, each
  mode multiplied by (1 - c lambda / 2) / (1 + c lambda / 2), c = dt K / dx^2.
* Second order in time: against the exact semi-discrete solution
  exp(-t c lambda / dt) per mode, halving dt divides the error by ~4
  (backward Euler: by ~2).
* The explicit-right-hand-side form equals twice the backward-Euler half step
  minus E^n (the route the library takes), with Dirichlet, Neumann and Robin
  walls and a source.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import spectral

TOL = 1e-13


def _box(n, K=1.0):
    lv = W.box_level(n // 2, n // 2, n // 2, 1.0 / n)
    rng = np.random.default_rng(n)
    xyz = lv.cell_xyz()
    E = 1.0 + np.cos(np.pi * (xyz[:, 0] + 0.5) / n) + 0.3 * rng.standard_normal(lv.n_cell)
    return lv, np.full(lv.n_cell, K), E, xyz


def _modal(lv, xyz, E, factor):
    n = int(xyz.max()) + 1
    g = np.zeros((n, n, n))
    g[xyz[:, 0], xyz[:, 1], xyz[:, 2]] = E
    Q = spectral.dct2_matrix(n)
    lam = spectral.neumann_eigenvalues(n)
    L = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    gh = np.einsum("ai,bj,ck,ijk->abc", Q, Q, Q, g, optimize=True)
    out = np.einsum("ai,bj,ck,abc->ijk", Q, Q, Q, factor(L) * gh, optimize=True)
    return out[xyz[:, 0], xyz[:, 1], xyz[:, 2]]


def test_cn_step_is_the_modal_factor():
    lv, K, E, xyz = _box(8)
    dx = lv.dx
    dt = 7.0 * dx * dx
    c = dt * 1.0 / (dx * dx)
    x, info = oracle.cn_step(lv, dt, K, E, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0
    ref = _modal(lv, xyz, E, lambda L: (1.0 - 0.5 * c * L) / (1.0 + 0.5 * c * L))
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_cn_is_second_order_in_time():
    """Smooth data (low modes): the asymptotic rate needs c lambda dt / 2 well
    below 1 on the modes present (for stiff modes the CN factor tends to -1
    instead of decaying)."""
    lv, K, _, xyz = _box(8)
    n = 8
    E = 1.0 + np.cos(np.pi * (xyz[:, 0] + 0.5) / n) + 0.5 * np.cos(2 * np.pi * (xyz[:, 1] + 0.5) / n)
    dx = lv.dx
    T = 4.0 * dx * dx
    exact = _modal(lv, xyz, E, lambda L: np.exp(-T / (dx * dx) * L))
    err = {}
    for name, step in (("cn", oracle.cn_step), ("be", None)):
        err[name] = []
        for n_steps in (4, 8, 16):
            dt = T / n_steps
            x = E.copy()
            for _ in range(n_steps):
                if step is None:
                    x, info = oracle.solve_level(lv, dt, K, x, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
                else:
                    x, info = step(lv, dt, K, x, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
                assert info["status"] == 0
            err[name].append(np.linalg.norm(x - exact))
    r_cn = [err["cn"][i] / err["cn"][i + 1] for i in range(2)]
    r_be = [err["be"][i] / err["be"][i + 1] for i in range(2)]
    assert all(3.5 < r < 4.5 for r in r_cn), r_cn
    assert all(1.7 < r < 2.3 for r in r_be), r_be


@pytest.mark.parametrize("seed", [1, 2])
def test_cn_equals_extrapolated_half_step(seed):
    rng = np.random.default_rng(seed)
    lv, st = W.random_box_solve(rng, 60, robin=True)
    src = rng.uniform(-0.1, 0.1, lv.n_cell)
    faces = dict(face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    x, info = oracle.cn_step(lv, st.dt, st.K, st.E, src=src, tol=TOL, stop_rule=oracle.STOP_CERTIFIED, **faces)
    assert info["status"] == 0
    half = dict(face_K=st.face_K, face_E=st.face_E,
                face_F=None if st.face_F is None else 0.5 * st.face_F)
    xh, info = oracle.solve_level(lv, 0.5 * st.dt, st.K, st.E, tol=TOL, stop_rule=oracle.STOP_CERTIFIED,
                                  src=0.5 * src, **half)
    assert info["status"] == 0
    np.testing.assert_allclose(x, 2.0 * xh - st.E, rtol=0, atol=1e-11 * np.max(np.abs(x)))
