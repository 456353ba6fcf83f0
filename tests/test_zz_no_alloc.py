"""The allocation-free entry point against the FP64 oracle and the regular solve.

ats_solve_noalloc serves callers that cannot allocate device memory: a
plug-in confined to a memory pool its host program owns, or a process whose
device memory belongs to another runtime's caching allocator.  It keeps its CG
scratch in one fixed device array inside the library.  The call is
synchronous (it synchronises its stream), so a stream under capture is
rejected.

This file runs last (pytest collects it after the other test files) so that a
run stopping at the first failure has already run everything else.  It must
pass alone in a fresh process and after the other tests.

Tolerance: the level matrix has lambda_min >= 1 (D >= I plus a weighted graph
Laplacian and non-negative interface terms), so ||x - x*|| <= ||b - A x||.
Each side's distance to the exact solution is bounded by its own FP64
residual: the no-alloc solve's res_norm, the oracle's certified residual and
the regular solve's certified 5e-11 ||x||.  The tests assert those bounds and
the relative L2 parity 1e-10 the other parity tests use.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

PAR = 1e-10       # relative L2 agreement, as in the other parity tests
NA_TOL = 1e-12    # residual reduction asked of the no-alloc solve
CERT = 5e-11      # certified rule of the regular solve and of the oracle reference


@pytest.fixture(scope="module")
def ats():
    from paper_1401_1112_gb300 import ats as A
    from paper_1401_1112_gb300 import build

    build.build()
    return A


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _faces(st):
    return dict(face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)


def _noalloc_inputs(lv, st):
    """b and the extra diagonal xd of the no-alloc call, both from the
    oracle's assembled matrix: b is its right-hand side, and since the only
    off-diagonal entries are the same-level leaf faces (-C each), the row sum
    of a leaf row is 1 + xd (coupling shift plus the interface terms)."""
    S = oracle.assemble(lv, st.dt, st.K, st.E, s=st.s, src=st.src, **_faces(st))
    leaf = lv.leaf_cells()
    xd = np.where(leaf, S.matvec(np.ones(lv.n_cell)) - 1.0, 0.0)
    K = np.where(leaf, st.K, -1.0)
    return S, S.b.copy(), xd, K


def _oracle_x(S, E):
    x, info = oracle.pcg(S, E, tol=1e-13, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0, info
    return x, info["residual"]


def _call(ats, lv, K, xd, b, x0, dt, stream=0):
    import torch

    dev = torch.device("cuda:0")
    h = 0.5 * dt / lv.dx ** 2
    nbr = torch.from_numpy(ats.ats_layout_neighbors(lv).reshape(-1).copy()).to(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    x = t(x0)
    code, st = ats.ats_solve_noalloc(0, stream, lv.n_oct, nbr, t(K), t(xd), h, t(b), x, tol=NA_TOL)
    assert code == 0, (st, ats.ats_last_error())
    assert st["res_norm"] <= NA_TOL * st["r0_norm"] * 1.0001
    return x.cpu().numpy(), st


def _walled_box(rng, dims, dx):
    lv = W.box_level(*dims, dx, [(W.DIRICHLET, 1.0), (W.ROBIN, 0.4), (W.NEUMANN, 0.0),
                                 (W.DIRICHLET, 1.0), (W.ROBIN, 0.7), None])
    N, nf = lv.n_cell, lv.n_face
    st = W.Step(dt=20.0 * dx ** 2 / 2.0, K=np.exp(rng.standard_normal(N)), E=rng.uniform(0.5, 1.5, N),
                s=rng.uniform(0.0, 2.0, N), face_K=np.exp(rng.standard_normal(nf)),
                face_E=rng.uniform(0.0, 2.0, nf), face_F=rng.uniform(-0.1, 0.1, nf))
    return lv, st


def _check_against_oracle_and_solve(ats, lv, st, x_na, na_stats, x_or, or_res):
    # against the oracle: both within their own residuals of the exact solution
    bound = na_stats["res_norm"] + or_res
    assert np.linalg.norm(x_na - x_or) <= bound * 1.0001 + 1e-14 * np.linalg.norm(x_or)
    assert _rel(x_na, x_or) <= PAR
    # against the regular entry point, certified to 5e-11 ||x||
    with ats.Context(0) as ctx:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, s=st.s, src=st.src, **_faces(st))
        x_ref = st.E.copy()
        code, st_ref = L.solve(x_ref, tol=CERT, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_FP64)
        assert code == 0, st_ref
        L.close()
    assert np.linalg.norm(x_na - x_ref) <= (na_stats["res_norm"] + st_ref["res_norm"]) * 1.0001 + \
        1e-14 * np.linalg.norm(x_ref)
    assert _rel(x_na, x_ref) <= PAR


def test_noalloc_two_calls_in_a_row_match_oracle_and_regular_solve(ats):
    """Two calls in a row on levels with Dirichlet / Robin / Neumann walls and
    a coupling shift, so xd and the interface part of b carry weight."""
    rng = np.random.default_rng(2024)
    for dims in ((9, 7, 6), (5, 11, 4)):
        lv, st = _walled_box(rng, dims, 1.0 / 22)
        S, b, xd, K = _noalloc_inputs(lv, st)
        x_or, or_res = _oracle_x(S, st.E)
        x_na, na = _call(ats, lv, K, xd, b, st.E, st.dt)
        _check_against_oracle_and_solve(ats, lv, st, x_na, na, x_or, or_res)


def test_noalloc_at_the_size_limit_then_smaller(ats):
    """A 64^3 level (exactly ATS_NOALLOC_MAX_CELLS, 128 work items), then a
    small level: the scratch array keeps the large call's contents, and the
    small call must give bitwise what it gives on a fresh array."""
    rng = np.random.default_rng(77)
    small_lv, small_st = _walled_box(rng, (6, 5, 7), 1.0 / 14)
    S_s, b_s, xd_s, K_s = _noalloc_inputs(small_lv, small_st)
    x_small_first, _ = _call(ats, small_lv, K_s, xd_s, b_s, small_st.E, small_st.dt)

    lv, st = _walled_box(rng, (32, 32, 32), 1.0 / 64)
    assert lv.n_cell == ats.ATS_NOALLOC_MAX_CELLS
    S, b, xd, K = _noalloc_inputs(lv, st)
    x_or, or_res = _oracle_x(S, st.E)
    x_na, na = _call(ats, lv, K, xd, b, st.E, st.dt)
    _check_against_oracle_and_solve(ats, lv, st, x_na, na, x_or, or_res)

    x_small_after, _ = _call(ats, small_lv, K_s, xd_s, b_s, small_st.E, small_st.dt)
    np.testing.assert_array_equal(x_small_after, x_small_first)
    x_or_s, _ = _oracle_x(S_s, small_st.E)
    assert _rel(x_small_after, x_or_s) <= PAR


@pytest.mark.parametrize("seed", [5, 9])
def test_noalloc_cells_that_are_not_unknowns(ats, seed):
    """Levels with refined (non-leaf) cells, marked by K < 0: their x is left
    exactly as given, the leaf cells match the oracle."""
    lv, st = W.random_amr_level(seed)
    leaf = lv.leaf_cells()
    assert (~leaf).sum() > 0
    S, b, xd, K = _noalloc_inputs(lv, st)
    x_or, or_res = _oracle_x(S, st.E)
    x0 = st.E.copy()
    x0[~leaf] = np.arange((~leaf).sum()) + 0.25   # arbitrary values to keep
    x_na, na = _call(ats, lv, K, xd, b, x0, st.dt)
    np.testing.assert_array_equal(x_na[~leaf], x0[~leaf])
    err = np.linalg.norm(x_na[leaf] - x_or[leaf])
    assert err <= (na["res_norm"] + or_res) * 1.0001 + 1e-14 * np.linalg.norm(x_or)
    assert err <= PAR * np.linalg.norm(x_or[leaf])


def test_noalloc_rejects_a_capturing_stream(ats):
    """The call synchronises its stream: under stream capture it must refuse
    (nothing enqueued, the capture left intact) instead of breaking it."""
    import torch

    rng = np.random.default_rng(3)
    lv, st = _walled_box(rng, (3, 3, 3), 0.1)
    S, b, xd, K = _noalloc_inputs(lv, st)
    x_or, _ = _oracle_x(S, st.E)
    # an ordinary call first: it also makes the once-per-device set-up, which
    # must not happen inside a capture
    x_na, _ = _call(ats, lv, K, xd, b, st.E, st.dt)
    assert _rel(x_na, x_or) <= PAR
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    nbr = torch.from_numpy(ats.ats_layout_neighbors(lv).reshape(-1).copy()).to(dev)
    Kd, xdd, bd, x = t(K), t(xd), t(b), t(st.E)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        y = x * 2.0   # something for the capture to hold
        code, _ = ats.ats_solve_noalloc(0, side.cuda_stream, lv.n_oct, nbr, Kd, xdd, 0.5 * st.dt / lv.dx ** 2,
                                        bd, x, tol=NA_TOL)
    assert code == ats.ATS_ERR_INVALID_ARG
    assert "captured" in ats.ats_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, x * 2.0)
    # the entry point still works on an ordinary stream afterwards
    x_again, _ = _call(ats, lv, K, xd, b, st.E, st.dt)
    np.testing.assert_array_equal(x_again, x_na)


def test_noalloc_rejects_oversize(ats):
    import torch

    dev = torch.device("cuda:0")
    n_oct = ats.ATS_NOALLOC_MAX_CELLS // 8 + 1
    t = torch.zeros(8, dtype=torch.float64, device=dev)
    nbr = torch.zeros(6, dtype=torch.int32, device=dev)
    code, _ = ats.ats_solve_noalloc(0, 0, n_oct, nbr, t, None, 1.0, t, t)
    assert code == ats.ATS_ERR_INVALID_ARG
    assert "scratch" in ats.ats_last_error()
