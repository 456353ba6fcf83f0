"""Crank-Nicolson steps on the GPU (the second-order integrator Sect. 3.3.5
names): the library builds the backward-Euler system of the half step, solves
it, and returns 2 x' - E^n; the oracle solves the Crank-Nicolson system
(I + dt/2 A) E^{n+1} = (I - dt/2 A) E^n + the step's face and source terms
directly.

Tolerance, derived per case: both sides stop on the certified rule
||b - M x|| <= tol ||x|| and both matrices have lambda_min >= 1, so the
library's half-step root is within tol ||x'|| of the exact one (doubled by the
extrapolation) and the oracle's E^{n+1} within tol ||E^{n+1}||:
||E_gpu - E_oracle|| <= 2 tol ||x'|| + tol ||E^{n+1}||.  With tol = 2.5e-11
that bound stays below 1e-10 ||E^{n+1}|| on these inputs (checked).

Crank-Nicolson does not keep positivity (its factor tends to -1 on stiff
modes), so a solve may end with the warning ATS_WARN_NEGATIVE: success is
a status >= 0.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 2.5e-11
PAR = 1e-10


@pytest.fixture(scope="module")
def ats():
    from paper_1401_1112_gb300 import ats as A
    from paper_1401_1112_gb300 import build

    build.build()
    return A


@pytest.fixture(scope="module")
def ctx(ats):
    c = ats.Context(0)
    yield c
    c.close()


def _faces(st):
    return dict(face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)


def _cn_oracle(lv, st, tol=TOL):
    x, info = oracle.cn_step(lv, st.dt, st.K, st.E, src=st.src, tol=tol, stop_rule=oracle.STOP_CERTIFIED,
                             **_faces(st))
    assert info["status"] == 0
    return x


def _be_oracle(lv, st, tol=TOL):
    S = oracle.assemble(lv, st.dt, st.K, st.E, src=st.src, **_faces(st))
    x, info = oracle.pcg(S, st.E, tol=tol, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0
    return x


def _check_cn(x, xr, E, tol=TOL):
    """x: library result, xr: oracle E^{n+1}, E: E^n."""
    half = 0.5 * (xr + E)
    bound = 2.0 * tol * np.linalg.norm(half) + tol * np.linalg.norm(xr)
    assert bound <= PAR * np.linalg.norm(xr)
    assert np.linalg.norm(x - xr) <= bound


def _with_src(st, seed):
    rng = np.random.default_rng(seed)
    st.src = rng.uniform(-0.2, 0.5, st.E.shape[0])
    return st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", [21, 22, 23])
def test_cn_level_matches_oracle(ats, ctx, prec, seed):
    """Irregular AMR level, Dirichlet / Neumann / Robin faces with flux F, a
    source: one Crank-Nicolson step against the oracle's."""
    lv, st = W.random_amr_level(seed)
    st = _with_src(st, seed)
    xr = _cn_oracle(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, src=st.src, integrator=ats.ATS_INTEGRATOR_CRANK_NICOLSON, **_faces(st))
    x = st.E.copy()
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED,
                          precision=ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED)
    assert code >= 0, stats
    _check_cn(x, xr, st.E)
    nl = ~lv.leaf_cells()
    np.testing.assert_array_equal(x[nl], st.E[nl])  # 2 E - E on cells the solve leaves alone
    # a backward-Euler build of the same level afterwards is backward Euler again
    L.build(st.dt, st.K, st.E, src=st.src, **_faces(st))
    x = st.E.copy()
    code, _ = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED)
    assert code >= 0
    xb = _be_oracle(lv, st)
    assert np.linalg.norm(x - xb) <= PAR * np.linalg.norm(xb)
    L.close()


def test_cn_initial_guess_is_a_guess_of_the_new_state(ats, ctx):
    """x on entry guesses E^{n+1}: starting from the oracle's answer the solve
    has almost nothing left to do, and the result still matches."""
    lv, st = W.random_amr_level(31)
    xr = _cn_oracle(lv, st, tol=1e-13)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, integrator=ats.ATS_INTEGRATOR_CRANK_NICOLSON, **_faces(st))
    x = st.E.copy()
    code, cold = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_FP64)
    assert code >= 0
    x = xr.copy()
    code, warm = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_FP64)
    assert code >= 0
    assert warm["iterations"] < cold["iterations"]
    assert warm["r0_norm"] < 1e-6 * cold["r0_norm"]
    _check_cn(x, xr, st.E)
    L.close()


@pytest.mark.parametrize("mem", ["host", "device"])
def test_cn_batch_mixed_integrators(ats, ctx, mem):
    """A batch whose levels alternate backward Euler and Crank-Nicolson, built
    through the batched build, started from E^n of the build (x0 = E_old):
    each level matches its own oracle and, bitwise, its solo solve."""
    import torch

    rng = np.random.default_rng(97)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (3, 60, 250, 9, 700)]
    integ = [ats.ATS_INTEGRATOR_CRANK_NICOLSON if k % 2 == 0 else ats.ATS_INTEGRATOR_BACKWARD_EULER
             for k in range(len(solves))]
    dev = torch.device("cuda:0")
    conv = (lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)) if mem == "device" \
        else (lambda a: a)
    M = ats.ATS_MEM_DEVICE if mem == "device" else ats.ATS_MEM_HOST
    levels = [ats.Level(ctx, lv) for lv, _ in solves]
    coefs = [dict(dt=st.dt, K=conv(st.K), E_old=conv(st.E), face_K=conv(st.face_K), face_E=conv(st.face_E),
                  face_F=conv(st.face_F), integrator=ig) for (_, st), ig in zip(solves, integ)]
    for L, c in zip(levels, coefs):  # a batch is made over built levels
        L.build(**c)
    torch.cuda.synchronize()
    B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, mem=M,
                  use_graph=1, x0=ats.ATS_X0_E_OLD)
    B.build_operators(B.prepare_coefs(coefs))
    xs = [conv(np.full(lv.n_cell, np.nan)) for lv, _ in solves]
    code, stats = B.solve(xs)
    assert code >= 0, stats
    got = [x.cpu().numpy() if mem == "device" else x for x in xs]
    B.close()
    for (lv, st), ig, x, L in zip(solves, integ, got, levels):
        if ig == ats.ATS_INTEGRATOR_CRANK_NICOLSON:
            _check_cn(x, _cn_oracle(lv, st), st.E)
        else:
            xb = _be_oracle(lv, st)
            assert np.linalg.norm(x - xb) <= PAR * np.linalg.norm(xb)
        L.build(st.dt, st.K, st.E, integrator=ig, **_faces(st))
        xo = st.E.copy()
        code, _ = L.solve(xo, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
        assert code >= 0
        np.testing.assert_array_equal(xo, x)
    for L in levels:
        L.close()


def test_cn_server_requests(ats):
    """Crank-Nicolson requests through the serving loop, with and without an
    initial guess, beside backward-Euler ones."""
    rng = np.random.default_rng(98)
    reqs = [W.random_box_solve(rng, o, robin=True) for o in (5, 40, 300, 12)]
    srv = ats.Server(0, precision=ats.ATS_PREC_MIXED, check_every=4)
    tickets = []
    for k, (lv, st) in enumerate(reqs):
        ig = ats.ATS_INTEGRATOR_CRANK_NICOLSON if k != 1 else ats.ATS_INTEGRATOR_BACKWARD_EULER
        x0 = st.E * 0.9 if k == 2 else None
        tickets.append((srv.submit(lv, st, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, x0=x0, integrator=ig), ig))
    for (lv, st), (t, ig) in zip(reqs, tickets):
        code, x, res = srv.wait(t, lv.n_cell)
        assert code >= 0, res
        if ig == ats.ATS_INTEGRATOR_CRANK_NICOLSON:
            _check_cn(x, _cn_oracle(lv, st), st.E)
        else:
            xb = _be_oracle(lv, st)
            assert np.linalg.norm(x - xb) <= PAR * np.linalg.norm(xb)
    srv.close()


def test_cn_rejects_a_shift_and_unknown_integrators(ats, ctx):
    lv, st = W.random_amr_level(41)
    L = ats.Level(ctx, lv)
    with pytest.raises(ats.AtsError) as e:
        L.build(st.dt, st.K, st.E, s=np.ones_like(st.K), integrator=ats.ATS_INTEGRATOR_CRANK_NICOLSON,
                **_faces(st))
    assert e.value.code == ats.ATS_ERR_INVALID_ARG
    with pytest.raises(ats.AtsError) as e:
        L.build(st.dt, st.K, st.E, integrator=7, **_faces(st))
    assert e.value.code == ats.ATS_ERR_INVALID_ARG
    L.close()
