"""GPU parity of the large work-item path against the FP64 oracle.

A level gets about one work item per CTA of the stencil kernel's resident
grid, so a level above ~155 k octs runs with 384..1024-oct items: several octs
per thread and per-item reductions of other sizes than the 256-oct items of
smaller levels.  These tests put that path against the oracle (the level
matrix of Eq. Er_imp1 with the interface rows of Sect. 3.2, Jacobi-PCG of
Sect. 3.3.4):

  * one level of 163 840 octs (64 x 64 x 40 octs, 1.31 M cells) with
    log-normal K and Dirichlet / Neumann / Robin walls, with the default item
    size and with explicit 384 / 512 / 1024-oct items, FP64 and mixed;
  * irregular AMR levels with every interface kind and ragged batches, at
    384 / 512 / 1024-oct items;
  * one coarse step of the 4-level radiation-matter workload (base 128^3)
    against the oracle's adaptive time-stepping driver, per level, for E and
    the gas temperature.

Tolerance: both sides stop on the certified rule ||b - A x|| <= 5e-11 ||x||;
lambda_min >= 1 bounds each solution's error by its residual, so one solve
differs by at most 1e-10 (relative L2).  A hierarchy step chains n solves:
n x 1e-10.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import driver, fld

pytestmark = pytest.mark.gpu

TOL = 5e-11
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _faces(st):
    return dict(face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)


def _oracle_x(lv, st):
    S = oracle.assemble(lv, st.dt, st.K, st.E, s=st.s, src=st.src, **_faces(st))
    x, info = oracle.pcg(S, st.E, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0, info
    return x


@pytest.fixture(scope="module")
def big_level():
    """64 x 64 x 40 octs (163 840 octs, above the ~155 k-oct threshold of
    384-oct items), K = exp(N(0,1)), dt = 30 explicit steps, walls of every
    kind with random ghost values and fluxes."""
    rng = np.random.default_rng(1311)
    dx = 1.0 / 128
    lv = W.box_level(64, 64, 40, dx, [(W.DIRICHLET, 1.0), (W.NEUMANN, 0.0), (W.ROBIN, 0.3),
                                      (W.DIRICHLET, 1.0), (W.ROBIN, 0.8), (W.NEUMANN, 0.0)])
    N, nf = lv.n_cell, lv.n_face
    st = W.Step(dt=30.0 * dx * dx / 2.0, K=np.exp(rng.standard_normal(N)), E=rng.uniform(0.5, 1.5, N),
                face_K=np.exp(rng.standard_normal(nf)), face_E=rng.uniform(0.0, 2.0, nf),
                face_F=rng.uniform(-0.05, 0.05, nf))
    return lv, st, _oracle_x(lv, st)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tile", [0, 384, 512, 1024])
def test_large_level_matches_oracle(ats, ctx, big_level, prec, tile):
    """The tick path at the default and explicit item sizes; with the default
    scheduler, mixed precision, the level (at most 1 100 octs per SM) takes
    the whole-GPU form, which must match too."""
    lv, st, xr = big_level
    assert lv.n_oct > 155_000
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    P = ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED
    scheds = [ats.ATS_SCHED_TICK] + ([ats.ATS_SCHED_AUTO] if tile == 0 else [])
    for sc in scheds:
        x = st.E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P, tile_octs=tile, sched=sc)
        assert code == 0, stats
        assert stats["err_bound"] <= TOL
        assert _rel(x, xr) <= PAR
    L.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tile", [384, 512, 1024])
@pytest.mark.parametrize("seed", [11, 12, 13])
def test_irregular_amr_levels_large_items(ats, ctx, prec, tile, seed):
    """The tick path on unions of random oct boxes (hundreds of octs, several passes per thread
    at these item sizes) with refined cells and every interface kind."""
    lv, st = W.random_amr_level(seed, n_box=4, box_hi=14)
    xr = _oracle_x(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    x = st.E.copy()
    P = ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P, tile_octs=tile,
                          sched=ats.ATS_SCHED_TICK)
    assert code == 0, stats
    assert _rel(x, xr) <= PAR
    nl = ~lv.leaf_cells()
    np.testing.assert_array_equal(x[nl], st.E[nl])
    L.close()


@pytest.mark.parametrize("tile", [384, 512, 1024])
def test_ragged_batch_large_items(ats, ctx, tile):
    """The tick path on a ragged batch at large item sizes: every solve matches the oracle and
    is bitwise the same alone and in the batch."""
    rng = np.random.default_rng(4242 + tile)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (1, 7, 100, 900, 2500, 5000)]
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    xs = [st.E.copy() for _, st in solves]
    B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                  use_graph=1, check_every=8, tile_octs=tile, sched=ats.ATS_SCHED_TICK)
    code, stats = B.solve(xs)
    assert code == 0, stats
    for (lv, st), x in zip(solves, xs):
        assert _rel(x, _oracle_x(lv, st)) <= PAR
    for k, ((lv, st), L) in enumerate(zip(solves, levels)):
        x = st.E.copy()
        code, _ = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                          tile_octs=tile, sched=ats.ATS_SCHED_TICK)
        assert code == 0
        np.testing.assert_array_equal(x, xs[k])
    B.close()
    for L in levels:
        L.close()


@pytest.mark.slow
def test_radiation_matter_full_size_coarse_step_matches_oracle(ats):
    """One coarse step of the 4-level radiation-matter workload at full size
    (base 128^3: 262 144 octs, 512-oct items by the size rule), fine first,
    mixed precision refined to the certified 5e-11, against the oracle's
    driver level by level: E and the gas temperature on the leaf cells."""
    with ats.Context(0) as ctx:
        levels, states, k0, cfl = W.radiation_matter_amr(n0=128)
        rho = [s[1] for s in states]
        T = [s[2] for s in states]
        K0, _, _ = fld.coefficients(levels[0], rho[0], T[0], states[0][0], 1.0, k0)
        dt = cfl * levels[0].dx ** 2 / (2.0 * np.median(K0[levels[0].leaf_cells()]))
        H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
        for l, (E, r, t) in enumerate(states):
            H.set_state(l, E, np.ones_like(E))
        for l, (E, r, t) in enumerate(states):
            H.set_fld(l, r, t, k0)
        code, st = H.advance(0, dt, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
        assert code == 0, st
        ref = driver.Hierarchy(levels, [(E, np.ones_like(E)) for E, _, _ in states], order="fine_first",
                               fld=(rho, T, k0))
        ref.advance(0, dt, tol=TOL)
        n_solves = sum(2 ** l for l in range(len(levels)))
        for l in range(len(levels)):
            assert _rel(H.state(l), ref.state(l)) <= n_solves * PAR, l
            leaf = levels[l].leaf_cells()
            assert _rel(H.temperature(l)[leaf], ref.fld[1][l][leaf]) <= n_solves * PAR, l
        H.close()
