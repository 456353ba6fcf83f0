"""GPU parity of the whole-GPU form of the resident solver against the oracle.

With ATS_SCHED_GRID, a level above res_max_octs (FP32 bulk) is solved by one
cooperative launch with one CTA per SM: the level is split into one
contiguous run per CTA, each run's K, z, p stay in that CTA's shared memory,
the neighbours' faces across runs come from the global arrays, and the
sums of each CG step (Dot2 pairs, merged in rank order) and the steps
themselves are ordered by a grid barrier with bounded waits.  The method is
that of the other paths -- the level matrix of Eq. Er_imp1 with the
interface rows of Sect. 3.2, Jacobi-PCG (Sect. 3.3.4) in FP32 with FP64
refinement -- so the same bound holds: both sides stop on the certified rule
||b - A x|| <= 5e-11 ||x||, lambda_min >= 1 bounds each solution's error by
its residual, and they differ by at most 1e-10 relative.

Covered: box levels with every wall kind from just above the limit to more
octs than the CTAs' shared memory holds (octs beyond it read and written in
global memory), irregular levels with non-leaf cells and every interface
kind split over more CTAs than octs (idle CTAs in every barrier and sum),
bitwise equality alone / in a batch / run to run, a batch mixing every
resident form, and the barrier's bounded wait.
"""
import numpy as np
import pytest

import oracle
import workloads as W

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


def _faces(st):
    return dict(face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _oracle_x(lv, st):
    S = oracle.assemble(lv, st.dt, st.K, st.E, s=st.s, src=st.src, **_faces(st))
    x, info = oracle.pcg(S, st.E, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0, info
    return x


def _box(rng, dims, dx, stiff=30.0):
    lv = W.box_level(*dims, dx, [(W.DIRICHLET, 1.0), (W.NEUMANN, 0.0), (W.ROBIN, 0.3),
                                 (W.DIRICHLET, 1.0), (W.ROBIN, 0.8), None])
    N, nf = lv.n_cell, lv.n_face
    st = W.Step(dt=stiff * dx * dx / 2.0, K=np.exp(rng.standard_normal(N)), E=rng.uniform(0.5, 1.5, N),
                face_K=np.exp(rng.standard_normal(nf)), face_E=rng.uniform(0.0, 2.0, nf),
                face_F=rng.uniform(-0.05, 0.05, nf))
    return lv, st


def _solve(ats, ctx, lv, st, **kw):
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    x = st.E.copy()
    kw.setdefault("sched", ats.ATS_SCHED_GRID)
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, **kw)
    L.close()
    return code, stats, x


@pytest.mark.parametrize("dims", [(32, 32, 17), (40, 40, 32), (70, 70, 64)],
                         ids=["just-above-limit", "51k-octs", "beyond-shared-capacity"])
def test_box_levels_match_oracle(ats, ctx, dims):
    """17 408, 51 200 and 313 600 octs: the largest splits into runs of 2 064
    octs, 16 more than a CTA keeps in shared memory.  Both forms of the CG
    step (the neighbours' p after a barrier, or their z with the q
    recurrence)."""
    rng = np.random.default_rng(sum(dims))
    lv, st = _box(rng, dims, 1.0 / (2 * max(dims)))
    assert lv.n_oct > 16384
    xr = _oracle_x(lv, st)
    for form in (1, 2):
        code, stats, x = _solve(ats, ctx, lv, st, cg_form=form)
        assert code == 0, stats
        assert stats["err_bound"] <= TOL
        assert _rel(x, xr) <= PAR


@pytest.mark.parametrize("form", [1, 2], ids=["q-from-p", "q-recurrence"])
@pytest.mark.parametrize("seed", [21, 22, 23])
def test_irregular_levels_more_ctas_than_octs(ats, ctx, seed, form):
    """Unions of random oct boxes (tens to hundreds of octs) with non-leaf
    cells and every interface kind, sent to the whole-GPU form by a limit of
    8 octs: most CTAs own one oct or none and still take part in every
    barrier and sum; non-leaf cells keep their values."""
    lv, st = W.random_amr_level(seed, n_box=4, box_hi=8)
    assert lv.n_oct > 8
    code, stats, x = _solve(ats, ctx, lv, st, res_max_octs=8, cg_form=form)
    assert code == 0, stats
    assert _rel(x, _oracle_x(lv, st)) <= PAR
    nl = ~lv.leaf_cells()
    np.testing.assert_array_equal(x[nl], st.E[nl])


def test_alone_in_batch_and_run_to_run_bitwise(ats, ctx):
    """A whole-GPU level gives the same bits alone, twice, and inside a batch
    that also holds one-CTA and cluster solves; every solve of the batch
    matches the oracle."""
    rng = np.random.default_rng(77)
    big_lv, big_st = _box(rng, (32, 32, 24), 1.0 / 64)
    others = [W.random_box_solve(rng, o, robin=True) for o in (60, 3000, 12000)]
    solves = [(big_lv, big_st)] + others
    opts = dict(tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, sched=ats.ATS_SCHED_GRID)
    _, _, x1 = _solve(ats, ctx, big_lv, big_st)
    _, _, x2 = _solve(ats, ctx, big_lv, big_st)
    np.testing.assert_array_equal(x1, x2)
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    xs = [st.E.copy() for _, st in solves]
    B = ats.Batch(ctx, levels, use_graph=1, **opts)
    code, stats = B.solve(xs)
    assert code == 0, stats
    np.testing.assert_array_equal(xs[0], x1)
    for (lv, st), x in zip(solves, xs):
        assert _rel(x, _oracle_x(lv, st)) <= PAR
    B.close()
    for L in levels:
        L.close()


def test_several_whole_gpu_levels_in_one_batch(ats, ctx):
    """Three levels above a limit of 1 000 octs run one after another in the
    same cooperative launch (the barrier and the partial sums carry over
    from one solve to the next); each matches the oracle and its solve
    alone."""
    rng = np.random.default_rng(5)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (1500, 4000, 9000)]
    opts = dict(tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, res_max_octs=1000,
                sched=ats.ATS_SCHED_GRID)
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    xs = [st.E.copy() for _, st in solves]
    B = ats.Batch(ctx, levels, use_graph=1, **opts)
    code, stats = B.solve(xs)
    assert code == 0, stats
    for k, (lv, st) in enumerate(solves):
        assert _rel(xs[k], _oracle_x(lv, st)) <= PAR
        x = st.E.copy()
        code, _ = levels[k].solve(x, **opts)
        assert code == 0
        np.testing.assert_array_equal(x, xs[k])
    B.close()
    for L in levels:
        L.close()


def test_grid_and_tick_paths_agree(ats, ctx):
    """A large level on the whole-GPU form (forced, and the default for a
    level whose runs keep all six arrays in shared memory) and on the tick
    path: each within the parity bound of the oracle (their arithmetic
    differs, so not bitwise); the default gives the forced form's bits."""
    rng = np.random.default_rng(8)
    lv, st = _box(rng, (32, 32, 20), 1.0 / 64)
    xr = _oracle_x(lv, st)
    xs = []
    for sched in (ats.ATS_SCHED_GRID, ats.ATS_SCHED_AUTO, ats.ATS_SCHED_TICK):
        code, stats, x = _solve(ats, ctx, lv, st, sched=sched)
        assert code == 0, stats
        assert _rel(x, xr) <= PAR
        xs.append(x)
    np.testing.assert_array_equal(xs[0], xs[1])


def test_grid_barrier_waits_are_bounded(ats):
    """The barrier on its own: with every CTA arriving, every wait ends
    normally; waiting for one CTA more than the launch has (an arrival that
    never comes), every wait gives up by itself within its bounded number of
    polls and raises the give-up flag -- the path that ends a solve with
    ATS_ERR_TIMEOUT -- and the device stays usable."""
    ok = ats.ats_grid_barrier_selftest(0, 0, 0)
    assert ok["gave_up"] == 0 and ok["normal"] > 0
    bad = ats.ats_grid_barrier_selftest(0, 8, 1)
    assert bad["normal"] == 0 and bad["gave_up"] == 8
    assert 1.0 < bad["ms"] < 5000.0
    again = ats.ats_grid_barrier_selftest(0, 0, 0)
    assert again["gave_up"] == 0
