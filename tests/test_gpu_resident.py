"""GPU parity of the resident solver against the FP64 oracle.

The resident solver runs a whole level solve inside one launch: a thread-block
cluster (per-step sums through distributed shared memory, steps ordered by
the hardware cluster barrier) or, for a small level, one CTA.  The method is
the same as on the tick path -- the level matrix of Eq. Er_imp1 with the
interface rows of Sect. 3.2, Jacobi-PCG (Sect. 3.3.4) in FP64 or in FP32 with
FP64 refinement -- so the same parity bound holds: both sides stop on the
certified rule ||b - A x|| <= 5e-11 ||x||, lambda_min >= 1 bounds each
solution's error by its residual, and they differ by at most 1e-10 relative.

Covered: every interface kind and non-leaf cells, every resident shape (one
CTA; clusters of 1, 2, 4, 8 and 16 CTAs; 256 and 512 threads), levels with
many octs per thread, ragged batches (bitwise alone vs in the batch, and run
to run), the FP32-scalar variant, both forms of the CG step (q from p, or by
recurrence), results written by the resident kernels into device, pinned and
pageable host memory, degenerate and capped solves.
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


def _prec(ats, name):
    return ats.ATS_PREC_FP64 if name == "fp64" else ats.ATS_PREC_MIXED


# (res_cta_octs, res_cluster, res_threads): one CTA per level, or clusters
SHAPES = [(1 << 30, 1, 512), (-1, 1, 256), (-1, 2, 512), (-1, 4, 256), (-1, 8, 512), (-1, 16, 256),
          (-1, 16, 512)]


PRECS = ["fp64", "mixed-shared", "mixed-global"]


def _popts(ats, name):
    """precision and where the mixed path keeps its CG state"""
    if name == "fp64":
        return dict(precision=ats.ATS_PREC_FP64)
    return dict(precision=ats.ATS_PREC_MIXED, res_state=0 if name == "mixed-shared" else 1)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"cta{s[0] > 0}-c{s[1]}-t{s[2]}")
@pytest.mark.parametrize("seed", [11, 12])
def test_irregular_levels_every_shape(ats, ctx, prec, shape, seed):
    """Unions of oct boxes with refined cells and Dirichlet / Neumann / Robin
    interface faces of every relation, a coupling shift and a source."""
    lv, st = W.random_amr_level(seed, n_box=4, box_hi=10)
    rng = np.random.default_rng(seed)
    st.s = rng.uniform(0, 2, lv.n_cell)
    st.src = rng.uniform(0, 0.5, lv.n_cell)
    xr = _oracle_x(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, s=st.s, src=st.src, **_faces(st))
    cta, cl, th = shape
    x = st.E.copy()
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, sched=ats.ATS_SCHED_RESIDENT,
                          res_cta_octs=cta, res_cluster=cl, res_threads=th, **_popts(ats, prec))
    assert code == 0, stats
    assert stats["err_bound"] <= TOL
    assert _rel(x, xr) <= PAR
    nl = ~lv.leaf_cells()
    np.testing.assert_array_equal(x[nl], st.E[nl])
    L.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 37), (33, 1, 1), (3, 5, 7), (17, 9, 5)])
def test_ragged_shapes_one_cta_and_cluster(ats, ctx, prec, dims):
    """One oct, strips, and oct counts that leave CTAs of a cluster empty or
    split unevenly."""
    rng = np.random.default_rng(sum(dims))
    lv = W.box_level(*dims, 0.05, [(W.DIRICHLET, 1.0), None, (W.ROBIN, 0.3), (W.NEUMANN, 0.0), None,
                                   (W.DIRICHLET, 1.0)])
    N, nf = lv.n_cell, lv.n_face
    st = W.Step(dt=3.0 * 0.05 ** 2, K=np.exp(rng.standard_normal(N)), E=rng.uniform(0.5, 1.5, N),
                face_K=np.exp(rng.standard_normal(nf)), face_E=rng.uniform(0, 2, nf),
                face_F=rng.uniform(-0.1, 0.1, nf))
    xr = _oracle_x(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    for cta, cl in ((1 << 30, 8), (-1, 8), (-1, 16)):
        x = st.E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, sched=ats.ATS_SCHED_RESIDENT,
                              res_cta_octs=cta, res_cluster=cl, **_popts(ats, prec))
        assert code == 0, stats
        assert _rel(x, xr) <= PAR
    L.close()


@pytest.mark.parametrize("prec", PRECS)
def test_many_octs_per_thread(ats, ctx, prec):
    """A 32 x 32 x 24-oct level (24 576 octs): 6 to 12 octs per thread on one
    cluster, 48 to 96 on one CTA; with the state in shared memory, more octs
    per CTA than its capacity, so the octs beyond it (and the faces they
    share) run from the global arrays."""
    rng = np.random.default_rng(321)
    lv = W.box_level(32, 32, 24, 1.0 / 64, [(W.DIRICHLET, 1.0), (W.NEUMANN, 0.0), (W.ROBIN, 0.5),
                                            (W.DIRICHLET, 1.0), None, (W.ROBIN, 0.9)])
    N, nf = lv.n_cell, lv.n_face
    st = W.Step(dt=20.0 / 64 ** 2 / 2.0, K=np.exp(rng.standard_normal(N)), E=rng.uniform(0.5, 1.5, N),
                face_K=np.exp(rng.standard_normal(nf)), face_E=rng.uniform(0, 2, nf),
                face_F=rng.uniform(-0.05, 0.05, nf))
    xr = _oracle_x(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    for cta, cl, th in ((-1, 8, 512), (-1, 4, 256), (1 << 30, 1, 512)):
        x = st.E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, sched=ats.ATS_SCHED_RESIDENT,
                              res_cta_octs=cta, res_cluster=cl, res_threads=th, **_popts(ats, prec))
        assert code == 0, stats
        assert _rel(x, xr) <= PAR
    L.close()


def test_state_in_shared_or_global_memory_same_bits(ats, ctx):
    """Where a CTA keeps K, z and p (shared memory, or the global arrays) does
    not enter the arithmetic: both forms give bitwise the same result, in
    one-CTA and cluster solves, within and beyond the shared capacity."""
    rng = np.random.default_rng(4040)
    for o, cta, cl in ((300, 1 << 30, 1), (5000, -1, 8), (24000, -1, 4), (24000, 1 << 30, 1)):
        lv, st = W.random_box_solve(rng, o, robin=True)
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        res = []
        for rs in (0, 1):
            x = st.E.copy()
            code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                                  sched=ats.ATS_SCHED_RESIDENT, res_cta_octs=cta, res_cluster=cl, res_state=rs)
            assert code == 0, stats
            res.append((x, stats["iterations"]))
        np.testing.assert_array_equal(res[0][0], res[1][0])
        assert res[0][1] == res[1][1]
        L.close()


@pytest.mark.parametrize("form", [1, 2], ids=["q-from-p", "q-recurrence"])
def test_cg_forms_match_oracle(ats, ctx, form):
    """Both forms of the CG step (q = (I + dt A) p after a group barrier, or
    q = (I + dt A) z + beta q_prev without one) on one CTA, 4- and 16-CTA
    clusters, within and beyond the shared capacity (24 000 octs on one CTA),
    with every interface kind and non-leaf cells: each refines to the
    certificate and matches the oracle; where the CTA keeps its state does not
    change the bits; the two forms' iteration counts stay close."""
    rng = np.random.default_rng(6060 + form)
    for o, cta, cl in ((60, 1 << 30, 1), (3000, -1, 4), (24000, -1, 16), (24000, 1 << 30, 1)):
        lv, st = W.random_box_solve(rng, o, dt_lo=10.0, dt_hi=100.0, robin=True)
        xr = _oracle_x(lv, st)
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        res = {}
        for f, rs in ((form, 0), (form, 1), (3 - form, 0)):
            x = st.E.copy()
            code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                                  sched=ats.ATS_SCHED_RESIDENT, res_cta_octs=cta, res_cluster=cl, res_state=rs,
                                  cg_form=f)
            assert code == 0, stats
            assert _rel(x, xr) <= PAR
            res[(f, rs)] = (x, stats["iterations"])
        np.testing.assert_array_equal(res[(form, 0)][0], res[(form, 1)][0])
        a, b = res[(form, 0)][1], res[(3 - form, 0)][1]
        assert abs(a - b) <= max(4, 0.1 * b), (a, b)
        L.close()
    lv, st = W.random_amr_level(31, n_box=4, box_hi=8)
    xr = _oracle_x(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    x = st.E.copy()
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                          sched=ats.ATS_SCHED_RESIDENT, res_cta_octs=-1, res_cluster=4, cg_form=form)
    assert code == 0, stats
    assert _rel(x, xr) <= PAR
    nl = ~lv.leaf_cells()
    np.testing.assert_array_equal(x[nl], st.E[nl])
    L.close()


@pytest.mark.parametrize("integ", ["backward-euler", "crank-nicolson"])
def test_results_written_where_each_solve_ends(ats, ctx, integ):
    """Each FP32-bulk resident solve writes its own result when it ends: into
    device x, straight into pinned host x (while the other solves still run),
    or into the staging buffer for pageable host x; k_final writes the
    results of the other solves (here a level on the whole-GPU form).  All
    three memory kinds give bitwise the same x (Crank-Nicolson: 2 x' - E^n),
    the same statuses (Crank-Nicolson may warn of a negative value, which the
    resident kernels flag as k_final does), and the backward-Euler results
    match the oracle."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(909)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (40, 3000, 12000, 24000)]
    I = ats.ATS_INTEGRATOR_BACKWARD_EULER if integ == "backward-euler" else ats.ATS_INTEGRATOR_CRANK_NICOLSON
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, integrator=I, **_faces(st))
        levels.append(L)
    opts = dict(tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, use_graph=1,
                res_max_octs=20000)
    outs, codes = [], []

    def run(B, xs):
        code, stats = B.solve(xs)
        assert code >= 0, stats
        codes.append((code, [st["status"] for st in stats]))

    B = ats.Batch(ctx, levels, mem=ats.ATS_MEM_HOST, **opts)
    xs = [st.E.copy() for _, st in solves]
    run(B, xs)
    outs.append(xs)
    sizes = [lv.n_cell for lv, _ in solves]
    buf = torch.empty(sum(sizes), dtype=torch.float64).pin_memory().numpy()
    views, at = [], 0
    for (lv, st), n in zip(solves, sizes):
        views.append(buf[at:at + n])
        views[-1][:] = st.E
        at += n
    for _ in range(2):  # the second run reuses the plan's pointer tables
        run(B, views)
        outs.append([v.copy() for v in views])
        for v, (_, st) in zip(views, solves):
            v[:] = st.E
    B.close()
    B = ats.Batch(ctx, levels, mem=ats.ATS_MEM_DEVICE, **opts)
    dx = [torch.from_numpy(st.E.copy()).cuda() for _, st in solves]
    run(B, dx)
    torch.cuda.synchronize()
    outs.append([t.cpu().numpy() for t in dx])
    B.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            np.testing.assert_array_equal(a, b)
    assert all(c == codes[0] for c in codes)
    if integ == "backward-euler":
        assert codes[0][0] == 0
        for (lv, st), x in zip(solves, outs[0]):
            assert _rel(x, _oracle_x(lv, st)) <= PAR
    for L in levels:
        L.close()


@pytest.mark.parametrize("prec", PRECS)
def test_batch_alone_and_in_batch_bitwise(ats, ctx, prec):
    """A ragged batch spanning one-CTA and cluster solves: every solve matches
    the oracle; each result is bitwise the same alone and in the batch, and
    run to run (the queue order and which cluster takes a solve do not
    enter its arithmetic)."""
    rng = np.random.default_rng(2077)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (1, 9, 130, 700, 2100, 4500, 12000, 3, 60)]
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    opts = dict(tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, sched=ats.ATS_SCHED_RESIDENT, **_popts(ats, prec))
    B = ats.Batch(ctx, levels, **opts)
    assert B.kernel_stats()["res_solves"] == len(solves)
    xs = [st.E.copy() for _, st in solves]
    code, stats = B.solve(xs)
    assert code == 0, stats
    for (lv, st), x in zip(solves, xs):
        assert _rel(x, _oracle_x(lv, st)) <= PAR
    for k, L in enumerate(levels):
        x = solves[k][1].E.copy()
        code, _ = L.solve(x, **opts)
        assert code == 0
        np.testing.assert_array_equal(x, xs[k])
    for _ in range(2):
        xs2 = [st.E.copy() for _, st in solves]
        code, stats2 = B.solve(xs2)
        assert code == 0
        for a, b in zip(xs, xs2):
            np.testing.assert_array_equal(a, b)
        assert [s["iterations"] for s in stats] == [s["iterations"] for s in stats2]
    B.close()
    for L in levels:
        L.close()


def test_cg_scalars_in_fp32_or_fp64(ats, ctx):
    """Mixed precision with the CG step's alpha, beta and inner test from the
    dot totals rounded to FP32 (default) or in FP64: both refine to the
    certificate and match the oracle, and the iteration counts stay close."""
    rng = np.random.default_rng(515)
    for o in (40, 3000):
        lv, st = W.random_box_solve(rng, o, dt_lo=10.0, dt_hi=100.0, robin=True)
        xr = _oracle_x(lv, st)
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        its = []
        for cs in (0, 1):
            x = st.E.copy()
            code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                                  sched=ats.ATS_SCHED_RESIDENT, cg_scalars=cs)
            assert code == 0, stats
            assert _rel(x, xr) <= PAR
            its.append(stats["iterations"])
        assert abs(its[0] - its[1]) <= max(3, 0.05 * its[1])
        L.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_degenerate_and_capped(ats, ctx, prec):
    """A constant state between zero-flux walls converges with no iteration
    (x = E^n bitwise) beside a solve that iterates; an iteration cap ends a
    resident solve with NOT_CONVERGED after exactly that many iterations;
    with one refinement pass allowed the mixed path stops near the FP32
    floor and reports it."""
    rng = np.random.default_rng(7)
    P = _prec(ats, prec)
    lv = W.box_level(5, 3, 4, 0.05)
    E = np.full(lv.n_cell, 0.7)
    L = ats.Level(ctx, lv)
    L.build(10.0 * 0.05 ** 2, np.exp(rng.standard_normal(lv.n_cell)), E)
    lv2, st2 = W.random_box_solve(rng, 3000, robin=True)
    L2 = ats.Level(ctx, lv2)
    L2.build(st2.dt, st2.K, st2.E, **_faces(st2))
    B = ats.Batch(ctx, [L, L2], tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P,
                  sched=ats.ATS_SCHED_RESIDENT)
    xs = [E.copy(), st2.E.copy()]
    code, stats = B.solve(xs)
    assert code == 0, stats
    assert stats[0]["iterations"] == 0 and stats[0]["res_norm"] == 0.0
    np.testing.assert_array_equal(xs[0], E)
    assert _rel(xs[1], _oracle_x(lv2, st2)) <= PAR
    B.close()
    x = st2.E.copy()
    code, s = L2.solve(x, tol=1e-14, precision=P, sched=ats.ATS_SCHED_RESIDENT, max_iter=5)
    assert code == ats.ATS_ERR_NOT_CONVERGED and s["iterations"] == 5
    if prec == "mixed":
        x = st2.E.copy()
        code, s = L2.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P, sched=ats.ATS_SCHED_RESIDENT,
                           max_refine=1, inner_rtol=1e-6)
        assert code == ats.ATS_ERR_NOT_CONVERGED and s["refinements"] == 2
        assert 1e-10 < _rel(x, _oracle_x(lv2, st2)) < 1e-4
    L.close()
    L2.close()


def test_tick_and_resident_agree(ats, ctx):
    """The same levels on both paths: each within the parity bound of the
    oracle (their arithmetic differs, so not bitwise)."""
    rng = np.random.default_rng(99)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (20, 800, 5000)]
    for lv, st in solves:
        xr = _oracle_x(lv, st)
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        for sched in (ats.ATS_SCHED_TICK, ats.ATS_SCHED_RESIDENT):
            x = st.E.copy()
            code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                                  sched=sched)
            assert code == 0, stats
            assert _rel(x, xr) <= PAR
        L.close()


def test_autotune_resident_shapes(ats, ctx):
    """The autotuner times the resident shapes (threads per CTA x cluster
    size x one-CTA limit) on a resident batch, keeps the fastest, and leaves
    a solution: each solve matches the oracle, and later solves are bitwise
    those of a batch created with the chosen options."""
    rng = np.random.default_rng(919)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (3, 90, 1500, 3000, 9000)]
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    opts = dict(tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, sched=ats.ATS_SCHED_RESIDENT)
    B = ats.Batch(ctx, levels, **opts)
    xs = [st.E.copy() for _, st in solves]
    r = B.autotune(xs, reps=1)
    assert r["candidates"] == 8  # the batch's own shape and the seven others
    assert r["res_threads"] in (256, 512) and r["res_cluster"] in (2, 4, 8, 16)
    assert r["res_cta_octs"] in (0, 1024, 2048) and r["chosen"]["res_cluster_big"] in (0, 8, 16, -1)
    assert 0.0 < r["ms"] <= r["ms_default"]
    for (lv, st), x in zip(solves, xs):
        assert _rel(x, _oracle_x(lv, st)) <= PAR
    xs2 = [st.E.copy() for _, st in solves]
    assert B.solve(xs2)[0] == 0
    B.close()
    B3 = ats.Batch(ctx, levels, res_threads=r["chosen"]["res_threads"], res_cluster=r["chosen"]["res_cluster"],
                   res_cta_octs=r["chosen"]["res_cta_octs"], res_cluster_big=r["chosen"]["res_cluster_big"], **opts)
    xs3 = [st.E.copy() for _, st in solves]
    assert B3.solve(xs3)[0] == 0
    for a, b in zip(xs2, xs3):
        np.testing.assert_array_equal(a, b)
    B3.close()
    for L in levels:
        L.close()


def test_two_cluster_sizes_in_one_batch(ats, ctx):
    """Levels of large estimated work (size x stiffness) on 16-CTA clusters,
    the others on 8-CTA clusters or single CTAs, as three concurrent
    launches: every solve matches the oracle and is bitwise the same alone
    (where it runs by itself on its shape) and in the batch."""
    rng = np.random.default_rng(5150)
    solves = [W.random_box_solve(rng, o, robin=True, dt_lo=lo, dt_hi=lo) for o, lo in
              ((5, 1.0), (600, 30.0), (2600, 1.0), (3100, 1.0), (5000, 80.0), (7000, 100.0), (40, 5.0), (2200, 2.0))]
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    opts = dict(tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, sched=ats.ATS_SCHED_RESIDENT,
                res_cta_octs=512, res_big_work=40000, res_cluster=8, res_cluster_big=16)
    B = ats.Batch(ctx, levels, **opts)
    xs = [st.E.copy() for _, st in solves]
    B.set_profiling(True)
    code, stats = B.solve(xs)
    assert code == 0, stats
    g = B.kernel_stats()["res_grids"]
    assert g[0] > 0 and g[1] > 0  # both cluster sizes ran
    for (lv, st), x in zip(solves, xs):
        assert _rel(x, _oracle_x(lv, st)) <= PAR
    for k, L in enumerate(levels):
        x = solves[k][1].E.copy()
        assert L.solve(x, **opts)[0] == 0
        np.testing.assert_array_equal(x, xs[k])
    B.close()
    for L in levels:
        L.close()
