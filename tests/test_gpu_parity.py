"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (stated per test):
  * operator / right-hand side: same FP64 arithmetic up to summation order,
    relative 1e-13 per element (the coefficients are O(1e3) sums of O(1) terms);
  * solves: both sides stop on the certified rule ||b - A x|| <= tol ||x||
    with tol = 5e-11; the level matrix has lambda_min >= 1, so each solution is
    within 5e-11 (relative) of the exact one and the two differ by <= 1e-10
    relative L2 -- the parity bound, for the FP64 and the refined mixed
    path alike.
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


def _oracle_solution(lv, st, tol=TOL):
    S = oracle.assemble(lv, st.dt, st.K, st.E, s=st.s, src=st.src, **_faces(st))
    x, info = oracle.pcg(S, st.E, tol=tol, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0
    return S, x


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_operator_and_rhs_match_oracle(ats, ctx, seed):
    lv, st = W.random_amr_level(seed)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    S = oracle.assemble(lv, st.dt, st.K, st.E, **_faces(st))
    b = L.rhs()
    np.testing.assert_allclose(b, S.b, rtol=1e-13, atol=1e-13 * np.abs(S.b).max())
    x = np.random.default_rng(seed).uniform(0.5, 1.5, lv.n_cell)
    y = L.apply(x)
    yr = S.matvec(x)
    leaf = lv.leaf_cells()
    scale = np.abs(S.val).max() * np.abs(x).max()
    np.testing.assert_allclose(y[leaf], yr[leaf], rtol=0, atol=1e-13 * scale)
    L.close()


@pytest.mark.parametrize("sched", ["auto", "tick"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_random_amr_levels_all_face_types(ats, ctx, prec, seed, sched):
    lv, st = W.random_amr_level(seed)
    _, xr = _oracle_solution(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    x = st.E.copy()
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED,
                          precision=ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED,
                          sched=ats.ATS_SCHED_TICK if sched == "tick" else ats.ATS_SCHED_AUTO)
    assert code == 0, stats
    assert stats["err_bound"] <= TOL
    assert _rel(x, xr) <= PAR
    nl = ~lv.leaf_cells()
    np.testing.assert_array_equal(x[nl], st.E[nl])  # non-leaf cells untouched
    L.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gaussian_32cube(ats, ctx, prec):
    """32^3 unit box, K = 1, dt = 10 dx^2 / 2K, Gaussian + floor, zero-flux walls."""
    lv, st = W.gaussian_32cube()
    _, xr = _oracle_solution(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E)
    x = st.E.copy()
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED,
                          precision=ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED)
    assert code == 0, stats
    assert _rel(x, xr) <= PAR
    # zero-flux walls conserve the total exactly (up to the solve tolerance)
    assert abs(x.sum() - st.E.sum()) <= 1e-10 * st.E.sum()
    L.close()


def test_gaussian_32cube_paper_stopping_rule(ats, ctx):
    """The paper's rule (L2 relative to r0 and L-inf relative change) at 1e-10."""
    lv, st = W.gaussian_32cube()
    S, xr = _oracle_solution(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E)
    x = st.E.copy()
    code, stats = L.solve(x, tol=1e-10, stop_rule=ats.ATS_STOP_PAPER, precision=ats.ATS_PREC_FP64)
    assert code == 0, stats
    assert stats["res_norm"] <= 1e-10 * stats["r0_norm"] * 1.0001
    # the L2 rule alone bounds the error by ||r|| <= 1e-10 ||r0||
    assert np.linalg.norm(x - xr) <= 1e-10 * stats["r0_norm"] + 5e-11 * np.linalg.norm(xr)
    L.close()


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 37), (33, 1, 1), (3, 5, 7), (8, 8, 9)])
def test_ragged_shapes_and_tails(ats, ctx, dims):
    """1 oct, strips, oct counts that are not multiples of the 32-oct pass or
    of the work-item tile."""
    rng = np.random.default_rng(sum(dims))
    lv, st = W.random_box_solve(rng, 1)
    lv = W.box_level(*dims, 0.05, [(W.DIRICHLET, 1.0), None, (W.ROBIN, 0.3), (W.NEUMANN, 0.0), None, (W.DIRICHLET, 1.0)])
    N, nf = lv.n_cell, lv.n_face
    st = W.Step(dt=3.0 * 0.05 ** 2, K=np.exp(rng.standard_normal(N)), E=rng.uniform(0.5, 1.5, N),
                face_K=np.exp(rng.standard_normal(nf)), face_E=rng.uniform(0, 2, nf), face_F=rng.uniform(-0.1, 0.1, nf))
    _, xr = _oracle_solution(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    for prec, tile, sched in ((ats.ATS_PREC_FP64, 0, ats.ATS_SCHED_AUTO), (ats.ATS_PREC_FP64, 0, ats.ATS_SCHED_TICK),
                              (ats.ATS_PREC_MIXED, 32, ats.ATS_SCHED_TICK), (ats.ATS_PREC_MIXED, 64, ats.ATS_SCHED_TICK)):
        x = st.E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=prec, tile_octs=tile,
                              sched=sched)
        assert code == 0, stats
        assert _rel(x, xr) <= PAR
    L.close()


def test_coupling_shift_and_source(ats, ctx):
    """Diagonal shift s and extra source (the linearised coupling terms)."""
    lv, st = W.random_amr_level(61)
    rng = np.random.default_rng(61)
    st.s = rng.uniform(0, 3, lv.n_cell)
    st.src = rng.uniform(0, 1, lv.n_cell)
    _, xr = _oracle_solution(lv, st)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, s=st.s, src=st.src, **_faces(st))
    for prec in (ats.ATS_PREC_FP64, ats.ATS_PREC_MIXED):
        x = st.E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=prec)
        assert code == 0, stats
        assert _rel(x, xr) <= PAR
    L.close()


def test_device_pointers_and_rhs_override(ats, ctx):
    import torch

    lv, st = W.random_amr_level(71)
    S, xr = _oracle_solution(lv, st)
    L = ats.Level(ctx, lv)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    L.build(st.dt, t(st.K), t(st.E), face_K=t(st.face_K), face_E=t(st.face_E), face_F=t(st.face_F))
    torch.cuda.synchronize()
    x = t(st.E.copy())
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED)
    assert code == 0
    assert _rel(x.cpu().numpy(), xr) <= PAR
    # explicit right-hand side: 2 b gives 2 x on the leaf cells (the others
    # keep their input value)
    xb = t(st.E.copy())
    code, _ = L.solve(xb, rhs=t(2 * S.b), tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED)
    assert code == 0
    leaf = lv.leaf_cells()
    assert _rel(xb.cpu().numpy()[leaf], 2 * xr[leaf]) <= PAR
    np.testing.assert_array_equal(xb.cpu().numpy()[~leaf], st.E[~leaf])
    L.close()


@pytest.mark.parametrize("sched", ["auto", "tick"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_oracle_and_is_invariant(ats, ctx, prec, sched):
    """A ragged batch: every solve matches the oracle, and each result is
    bitwise the same alone and inside the batch (same work-item tiling,
    fixed-order reductions)."""
    rng = np.random.default_rng(77)
    solves = [W.random_box_solve(rng, o) for o in (1, 7, 64, 100, 333, 900, 2)]
    P = ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    xs = [st.E.copy() for _, st in solves]
    SC = ats.ATS_SCHED_TICK if sched == "tick" else ats.ATS_SCHED_AUTO
    B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P, use_graph=1, check_every=8,
                  sched=SC)
    code, stats = B.solve(xs)
    assert code == 0, stats
    for (lv, st), x, s in zip(solves, xs, stats):
        _, xr = _oracle_solution(lv, st)
        assert _rel(x, xr) <= PAR, s
    for k, ((lv, st), L) in enumerate(zip(solves, levels)):
        x = st.E.copy()
        code, _ = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P, sched=SC)
        assert code == 0
        np.testing.assert_array_equal(x, xs[k])
    # run the batch a second time: identical results (deterministic)
    xs2 = [st.E.copy() for _, st in solves]
    B.solve(xs2)
    for a, b in zip(xs, xs2):
        np.testing.assert_array_equal(a, b)
    B.close()
    for L in levels:
        L.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_state_already_converged(ats, ctx, prec):
    """Degenerate case: a constant state between zero-flux walls is its own
    backward-Euler step (every face flux C (x_i - x_j) is exactly zero), so
    the first FP64 residual is zero and every stopping rule ends the solve
    there: no CG iteration, x = E^n bitwise.  Beside a solve that does
    iterate, in one batch, neither result changes."""
    rng = np.random.default_rng(91)
    P = ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED
    lv = W.box_level(5, 3, 4, 0.05)
    K = np.exp(rng.standard_normal(lv.n_cell))
    E = np.full(lv.n_cell, 0.7)
    L = ats.Level(ctx, lv)
    L.build(10.0 * 0.05 ** 2, K, E)
    for rule in (ats.ATS_STOP_CERTIFIED, ats.ATS_STOP_RESIDUAL, ats.ATS_STOP_PAPER):
        x = E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=rule, precision=P)
        assert code == 0, stats
        assert stats["iterations"] == 0 and stats["res_norm"] == 0.0
        np.testing.assert_array_equal(x, E)
    lv2, st2 = W.random_box_solve(rng, 50)
    L2 = ats.Level(ctx, lv2)
    L2.build(st2.dt, st2.K, st2.E, **_faces(st2))
    _, xr2 = _oracle_solution(lv2, st2)
    B = ats.Batch(ctx, [L, L2], tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P, use_graph=1, check_every=8)
    xs = [E.copy(), st2.E.copy()]
    code, stats = B.solve(xs)
    assert code == 0, stats
    assert stats[0]["iterations"] == 0 and stats[1]["iterations"] > 0
    np.testing.assert_array_equal(xs[0], E)
    assert _rel(xs[1], xr2) <= PAR
    B.close()
    L2.close()
    L.close()


def test_bad_input_and_caps(ats, ctx):
    lv, st = W.random_amr_level(81)
    L = ats.Level(ctx, lv)
    K = st.K.copy()
    K[np.nonzero(lv.leaf_cells())[0][0]] = -1.0
    L.build(st.dt, K, st.E, **_faces(st))
    x = st.E.copy()
    code, _ = L.solve(x)
    assert code == ats.ATS_ERR_BAD_INPUT
    L.build(st.dt, st.K, st.E, **_faces(st))
    x = st.E.copy()
    code, stats = L.solve(x, tol=1e-14, max_iter=3)
    assert code == ats.ATS_ERR_NOT_CONVERGED
    assert stats["iterations"] == 3
    L.close()


def test_memory_budget(ats):
    c = ats.Context(0, mem_budget_bytes=64 * 1024)
    lv, st = W.gaussian_32cube()
    with pytest.raises(ats.AtsError) as e:
        ats.Level(c, lv)
    assert e.value.code == ats.ATS_ERR_OVER_BUDGET
    c.close()


def test_batched_operator_build_matches_per_level(ats, ctx):
    """One-launch operator build of a batch gives bitwise the per-level
    right-hand sides and the same solves."""
    import torch

    rng = np.random.default_rng(91)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (1, 5, 40, 300)]
    solves.append(W.random_amr_level(92))
    levels = [ats.Level(ctx, lv) for lv, _ in solves]
    for L, (lv, st) in zip(levels, solves):
        L.build(st.dt, st.K, st.E, **_faces(st))
    ref_b = [L.rhs() for L in levels]
    B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                  mem=ats.ATS_MEM_DEVICE, use_graph=1)
    dev = torch.device("cuda:0")
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    # zero the operators, then rebuild them all in one launch from device arrays
    for L, (lv, st) in zip(levels, solves):
        L.build(st.dt, np.ones(lv.n_cell), np.zeros(lv.n_cell))
    keep = [dict(dt=st.dt, K=t(st.K), E_old=t(st.E), face_K=t(st.face_K), face_E=t(st.face_E), face_F=t(st.face_F))
            for _, st in solves]
    prepared = B.prepare_coefs(keep)
    B.build_operators(prepared)
    torch.cuda.synchronize()
    for L, b in zip(levels, ref_b):
        np.testing.assert_array_equal(L.rhs(), b)
    xs = [t(st.E.copy()) for _, st in solves]
    code, stats = B.solve(xs)
    assert code == 0, stats
    for (lv, st), x in zip(solves, xs):
        _, xr = _oracle_solution(lv, st)
        assert _rel(x.cpu().numpy(), xr) <= PAR
    B.close()
    for L in levels:
        L.close()


def test_batched_host_inputs_from_one_buffer(ats, ctx):
    """Host inputs given as views of one contiguous buffer per array kind, and
    x as views of one buffer, are staged with one copy per contiguous run;
    the batch results equal the per-level builds and solves bitwise."""
    rng = np.random.default_rng(93)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (3, 50, 200, 8)]
    n = len(solves)
    off = np.concatenate([[0], np.cumsum([lv.n_cell for lv, _ in solves])])
    foff = np.concatenate([[0], np.cumsum([lv.n_face for lv, _ in solves])])
    def cat(key):
        parts = [getattr(st, key) for _, st in solves]
        return None if any(p is None for p in parts) else np.concatenate(parts)

    Kb, Eb = cat("K"), cat("E")
    fKb, fEb, fFb = cat("face_K"), cat("face_E"), cat("face_F")

    def fview(a, k):
        return a[foff[k]:foff[k + 1]] if a is not None and foff[k + 1] > foff[k] else None

    levels = [ats.Level(ctx, lv) for lv, _ in solves]
    for L, (lv, st) in zip(levels, solves):  # plan needs built operators
        L.build(st.dt, st.K, st.E, **_faces(st))
    B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                  mem=ats.ATS_MEM_HOST, use_graph=1)
    coefs = B.prepare_coefs([dict(dt=solves[k][1].dt, K=Kb[off[k]:off[k + 1]], E_old=Eb[off[k]:off[k + 1]],
                                  face_K=fview(fKb, k), face_E=fview(fEb, k), face_F=fview(fFb, k))
                             for k in range(n)])
    B.build_operators(coefs)
    xb = Eb.copy()
    code, stats = B.solve([xb[off[k]:off[k + 1]] for k in range(n)])
    assert code == 0, stats
    for k, ((lv, st), L) in enumerate(zip(solves, levels)):
        L.build(st.dt, st.K, st.E, **_faces(st))
        x = st.E.copy()
        code, _ = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
        assert code == 0
        np.testing.assert_array_equal(x, xb[off[k]:off[k + 1]])
        _, xr = _oracle_solution(lv, st)
        assert _rel(x, xr) <= PAR
    B.close()
    for L in levels:
        L.close()


@pytest.mark.parametrize("mem", ["host", "device"])
def test_initial_guess_from_build(ats, ctx, mem):
    """x0 = E^n of the last operator build (ATS_X0_E_OLD) gives bitwise the
    result of passing x = E^n as the initial guess."""
    import torch

    rng = np.random.default_rng(95)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (4, 70, 9)]
    levels = [ats.Level(ctx, lv) for lv, _ in solves]
    dev = torch.device("cuda:0")
    conv = (lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)) if mem == "device" \
        else (lambda a: a)
    M = ats.ATS_MEM_DEVICE if mem == "device" else ats.ATS_MEM_HOST
    coefs = [dict(dt=st.dt, K=conv(st.K), E_old=conv(st.E), face_K=conv(st.face_K), face_E=conv(st.face_E),
                  face_F=conv(st.face_F)) for _, st in solves]
    for L, c in zip(levels, coefs):
        L.build(**c)
    torch.cuda.synchronize()
    outs = []
    for x0 in (ats.ATS_X0_GIVEN, ats.ATS_X0_E_OLD):
        B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                      mem=M, use_graph=1, x0=x0)
        prepared = B.prepare_coefs(coefs)
        B.build_operators(prepared)
        xs = [conv(st.E.copy()) if x0 == ats.ATS_X0_GIVEN else conv(np.full(lv.n_cell, np.nan)) for lv, st in solves]
        code, stats = B.solve(xs)
        assert code == 0, stats
        outs.append([x.cpu().numpy() if mem == "device" else x for x in xs])
        B.close()
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    for L in levels:
        L.close()


@pytest.mark.parametrize("mem", ["host", "device"])
def test_autotune_keeps_a_valid_fastest_plan(ats, ctx, mem):
    """The autotuner times every (tile, poll interval) candidate on the batch's
    own solves, keeps the fastest plan, and leaves a solution in x: each solve
    matches the oracle, and later solves of the batch are bitwise those of a
    batch created with the chosen options."""
    import torch

    rng = np.random.default_rng(83)
    solves = [W.random_box_solve(rng, o) for o in (1, 7, 64, 100, 333, 900, 2)]
    dev = torch.device("cuda:0")
    conv = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)) if mem == "device" else (lambda a: a)
    back = (lambda t: t.cpu().numpy()) if mem == "device" else (lambda a: a)
    M = ats.ATS_MEM_DEVICE if mem == "device" else ats.ATS_MEM_HOST
    x0 = ats.ATS_X0_E_OLD if mem == "device" else ats.ATS_X0_GIVEN
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    opts = dict(tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, use_graph=1, mem=M, x0=x0,
                sched=ats.ATS_SCHED_TICK)
    B = ats.Batch(ctx, levels, check_every=16, **opts)
    xs = [conv(st.E.copy()) for _, st in solves]
    r = B.autotune(xs, tiles=(0, 64, 256), checks=(4, 16), reps=1)
    assert r["candidates"] == 6  # the batch's own options (0, 16) are timed once
    assert r["tile_octs"] in (0, 64, 256) and r["check_every"] in (4, 16)
    assert 0.0 < r["ms"] <= r["ms_default"]
    for (lv, st), x in zip(solves, xs):
        _, xr = _oracle_solution(lv, st)
        assert _rel(back(x), xr) <= PAR
    xs2 = [conv(st.E.copy()) for _, st in solves]
    code, _ = B.solve(xs2)
    assert code == 0
    B.close()
    B3 = ats.Batch(ctx, levels, check_every=r["check_every"], tile_octs=r["tile_octs"], **opts)
    xs3 = [conv(st.E.copy()) for _, st in solves]
    code, _ = B3.solve(xs3)
    assert code == 0
    for a, b in zip(xs2, xs3):
        np.testing.assert_array_equal(back(a), back(b))
    B3.close()
    with pytest.raises(ats.AtsError) as e:
        B3 = ats.Batch(ctx, levels, **opts)
        try:
            B3.autotune([conv(st.E.copy()) for _, st in solves], tiles=(-32,), reps=1)
        finally:
            B3.close()
    assert e.value.code == ats.ATS_ERR_INVALID_ARG
    for L in levels:
        L.close()


def test_unrefined_fp32_error_and_refinement(ats, ctx):
    """The mixed path without FP64 refinement (one FP32 inner solve from the
    FP64 residual of x0, max_refine = 1) stops near the FP32 floor: its error
    against the oracle lies between 1e-10 and 1e-4 and the final true-residual
    pass reports it (status NOT_CONVERGED); with refinement the same solves
    reach the 1e-10 bound."""
    rng = np.random.default_rng(91)
    for o in (8, 120, 700):
        # large steps (10..100 explicit steps): the correction x - E^n is a
        # sizeable part of x, so the FP32 floor shows in the result
        lv, st = W.random_box_solve(rng, o, dt_lo=10.0, dt_hi=100.0, robin=True)
        _, xr = _oracle_solution(lv, st)
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        x = st.E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                              max_refine=1, inner_rtol=1e-6)
        assert code == ats.ATS_ERR_NOT_CONVERGED, stats
        assert stats["refinements"] == 2
        e_un = _rel(x, xr)
        assert 1e-10 < e_un < 1e-4, e_un
        assert stats["err_bound"] > TOL
        x = st.E.copy()
        code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
        assert code == 0, stats
        assert _rel(x, xr) <= PAR
        L.close()


def test_full_size_batch_sampled_parity(ats, ctx):
    """The benchmark's workload at full size and in its launch configuration
    (512 solves, 21 M cells, device arrays, mixed precision, graph-replayed
    ticks of 16, certified 5e-11): every solve ends OK with its FP64
    certificate <= 5e-11, and sampled solves (the smallest, the largest and
    six drawn at random) match the oracle to 1e-10."""
    import torch

    solves = W.ragged_batch(n_solves=512, seed=1404)
    dev = torch.device("cuda:0")
    sizes = [lv.n_cell for lv, _ in solves]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    K_d = torch.from_numpy(np.concatenate([st.K for _, st in solves])).to(dev)
    E_d = torch.from_numpy(np.concatenate([st.E for _, st in solves])).to(dev)
    x_d = E_d.clone()
    levels, coefs = [], []
    for k, (lv, st) in enumerate(solves):
        L = ats.Level(ctx, lv)
        c = dict(dt=st.dt, K=K_d[offs[k]:offs[k + 1]], E_old=E_d[offs[k]:offs[k + 1]],
                 face_E=None if st.face_E is None else torch.from_numpy(st.face_E).to(dev),
                 face_F=None if st.face_F is None else torch.from_numpy(st.face_F).to(dev))
        L.build(**c)
        levels.append(L)
        coefs.append(c)
    torch.cuda.synchronize()
    B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                  use_graph=1, check_every=16, mem=ats.ATS_MEM_DEVICE)
    B.build_operators(B.prepare_coefs(coefs))
    xs = [x_d[offs[k]:offs[k + 1]] for k in range(len(solves))]
    code, stats = B.solve(xs)
    assert code == 0
    assert all(s["status"] == 0 and s["err_bound"] <= TOL for s in stats)
    x = x_d.cpu().numpy()
    rng = np.random.default_rng(5)
    sample = {int(np.argmin(sizes)), int(np.argmax(sizes))} | set(int(i) for i in rng.choice(len(solves), 6, False))
    for k in sorted(sample):
        lv, st = solves[k]
        _, xr = _oracle_solution(lv, st)
        assert _rel(x[offs[k]:offs[k + 1]], xr) <= PAR, k
    B.close()
    for L in levels:
        L.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_loop_matches_host_polled(ats, ctx, prec):
    """The tick path: a ragged batch and a solo solve with the whole tick loop in one graph
    (use_graph = 2, a WHILE conditional node) give bitwise the results and
    statistics of host-polled graphs (use_graph = 1); an iteration cap still
    ends the loop with NOT_CONVERGED."""
    rng = np.random.default_rng(61)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (2, 40, 300, 1100, 9)]
    P = ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)
    res = {}
    for g in (1, 2):
        B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=P, use_graph=g, check_every=4,
                      sched=ats.ATS_SCHED_TICK)
        xs = [st.E.copy() for _, st in solves]
        code, stats = B.solve(xs)
        assert code == 0, stats
        xs2 = [st.E.copy() for _, st in solves]
        code, stats2 = B.solve(xs2)  # the graph is reused
        assert code == 0
        for a, b in zip(xs, xs2):
            np.testing.assert_array_equal(a, b)
        res[g] = (xs, [(s["iterations"], s["refinements"], s["ticks"]) for s in stats])
        B.close()
    for a, b in zip(res[1][0], res[2][0]):
        np.testing.assert_array_equal(a, b)
    assert res[1][1] == res[2][1]
    for (lv, st), x in zip(solves, res[2][0]):
        _, xr = _oracle_solution(lv, st)
        assert _rel(x, xr) <= PAR
    lv, st = solves[3]
    x = st.E.copy()
    code, s = levels[3].solve(x, tol=1e-14, precision=P, use_graph=2, check_every=4, max_iter=5,
                              sched=ats.ATS_SCHED_TICK)
    assert code == ats.ATS_ERR_NOT_CONVERGED
    assert s["iterations"] == 5
    for L in levels:
        L.close()


def test_negative_energy_warning(ats, ctx):
    """A result with a negative value (here from a strong sink) is still the
    solution (matches the oracle) and carries the warning ATS_WARN_NEGATIVE,
    alone and in a batch beside solves without it (the batch returns the
    warning, each solve its own status)."""
    rng = np.random.default_rng(17)
    solves = [W.random_box_solve(rng, o) for o in (30, 200)]
    (lv, st), (lv2, st2) = solves
    src = np.full(lv.n_cell, -50.0)
    S = oracle.assemble(lv, st.dt, st.K, st.E, src=src, **_faces(st))
    xr, info = oracle.pcg(S, st.E, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0 and np.min(xr) < 0.0
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, src=src, **_faces(st))
    x = st.E.copy()
    code, stats = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
    assert code == ats.ATS_WARN_NEGATIVE and stats["status"] == ats.ATS_WARN_NEGATIVE
    assert _rel(x, xr) <= PAR
    L2 = ats.Level(ctx, lv2)
    L2.build(st2.dt, st2.K, st2.E, **_faces(st2))
    B = ats.Batch(ctx, [L2, L], tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, use_graph=1)
    xs = [st2.E.copy(), st.E.copy()]
    code, bstats = B.solve(xs)
    assert code == ats.ATS_WARN_NEGATIVE
    assert [s["status"] for s in bstats] == [0, ats.ATS_WARN_NEGATIVE]
    np.testing.assert_array_equal(xs[1], x)
    B.close()
    L.close()
    L2.close()


def test_prefetched_inputs_give_the_same_results(ats, ctx):
    """Host inputs copied ahead on the batch's copy stream (while a solve
    runs) give bitwise the results of plain builds; a prefetch of other
    arrays than the next build's is dropped."""
    rng = np.random.default_rng(29)
    solves = [W.random_box_solve(rng, o, robin=True) for o in (5, 80, 300)]
    levels = []
    for lv, st in solves:
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, **_faces(st))
        levels.append(L)

    def coefs(scale):
        return [dict(dt=st.dt, K=st.K.copy(), E_old=st.E * scale, face_K=st.face_K, face_E=st.face_E,
                     face_F=st.face_F) for _, st in solves]

    B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                  mem=ats.ATS_MEM_HOST, x0=ats.ATS_X0_E_OLD, use_graph=2)
    A, Bc = B.prepare_coefs(coefs(1.0)), B.prepare_coefs(coefs(1.1))

    def solve():
        xs = [np.empty(lv.n_cell) for lv, _ in solves]
        code, _ = B.solve(xs)
        assert code == 0
        return xs

    B.build_operators(A)
    xa = solve()
    B.build_operators(Bc)
    xb = solve()
    B.build_operators(A)
    B.prefetch_operators(Bc)   # copies overlap the next solve
    xa2 = solve()
    B.build_operators(Bc)      # from the prefetched copies
    xb2 = solve()
    B.prefetch_operators(Bc)
    B.build_operators(A)       # other arrays: the prefetch is dropped
    xa3 = solve()
    for u, v in zip(xa, xa2):
        np.testing.assert_array_equal(u, v)
    for u, v in zip(xb, xb2):
        np.testing.assert_array_equal(u, v)
    for u, v in zip(xa, xa3):
        np.testing.assert_array_equal(u, v)
    for (lv, st), x in zip(solves, xb):
        S = oracle.assemble(lv, st.dt, st.K, st.E * 1.1, **_faces(st))
        xr, info = oracle.pcg(S, st.E * 1.1, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
        assert _rel(x, xr) <= PAR
    B.close()
    for L in levels:
        L.close()
