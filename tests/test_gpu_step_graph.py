"""The whole coarse step as one graph (ats_level_advance, use_graph = 3).

Sect. 2.2's recursion (a level's step is two substeps of the next finer
level and its own solve) with Sect. 3.3's interface handling runs, per
coarse step, restriction, ghost gathers, operator builds, 2^L - 1 level
solves and flux stores.  With use_graph = 3 the first call takes the step
with deferred solves (use_graph = 2) and captures it; later calls replay the
captured graph: one launch and one host wait per step.

Every kernel of a replay is the kernel the deferred path launches, with the
same arguments, so the states and the per-step statistics must be bitwise
those of use_graph = 2 -- on small random hierarchies (resident and tick-path
level solves, both orders), on the two-level 64^3 workload with every
coarse-to-fine row, and on the 4-level radiation-matter workload (base
128^3).  The graph must be replaced when the step's arguments or the
hierarchy's configuration change, and a failure inside a replayed step must
be reported.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fld

pytestmark = pytest.mark.gpu
TOL = 5e-11


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


def _steps(ats, ctx, levels, states, order, dts, use_graph, between=None, **kw):
    """Take one step per entry of dts from level 0; returns the per-step
    (code, iterations, refinements, ticks), the final states and the
    hierarchy's graph statistics."""
    H = ats.Hierarchy(ctx, levels, order)
    try:
        for l, (E, K) in enumerate(states):
            H.set_state(l, E, K)
        rows = []
        for k, dt in enumerate(dts):
            if between is not None:
                between(H, k)
            code, st = H.advance(0, dt, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                                 use_graph=use_graph, **kw)
            rows.append((code, st["iterations"], st["refinements"], st["ticks"], st["status"]))
        return rows, [H.state(l).copy() for l in range(len(levels))], H.graph_stats()
    finally:
        H.close()


def _assert_same(a, b):
    rows_a, states_a, _ = a
    rows_b, states_b, _ = b
    assert rows_a == rows_b
    for x, y in zip(states_a, states_b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("order", ["fine_first", "coarse_first"])
@pytest.mark.parametrize("sched", ["auto", "tick"])
def test_step_graph_is_bitwise_the_deferred_step(ats, ctx, order, sched):
    """Three-level random hierarchies: four coarse steps, the first captured,
    three replayed; with the automatic scheduler the small levels run on the
    resident solver, with the tick scheduler every solve runs the device
    loop (a WHILE node inside the step graph)."""
    levels, states, dt = W.random_hierarchy(6, n0=8, n_levels=3)
    o = ats.ATS_ORDER_FINE_FIRST if order == "fine_first" else ats.ATS_ORDER_COARSE_FIRST
    s = ats.ATS_SCHED_AUTO if sched == "auto" else ats.ATS_SCHED_TICK
    for check in (16, 3):
        ref = _steps(ats, ctx, levels, states, o, [dt] * 4, 2, sched=s, check_every=check)
        got = _steps(ats, ctx, levels, states, o, [dt] * 4, 3, sched=s, check_every=check)
        assert all(r[0] == 0 for r in ref[0]), ref[0]
        _assert_same(ref, got)
        assert got[2] == {"held": True, "captures": 1, "replays": 3}


def test_step_graph_follows_changes(ats, ctx):
    """A new dt, a new set of options or a new interface row replaces the
    graph (the step is taken deferred and captured again); new state values
    keep it (the graph reads E and K in place)."""
    levels, states, dt = W.random_hierarchy(7, n0=8, n_levels=3)
    rng = np.random.default_rng(7)
    E2 = [E * rng.uniform(0.9, 1.1, E.shape) for E, _ in states]

    def between(H, k):
        if k == 2:  # new values in place: the graph stays
            for l, (E, K) in enumerate(states):
                H.set_state(l, E2[l], K)
        if k == 5:  # another interface row: a configuration change
            H.set_interface(ats.ATS_FACE_ROBIN, 0.5)

    dts = [dt, dt, dt, 0.5 * dt, 0.5 * dt, 0.5 * dt, 0.5 * dt]
    ref = _steps(ats, ctx, levels, states, ats.ATS_ORDER_FINE_FIRST, dts, 2, between=between)
    got = _steps(ats, ctx, levels, states, ats.ATS_ORDER_FINE_FIRST, dts, 3, between=between)
    _assert_same(ref, got)
    # captures at steps 0 (first), 3 (new dt), 5 (new interface row)
    assert got[2] == {"held": True, "captures": 3, "replays": 4}


def test_step_graph_reports_a_failing_replay(ats, ctx):
    """A non-finite value put into a level between steps makes that level's
    operator build flag bad input inside the replayed graph: the call
    returns ATS_ERR_BAD_INPUT as the deferred path does.  A step whose
    solves fail is not captured."""
    levels, states, dt = W.random_hierarchy(8, n0=8, n_levels=3)

    def poison(H, k):
        if k == 2:
            E = states[1][0].copy()
            E[5] = np.nan
            H.set_state(1, E, states[1][1])

    ref = _steps(ats, ctx, levels, states, ats.ATS_ORDER_FINE_FIRST, [dt] * 3, 2, between=poison)
    got = _steps(ats, ctx, levels, states, ats.ATS_ORDER_FINE_FIRST, [dt] * 3, 3, between=poison)
    assert ref[0][2][0] == ats.ATS_ERR_BAD_INPUT
    assert [r[0] for r in got[0]] == [r[0] for r in ref[0]]
    assert got[2]["replays"] == 2
    # a step that fails is not captured: max_iter = 2 cannot reach 1e-14
    H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
    for l, (E, K) in enumerate(states):
        H.set_state(l, E, K)
    for _ in range(2):
        code, st = H.advance(0, dt, tol=1e-14, precision=ats.ATS_PREC_FP64, use_graph=3, max_iter=2)
        assert code == ats.ATS_ERR_NOT_CONVERGED
    assert H.graph_stats() == {"held": False, "captures": 0, "replays": 0}
    H.close()


@pytest.mark.parametrize("kind", ["dirichlet", "neumann", "robin"])
def test_two_level_64cube_step_graph(ats, ctx, kind):
    """The two-level workload (base 64^3, 64^3 fine cells on the central
    1/8), fine first, each coarse-to-fine row: three coarse steps."""
    levels, states, dt = W.two_level_gaussian_64cube(n0=64)
    k, a = {"dirichlet": (ats.ATS_FACE_DIRICHLET, 1.0), "neumann": (ats.ATS_FACE_NEUMANN, 0.0),
            "robin": (ats.ATS_FACE_ROBIN, 0.5)}[kind]

    def iface(H, step):
        if step == 0:
            H.set_interface(k, a)

    ref = _steps(ats, ctx, levels, states, ats.ATS_ORDER_FINE_FIRST, [dt] * 3, 2, between=iface)
    got = _steps(ats, ctx, levels, states, ats.ATS_ORDER_FINE_FIRST, [dt] * 3, 3, between=iface)
    _assert_same(ref, got)
    assert got[2] == {"held": True, "captures": 1, "replays": 2}


@pytest.mark.slow
def test_radiation_matter_step_graph(ats, ctx):
    """The 4-level radiation-matter workload (base 128^3, flux-limited
    coefficients and gas coupling before and after every level solve, 15
    solves per coarse step): two coarse steps, the second replayed; E and the
    gas temperature of every level bitwise those of the deferred path."""
    levels, states, k0, cfl = W.radiation_matter_amr(n0=128)
    rho = [s[1] for s in states]
    K0, _, _ = fld.coefficients(levels[0], rho[0], states[0][2], states[0][0], 1.0, k0)
    dt = cfl * levels[0].dx ** 2 / (2.0 * np.median(K0[levels[0].leaf_cells()]))
    out = []
    for ug in (2, 3):
        H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
        for l, (E, r, t) in enumerate(states):
            H.set_state(l, E, np.ones_like(E))
        for l, (E, r, t) in enumerate(states):
            H.set_fld(l, r, t, k0)
        rows = []
        for _ in range(2):
            code, st = H.advance(0, dt, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                                 use_graph=ug)
            assert code >= 0, st
            rows.append((code, st["iterations"], st["refinements"], st["ticks"]))
        out.append((rows, [H.state(l).copy() for l in range(len(levels))],
                    [H.temperature(l).copy() for l in range(len(levels))], H.graph_stats()))
        H.close()
    (r2, e2, t2, _), (r3, e3, t3, g3) = out
    assert r2 == r3
    for a, b in zip(e2 + t2, e3 + t3):
        np.testing.assert_array_equal(a, b)
    assert g3 == {"held": True, "captures": 1, "replays": 1}
