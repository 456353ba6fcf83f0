"""GPU parity of the radiation-matter (flux-limited diffusion) workload on a
4-level AMR grid: per-level FLD coefficients, linearised coupling and the
temperature update, driven fine-first (the paper's order), mixed precision
refined to 5e-11, against the oracle's driver.  Tolerance as for the other
hierarchy tests: n solves x 1e-10 relative."""
import numpy as np
import pytest

import workloads as W
from oracle import driver, fld

pytestmark = pytest.mark.gpu
TOL = 5e-11


@pytest.fixture(scope="module")
def ats():
    from paper_1401_1112_gb300 import ats as A
    from paper_1401_1112_gb300 import build

    build.build()
    return A


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _setup(ats, ctx, n0):
    levels, states, k0, cfl = W.radiation_matter_amr(n0=n0)
    rho = [s[1] for s in states]
    T = [s[2] for s in states]
    K0, _, _ = fld.coefficients(levels[0], rho[0], T[0], states[0][0], 1.0, k0)
    dt = cfl * levels[0].dx ** 2 / (2.0 * np.median(K0[levels[0].leaf_cells()]))
    H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
    for l, (E, r, t) in enumerate(states):
        H.set_state(l, E, np.ones_like(E))
    for l, (E, r, t) in enumerate(states):
        H.set_fld(l, r, t, k0)
    ref = driver.Hierarchy(levels, [(E, np.ones_like(E)) for E, _, _ in states], order="fine_first",
                           fld=(rho, T, k0))
    return levels, H, ref, dt


@pytest.mark.parametrize("n0,steps", [(32, 2), (64, 1)])
def test_fld_hierarchy_matches_oracle(ats, n0, steps):
    with ats.Context(0) as ctx:
        levels, H, ref, dt = _setup(ats, ctx, n0)
        for _ in range(steps):
            code, st = H.advance(0, dt, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
            assert code == 0, st
            ref.advance(0, dt, tol=TOL)
        n_solves = steps * sum(2 ** l for l in range(len(levels)))
        for l in range(len(levels)):
            assert _rel(H.state(l), ref.state(l)) <= n_solves * 1e-10, l
            leaf = levels[l].leaf_cells()
            assert _rel(H.temperature(l)[leaf], ref.fld[1][l][leaf]) <= n_solves * 1e-10, l
        H.close()


def test_fld_full_size_converges(ats):
    """The full workload (base 128^3, 4 levels): every level solve of one
    coarse step reaches the certified FP64 residual bound."""
    with ats.Context(0) as ctx:
        levels, states, k0, cfl = W.radiation_matter_amr(n0=128)
        rho = [s[1] for s in states]
        H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
        for l, (E, r, t) in enumerate(states):
            H.set_state(l, E, np.ones_like(E))
        for l, (E, r, t) in enumerate(states):
            H.set_fld(l, r, t, k0)
        # dt: 30 x the explicit step at the median base-level K (K = lambda / (k0 rho^2), lambda ~ 1/3)
        kmed = np.median((1.0 / 3.0) / (k0 * rho[0] ** 2))
        dt = cfl * levels[0].dx ** 2 / (2.0 * kmed)
        code, st = H.advance(0, dt, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
        assert code == 0, st
        assert st["err_bound"] <= TOL
        for l in range(len(levels)):
            assert np.all(np.isfinite(H.state(l)))
        H.close()
