"""The equilibrium test with a nonlinear diffusion coefficient (Sect. 4.2) on
the GPU: the device-side coefficient K = K0 E^a, lagged backward-Euler steps
through the library, relaxed to the steady state, against the oracle's
relaxed state and the closed form.

Tolerance: both sides stop when a step changes E by less than 1e-10
(relative, max norm) and certify every solve at 5e-11; a step contracts the
distance to the discrete steady state by at least ~0.75 here, so each side
is within ~5e-10 of it and the two differ by at most ~1e-9 (1e-8 is used).
"""
import numpy as np
import pytest

import workloads as W
from oracle import equilibrium as Q

pytestmark = pytest.mark.gpu


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


def test_power_law_coefficient_kernel(ats, ctx):
    import torch

    E = torch.linspace(0.25, 6.0, 1001, dtype=torch.float64, device="cuda")
    K = torch.empty_like(E)
    ats.ats_power_law_K(ctx.handle, E, 1.7, 1.5, K)
    torch.cuda.synchronize()
    ref = Q.power_law_K(E.cpu().numpy(), 1.7, 1.5)
    np.testing.assert_allclose(K.cpu().numpy(), ref, rtol=4e-15)
    with pytest.raises(ValueError):
        ats.ats_power_law_K(ctx.handle, E, 1.0, 1.5, K[:10])
    assert ats.lib().ats_power_law_K(ctx.handle, -1, None, 1.0, 1.0, None) == ats.ATS_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_relaxed_states_match_the_oracle(ats, ctx, prec):
    from paper_1401_1112_gb300 import equilibrium as G

    P = ats.ATS_PREC_FP64 if prec == "fp64" else ats.ATS_PREC_MIXED
    l2 = []
    for n in (8, 16, 32, 64, 128):
        lv, E, fE, _ = W.equilibrium_column(n)
        Eg, steps, ok, _ = G.relax(ctx, lv, E, fE, precision=P)
        assert ok, (n, steps)
        Eo, _, ok_o = Q.relax(lv, E, fE)
        assert ok_o
        assert np.max(np.abs(Eg - Eo)) <= 1e-8 * np.max(Eo), n
        l2.append(G.l2_error(lv, Eg))
        assert l2[-1] == pytest.approx(Q.l2_error(lv, Eo), rel=1e-6)
    ratios = [l2[i] / l2[i + 1] for i in range(len(l2) - 1)]
    assert all(3.0 <= r <= 4.5 for r in ratios), ratios


@pytest.mark.parametrize("l_max", [0, 1, 2, 3])
def test_adaptive_runs_match_the_oracle(ats, ctx, l_max):
    """The adaptive-time-step runs (static mesh refined toward the steep end,
    Dirichlet sides on every level touching them, K = E^1.5 from each
    level's own E^n, fine levels first): relaxed leaf values within 1e-8 of
    the oracle's driver, the same L2 norm."""
    from paper_1401_1112_gb300 import equilibrium as G

    levels, E_init, walls = W.equilibrium_amr(l_max)
    Eg, steps, ok, _ = G.relax_amr(ctx, levels, E_init, walls)
    assert ok, steps
    Eo, steps_o, ok_o = Q.relax_amr(levels, E_init, walls)
    assert ok_o
    scale = max(float(np.max(e)) for e in Eo)
    for lv, a, b in zip(levels, Eg, Eo):
        leaf = lv.leaf_cells()
        assert np.max(np.abs(a[leaf] - b[leaf])) <= 1e-8 * scale
    n_eff = 8 * 2 ** l_max
    assert G.l2_error_amr(levels, Eg, n_eff) == pytest.approx(Q.l2_error_amr(levels, Eo, n_eff), rel=1e-6)


def test_walled_hierarchy_linear_steady_state(ats, ctx):
    """Constant K, Dirichlet sides, interior refinement: the exact linear
    profile through the ghost values on every leaf (as the oracle's pin)."""
    from paper_1401_1112_gb300 import equilibrium as G

    levels = W.column_hierarchy(8, [[3, 4], [7, 8]])
    E0, E1 = 3.0, 1.0
    Es, steps, ok, _ = G.relax_amr(ctx, levels, [np.full(lv.n_cell, 2.0) for lv in levels], {0: E0, 1: E1},
                                   K0=1.0, a=0.0, precision=ats.ATS_PREC_FP64)
    assert ok, steps
    dx0 = levels[0].dx
    for lv, E in zip(levels, Es):
        x = (lv.cell_xyz()[:, 0] + 0.5) * lv.dx
        lin = E0 + (E1 - E0) * (x + 0.5 * dx0) / (1.0 + dx0)
        leaf = lv.leaf_cells()
        assert np.max(np.abs(E[leaf] - lin[leaf])) <= 1e-8
