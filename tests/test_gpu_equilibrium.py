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
