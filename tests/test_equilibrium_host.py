"""Host side of the library's nonlinear-equilibrium driver (Sect. 4.2)
against the oracle's independent version (CPU): the closed-form profile and
the paper's L2 norms, uniform and adaptive, agree to round-off on states
that are not the equilibrium."""
import numpy as np
import pytest

import workloads as W
from oracle import equilibrium as OE
from paper_1401_1112_gb300 import equilibrium as LE


def test_closed_form_matches_the_oracle():
    x = np.linspace(0.0, 1.0, 1001)
    np.testing.assert_allclose(LE.closed_form(x), OE.analytic(x), rtol=1e-15, atol=0.0)
    assert LE.closed_form(0.0) == pytest.approx(4.0, rel=1e-15)
    assert LE.closed_form(1.0) == pytest.approx(0.5, rel=1e-15)


@pytest.mark.parametrize("n", [8, 32])
def test_uniform_l2_norm_matches_the_oracle(n):
    lv, E0, _, _ = W.equilibrium_column(n)
    rng = np.random.default_rng(n)
    E = np.asarray(E0) * rng.uniform(0.9, 1.1, len(E0))
    assert LE.l2_error(lv, E) == pytest.approx(OE.l2_error(lv, E), rel=1e-13)


@pytest.mark.parametrize("l_max", [1, 2])
def test_adaptive_l2_norm_matches_the_oracle(l_max):
    levels, E_init, _ = W.equilibrium_amr(l_max)
    rng = np.random.default_rng(l_max)
    E = [np.asarray(e) * rng.uniform(0.9, 1.1, len(e)) for e in E_init]
    n_eff = 8 * 2 ** l_max
    assert LE.l2_error_amr(levels, E, n_eff) == pytest.approx(OE.l2_error_amr(levels, E, n_eff), rel=1e-13)
