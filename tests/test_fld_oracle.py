"""Pins of the oracle's flux-limited-diffusion coefficients and linearised
coupling (CPU)."""
import numpy as np

import workloads as W
from oracle import fld


def test_limiter_limits():
    # optically thick: lambda -> 1/3 (the diffusion limit of Sect. 4); streaming:
    # lambda R -> 1 so the flux |F| = c lambda |grad E| / (rho kappa) -> c E
    assert abs(fld.limiter(0.0) - 1.0 / 3.0) < 1e-15
    R = np.array([1e6, 1e8])
    assert np.allclose(fld.limiter(R) * R, 1.0, rtol=1e-5)
    r = np.linspace(0, 50, 1001)
    assert np.all(np.diff(fld.limiter(r)) < 0)   # monotone


def test_gradient_exact_for_linear_fields():
    lv = W.box_level(3, 2, 4, 0.25)
    xyz = W.cell_centres(lv, (0.0, 0.0, 0.0))
    a = np.array([0.3, -1.2, 2.0])
    E = 5.0 + xyz @ a
    g = fld.grad_norm(lv, E)
    np.testing.assert_allclose(g, np.linalg.norm(a), rtol=1e-12)


def test_coupling_conserves_total_energy_without_diffusion():
    """With no diffusion the radiation row is (1 + s) E = E_n + s a_R T_n^4 and
    the gas update is T = T_n + sigma (E - a_R T_n^4) / (rho c_v (1 + sigma mu));
    E + rho c_v T is then exactly conserved (the linearisation exchanges energy
    between the two reservoirs only)."""
    rng = np.random.default_rng(5)
    lv = W.box_level(2, 2, 2, 0.1)
    rho = rng.uniform(0.2, 5.0, lv.n_cell)
    T = rng.uniform(0.5, 2.0, lv.n_cell)
    E = rng.uniform(0.1, 20.0, lv.n_cell)
    for dt in (1e-6, 1e-2, 10.0):
        _, s, src = fld.coefficients(lv, rho, T, E, dt, k0=3.0)
        E1 = (E + src) / (1.0 + s)
        T1 = fld.update_temperature(rho, T, E1, dt, k0=3.0)
        np.testing.assert_allclose(E1 + rho * fld.C_V * T1, E + rho * fld.C_V * T, rtol=1e-13)
        assert np.all(s >= 0)


def test_equilibrium_is_a_fixed_point():
    """E = a_R T^4 and uniform fields: nothing changes."""
    lv = W.box_level(2, 2, 2, 0.1)
    T = np.full(lv.n_cell, 1.7)
    E = fld.A_R * T ** 4
    rho = np.full(lv.n_cell, 2.0)
    K, s, src = fld.coefficients(lv, rho, T, E, 0.5, k0=1.0)
    E1 = (E + src) / (1.0 + s)
    np.testing.assert_allclose(E1, E, rtol=1e-14)
    np.testing.assert_allclose(fld.update_temperature(rho, T, E1, 0.5, 1.0), T, rtol=1e-14)
