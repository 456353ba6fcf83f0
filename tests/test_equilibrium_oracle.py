"""Equilibrium test with a nonlinear diffusion coefficient (Sect. 4.2) on
uniform grids: pins of the oracle's steady states that do not depend on the
implementation.

* The closed-form profile holds the wall values and carries a constant flux
  K(E) dE/dx (it is the steady state of the law K = K0 E^a).
* The relaxed state is the discrete equilibrium: every face flux, the two
  wall faces (ghost value one cell width away) included, is the same.
* The relaxed state does not depend on the time step (it is the fixed point
  of the lagged steps).
* Against the closed form, the paper's L2 norm falls by close to 4 per
  halving of dx (the paper: close to second order on uniform grids).
"""
import numpy as np
import pytest

import workloads as W
from oracle import equilibrium as Q

RESOLUTIONS = (8, 16, 32, 64, 128)


@pytest.fixture(scope="module")
def relaxed():
    out = {}
    for n in RESOLUTIONS:
        lv, E, fE, _ = W.equilibrium_column(n)
        Es, steps, ok = Q.relax(lv, E, fE)
        assert ok, (n, steps)
        out[n] = (lv, Es, fE)
    return out


def test_closed_form_holds_the_walls_and_a_constant_flux():
    a = Q.A_EXP
    assert Q.analytic(0.0) == pytest.approx(Q.E_LEFT, rel=1e-15)
    assert Q.analytic(1.0) == pytest.approx(Q.E_RIGHT, rel=1e-15)
    x = np.linspace(0.05, 0.95, 37)
    h = 2e-4
    # fourth-order central difference of the closed form
    d = (-Q.analytic(x + 2 * h) + 8 * Q.analytic(x + h) - 8 * Q.analytic(x - h) + Q.analytic(x - 2 * h)) / (12 * h)
    flux = Q.power_law_K(Q.analytic(x), 1.0, a) * d
    assert np.max(np.abs(flux - flux[0])) <= 1e-8 * abs(flux[0])
    assert flux[0] < 0.0  # energy flows from the hot wall at x = 0


def test_relaxed_state_is_the_discrete_equilibrium(relaxed):
    lv, E, fE = relaxed[32]
    xyz = lv.cell_xyz()
    for ix in range(32):  # uniform in y and z
        col = E[xyz[:, 0] == ix]
        assert np.max(col) - np.min(col) <= 1e-12 * np.max(col)
    _, e = Q.profile(lv, E)
    dx = lv.dx
    K = Q.power_law_K(e)
    inner = 0.5 * (K[1:] + K[:-1]) * (e[1:] - e[:-1]) / dx
    left = 0.5 * (K[0] + Q.power_law_K(Q.E_LEFT)) * (e[0] - Q.E_LEFT) / dx
    right = 0.5 * (K[-1] + Q.power_law_K(Q.E_RIGHT)) * (Q.E_RIGHT - e[-1]) / dx
    flux = np.concatenate([[left], inner, [right]])
    assert np.max(np.abs(flux - flux.mean())) <= 1e-7 * abs(flux.mean())


def test_relaxed_state_does_not_depend_on_the_step(relaxed):
    lv, E, fE = relaxed[16]
    _, E0, _, _ = W.equilibrium_column(16)
    E_big, _, ok = Q.relax(lv, E0, fE, dt=2.0)
    assert ok
    assert np.max(np.abs(E_big - E)) <= 1e-8 * np.max(E)


def test_uniform_grids_converge_at_close_to_second_order(relaxed):
    l2 = [Q.l2_error(relaxed[n][0], relaxed[n][1]) for n in RESOLUTIONS]
    ratios = [l2[i] / l2[i + 1] for i in range(len(l2) - 1)]
    assert all(3.0 <= r <= 4.5 for r in ratios), ratios
    assert ratios[-1] >= 3.5, ratios
