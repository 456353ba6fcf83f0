"""Flux-limited diffusion coefficients and the linearised gas-radiation
coupling (TEST INFRASTRUCTURE ONLY).

Sect. 2.1: the radiative energy diffuses with K = c lambda / (rho kappa_R)
and exchanges energy with the gas through kappa_P rho c (a_R T^4 - E_r).  The
limiter lambda and the linearisation are in the paper's Paper I, not in this
paper; the readings used are:
  * Levermore-Pomraning limiter lambda(R) = (2 + R) / (6 + 3R + R^2),
    R = |grad E| / (rho kappa_R E), lambda -> 1/3 for R -> 0;
  * kappa_R = kappa_P = k0 rho / T (per unit mass), so rho kappa_R = k0 rho^2 / T;
  * grad E by central differences over same-level cells (leaf or refined),
    one-sided where one neighbour is missing, 0 where both are;
  * emission linearised about T_n: with sigma = dt kappa_P rho c and
    mu = 4 a_R T_n^3 / (rho c_v), the matter equation is eliminated and the
    radiation row gets the diagonal shift s = sigma / (1 + sigma mu) and the
    source s a_R T_n^4; after the solve T = T_n + sigma (E - a_R T_n^4) /
    (rho c_v (1 + sigma mu)).
Code units c = a_R = c_v = 1.
"""
from __future__ import annotations

import numpy as np

C = 1.0
A_R = 1.0
C_V = 1.0


def limiter(R):
    R = np.asarray(R, dtype=np.float64)
    return (2.0 + R) / (6.0 + 3.0 * R + R * R)


def grad_norm(level, E):
    """|grad E| per cell by central / one-sided differences over the cells of
    the same level (leaf or refined); plain loops over a coordinate dict."""
    cell_of = {}
    for o, (x, y, z) in enumerate(level.oct_xyz.tolist()):
        for c in range(8):
            cell_of[(2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1))] = 8 * o + c
    N = 8 * len(level.oct_xyz)
    g2 = np.zeros(N)
    for p, i in cell_of.items():
        for a in range(3):
            pm = list(p); pm[a] -= 1
            pp = list(p); pp[a] += 1
            jm = cell_of.get(tuple(pm))
            jp = cell_of.get(tuple(pp))
            if jm is not None and jp is not None:
                g = (E[jp] - E[jm]) / (2.0 * level.dx)
            elif jp is not None:
                g = (E[jp] - E[i]) / level.dx
            elif jm is not None:
                g = (E[i] - E[jm]) / level.dx
            else:
                g = 0.0
            g2[i] += g * g
    return np.sqrt(g2)


def coefficients(level, rho, T, E, dt, k0):
    """(K, s, src) per cell from the gas state and E^n."""
    kr = k0 * rho * rho / T                     # rho kappa_R
    R = grad_norm(level, E) / (kr * E)
    K = C * limiter(R) / kr
    sigma = dt * kr * C                         # dt kappa_P rho c with kappa_P = kappa_R
    mu = 4.0 * A_R * T ** 3 / (rho * C_V)
    s = sigma / (1.0 + sigma * mu)
    src = s * A_R * T ** 4
    return K, s, src


def update_temperature(rho, T, E_new, dt, k0):
    kr = k0 * rho * rho / T
    sigma = dt * kr * C
    mu = 4.0 * A_R * T ** 3 / (rho * C_V)
    return T + sigma * (E_new - A_R * T ** 4) / (rho * C_V * (1.0 + sigma * mu))
