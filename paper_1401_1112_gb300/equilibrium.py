"""The equilibrium test with a nonlinear diffusion coefficient (Sect. 4.2)
through the library: a level with Dirichlet walls holding E = 4 at x = 0 and
E = 0.5 at x = 1 relaxes, by backward-Euler steps whose coefficient K = K0
E^a is evaluated at E^n on the device (``ats_power_law_K``), to the steady
state E(x) = [(E1^(a+1) - E0^(a+1)) x + E0^(a+1)]^(1/(a+1)) (a = 3/2, the
exponent printed as 1/(n+1) read as 1/(a+1), with the law K ~ E^a that makes
it the steady state).  Every array stays on the device; the host only checks
the change of each step.
"""
from __future__ import annotations

import numpy as np

from . import ats as A

A_EXP = 1.5
E_LEFT, E_RIGHT = 4.0, 0.5


def closed_form(x, E0=E_LEFT, E1=E_RIGHT, a=A_EXP):
    x = np.asarray(x, dtype=np.float64)
    return (E0 ** (a + 1) + (E1 ** (a + 1) - E0 ** (a + 1)) * x) ** (1.0 / (a + 1))


def relax(ctx, level_desc, E_init, face_E, K0=1.0, a=A_EXP, dt=0.1, tol_step=1e-10, max_steps=2000,
          precision=A.ATS_PREC_MIXED, tol=5e-11, use_graph=2):
    """Steps of dt until the largest relative change of a step is below
    tol_step.  E_init, face_E: host arrays.  Returns (E on the host, steps,
    converged, seconds per step)."""
    import time

    import torch

    dev = torch.device("cuda", ctx.device)
    # torch's copies and reductions run on torch's stream, the library on the
    # context's: each hand-over waits for the torch side to finish
    E = torch.from_numpy(np.ascontiguousarray(E_init, dtype=np.float64)).to(dev)
    x = torch.empty_like(E)
    K = torch.empty_like(E)
    fE = torch.from_numpy(np.ascontiguousarray(face_E, dtype=np.float64)).to(dev)
    fK = torch.empty_like(fE)
    torch.cuda.synchronize(dev)
    A.ats_power_law_K(ctx.handle, fE, K0, a, fK)  # the ghosts' K at the wall values
    L = A.Level(ctx, level_desc)
    steps, ok = 0, False
    t0 = time.perf_counter()
    try:
        for steps in range(1, max_steps + 1):
            A.ats_power_law_K(ctx.handle, E, K0, a, K)
            L.build(dt, K, E, face_K=fK, face_E=fE)
            x.copy_(E)
            torch.cuda.synchronize(dev)
            code, st = L.solve(x, tol=tol, stop_rule=A.ATS_STOP_CERTIFIED, precision=precision,
                               mem=A.ATS_MEM_DEVICE, use_graph=use_graph)
            if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                raise RuntimeError(f"equilibrium step {steps} failed: {code} {st}")
            change = float((x - E).abs().max() / E.abs().max())  # the solve has returned: x is final
            E.copy_(x)
            torch.cuda.synchronize(dev)
            if change < tol_step:
                ok = True
                break
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
    finally:
        L.close()
    return E.cpu().numpy(), steps, ok, el / max(1, steps)


def l2_error(level_desc, E):
    """The paper's L2 norm against the closed form on a uniform level:
    sqrt(sum_i [(E_i - E(x_i)) dx]^2 / N) over the cells of the y = z = 0
    row (the column is uniform in y and z), N the cells in x."""
    xyz = level_desc.cell_xyz()
    row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0)
    dx = level_desc.dx
    xc = (xyz[row, 0] + 0.5) * dx
    err = (np.asarray(E)[row] - closed_form(xc)) * dx
    return float(np.sqrt(np.sum(err * err) / row.sum()))


def relax_amr(ctx, levels, E_init, walls, K0=1.0, a=A_EXP, dt=0.1, tol_step=1e-10, max_steps=2000,
              precision=A.ATS_PREC_MIXED, tol=5e-11, use_graph=2):
    """The same relaxation on an AMR hierarchy with adaptive time steps
    (fine levels first, Sect. 2.2): coarse steps of dt until the largest
    relative change of the leaf values over a coarse step is below tol_step.
    walls: {side: E_wall} Dirichlet sides; the ghosts' K is K0 E_wall^a.
    Returns (per-level E on the host, coarse steps, converged, seconds per
    coarse step)."""
    import time

    H = A.Hierarchy(ctx, levels, A.ATS_ORDER_FINE_FIRST,
                    walls={side: (e, K0 * e ** a) for side, e in walls.items()})
    leaves = [lv.leaf_cells() for lv in levels]
    try:
        H.set_power_law(K0, a)
        for l, e in enumerate(E_init):
            e = np.ascontiguousarray(e, dtype=np.float64)
            H.set_state(l, e, K0 * e ** a)
        prev = [H.state(l)[leaves[l]] for l in range(len(levels))]
        steps, ok = 0, False
        t0 = time.perf_counter()
        for steps in range(1, max_steps + 1):
            code, st = H.advance(0, dt, tol=tol, stop_rule=A.ATS_STOP_CERTIFIED, precision=precision,
                                 use_graph=use_graph)
            if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                raise RuntimeError(f"equilibrium coarse step {steps} failed: {code} {st}")
            cur = [H.state(l)[leaves[l]] for l in range(len(levels))]
            scale = max(float(np.max(np.abs(c))) for c in cur)
            change = max(float(np.max(np.abs(c - p))) for c, p in zip(cur, prev)) / scale
            prev = cur
            if change < tol_step:
                ok = True
                break
        el = time.perf_counter() - t0
        return [H.state(l) for l in range(len(levels))], steps, ok, el / max(1, steps)
    finally:
        H.close()


def l2_error_amr(levels, E_levels, n_eff):
    """The paper's L2 norm over the leaves of the y = z = 0 row of every
    level, each with its own dx, divided by N_eff (the cells at the finest
    resolution)."""
    tot = 0.0
    for lv, E in zip(levels, E_levels):
        xyz = lv.cell_xyz()
        row = (xyz[:, 1] == 0) & (xyz[:, 2] == 0) & lv.leaf_cells()
        err = (np.asarray(E)[row] - closed_form((xyz[row, 0] + 0.5) * lv.dx)) * lv.dx
        tot += float(np.sum(err * err))
    return float(np.sqrt(tot / n_eff))
