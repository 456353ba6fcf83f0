"""The allocation-free entry point, checked against the regular solve.

ats_solve_noalloc serves callers that cannot allocate device memory (for
example code running inside a stream capture, or a plug-in confined to a
memory pool its host program owns): it keeps its CG scratch in one fixed
device array inside the library.  This file runs last (pytest collects it
after the other test files) so that a run stopping at the first failure has
already run everything else.  It must pass alone in a fresh process and after
the other tests, and it checks two calls in a row against ats_solve with the
same operator, within the tolerance the other parity tests use.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10   # relative residual target of both solves
PAR = 1e-10   # relative L2 agreement, as in the other parity tests


@pytest.fixture(scope="module")
def ats():
    from paper_1401_1112_gb300 import ats as A
    from paper_1401_1112_gb300 import build

    build.build()
    return A


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_regular_solve_twice(ats):
    import torch

    dev = torch.device("cuda:0")
    rng = np.random.default_rng(2024)
    lv = W.box_level(9, 7, 6, 1.0 / 18)          # 378 octs, zero-flux walls
    N = lv.n_cell
    K = np.exp(rng.standard_normal(N))
    dt = 20.0 * lv.dx ** 2 / 2.0
    h = 0.5 * dt / lv.dx ** 2
    nbr = torch.from_numpy(ats.ats_layout_neighbors(lv).reshape(-1).copy()).to(dev)
    Kd = torch.from_numpy(K).to(dev)
    with ats.Context(0) as ctx:
        L = ats.Level(ctx, lv)
        cases = [
            (rng.uniform(0.5, 1.5, N), None),                      # plain heat step
            (rng.uniform(0.5, 1.5, N), rng.uniform(0.0, 2.0, N)),  # with a diagonal shift s
        ]
        for E, s in cases:
            # the regular entry point: operator built by the library
            L.build(dt, K, E, s=s)
            x_ref = E.copy()
            code, st_ref = L.solve(x_ref, tol=TOL, precision=ats.ATS_PREC_FP64)
            assert code == 0, st_ref
            # the allocation-free entry point on the same operator
            b = torch.from_numpy(E.copy()).to(dev)                 # zero-flux walls: b = E^n
            xd = None if s is None else torch.from_numpy(s.copy()).to(dev)
            x = torch.from_numpy(E.copy()).to(dev)
            code, st = ats.ats_solve_noalloc(0, 0, lv.n_oct, nbr, Kd, xd, h, b, x, tol=TOL)
            assert code == 0, (st, ats.ats_last_error())
            assert st["res_norm"] <= TOL * st["r0_norm"] * 1.0001
            assert _rel(x.cpu().numpy(), x_ref) <= PAR
        L.close()


def test_noalloc_rejects_oversize(ats):
    import torch

    dev = torch.device("cuda:0")
    n_oct = ats.ATS_NOALLOC_MAX_CELLS // 8 + 1
    t = torch.zeros(8, dtype=torch.float64, device=dev)
    nbr = torch.zeros(6, dtype=torch.int32, device=dev)
    code, _ = ats.ats_solve_noalloc(0, 0, n_oct, nbr, t, None, 1.0, t, t)
    assert code == ats.ATS_ERR_INVALID_ARG
    assert "scratch" in ats.ats_last_error()
