"""Linear diffusion (Dirac) test of Sect. 4.1 on the GPU with the mesh
following the 25 % criterion before every coarse step, for each interface
row: the library's runs against the oracle's.

Tolerance: every level solve on both sides is certified at 5e-11 (relative
error); the level matrices are M-matrices with lambda_min >= 1, so errors are
not amplified from solve to solve and after n solves the two sides differ by
at most about n * 1e-10 (relative L2).  8 coarse steps of up to 15 level
solves: 1.2e-8; 2e-8 is used.  Both sides take the same refinement
decisions (compared).
"""
import numpy as np
import pytest

from oracle import dirac as D

pytestmark = pytest.mark.gpu
STEPS = 8


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


@pytest.mark.parametrize("row", ["dirichlet", "robin", "neumann"])
def test_pulse_runs_match_the_oracle(ats, ctx, row):
    from paper_1401_1112_gb300 import amr1d as G

    kind, alpha = {"dirichlet": (ats.ATS_FACE_DIRICHLET, 1.0), "robin": (ats.ATS_FACE_ROBIN, 0.5),
                   "neumann": (ats.ATS_FACE_NEUMANN, 0.0)}[row]
    levels, E, energies, x0, _ = G.run_pulse(ctx, kind, alpha, n_steps=STEPS)
    lo, Eo, en_o, x0o = D.run(row, alpha, n_steps=STEPS)
    assert x0 == pytest.approx(x0o)
    x, dx, e = G.leaf_row(levels, E)
    xo, dxo, eo = D.leaf_profile(lo, Eo)
    np.testing.assert_array_equal(x, xo)      # the same mesh
    np.testing.assert_array_equal(dx, dxo)
    assert np.linalg.norm(e - eo) <= 2e-8 * np.linalg.norm(eo)
    np.testing.assert_allclose(energies, en_o, rtol=2e-8)
    if row == "neumann":
        assert np.max(np.abs(energies / energies[0] - 1.0)) <= 1e-9
