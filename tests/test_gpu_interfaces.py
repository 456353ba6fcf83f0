"""Energy-conserving interfaces on the GPU (Sect. 3.3.1 - 3.3.2): the stored
fine-side flux feeds Neumann or Robin coarse-to-fine rows.  Parity with the
oracle's driver for every row kind, and exact energy conservation of the
GPU result with Neumann rows in a closed hierarchy.

Tolerance as for the hierarchy driver: every level solve stops on the
certified rule ||b - Ax|| <= 5e-11 ||x||; the stored energies are sums of
fine-side fluxes of such solutions, so after n solves the two sides differ by
at most about n * 1e-10 (relative L2)."""
import numpy as np
import pytest

import workloads as W
from oracle import driver

pytestmark = pytest.mark.gpu
TOL = 5e-11


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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _energy(levels, states):
    return sum(float(np.sum(E[lv.leaf_cells()])) * lv.dx ** 3 for lv, E in zip(levels, states))


@pytest.mark.parametrize("interface,alpha", [("dirichlet", 1.0), ("neumann", 0.0), ("robin", 0.4)])
@pytest.mark.parametrize("seed", [1, 4])
def test_interfaces_match_oracle(ats, ctx, seed, interface, alpha):
    levels, states, dt = W.random_hierarchy(seed, n0=8, n_levels=3)
    H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
    kind = {"dirichlet": ats.ATS_FACE_DIRICHLET, "neumann": ats.ATS_FACE_NEUMANN, "robin": ats.ATS_FACE_ROBIN}
    H.set_interface(kind[interface], alpha)
    for l, (E, K) in enumerate(states):
        H.set_state(l, E, K)
    ref = driver.Hierarchy(levels, states, order="fine_first", interface=interface, alpha=alpha)
    steps = 2
    for _ in range(steps):
        code, st = H.advance(0, dt, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED)
        ref.advance(0, dt, tol=TOL)
        # negative energies, the failure Sect. 4.2 reports for Neumann
        # interfaces, come with the warning
        negative = any(float(np.min(ref.E[l][lv.leaf_cells()])) < 0.0 for l, lv in enumerate(levels))
        assert code == (ats.ATS_WARN_NEGATIVE if negative else 0), st
    bound = steps * 7 * 1e-10
    for l in range(len(levels)):
        assert _rel(H.state(l), ref.state(l)) <= bound, l
    H.close()


def test_neumann_interfaces_conserve_energy_on_gpu(ats, ctx):
    levels, states, dt = W.random_hierarchy(6, n0=8, n_levels=3)
    H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
    H.set_interface(ats.ATS_FACE_NEUMANN)
    for l, (E, K) in enumerate(states):
        H.set_state(l, E, K)
    e0 = _energy(levels, [E for E, _ in states])
    for _ in range(3):
        code, st = H.advance(0, dt, tol=1e-12, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_FP64)
        assert code >= 0, st  # Neumann interfaces may leave negative energies (ATS_WARN_NEGATIVE)
    e1 = _energy(levels, [H.state(l) for l in range(len(levels))])
    assert abs(e1 - e0) <= 1e-10 * e0, (e0, e1)


def test_stored_fluxes_need_fine_first(ats, ctx):
    levels, _, _ = W.random_hierarchy(2, n0=8, n_levels=2)
    H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_COARSE_FIRST)
    with pytest.raises(ats.AtsError) as e:
        H.set_interface(ats.ATS_FACE_NEUMANN)
    assert e.value.code == ats.ATS_ERR_INVALID_ARG
    H.set_interface(ats.ATS_FACE_DIRICHLET)  # allowed in either order
    H.close()
    H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
    with pytest.raises(ats.AtsError):
        H.set_interface(ats.ATS_FACE_ROBIN, 1.5)
    H.close()
