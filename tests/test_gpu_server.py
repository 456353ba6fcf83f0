"""Serving loop (continuous batching): requests of mixed sizes, walls
(Dirichlet / Neumann / Robin), tolerances and time steps arrive from several
threads while others are on the GPU; every result matches the oracle, and is
bitwise the same as the same solve alone (its arithmetic involves no other
solve)."""
import threading
import time

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ats():
    from paper_1401_1112_gb300 import ats as A
    from paper_1401_1112_gb300 import build

    build.build()
    return A


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        o = float(np.exp(rng.uniform(np.log(8), np.log(4096))))
        lv, st = W.random_box_solve(rng, o, robin=True)
        tol = 5e-11 if rng.uniform() < 0.5 else 1e-6
        out.append((lv, st, tol))
    return out


def _oracle(lv, st, tol):
    S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    x, info = oracle.pcg(S, st.E, tol=tol, stop_rule=oracle.STOP_CERTIFIED)
    assert info["status"] == 0
    return x


def test_continuous_batching_mix_matches_alone_and_oracle(ats):
    reqs = _requests(40, 77)
    srv = ats.Server(0, precision=ats.ATS_PREC_MIXED, check_every=4)
    tickets = [None] * len(reqs)

    def producer(idx):
        for k in idx:
            lv, st, tol = reqs[k]
            tickets[k] = srv.submit(lv, st, tol=tol, stop_rule=ats.ATS_STOP_CERTIFIED)
            time.sleep(0.002)

    th = [threading.Thread(target=producer, args=(list(range(j, len(reqs), 2)),)) for j in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    results = []
    for k, (lv, st, tol) in enumerate(reqs):
        code, x, res = srv.wait(tickets[k], lv.n_cell)
        assert code == 0, res
        assert res["stats"]["err_bound"] <= tol
        results.append(x)
    stats = srv.stats()
    assert stats["completed"] == len(reqs)
    assert stats["peak_resident"] > 1  # solves really overlapped on the device
    srv.close()
    # alone: each request through a fresh server, one at a time -> bitwise equal
    alone = ats.Server(0, precision=ats.ATS_PREC_MIXED, check_every=4)
    for k in (0, 7, 13, 21, 39):
        lv, st, tol = reqs[k]
        t = alone.submit(lv, st, tol=tol, stop_rule=ats.ATS_STOP_CERTIFIED)
        code, x, _ = alone.wait(t, lv.n_cell)
        assert code == 0
        np.testing.assert_array_equal(x, results[k])
    alone.close()
    # and against the oracle (certified on both sides: difference <= 2 tol)
    for k in range(0, len(reqs), 3):
        lv, st, tol = reqs[k]
        xr = _oracle(lv, st, tol)
        assert np.linalg.norm(results[k] - xr) <= 2.0 * tol * np.linalg.norm(xr)


def test_memory_budget_admission_and_rejection(ats):
    reqs = _requests(12, 5)
    # a budget that holds only a few requests at a time: the rest wait
    srv = ats.Server(0, mem_budget_bytes=64 << 20, precision=ats.ATS_PREC_MIXED, check_every=4)
    tickets = [srv.submit(lv, st, tol=tol, stop_rule=ats.ATS_STOP_CERTIFIED) for lv, st, tol in reqs]
    for (lv, st, tol), t in zip(reqs, tickets):
        code, x, res = srv.wait(t, lv.n_cell)
        assert code == 0
    # a request that can never fit is rejected, not left waiting
    lv, st = W.random_box_solve(np.random.default_rng(1), 128 ** 3 / 8)  # ~190 MB resident > 64 MB
    t = srv.submit(lv, st)
    code, _, res = srv.wait(t, lv.n_cell, timeout_us=60_000_000)
    assert code == ats.ATS_ERR_OVER_BUDGET
    srv.close()
