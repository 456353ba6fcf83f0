"""Ordering with the caller's stream.  The library runs on the stream it is
given, so torch work queued on that stream before a call (here hundreds of
small copies resetting x0 = E^n) is complete when the call's kernels read it:
every step of a repeated batch starts from the same x0 and so reports the same
FP64 initial residual."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_batch_is_ordered_after_caller_stream_work():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1401_1112_gb300 import ats, build

    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    solves = W.ragged_batch(n_solves=192, seed=77, lo_oct=64, hi_oct=1024)
    n = len(solves)
    with torch.cuda.stream(stream), ats.Context(0) as ctx:
        ctx.set_stream(stream.cuda_stream)
        levels = [ats.Level(ctx, lv) for lv, _ in solves]
        K = [torch.from_numpy(st.K).to(dev) for _, st in solves]
        E = [torch.from_numpy(st.E).to(dev) for _, st in solves]
        fE = [torch.from_numpy(st.face_E).to(dev) if lv.n_face else None for lv, st in solves]
        fF = [torch.from_numpy(st.face_F).to(dev) if lv.n_face else None for lv, st in solves]
        xs = [torch.empty_like(e) for e in E]
        kw = [dict(dt=st.dt, K=K[k], E_old=E[k], face_E=fE[k], face_F=fF[k]) for k, (_, st) in enumerate(solves)]
        for k in range(n):
            levels[k].build(**kw[k])
        batch = ats.Batch(ctx, levels, tol=1e-10, stop_rule=ats.ATS_STOP_RESIDUAL, precision=ats.ATS_PREC_MIXED,
                          use_graph=1, check_every=16, mem=ats.ATS_MEM_DEVICE)
        coefs = batch.prepare_coefs(kw)
        r0 = None
        for _ in range(3):
            for k in range(n):  # many small copies queued right before the solve
                xs[k].copy_(E[k])
            batch.build_operators(coefs)
            code, stats = batch.solve(xs)
            assert code == 0, ats.ats_last_error()
            now = np.array([s["r0_norm"] for s in stats])
            assert np.all(now > 0.0)
            if r0 is None:
                r0 = now
            else:
                np.testing.assert_allclose(now, r0, rtol=1e-12, atol=0.0)
