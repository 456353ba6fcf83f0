"""Cases run on both builds of the library by test_gpu_bounds_checked.py:
ragged batches (FP64 and mixed), a level with every interface kind, a
served request and a 4-level radiation-matter
coarse step (flux-limited coefficients, interfaces, restriction, stored
fluxes).  ``main(path)`` writes every result to an .npz file together with
the library's bounds-violation count.  Run as a script in a fresh process,
so that the library build the process loads is the one ATS_BOUNDS_CHECK
selects."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

TOL = 5e-11


def _faces(st):
    return dict(face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)


def run(ats):
    out = {}
    ctx = ats.Context(0)
    rng = np.random.default_rng(2024)
    solves = [W.random_box_solve(rng, o) for o in (1, 7, 64, 100, 333, 900, 2)]
    for name, prec in (("fp64", ats.ATS_PREC_FP64), ("mixed", ats.ATS_PREC_MIXED)):
        levels = []
        for lv, st in solves:
            L = ats.Level(ctx, lv)
            L.build(st.dt, st.K, st.E, **_faces(st))
            levels.append(L)
        xs = [st.E.copy() for _, st in solves]
        B = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=prec, use_graph=1,
                      check_every=8)
        code, _ = B.solve(xs)
        out[f"batch_{name}_code"] = np.array(code)
        for k, x in enumerate(xs):
            out[f"batch_{name}_{k}"] = x
        B.close()
        for L in levels:
            L.close()
    lv, st = W.random_amr_level(13)
    L = ats.Level(ctx, lv)
    L.build(st.dt, st.K, st.E, **_faces(st))
    x = st.E.copy()
    code, _ = L.solve(x, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, use_graph=2)
    out["amr_code"] = np.array(code)
    out["amr"] = x
    L.close()
    srv = ats.Server(0, precision=ats.ATS_PREC_MIXED, check_every=4)
    lv, st = W.random_box_solve(rng, 300, robin=True)
    t = srv.submit(lv, st, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED)
    code, x, _ = srv.wait(t, lv.n_cell)
    out["served_code"] = np.array(code)
    out["served"] = x
    srv.close()
    levels, states, k0, cfl = W.radiation_matter_amr(n0=32)
    H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
    for l, (E, r, T) in enumerate(states):
        H.set_state(l, E, np.ones_like(E))
    for l, (E, r, T) in enumerate(states):
        H.set_fld(l, r, T, k0)
    code, _ = H.advance(0, 30.0 * levels[0].dx ** 2, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED,
                        precision=ats.ATS_PREC_MIXED, use_graph=2)
    out["fld_code"] = np.array(code)
    for l in range(len(levels)):
        out[f"fld_{l}"] = H.state(l)
    H.close()
    ctx.close()
    out["violations"] = np.array(ats.ats_bounds_violations(0))
    return out


def main(path):
    from paper_1401_1112_gb300 import ats

    np.savez(path, **run(ats))


if __name__ == "__main__":
    main(sys.argv[1])
