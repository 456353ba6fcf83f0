"""Thin ctypes binding of the C ABI in include/ats.h (argument marshalling only).

Every function named ``ats_*`` here calls the C entry point of the same name.
Arrays are either numpy arrays (host memory, ``ATS_MEM_HOST``) or CUDA torch
tensors (device memory, ``ATS_MEM_DEVICE``); the binding passes their raw
pointers and never computes anything of the method itself.  The classes
``Context``, ``Level`` and ``Batch`` only own the C handles.

The library must be built (``paper_1401_1112_gb300.build.build()``); when it
is missing, ``lib()`` raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ATS_BOUNDS_CHECK=1 selects the bounds-checked build of the same library
# (paper_1401_1112_gb300.build.build(checked=True)).
LIB_PATH = os.path.join(_HERE, "_build_checked" if os.environ.get("ATS_BOUNDS_CHECK") == "1" else "_build",
                        "libats.so")

ATS_OK = 0
ATS_ERR_INVALID_ARG = -1
ATS_ERR_OOM = -2
ATS_ERR_OVER_BUDGET = -3
ATS_ERR_NOT_CONVERGED = -4
ATS_ERR_BREAKDOWN = -5
ATS_ERR_TIMEOUT = -6
ATS_ERR_CUDA = -7
ATS_ERR_NO_DEVICE = -8
ATS_ERR_BAD_INPUT = -9
ATS_WARN_NEGATIVE = 1

ATS_FACE_DIRICHLET, ATS_FACE_NEUMANN, ATS_FACE_ROBIN = 0, 1, 2
ATS_REL_SAME, ATS_REL_COARSER, ATS_REL_FINER = 0, 1, 2
ATS_MEM_HOST, ATS_MEM_DEVICE = 0, 1
ATS_STOP_RESIDUAL, ATS_STOP_CERTIFIED, ATS_STOP_PAPER = 0, 1, 2
ATS_PREC_FP64, ATS_PREC_MIXED = 0, 1
ATS_X0_GIVEN, ATS_X0_E_OLD = 0, 1
ATS_INTEGRATOR_BACKWARD_EULER, ATS_INTEGRATOR_CRANK_NICOLSON = 0, 1

P = ctypes.c_void_p


class ats_level_desc(ctypes.Structure):
    _fields_ = [
        ("n_oct", ctypes.c_int64), ("oct_xyz", P), ("leaf_mask", P), ("dx", ctypes.c_double),
        ("n_face", ctypes.c_int64), ("face_cell", P), ("face_dir", P), ("face_kind", P),
        ("face_rel", P), ("face_alpha", P),
    ]


class ats_coef_desc(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("mem", ctypes.c_int), ("K", P), ("E_old", P), ("s", P),
        ("src", P), ("face_K", P), ("face_E", P), ("face_F", P), ("integrator", ctypes.c_int),
    ]


class ats_solve_opts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double), ("stop_rule", ctypes.c_int), ("precision", ctypes.c_int),
        ("max_iter", ctypes.c_int), ("max_refine", ctypes.c_int), ("inner_rtol", ctypes.c_double),
        ("tile_octs", ctypes.c_int), ("check_every", ctypes.c_int), ("use_graph", ctypes.c_int),
        ("mem", ctypes.c_int), ("x0", ctypes.c_int), ("sched", ctypes.c_int), ("res_threads", ctypes.c_int),
        ("res_cluster", ctypes.c_int), ("res_cta_octs", ctypes.c_int), ("res_max_octs", ctypes.c_int),
        ("cg_scalars", ctypes.c_int), ("res_state", ctypes.c_int), ("res_cluster_big", ctypes.c_int),
        ("res_big_work", ctypes.c_int),
        ("res_cluster_mid", ctypes.c_int), ("cg_form", ctypes.c_int),
    ]


class ats_hierarchy_desc(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("levels", ctypes.POINTER(ats_level_desc)), ("order", ctypes.c_int),
                ("wall_kind", P), ("wall_E", P), ("wall_K", P)]


ATS_ORDER_FINE_FIRST, ATS_ORDER_COARSE_FIRST = 0, 1
ATS_SCHED_AUTO, ATS_SCHED_TICK, ATS_SCHED_RESIDENT, ATS_SCHED_GRID = 0, 1, 2, 3


class ats_kernel_stats(ctypes.Structure):
    _fields_ = [
        ("op_ms", ctypes.c_double), ("op_bytes", ctypes.c_double), ("ref_ms", ctypes.c_double),
        ("ref_bytes", ctypes.c_double), ("upd_ms", ctypes.c_double), ("upd_bytes", ctypes.c_double),
        ("launches", ctypes.c_int), ("ticks", ctypes.c_int), ("res_ms", ctypes.c_double),
        ("res_bytes", ctypes.c_double), ("res_launches", ctypes.c_int), ("res_solves", ctypes.c_int),
        ("res_span_ms", ctypes.c_double), ("res_longest_ms", ctypes.c_double), ("res_occupancy", ctypes.c_double),
        ("res_longest", ctypes.c_int), ("res_grid", ctypes.c_int), ("res_end_ms", ctypes.c_double * 3),
        ("res_grids", ctypes.c_int * 3),
    ]


class ats_tune_result(ctypes.Structure):
    _fields_ = [("tile_octs", ctypes.c_int), ("check_every", ctypes.c_int), ("ms", ctypes.c_double),
                ("ms_default", ctypes.c_double), ("candidates", ctypes.c_int), ("res_threads", ctypes.c_int),
                ("res_cluster", ctypes.c_int), ("res_cta_octs", ctypes.c_int), ("chosen", ats_solve_opts)]


class ats_solve_stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iterations", ctypes.c_int), ("refinements", ctypes.c_int),
        ("ticks", ctypes.c_int), ("r0_norm", ctypes.c_double), ("res_norm", ctypes.c_double),
        ("x_norm", ctypes.c_double), ("err_bound", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ats_server_opts(ctypes.Structure):
    _fields_ = [("solve", ats_solve_opts), ("max_slots", ctypes.c_int), ("max_items", ctypes.c_int)]


class ats_request(ctypes.Structure):
    _fields_ = [("level", ctypes.POINTER(ats_level_desc)), ("coef", ctypes.POINTER(ats_coef_desc)), ("x0", P),
                ("tol", ctypes.c_double), ("stop_rule", ctypes.c_int)]


class ats_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("stats", ats_solve_stats), ("latency_us", ctypes.c_double),
                ("queue_us", ctypes.c_double)]


class ats_server_counters(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("ticks", ctypes.c_int64),
                ("peak_resident", ctypes.c_int), ("resident_bytes", ctypes.c_size_t)]


# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("ats_context_create", ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(P)]),
    ("ats_context_destroy", ctypes.c_int, [P]),
    ("ats_context_set_stream", ctypes.c_int, [P, P]),
    ("ats_context_memory", ctypes.c_int, [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    ("ats_level_create", ctypes.c_int, [P, ctypes.POINTER(ats_level_desc), ctypes.POINTER(P)]),
    ("ats_level_destroy", ctypes.c_int, [P]),
    ("ats_level_size", ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("ats_level_build_operator", ctypes.c_int, [P, ctypes.POINTER(ats_coef_desc)]),
    ("ats_level_get_rhs", ctypes.c_int, [P, P, ctypes.c_int]),
    ("ats_level_apply", ctypes.c_int, [P, P, P, ctypes.c_int]),
    ("ats_solve", ctypes.c_int, [P, P, P, ctypes.POINTER(ats_solve_opts), ctypes.POINTER(ats_solve_stats)]),
    ("ats_batch_create", ctypes.c_int, [P, ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(ats_solve_opts), ctypes.POINTER(P)]),
    ("ats_batch_solve", ctypes.c_int, [P, ctypes.POINTER(P), ctypes.POINTER(ats_solve_stats)]),
    ("ats_batch_destroy", ctypes.c_int, [P]),
    ("ats_batch_run", ctypes.c_int, [P, ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(ats_solve_opts), ctypes.POINTER(ats_solve_stats)]),
    ("ats_batch_build_operators", ctypes.c_int, [P, ctypes.POINTER(ats_coef_desc)]),
    ("ats_batch_set_profiling", ctypes.c_int, [P, ctypes.c_int]),
    ("ats_batch_kernel_stats", ctypes.c_int, [P, ctypes.POINTER(ats_kernel_stats)]),
    ("ats_power_law_K", ctypes.c_int, [P, ctypes.c_int64, P, ctypes.c_double, ctypes.c_double, P]),
    ("ats_batch_prefetch_operators", ctypes.c_int, [P, ctypes.POINTER(ats_coef_desc)]),
    ("ats_batch_autotune", ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ats_tune_result)]),
    ("ats_default_opts", None, [ctypes.POINTER(ats_solve_opts)]),
    ("ats_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("ats_last_error", ctypes.c_char_p, []),
    ("ats_layout_neighbors", ctypes.c_int, [ctypes.POINTER(ats_level_desc), P]),
    ("ats_hierarchy_create", ctypes.c_int, [P, ctypes.POINTER(ats_hierarchy_desc), ctypes.POINTER(P)]),
    ("ats_hierarchy_destroy", ctypes.c_int, [P]),
    ("ats_hierarchy_set_interface", ctypes.c_int, [P, ctypes.c_int, ctypes.c_double]),
    ("ats_hierarchy_level", ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(P)]),
    ("ats_hierarchy_set_state", ctypes.c_int, [P, ctypes.c_int, P, P, ctypes.c_int]),
    ("ats_hierarchy_get_state", ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int]),
    ("ats_level_advance", ctypes.c_int, [P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ats_solve_opts),
                                         ctypes.POINTER(ats_solve_stats)]),
    ("ats_hierarchy_set_fld", ctypes.c_int, [P, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int]),
    ("ats_hierarchy_graph_stats", ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_int64)]),
    ("ats_hierarchy_get_temperature", ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int]),
    ("ats_hierarchy_set_power_law", ctypes.c_int, [P, ctypes.c_double, ctypes.c_double]),
    ("ats_hierarchy_plan_faces", ctypes.c_int, [ctypes.POINTER(ats_hierarchy_desc), ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_int64), P, P, P, P]),
    ("ats_server_create", ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(ats_server_opts),
                                         ctypes.POINTER(P)]),
    ("ats_server_destroy", ctypes.c_int, [P]),
    ("ats_server_submit", ctypes.c_int, [P, ctypes.POINTER(ats_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("ats_server_wait", ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_int64, P, ctypes.POINTER(ats_result)]),
    ("ats_server_stats", ctypes.c_int, [P, ctypes.POINTER(ats_server_counters)]),
    ("ats_solve_noalloc", ctypes.c_int, [ctypes.c_int, P, ctypes.c_int64, P, P, P, ctypes.c_double, P, P,
                                         ctypes.c_double, ctypes.c_int, ctypes.POINTER(ats_solve_stats)]),
    ("ats_bounds_violations", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]),
    ("ats_grid_barrier_selftest", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
]

ATS_NOALLOC_MAX_CELLS = 262144

_lib = None
_lock = threading.Lock()


def lib():
    """Load the built library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library not built: {LIB_PATH} is missing "
                    "(run paper_1401_1112_gb300.build.build())"
                )
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in _SIGS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class AtsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().ats_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib().ats_status_string(code).decode()} ({code}): {msg}")


def _check(code, where):
    if code < 0:
        raise AtsError(code, where)
    return code


# ---------------------------------------------------------------------------
# pointer marshalling
# ---------------------------------------------------------------------------

def _is_torch_cuda(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _mem_of(*arrays) -> int:
    kinds = {(_is_torch_cuda(a)) for a in arrays if a is not None}
    if len(kinds) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return ATS_MEM_DEVICE if kinds == {True} else ATS_MEM_HOST


def _ptr(a, dtype=np.float64, keep=None):
    """Raw pointer of a numpy array (converted to a contiguous ``dtype``
    array, kept alive in ``keep``) or of a CUDA torch tensor."""
    if a is None:
        return None
    if _is_torch_cuda(a):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    arr = np.ascontiguousarray(a, dtype=dtype)
    if keep is not None:
        keep.append(arr)
    return arr.ctypes.data_as(ctypes.c_void_p)


def _level_desc(level, keep):
    d = ats_level_desc()
    d.n_oct = int(level.oct_xyz.shape[0])
    d.oct_xyz = _ptr(level.oct_xyz, np.int32, keep)
    d.leaf_mask = _ptr(level.leaf, np.uint8, keep) if level.leaf is not None else None
    d.dx = float(level.dx)
    d.n_face = int(len(level.face_cell))
    if d.n_face:
        d.face_cell = _ptr(level.face_cell, np.int32, keep)
        d.face_dir = _ptr(level.face_dir, np.int8, keep)
        d.face_kind = _ptr(level.face_kind, np.int8, keep)
        d.face_rel = _ptr(level.face_rel, np.int8, keep)
        d.face_alpha = _ptr(level.face_alpha, np.float64, keep)
    return d


def make_opts(tol=1e-10, stop_rule=ATS_STOP_RESIDUAL, precision=ATS_PREC_FP64, max_iter=0, max_refine=0,
              inner_rtol=0.0, tile_octs=0, check_every=0, use_graph=0, mem=ATS_MEM_HOST,
              x0=ATS_X0_GIVEN, sched=ATS_SCHED_AUTO, res_threads=0, res_cluster=0, res_cta_octs=0,
              res_max_octs=0, cg_scalars=0, res_state=0, res_cluster_big=0, res_big_work=0,
              res_cluster_mid=0, cg_form=0) -> ats_solve_opts:
    o = ats_solve_opts()
    lib().ats_default_opts(ctypes.byref(o))
    o.tol = tol
    o.stop_rule = stop_rule
    o.precision = precision
    if max_iter:
        o.max_iter = max_iter
    if max_refine:
        o.max_refine = max_refine
    if inner_rtol:
        o.inner_rtol = inner_rtol
    o.tile_octs = tile_octs
    if check_every:
        o.check_every = check_every
    o.use_graph = use_graph
    o.mem = mem
    o.x0 = x0
    o.sched = sched
    o.res_threads = res_threads
    o.res_cluster = res_cluster
    o.res_cta_octs = res_cta_octs
    o.res_max_octs = res_max_octs
    o.cg_scalars = cg_scalars
    o.res_state = res_state
    o.res_cluster_big = res_cluster_big
    o.res_big_work = res_big_work
    o.res_cluster_mid = res_cluster_mid
    o.cg_form = cg_form
    return o


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------

def ats_context_create(device: int = 0, mem_budget_bytes: int = 0):
    h = P()
    _check(lib().ats_context_create(device, mem_budget_bytes, ctypes.byref(h)), "ats_context_create")
    return h


def ats_context_destroy(ctx):
    return _check(lib().ats_context_destroy(ctx), "ats_context_destroy")


def ats_context_set_stream(ctx, stream_handle: Optional[int]):
    """``stream_handle``: a cudaStream_t (e.g. ``torch.cuda.Stream().cuda_stream``),
    or None for the context's own stream.  0 (the legacy default stream, which
    is what ``torch.cuda.current_stream()`` returns unless a stream was made
    current) is rejected: the C call would take it as "own stream" and run
    unordered with the caller's work, and the library's CUDA graphs cannot be
    captured on the legacy stream."""
    if stream_handle is not None and int(stream_handle) == 0:
        raise ValueError("stream handle 0 is the legacy default stream: pass a non-default stream "
                         "(torch.cuda.Stream) or None for the context's own stream")
    return _check(lib().ats_context_set_stream(ctx, ctypes.c_void_p(stream_handle) if stream_handle else None),
                  "ats_context_set_stream")


def ats_context_memory(ctx):
    u, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().ats_context_memory(ctx, ctypes.byref(u), ctypes.byref(b)), "ats_context_memory")
    return u.value, b.value


def ats_level_create(ctx, level):
    keep = []
    d = _level_desc(level, keep)
    h = P()
    _check(lib().ats_level_create(ctx, ctypes.byref(d), ctypes.byref(h)), "ats_level_create")
    return h


def ats_level_destroy(lvl):
    return _check(lib().ats_level_destroy(lvl), "ats_level_destroy")


def ats_level_size(lvl):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ats_level_size(lvl, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "ats_level_size")
    return a.value, b.value, c.value


def coef_desc(dt, K, E_old, s=None, src=None, face_K=None, face_E=None, face_F=None, keep=None,
              integrator=ATS_INTEGRATOR_BACKWARD_EULER):
    """Fill an ats_coef_desc (``keep`` collects converted host arrays that
    must outlive the call)."""
    keep = [] if keep is None else keep
    c = ats_coef_desc()
    c.dt = float(dt)
    c.integrator = int(integrator)
    c.mem = _mem_of(K, E_old, s, src, face_K, face_E, face_F)
    c.K = _ptr(K, keep=keep)
    c.E_old = _ptr(E_old, keep=keep)
    c.s = _ptr(s, keep=keep)
    c.src = _ptr(src, keep=keep)
    c.face_K = _ptr(face_K, keep=keep)
    c.face_E = _ptr(face_E, keep=keep)
    c.face_F = _ptr(face_F, keep=keep)
    return c


def ats_level_build_operator(lvl, dt, K, E_old, s=None, src=None, face_K=None, face_E=None, face_F=None,
                             integrator=ATS_INTEGRATOR_BACKWARD_EULER):
    keep = []
    c = coef_desc(dt, K, E_old, s=s, src=src, face_K=face_K, face_E=face_E, face_F=face_F, keep=keep,
                  integrator=integrator)
    return _check(lib().ats_level_build_operator(lvl, ctypes.byref(c)), "ats_level_build_operator")


def ats_level_get_rhs(lvl, out):
    mem = _mem_of(out)
    return _check(lib().ats_level_get_rhs(lvl, _ptr(out), mem), "ats_level_get_rhs")


def ats_level_apply(lvl, x, y):
    mem = _mem_of(x, y)
    keep = []
    return _check(lib().ats_level_apply(lvl, _ptr(x, keep=keep), _ptr(y), mem), "ats_level_apply")


def ats_solve(lvl, x_inout, rhs=None, opts: Optional[ats_solve_opts] = None):
    """x_inout: float64 numpy array (host, updated in place) or CUDA tensor."""
    if isinstance(x_inout, np.ndarray) and (x_inout.dtype != np.float64 or not x_inout.flags.c_contiguous):
        raise ValueError("x_inout must be a contiguous float64 array")
    o = opts if opts is not None else make_opts()
    o.mem = _mem_of(x_inout, rhs)
    keep = []
    st = ats_solve_stats()
    code = lib().ats_solve(lvl, _ptr(rhs, keep=keep), _ptr(x_inout), ctypes.byref(o), ctypes.byref(st))
    return code, st.as_dict()


def ats_batch_create(ctx, levels: Sequence, opts: Optional[ats_solve_opts] = None):
    arr = (P * len(levels))(*[l.handle if isinstance(l, Level) else l for l in levels])
    o = opts if opts is not None else make_opts()
    h = P()
    _check(lib().ats_batch_create(ctx, arr, len(levels), ctypes.byref(o), ctypes.byref(h)), "ats_batch_create")
    return h


def ats_batch_solve(batch, xs: Sequence):
    arr = (P * len(xs))(*[_ptr(x) for x in xs])
    st = (ats_solve_stats * len(xs))()
    code = lib().ats_batch_solve(batch, arr, st)
    return code, [s.as_dict() for s in st]


def ats_batch_destroy(batch):
    return _check(lib().ats_batch_destroy(batch), "ats_batch_destroy")


def ats_batch_run(ctx, levels: Sequence, xs: Sequence, opts: Optional[ats_solve_opts] = None):
    arr = (P * len(levels))(*[l.handle if isinstance(l, Level) else l for l in levels])
    xa = (P * len(xs))(*[_ptr(x) for x in xs])
    o = opts if opts is not None else make_opts()
    st = (ats_solve_stats * len(xs))()
    code = lib().ats_batch_run(ctx, arr, len(levels), xa, ctypes.byref(o), st)
    return code, [s.as_dict() for s in st]


def ats_batch_build_operators(batch, coefs):
    """coefs: a ctypes array of ats_coef_desc (see ``coef_desc``), one per level."""
    return _check(lib().ats_batch_build_operators(batch, coefs), "ats_batch_build_operators")


def ats_batch_prefetch_operators(batch, coefs):
    """coefs: a ctypes array of ats_coef_desc; their host arrays are copied
    to the device without waiting (see the C header)."""
    return _check(lib().ats_batch_prefetch_operators(batch, coefs), "ats_batch_prefetch_operators")


def ats_batch_set_profiling(batch, on: bool):
    return _check(lib().ats_batch_set_profiling(batch, 1 if on else 0), "ats_batch_set_profiling")


def ats_batch_kernel_stats(batch):
    k = ats_kernel_stats()
    _check(lib().ats_batch_kernel_stats(batch, ctypes.byref(k)), "ats_batch_kernel_stats")
    out = {}
    for name, _ in k._fields_:
        v = getattr(k, name)
        out[name] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def ats_batch_autotune(batch, xs: Sequence, tiles: Sequence[int] = (), checks: Sequence[int] = (), reps: int = 2):
    """Time the batch's solve per (tile_octs, check_every) candidate and keep
    the fastest; xs as in ``ats_batch_solve`` (holds a solution on return)."""
    arr = (P * len(xs))(*[_ptr(x) for x in xs])
    ta = (ctypes.c_int * max(1, len(tiles)))(*tiles)
    ca = (ctypes.c_int * max(1, len(checks)))(*checks)
    r = ats_tune_result()
    _check(lib().ats_batch_autotune(batch, arr, ta, len(tiles), ca, len(checks), int(reps), ctypes.byref(r)),
           "ats_batch_autotune")
    out = {name: getattr(r, name) for name, _ in r._fields_ if name != "chosen"}
    out["chosen"] = {name: getattr(r.chosen, name) for name, _ in r.chosen._fields_}
    return out


def ats_power_law_K(ctx, E, K0, p, K):
    """K = K0 E^p on the device (E, K: CUDA tensors of float64)."""
    for t in (E, K):
        if _mem_of(t) != ATS_MEM_DEVICE:
            raise ValueError("ats_power_law_K takes device arrays")
    n = int(E.numel())
    if int(K.numel()) != n:
        raise ValueError("E and K differ in size")
    return _check(lib().ats_power_law_K(ctx, n, _ptr(E), float(K0), float(p), _ptr(K)), "ats_power_law_K")


def ats_default_opts() -> ats_solve_opts:
    o = ats_solve_opts()
    lib().ats_default_opts(ctypes.byref(o))
    return o


def ats_status_string(code: int) -> str:
    return lib().ats_status_string(code).decode()


def ats_last_error() -> str:
    return lib().ats_last_error().decode(errors="replace")


def ats_grid_barrier_selftest(device: int = 0, ctas: int = 0, extra: int = 0):
    """One grid barrier of the whole-GPU resident solver alone: {"normal",
    "gave_up", "ms"} (CTAs whose wait ended normally / gave up)."""
    a, b, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().ats_grid_barrier_selftest(device, ctas, extra, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)),
           "ats_grid_barrier_selftest")
    return {"normal": a.value, "gave_up": b.value, "ms": t.value}


def ats_bounds_violations(device: int = 0) -> int:
    """Out-of-range gathered indices counted since the last call by a
    bounds-checked build (the count restarts); -1 from the default build."""
    n = ctypes.c_longlong(0)
    _check(lib().ats_bounds_violations(device, ctypes.byref(n)), "ats_bounds_violations")
    return int(n.value)


def ats_layout_neighbors(level) -> np.ndarray:
    keep = []
    d = _level_desc(level, keep)
    out = np.empty(6 * d.n_oct, dtype=np.int32)
    _check(lib().ats_layout_neighbors(ctypes.byref(d), out.ctypes.data_as(ctypes.c_void_p)), "ats_layout_neighbors")
    return out.reshape(-1, 6)


def ats_solve_noalloc(device, stream, n_oct, nbr, K, xd, h, b, x, tol=1e-10, max_iter=0):
    """The allocation-free solve (see include/ats.h): every array is a CUDA
    tensor (nbr int32, the others float64), ``stream`` a cudaStream_t handle
    or 0.  Returns (status, stats dict)."""
    for name, t in (("nbr", nbr), ("K", K), ("b", b), ("x", x)) + ((("xd", xd),) if xd is not None else ()):
        if not _is_torch_cuda(t):
            raise ValueError(f"{name} must be a CUDA tensor")
    st = ats_solve_stats()
    code = lib().ats_solve_noalloc(int(device), ctypes.c_void_p(stream) if stream else None, int(n_oct),
                                   _ptr(nbr), _ptr(K), _ptr(xd), float(h), _ptr(b), _ptr(x), float(tol),
                                   int(max_iter), ctypes.byref(st))
    return code, st.as_dict()


def _hierarchy_desc(levels, order, keep, walls=None):
    """walls: None (zero-flux domain) or {side: (E_ghost, K_ghost)} for the
    Dirichlet sides (0..5 = -x, +x, -y, +y, -z, +z)."""
    arr = (ats_level_desc * len(levels))(*[_level_desc(l, keep) for l in levels])
    keep.append(arr)
    d = ats_hierarchy_desc()
    d.n_levels = len(levels)
    d.levels = ctypes.cast(arr, ctypes.POINTER(ats_level_desc))
    d.order = order
    if walls:
        kind = np.full(6, -1, dtype=np.int8)
        wE = np.zeros(6)
        wK = np.ones(6)
        for side, (e, k) in walls.items():
            kind[side] = ATS_FACE_DIRICHLET
            wE[side] = e
            wK[side] = k
        keep += [kind, wE, wK]
        d.wall_kind = kind.ctypes.data_as(P)
        d.wall_E = wE.ctypes.data_as(P)
        d.wall_K = wK.ctypes.data_as(P)
    return d


def ats_hierarchy_create(ctx, levels, order=ATS_ORDER_FINE_FIRST, walls=None):
    keep = []
    d = _hierarchy_desc(levels, order, keep, walls)
    h = P()
    _check(lib().ats_hierarchy_create(ctx, ctypes.byref(d), ctypes.byref(h)), "ats_hierarchy_create")
    return h


def ats_hierarchy_destroy(h):
    return _check(lib().ats_hierarchy_destroy(h), "ats_hierarchy_destroy")


def ats_hierarchy_set_power_law(h, K0, a):
    return _check(lib().ats_hierarchy_set_power_law(h, float(K0), float(a)), "ats_hierarchy_set_power_law")


def ats_hierarchy_set_interface(h, kind, alpha=1.0):
    return _check(lib().ats_hierarchy_set_interface(h, int(kind), float(alpha)), "ats_hierarchy_set_interface")


def ats_hierarchy_level(h, level):
    out = P()
    _check(lib().ats_hierarchy_level(h, level, ctypes.byref(out)), "ats_hierarchy_level")
    return out


def ats_hierarchy_set_state(h, level, E, K):
    keep = []
    mem = _mem_of(E, K)
    return _check(lib().ats_hierarchy_set_state(h, level, _ptr(E, keep=keep), _ptr(K, keep=keep), mem),
                  "ats_hierarchy_set_state")


def ats_hierarchy_get_state(h, level, out):
    mem = _mem_of(out)
    return _check(lib().ats_hierarchy_get_state(h, level, _ptr(out), mem), "ats_hierarchy_get_state")


def ats_hierarchy_set_fld(h, level, rho, T, k0):
    keep = []
    mem = _mem_of(rho, T)
    return _check(lib().ats_hierarchy_set_fld(h, level, _ptr(rho, keep=keep), _ptr(T, keep=keep), float(k0), mem),
                  "ats_hierarchy_set_fld")


def ats_hierarchy_get_temperature(h, level, out):
    mem = _mem_of(out)
    return _check(lib().ats_hierarchy_get_temperature(h, level, _ptr(out), mem), "ats_hierarchy_get_temperature")


def ats_level_advance(h, level, dt, opts: Optional[ats_solve_opts] = None):
    o = opts if opts is not None else make_opts()
    st = ats_solve_stats()
    code = lib().ats_level_advance(h, level, float(dt), ctypes.byref(o), ctypes.byref(st))
    return code, st.as_dict()


def ats_hierarchy_graph_stats(h):
    """The step graph of use_graph = 3: {"held", "captures", "replays"}."""
    held, cap, rep = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ats_hierarchy_graph_stats(h, ctypes.byref(held), ctypes.byref(cap), ctypes.byref(rep)),
           "ats_hierarchy_graph_stats")
    return {"held": bool(held.value), "captures": cap.value, "replays": rep.value}


def ats_hierarchy_plan_faces(levels, level, order=ATS_ORDER_FINE_FIRST, walls=None):
    """Host-only: (cell, dir, rel, src_cell) arrays of the interface faces the
    library derives for one level."""
    keep = []
    d = _hierarchy_desc(levels, order, keep, walls)
    n = ctypes.c_int64()
    _check(lib().ats_hierarchy_plan_faces(ctypes.byref(d), level, ctypes.byref(n), None, None, None, None),
           "ats_hierarchy_plan_faces")
    cell = np.empty(n.value, np.int32)
    dr = np.empty(n.value, np.int8)
    rel = np.empty(n.value, np.int8)
    src = np.empty(n.value, np.int32)
    _check(lib().ats_hierarchy_plan_faces(ctypes.byref(d), level, ctypes.byref(n), cell.ctypes.data_as(P),
                                          dr.ctypes.data_as(P), rel.ctypes.data_as(P), src.ctypes.data_as(P)),
           "ats_hierarchy_plan_faces")
    return cell, dr, rel, src


def ats_server_create(device=0, mem_budget_bytes=0, opts: Optional[ats_solve_opts] = None, max_slots=0,
                      max_items=0):
    so = ats_server_opts()
    so.solve = opts if opts is not None else make_opts()
    so.max_slots = max_slots
    so.max_items = max_items
    h = P()
    _check(lib().ats_server_create(device, mem_budget_bytes, ctypes.byref(so), ctypes.byref(h)), "ats_server_create")
    return h


def ats_server_destroy(server):
    return _check(lib().ats_server_destroy(server), "ats_server_destroy")


def ats_server_submit(server, level, dt, K, E_old, tol=1e-10, stop_rule=ATS_STOP_RESIDUAL, x0=None, s=None,
                      src=None, face_K=None, face_E=None, face_F=None, integrator=ATS_INTEGRATOR_BACKWARD_EULER):
    """Submit one level solve (host arrays, copied by the call); returns the ticket."""
    keep = []
    d = _level_desc(level, keep)
    c = coef_desc(dt, K, E_old, s=s, src=src, face_K=face_K, face_E=face_E, face_F=face_F, keep=keep,
                  integrator=integrator)
    if c.mem != ATS_MEM_HOST:
        raise ValueError("server requests take host arrays")
    r = ats_request()
    r.level = ctypes.pointer(d)
    r.coef = ctypes.pointer(c)
    r.x0 = _ptr(x0, keep=keep)
    r.tol = float(tol)
    r.stop_rule = int(stop_rule)
    t = ctypes.c_uint64()
    _check(lib().ats_server_submit(server, ctypes.byref(r), ctypes.byref(t)), "ats_server_submit")
    return t.value


def ats_server_wait(server, ticket, n_cell, timeout_us=-1):
    """Returns (status, x, result dict with stats, latency_us, queue_us)."""
    x = np.empty(n_cell)
    res = ats_result()
    code = lib().ats_server_wait(server, ctypes.c_uint64(ticket), int(timeout_us), x.ctypes.data_as(P),
                                 ctypes.byref(res))
    out = {"status": res.status, "stats": res.stats.as_dict(), "latency_us": res.latency_us,
           "queue_us": res.queue_us}
    return code, x, out


def ats_server_stats(server):
    c = ats_server_counters()
    _check(lib().ats_server_stats(server, ctypes.byref(c)), "ats_server_stats")
    return {k: getattr(c, k) for k, _ in c._fields_}


# ---------------------------------------------------------------------------
# handle owners
# ---------------------------------------------------------------------------

class Context:
    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream: Optional[int] = None):
        self.device = device
        self.handle = ats_context_create(device, mem_budget_bytes)
        if stream is not None:
            ats_context_set_stream(self.handle, stream)

    def set_stream(self, stream_handle):
        ats_context_set_stream(self.handle, stream_handle)

    def memory(self):
        return ats_context_memory(self.handle)

    def close(self):
        if self.handle:
            ats_context_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Level:
    def __init__(self, ctx: Context, level_desc):
        self.ctx = ctx
        self.desc = level_desc
        self.handle = ats_level_create(ctx.handle, level_desc)
        self.n_cell = 8 * int(level_desc.oct_xyz.shape[0])

    def build(self, dt, K, E_old, s=None, src=None, face_K=None, face_E=None, face_F=None,
              integrator=ATS_INTEGRATOR_BACKWARD_EULER):
        return ats_level_build_operator(self.handle, dt, K, E_old, s=s, src=src, face_K=face_K, face_E=face_E,
                                        face_F=face_F, integrator=integrator)

    def rhs(self):
        out = np.empty(self.n_cell)
        ats_level_get_rhs(self.handle, out)
        return out

    def apply(self, x):
        y = np.empty(self.n_cell) if not _is_torch_cuda(x) else x.new_empty(x.shape)
        ats_level_apply(self.handle, x, y)
        return y

    def solve(self, x_inout, rhs=None, **opts):
        return ats_solve(self.handle, x_inout, rhs=rhs, opts=make_opts(**opts))

    def close(self):
        if self.handle:
            ats_level_destroy(self.handle)
            self.handle = None


class Hierarchy:
    def __init__(self, ctx: Context, levels, order=ATS_ORDER_FINE_FIRST, walls=None):
        self.ctx = ctx
        self.levels = levels
        self.handle = ats_hierarchy_create(ctx.handle, levels, order, walls)

    def set_power_law(self, K0, a):
        ats_hierarchy_set_power_law(self.handle, K0, a)

    def set_state(self, level, E, K):
        ats_hierarchy_set_state(self.handle, level, E, K)

    def state(self, level):
        out = np.empty(self.levels[level].n_cell)
        ats_hierarchy_get_state(self.handle, level, out)
        return out

    def set_fld(self, level, rho, T, k0):
        ats_hierarchy_set_fld(self.handle, level, rho, T, k0)

    def set_interface(self, kind, alpha=1.0):
        """Row of the coarse-to-fine faces: ATS_FACE_DIRICHLET (restriction),
        ATS_FACE_NEUMANN (stored fine-side flux) or ATS_FACE_ROBIN (alpha)."""
        ats_hierarchy_set_interface(self.handle, kind, alpha)

    def temperature(self, level):
        out = np.empty(self.levels[level].n_cell)
        ats_hierarchy_get_temperature(self.handle, level, out)
        return out

    def advance(self, level, dt, **opts):
        return ats_level_advance(self.handle, level, dt, make_opts(**opts))

    def graph_stats(self):
        return ats_hierarchy_graph_stats(self.handle)

    def close(self):
        if self.handle:
            ats_hierarchy_destroy(self.handle)
            self.handle = None


class Server:
    def __init__(self, device=0, mem_budget_bytes=0, max_slots=0, max_items=0, **opts):
        self.handle = ats_server_create(device, mem_budget_bytes, make_opts(**opts), max_slots, max_items)

    def submit(self, level, step, tol=1e-10, stop_rule=ATS_STOP_RESIDUAL, x0=None,
               integrator=ATS_INTEGRATOR_BACKWARD_EULER):
        return ats_server_submit(self.handle, level, step.dt, step.K, step.E, tol=tol, stop_rule=stop_rule, x0=x0,
                                 s=step.s, src=step.src, face_K=step.face_K, face_E=step.face_E,
                                 face_F=step.face_F, integrator=integrator)

    def wait(self, ticket, n_cell, timeout_us=-1):
        return ats_server_wait(self.handle, ticket, n_cell, timeout_us)

    def stats(self):
        return ats_server_stats(self.handle)

    def close(self):
        if self.handle:
            ats_server_destroy(self.handle)
            self.handle = None


class Batch:
    def __init__(self, ctx: Context, levels: Sequence[Level], **opts):
        self.ctx = ctx
        self.levels = list(levels)
        self.opts = make_opts(**opts)
        self.handle = ats_batch_create(ctx.handle, self.levels, self.opts)

    def solve(self, xs):
        return ats_batch_solve(self.handle, xs)

    def prepare_coefs(self, per_level):
        """per_level: list of dicts of ``coef_desc`` keyword arguments.  The
        returned object can be passed to ``build_operators`` repeatedly."""
        keep = []
        arr = (ats_coef_desc * len(per_level))(*[coef_desc(keep=keep, **kw) for kw in per_level])
        return (arr, keep)

    def build_operators(self, prepared):
        return ats_batch_build_operators(self.handle, prepared[0])

    def prefetch_operators(self, prepared):
        return ats_batch_prefetch_operators(self.handle, prepared[0])

    def set_profiling(self, on=True):
        ats_batch_set_profiling(self.handle, on)

    def kernel_stats(self):
        return ats_batch_kernel_stats(self.handle)

    def autotune(self, xs, tiles=(), checks=(), reps=2):
        return ats_batch_autotune(self.handle, xs, tiles=tiles, checks=checks, reps=reps)

    def close(self):
        if self.handle:
            ats_batch_destroy(self.handle)
            self.handle = None
