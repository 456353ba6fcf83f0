"""Plain FP64 CPU oracle for the per-level implicit diffusion solve.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import
this package.  The CUDA product path never imports it, and it never imports
the product path.

Contents
  * ``assemble`` / ``pcg`` / ``residual`` -- ctypes front end of the C oracle
    (``ats_oracle.c``): the level matrix of Eq. (Er_imp1) with the interface
    rows of Sect. 3.2, and the diagonal-preconditioned CG of Sect. 3.3.4.
  * ``dense``    -- dense matrix of a level and a dense Cholesky solve.
  * ``spectral`` -- DCT-II closed-form solve for constant K with zero-flux
    walls (the exact discrete solution, independent of CG).
  * ``fld``      -- flux-limited-diffusion coefficients and the linearised
    gas-radiation coupling (Sect. 2.1; the paper leaves the limiter and the
    coupling to its Paper I, and the module docstring states the forms taken).
  * ``equilibrium`` -- the equilibrium test with a nonlinear diffusion
    coefficient (Sect. 4.2) on uniform grids: closed form, lagged steps to
    the steady state, the paper's L2 norm.
  * ``dirac``    -- the linear diffusion test (Sect. 4.1): a pulse on a 1D
    column whose mesh follows the 25 % gradient criterion before every
    coarse step, with each interface row.
  * ``driver``   -- the two-level / multi-level adaptive time-stepping driver
    (Sect. 2.2 and Sect. 3.3), level by level, on top of assemble + pcg.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libats_oracle.so")
_lock = threading.Lock()
_lib = None

DIRICHLET, NEUMANN, ROBIN = 0, 1, 2
REL_SAME, REL_COARSER, REL_FINER = 0, 1, 2
STOP_RESIDUAL, STOP_CERTIFIED, STOP_PAPER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build (plain -O2, FP64,
    no fast-math so every operation rounds as written)."""
    src = os.path.join(_HERE, "ats_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, src, "-lm"]
    )
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_assemble.restype = ctypes.c_int
            lib.oracle_assemble.argtypes = [
                ctypes.c_int64, P, P, ctypes.c_double, ctypes.c_double, P, P, P, P,
                ctypes.c_int64, P, P, P, P, P, P, P, P, P, P, P, P, P,
            ]
            lib.oracle_residual.restype = ctypes.c_double
            lib.oracle_residual.argtypes = [ctypes.c_int64, P, P, P, P, P, P]
            lib.oracle_pcg.restype = ctypes.c_int
            lib.oracle_pcg.argtypes = [
                ctypes.c_int64, P, P, P, P, P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int64, P,
            ]
            lib.oracle_matvec.restype = None
            lib.oracle_matvec.argtypes = [ctypes.c_int64, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class System:
    """An assembled level system (CSR over all 8*n_oct cells; non-leaf rows empty)."""

    def __init__(self, N, row_ptr, col, val, b, diag):
        self.N = N
        self.row_ptr, self.col, self.val, self.b, self.diag = row_ptr, col, val, b, diag

    @property
    def leaf(self):
        return self.row_ptr[1:] > self.row_ptr[:-1]

    def matvec(self, x):
        x = _f64(x)
        y = np.empty(self.N)
        _load().oracle_matvec(self.N, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val), _ptr(x), _ptr(y))
        return y

    def residual(self, x, b=None):
        """(r, ||r||_2) with r = b - A x, compensated sums."""
        x = _f64(x)
        b = self.b if b is None else _f64(b)
        r = np.empty(self.N)
        n = _load().oracle_residual(
            self.N, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val), _ptr(b), _ptr(x), _ptr(r)
        )
        return r, n

    def to_scipy(self):
        import scipy.sparse as sp

        nnz = int(self.row_ptr[-1])
        return sp.csr_matrix((self.val[:nnz], self.col[:nnz], self.row_ptr), shape=(self.N, self.N))


def assemble(level, dt, K, E_old, s=None, src=None, face_K=None, face_E=None, face_F=None) -> System:
    """Assemble the level system of Eq. (Er_imp1) with the face rules of
    Sect. 3.1-3.2.  ``level`` is a ``workloads.LevelDesc``-like object with
    ``oct_xyz``, ``leaf``, ``dx``, ``face_cell``, ``face_dir``, ``face_kind``,
    ``face_rel``, ``face_alpha``."""
    lib = _load()
    n_oct = int(level.oct_xyz.shape[0])
    N = 8 * n_oct
    oct_xyz = np.ascontiguousarray(level.oct_xyz, dtype=np.int32)
    leaf = None if level.leaf is None else np.ascontiguousarray(level.leaf, dtype=np.uint8)
    nf = int(len(level.face_cell))
    fc = np.ascontiguousarray(level.face_cell, dtype=np.int32)
    fd = np.ascontiguousarray(level.face_dir, dtype=np.int8)
    fk = np.ascontiguousarray(level.face_kind, dtype=np.int8)
    fr = np.ascontiguousarray(level.face_rel, dtype=np.int8)
    fa = _f64(level.face_alpha)
    K, E_old, s, src = _f64(K), _f64(E_old), _f64(s), _f64(src)
    face_K, face_E, face_F = _f64(face_K), _f64(face_E), _f64(face_F)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(max(7 * N, 1), dtype=np.int32)
    val = np.zeros(max(7 * N, 1), dtype=np.float64)
    b = np.zeros(N)
    diag = np.zeros(N)
    rc = lib.oracle_assemble(
        n_oct, _ptr(oct_xyz), _ptr(leaf), float(level.dx), float(dt), _ptr(K), _ptr(s), _ptr(src),
        _ptr(E_old), nf, _ptr(fc), _ptr(fd), _ptr(fk), _ptr(fr), _ptr(fa), _ptr(face_K),
        _ptr(face_E), _ptr(face_F), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b), _ptr(diag),
    )
    if rc != 0:
        raise ValueError("oracle_assemble: invalid level description")
    return System(N, row_ptr, col, val, b, diag)


def pcg(system: System, x0, tol=1e-10, stop_rule=STOP_RESIDUAL, max_iter=100000, b=None):
    """Jacobi-PCG (Sect. 3.3.4).  Returns (x, info dict)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    b = system.b if b is None else _f64(b)
    info = np.zeros(5)
    rc = _load().oracle_pcg(
        system.N, _ptr(system.row_ptr), _ptr(system.col), _ptr(system.val), _ptr(system.diag),
        _ptr(b), _ptr(x), float(tol), int(stop_rule), int(max_iter), _ptr(info),
    )
    return x, {
        "status": rc,
        "iterations": int(info[0]),
        "r0": info[1],
        "residual": info[2],
        "x_norm": info[3],
        "max_change": info[4],
    }


def cn_step(level, dt, K, E_old, src=None, face_K=None, face_E=None, face_F=None, tol=1e-10,
            stop_rule=STOP_RESIDUAL, max_iter=100000):
    """Crank-Nicolson step (the second-order integrator Sect. 3.3.5 names as
    the remedy for the first-order backward Euler): the same SPD matrix with
    dt/2, M' = I + (dt/2) A, and the explicit half step on the right-hand side,
    M' E^{n+1} = (I - (dt/2) A) E^n + the step's face and source terms:
    b_CN = 2 b' - M' E^n with b' the right-hand side assembled for dt/2 (its
    source terms at half weight, F and src being amounts over the full step).
    x0 = E^n.  Returns (x, info)."""
    half = lambda a: None if a is None else 0.5 * np.asarray(a, dtype=np.float64)
    S = assemble(level, 0.5 * dt, K, E_old, src=half(src), face_K=face_K, face_E=face_E, face_F=half(face_F))
    b_cn = 2.0 * S.b - S.matvec(E_old)
    return pcg(S, E_old, tol=tol, stop_rule=stop_rule, max_iter=max_iter, b=b_cn)


def solve_level(level, dt, K, E_old, x0=None, tol=1e-10, stop_rule=STOP_RESIDUAL, max_iter=100000,
                **faces):
    """assemble + pcg in one call; x0 defaults to E^n (Sect. 3.3.4)."""
    sys_ = assemble(level, dt, K, E_old, **faces)
    x0 = E_old if x0 is None else x0
    return pcg(sys_, x0, tol=tol, stop_rule=stop_rule, max_iter=max_iter)
