"""Host-side checks of the C ABI (no GPU needed): the library builds and
exports every entry point include/ats.h declares, the layout builder (oct
neighbour table, descriptor validation) matches brute force, and status codes
have messages."""
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1401_1112_gb300 import build

    build.build()
    from paper_1401_1112_gb300 import ats

    return ats


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "ats.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ats_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(built):
    names = _declared_functions()
    assert len(names) >= 20
    L = built.lib()
    for n in names:
        assert hasattr(L, n), f"missing export {n}"
    # and the binding wraps each of them under the same name
    for n in names:
        assert hasattr(built, n), f"binding lacks {n}"


def test_nm_exports(built):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", built.LIB_PATH], capture_output=True, text=True).stdout
    for n in _declared_functions():
        assert re.search(rf"\bT {n}\b", out), n


def _brute_neighbors(oct_xyz):
    idx = {tuple(map(int, c)): i for i, c in enumerate(oct_xyz)}
    out = np.full((len(oct_xyz), 6), -1, dtype=np.int32)
    for i, c in enumerate(oct_xyz):
        for d in range(6):
            q = list(map(int, c))
            q[d // 2] += -1 if d % 2 == 0 else 1
            out[i, d] = idx.get(tuple(q), -1)
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_layout_neighbors_match_brute_force(built, seed):
    lv, _ = W.random_amr_level(seed)
    nb = built.ats_layout_neighbors(lv)
    np.testing.assert_array_equal(nb, _brute_neighbors(lv.oct_xyz))


def test_layout_box_and_strip(built):
    for dims in [(1, 1, 1), (1, 1, 9), (3, 4, 5)]:
        lv = W.box_level(*dims, 0.1)
        np.testing.assert_array_equal(built.ats_layout_neighbors(lv), _brute_neighbors(lv.oct_xyz))


def test_layout_rejects_bad_descriptions(built):
    lv, _ = W.random_amr_level(7)
    # duplicate oct
    dup = W.LevelDesc(np.concatenate([lv.oct_xyz, lv.oct_xyz[:1]]), None, lv.dx, *(np.zeros(0, t) for t in (np.int32, np.int8, np.int8, np.int8, np.float64)))
    with pytest.raises(built.AtsError):
        built.ats_layout_neighbors(dup)
    # descriptor on an interior face
    box = W.box_level(2, 2, 2, 0.1)
    bad = W.LevelDesc(box.oct_xyz, None, 0.1, np.array([0], np.int32), np.array([1], np.int8), np.array([0], np.int8), np.array([0], np.int8), np.array([1.0]))
    with pytest.raises(built.AtsError, match="interior"):
        built.ats_layout_neighbors(bad)
    # alpha outside [0, 1]
    walls = W.box_level(1, 1, 1, 0.1, [(W.ROBIN, 0.5)] * 6)
    walls.face_alpha = walls.face_alpha.copy()
    walls.face_alpha[0] = 1.5
    with pytest.raises(built.AtsError, match="alpha"):
        built.ats_layout_neighbors(walls)
    # a level without octs
    empty = W.LevelDesc(np.zeros((0, 3), np.int32), None, 0.1,
                        *(np.zeros(0, t) for t in (np.int32, np.int8, np.int8, np.int8, np.float64)))
    with pytest.raises(built.AtsError, match="no octs"):
        built.ats_layout_neighbors(empty)
    # descriptor on a non-leaf cell
    lv2 = W.box_level(1, 1, 1, 0.1, [(W.DIRICHLET, 1.0)] * 6)
    lv2.leaf = np.array([0xFE], np.uint8)
    with pytest.raises(built.AtsError, match="non-leaf"):
        built.ats_layout_neighbors(lv2)


def test_bounds_checked_build_exports_the_same_entry_points(built):
    """The bounds-checked build compiles from the same sources and exports
    every declared entry point; the default build reports that it has no
    checks (-1) without touching a device."""
    import ctypes

    from paper_1401_1112_gb300 import build

    checked = ctypes.CDLL(build.build(checked=True))
    for n in _declared_functions():
        assert hasattr(checked, n), f"checked build lacks {n}"
    assert built.ats_bounds_violations(0) == -1


def test_status_strings(built):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9, 1):
        assert built.ats_status_string(code) != "unknown status"


def test_no_device_is_reported_not_faked(built):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(built.AtsError) as e:
        built.ats_context_create(0, 0)
    assert e.value.code == built.ATS_ERR_NO_DEVICE


def test_noalloc_rejects_misaligned_arrays(built):
    """The allocation-free entry point checks the 32-byte alignment of its
    FP64 arrays before any CUDA call (the kernels move an oct as two 32-byte
    accesses)."""
    import ctypes

    st = built.ats_solve_stats()
    V = ctypes.c_void_p
    code = built.lib().ats_solve_noalloc(0, None, 8, V(0x1000), V(0x2008), None, 0.5, V(0x3000), V(0x4000),
                                         1e-10, 0, ctypes.byref(st))
    assert code == built.ATS_ERR_INVALID_ARG
    assert "32-byte" in built.ats_last_error()


def test_legacy_default_stream_is_rejected(built):
    """Stream handle 0 (the legacy default stream) would be taken as "the
    context's own stream" and run unordered with the caller's work; the
    binding rejects it before any CUDA call."""
    with pytest.raises(ValueError, match="legacy default stream"):
        built.ats_context_set_stream(None, 0)
