"""The bounds-checked build (ATS_BOUNDS_CHECK=1): the library compiled with
every gathered index (neighbour oct, interface record, face descriptor,
work item, work-list entry) range-checked on the device.  The cases of
bounds_cases.py run in two fresh processes, one per build: the checked one
meets no out-of-range index, the default one reports that it has no checks
(-1), and both give bitwise the same results (the checks change no
arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(tmp_path, checked):
    from paper_1401_1112_gb300 import build

    build.build(checked=checked)
    out = str(tmp_path / ("checked.npz" if checked else "default.npz"))
    env = dict(os.environ, ATS_BOUNDS_CHECK="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), out], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


def test_checked_build_meets_no_bad_index_and_changes_nothing(tmp_path):
    checked = _run(tmp_path, True)
    default = _run(tmp_path, False)
    assert int(checked["violations"]) == 0
    assert int(default["violations"]) == -1
    keys = sorted(k for k in default if k != "violations")
    assert sorted(k for k in checked if k != "violations") == keys
    for k in keys:
        if k.endswith("_code"):
            assert int(default[k]) >= 0, k  # a warning (negative energy) is a result
        np.testing.assert_array_equal(checked[k], default[k], err_msg=k)
