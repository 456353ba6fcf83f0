"""bench.py's clock sampler against a stand-in nvidia-smi (CPU): sampling is
live before the timed region starts, only the lines that arrive inside the
region are summarised, and throttle reasons marked Active are reported."""
import importlib.util
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!{py}
import sys, time
# the sampler must name the GPU by a stable identifier, not a CUDA ordinal
ids = [a for a in sys.argv[1:] if a.startswith("--id=")]
with open({log!r}, "w") as f:
    f.write(ids[0][5:] if ids else "")
# one CSV line every 20 ms: SM clock 1000 MHz for 0.3 s, then 2000 MHz with
# the power cap active, as the real query prints them (noheader, nounits)
t0 = time.time()
while True:
    hot = time.time() - t0 > 0.3
    print("0, %d, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, %s" %
          (2000 if hot else 1000, "Active" if hot else "Not Active"), flush=True)
    time.sleep(0.02)
"""


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sampler_keeps_the_region_only(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    log = tmp_path / "id.txt"
    exe.write_text(FAKE.format(py=sys.executable, log=str(log)))
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    bench = _bench()
    uuid = "GPU-6f1e2d3c-0000-1111-2222-333344445555"
    s = bench.ClockSampler(uuid)
    s.start()
    assert s.lines, "the first sample is awaited before the region"
    time.sleep(0.45)  # past the switch to 2000 MHz
    t0 = time.perf_counter()
    time.sleep(0.2)
    out = s.stop(t0, time.perf_counter())
    assert out["samples_in_region"] >= 5
    assert out["sm_mhz"] == 2000.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["gpu"] == uuid
    assert log.read_text() == uuid


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    bench = _bench()
    s = bench.ClockSampler("GPU-x")
    s.start()
    assert s.stop(0.0, 1.0)["reasons"] == ["nvidia-smi unavailable"]
