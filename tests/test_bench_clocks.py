"""The benchmark's clock sampler (CPU): a fake nvidia-smi on PATH that, like
the real one, starts printing only after a delay.  A timed region of a few
milliseconds must still get a sample taken after it began, and the
throttle-reason columns must be read by name."""
import os
import sys
import time

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

FAKE = """#!{py}
import sys, time
time.sleep(0.3)                    # nvidia-smi's start-up
while True:
    print("0, 1965, 2070, 1012.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active", flush=True)
    time.sleep(0.02)
"""


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(py=sys.executable))
    exe.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    return exe


def test_short_region_gets_a_sample(fake_smi):
    import bench
    with bench.ClockSampler(0) as clk:
        time.sleep(0.005)          # a region far shorter than the start-up delay
    s = clk.summary()
    assert s["samples"] >= 1
    assert s["sm_mhz"] == 1965.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_unsampled_when_disabled():
    import bench
    with bench.ClockSampler(-1) as clk:
        pass
    assert clk.summary()["samples"] == 0
