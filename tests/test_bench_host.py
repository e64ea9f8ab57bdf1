"""Host logic of bench.py that needs no GPU: the clock sampler keeps only the
samples taken inside the timed window and reports throttle reasons; it
degrades to no record when nvidia-smi is absent.  A fake nvidia-smi (a
shell script writing numbered lines) stands in for the real one."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_smi(tmp_path, power_cap="Not Active"):
    script = tmp_path / "nvidia-smi"
    script.write_text(
        "#!/bin/bash\n"
        "i=0\n"
        "while true; do\n"
        f'  echo "0, $((1000+i)), 2070, 500.0, 0x0, Not Active, Not Active, Not Active, {power_cap}"\n'
        "  i=$((i+1)); sleep 0.05\n"
        "done\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def _lines(path):
    with open(path) as f:
        return f.read().count("\n")


def _wait_lines(path, n, limit=10.0):
    t0 = time.time()
    while _lines(path) < n and time.time() - t0 < limit:
        time.sleep(0.02)
    assert _lines(path) >= n


@pytest.mark.parametrize("cap", ["Not Active", "Active"])
def test_clock_samples_from_the_window_only(tmp_path, monkeypatch, cap):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, cap) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler("GPU-test")
    assert c.proc is not None
    _wait_lines(c.path, 3)        # lines 0..2 come before the window
    c.begin()
    before = _lines(c.path)
    _wait_lines(c.path, before + 3)
    rec = c.stop()
    assert rec["samples"] >= 3
    assert rec["sm_mhz"] >= 1000 + before   # nothing from before begin()
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ([] if cap == "Not Active" else ["sw_power_cap"])
    assert not os.path.exists(c.path)


def test_no_nvidia_smi_gives_no_record(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))   # an empty directory
    c = bench.ClockSampler(None)
    c.begin()
    assert c.stop() is None


class _FakeGrid:
    """Stands in for ItpGrid: energies approach the oscillator values as
    2^-steps, returned in descending order (the leg sorts them)."""

    def __init__(self, nx, ny, nz, lx, ly, lz, n_states, n_guard, precision):
        self.n, self.k, self.closed = n_states, 0, False

    def set_potential(self, V):
        pass

    def set_states(self, psi):
        self.k = 0

    def synchronize(self):
        pass

    def step_graph(self, order, tau):
        self.k += 1
        return (bench.ho_closed_shells(self.n) + 0.5 ** self.k)[::-1].copy()

    def close(self):
        self.closed = True


def test_osc32_gpu_leg_logic():
    import types
    made = []

    def grid(*a):
        made.append(_FakeGrid(*a))
        return made[-1]

    r = bench.osc32_gpu(types.SimpleNamespace(ItpGrid=grid, ITP_FP64=0))
    assert r["reached"] and r["steps"] == 34   # 2^-34 < 1e-10 <= 2^-33
    assert made[0].closed


def test_steps_to_tol_stops_at_the_limit():
    steps, err = bench.steps_to_tol(lambda: [2.0], [1.0], 1e-10, 5)
    assert steps == 5 and err == 1.0


def test_osc32_oracle_leg_reaches_the_spectrum():
    r = bench.osc32_oracle()
    assert r["reached"] and r["steps"] < bench.OSC32["max_steps"]
    assert r["max_abs_error_ha"] < 1e-10


def test_oracle_extrapolation():
    cpu = {"value": 1.1}
    ttt = {"fp64": {"fp64_steps": 23}}
    r = bench.extrapolate_oracle(cpu, ttt, 128)
    assert r["value_s"] == round(128 * 23 / 1.1, 1)
    assert "not measured" in r["how"]
    for c, t in ((None, ttt), ({"value": None}, ttt), (cpu, None), (cpu, {"fp64": {}})):
        assert bench.extrapolate_oracle(c, t, 128) is None


def test_all_cores_oracle_sample_logic():
    """Spawned single-threaded oracle processes start together and their
    rates add up (a tiny grid stands in for the workload)."""
    w = {"n": 16, "box": 8.0, "potential": "ho", "seed": 5, "order": 4, "tau": 0.1}
    rate, started = bench._cpu_worker((w, time.time() - 1.0, 2))
    assert rate > 0 and started > 0
    r = bench.cpu_sample_all_cores(w, steps=2, setup_s=4.0)
    assert r["cores"] == len(os.sched_getaffinity(0))
    assert r["value"] > 0 and r["per_core_median"] > 0
    assert r["start_skew_s"] < 1.0
