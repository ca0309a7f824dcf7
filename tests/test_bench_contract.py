"""The benchmark's reference arm (the oracle on the host cores) prints one JSON line with the
contract's keys; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "10",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "dtype",
              "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_samples_and_throttle_decision():
    """nvidia-smi CSV lines (clocks.sm, clocks.max.sm, power.draw, hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap): median clock, maximum clock and
    reasons; only the hardware and thermal slowdowns make the bench take the timing again."""
    b = _bench()
    lines = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
             "1995, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
             "2055, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active",
             "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
             "garbled"]
    c = b.parse_clock_lines(lines)
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"] and not b.throttled(c)
    for col, name in zip(range(3, 6), ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")):
        f = lines[0].split(", ")
        f[col] = "Active"
        c = b.parse_clock_lines([", ".join(f)])
        assert c["reasons"] == [name] and b.throttled(c)
    assert b.parse_clock_lines([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    assert not b.throttled({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})


def test_accuracy_check_of_the_timed_steps():
    """The bench's accuracy check: the oracle's outputs on sampled instances over the warm-up and
    timed load steps (the CPU-baseline leg) against the GPU's outputs of the timed steps.  Fed the
    oracle's own outputs it reports zero error; a planted Pbar error above 1e-7 makes the line
    inadmissible; an instance whose convergence status differs leaves the comparison from that
    load step on (its histories differ from there)."""
    import argparse
    import numpy as np
    b = _bench()
    args = argparse.Namespace(workload="c2", batch=None)
    idx = np.array([0, 3, 7])
    W, K = 2, 3
    cb = b.cpu_baseline(args, idx=idx, n_steps=W + K, budget_s=None, keep=True)
    ref = cb.pop("_out")
    assert ref["steps"] == W + K and ref["Pbar"].shape == (W + K, 3, 2, 2) and cb["kind"] == "oracle"
    assert "instances 0,3,7" in cb["sample"]
    check = dict(idx=idx, Pbar=ref["Pbar"][W:].copy(), Abar=ref["Abar"][W:].copy(), status=ref["status"][W:].copy(),
                 a=ref["q"].copy(), xi=ref["xi"].copy())
    acc = b.accuracy(check, ref, W, K)
    assert acc["checked"] and acc["admissible"] and acc["pbar_rel_err"] == 0.0 and acc["q_rel_err"] == 0.0
    bad = dict(check, Pbar=check["Pbar"].copy())
    bad["Pbar"][1, 2] *= 1 + 1e-6
    acc = b.accuracy(bad, ref, W, K)
    assert not acc["admissible"] and 5e-7 < acc["pbar_rel_err"] < 2e-6
    bad = dict(check, status=check["status"].copy(), Pbar=check["Pbar"].copy())
    bad["status"][1, 0] = 5
    bad["Pbar"][2, 0] *= 2.0          # after the split: not compared
    acc = b.accuracy(bad, ref, W, K)
    assert acc["admissible"] and acc["split"] == [0] and acc["instance_steps_compared"] == 3 * K - 2
    assert not b.accuracy(check, dict(ref, steps=W + K - 1), W, K)["checked"]


def test_sample_indices():
    b = _bench()
    s = b.sample_indices(16384, 16)
    assert len(s) == 16 and s[0] == 0 and s[-1] == 16383 and (s[1:] > s[:-1]).all()
    assert list(b.sample_indices(3, 16)) == [0, 1, 2]
