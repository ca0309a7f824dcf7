"""The benchmark's per-kernel roofline arithmetic (host logic, no GPU): achieved = algorithmic
FLOPs / time, frac = achieved / peak, the unit that bounds each kernel group, and the traffic
from the measured DRAM bytes per point."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_rooflines_c3_tf32(bench):
    # one second of each group, with known FLOP counts
    kin = 2.0 * 600 * 9 * 64
    points = 1.0e6
    prof = {"start": (0.0, 1, 0.0), "constitutive": (1000.0, 10, points / 600 * kin),
            "assemble": (1000.0, 10, 2.0e14), "solve": (1000.0, 10, 1.0e12), "finalize": (0.0, 1, 0.0),
            "bookkeeping": (0.0, 1, 0.0), "learned_start": (0.0, 0, 0.0), "force": (1000.0, 10, 3.0e12),
            "sensitivity": (0.0, 0, 0.0)}
    r = dict(workload="c3", prof=prof, prec="tf32", fp64_residual=False)
    out = bench.kernel_rooflines(r, {"bf16_tflops": 2000.0})
    c = out["constitutive"]
    per_point = bench.CONST_FP64_FLOP_PER_POINT[(3, "mixed")]
    assert 1000.0 < per_point < 2000.0                                # FP64 FLOP per 3D mixed point (ncu)
    assert c["bound"] == "alu" and abs(c["achieved"] - points * per_point / 1e12) < 1e-9
    assert abs(c["frac"] - c["achieved"] / bench.FP64_PEAK_TFLOPS) < 1e-12
    assert abs(c["traffic"] - points / 10 * bench.CONST_DRAM_BYTES_PER_POINT[(3, "mixed")]) < 1e-3   # bytes per launch
    a = out["assemble"]
    assert a["bound"] == "tensor" and abs(a["peak"] - 1000.0) < 1e-9 and abs(a["achieved"] - 200.0) < 1e-9
    f = out["force"]
    assert abs(f["peak"] - bench.FP32_PEAK_TFLOPS / 12) < 1e-12 and abs(f["achieved"] - 3.0) < 1e-9
    r["fp64_residual"] = True
    assert abs(bench.kernel_rooflines(r, {})["force"]["peak"] - bench.FP64_PEAK_TFLOPS) < 1e-12


def test_rooflines_c2_fp32_on_tensor_cores(bench):
    """The 2D FP32 stiffness runs on the tensor cores (TF32 hi/lo split): its roofline is the
    TF32 rate by algorithmic FLOPs, and the 2D mixed constitutive count applies."""
    kin = 2.0 * 160 * 4 * 24
    points = 2.0e6
    prof = {"start": (0.0, 1, 0.0), "constitutive": (1000.0, 10, points / 160 * kin),
            "assemble": (1000.0, 10, 1.0e14), "solve": (1000.0, 10, 1.0e11), "finalize": (0.0, 1, 0.0),
            "bookkeeping": (0.0, 1, 0.0), "learned_start": (0.0, 0, 0.0), "force": (1000.0, 10, 1.0e12),
            "sensitivity": (0.0, 0, 0.0)}
    out = bench.kernel_rooflines(dict(workload="c2", prof=prof, prec="fp32", fp64_residual=False), {"bf16_tflops": 2000.0})
    a = out["assemble"]
    assert a["bound"] == "tensor" and abs(a["peak"] - 1000.0) < 1e-9 and abs(a["achieved"] - 100.0) < 1e-9
    c = out["constitutive"]
    assert abs(c["achieved"] - points * bench.CONST_FP64_FLOP_PER_POINT[(2, "mixed")] / 1e12) < 1e-9


@pytest.mark.parametrize("d,name", [(3, "k_constitutive_c3_mixed_b2048.md"), (2, "k_constitutive_c2_mixed_b4096.md")])
def test_constants_match_the_committed_captures(bench, d, name):
    """The per-point FP64 FLOP and DRAM constants the bench multiplies by are the ones the
    committed ncu summaries of the constitutive kernels report, so a re-measured capture and the
    bench cannot drift apart silently."""
    import re
    text = open(os.path.join(ROOT, "profiles", name)).read()
    row = re.search(r"\| FP64 FLOP per point[^|]*\| ([0-9.]+) \| ([0-9.]+) \|", text)
    assert row, "FLOP-per-point row missing in " + name
    assert float(row.group(1)) == bench.CONST_FP64_FLOP_PER_POINT[(d, "mixed")]
    assert float(row.group(2)) == bench.CONST_FP64_FLOP_PER_POINT[(d, "fp64")]
    dram = re.search(r"\| DRAM read / write \| [0-9.]+ MB / [0-9.]+ MB = ([0-9.]+) B per point", text)
    assert dram, "DRAM row missing in " + name
    assert abs(float(dram.group(1)) - bench.CONST_DRAM_BYTES_PER_POINT[(d, "mixed")]) < 1.0
