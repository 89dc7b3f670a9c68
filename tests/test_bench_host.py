"""Host-side logic of bench.py on the CPU: the roofline arithmetic, the
time-to-solution formula, the workload recipes, the oracle's sampling plan
and the reference arm's JSON line (the oracle on the host cores)."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_tc_roofline_flops_per_form():
    """Two E4M3 GEMMs (4 n^2 R) against 2 x the BF16 peak for FP8 with S in
    two terms; one GEMM (2 n^2 R) for BF16, one-term FP8 and PA's FP8."""
    peaks, _ = bench._peaks()
    n, R, ms = 8192, 1024, 0.07
    bf = bench.tc_roofline(1, "bsb", n, R, ms)
    f8 = bench.tc_roofline(2, "bsb", n, R, ms)
    ot = bench.tc_roofline(3, "bsb", n, R, ms)
    pa = bench.tc_roofline(2, "pa", n, R, ms)
    assert bf["algorithmic_flops_per_launch"] == 2.0 * n * n * R
    assert f8["algorithmic_flops_per_launch"] == 4.0 * n * n * R
    assert ot["algorithmic_flops_per_launch"] == pa["algorithmic_flops_per_launch"] == 2.0 * n * n * R
    assert bf["peak"] == peaks["bf16_tflops"] and f8["peak"] == 2.0 * peaks["bf16_tflops"]
    for r in (bf, f8, ot, pa):
        assert math.isclose(r["achieved"], r["algorithmic_flops_per_launch"] / (ms / 1e3) / 1e12)
        assert math.isclose(r["frac"], r["achieved"] / r["peak"])
    # the two-term form's fraction equals 2 n^2 R against the BF16 peak
    assert math.isclose(f8["frac"], bf["frac"])


def test_tts99_formula():
    assert bench._tts99(10.0, 0.0) is None
    assert bench._tts99(10.0, 0.995) == 10.0
    assert math.isclose(bench._tts99(10.0, 0.5), 10.0 * math.log(0.01) / math.log(0.5))
    # monotone: a lower success probability needs more runs
    assert bench._tts99(10.0, 0.2) > bench._tts99(10.0, 0.6)


@pytest.mark.parametrize("name", ["dense_n20", "chimera_c16", "sk_n8192_fp8", "wishart_b128_k50",
                                  "pegasus_p16", "zephyr_z12", "xorsat_3r3x_1e5",
                                  "tile_planting_l300"])
def test_workload_recipes(name):
    """Each workload states its sizes, replicas and steps consistently with
    the instance it builds."""
    w = bench.workload(name)
    assert w["name"] == name and w["R"] >= 1 and w["K"] >= 1 and w["desc"]
    if "Q" in w:
        assert w["Q"].shape == (w["n"], w["n"])
    if "sp" in w:
        assert w["sp"].n == w["n"] and w["sp"].rowptr.shape[0] == w["n"] + 1
    if w["kind"] == "batch":
        assert w["n"] == int(np.sum(w["sizes"])) and len(w["sizes"]) == 128
    if "E0_ising" in w:
        assert w["n"] == 300 * 300 and w["E0_ising"] < 0


def test_oracle_samples_of_the_largest_workloads_are_bounded():
    """The oracle's sample of the workloads too large for the host is a
    smaller instance of the same recipe, and the memory-aware process count
    is at least one."""
    z = bench.workload("zephyr_z1750", for_oracle=True)
    assert "sp" not in z and z["oracle_graph_m"] == 50 and z["n"] > 9.8e7
    h = bench.workload("hubo_chain_5e7", for_oracle=True)
    assert h["hubo"] is None and h["oracle_chain"] == 10 ** 6
    assert bench.oracle_procs(z, 2) >= 1 and bench.oracle_procs(h, 8) >= 1


def test_reference_arm_json_line():
    """`--impl reference` on the small dense workload prints one JSON line
    with the oracle's rate, its sample, and e2e equal to the line's value."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "dense_n20",
           "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "spin-updates/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"] == "dense_n20" and d["higher_is_better"] is True
