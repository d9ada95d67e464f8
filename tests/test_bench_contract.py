"""bench.py's host side without a GPU: the algorithmic bytes match the
per-op byte counts of the streaming operations at the benchmark's sizes, and
the reference arm (the oracle on the host cores) prints one JSON line with
the keys the measurement contract names."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_at_the_benchmark_sizes():
    n, NL, NG = 1 << 28, 56623104, 38272753  # n = 2^28; N = 7 on 48^3
    b = bench.alg_bytes(n, NL, NG)
    assert b["copy"] == 16 * n and b["axpy"] == 24 * n and b["norm"] == 8 * n
    assert b["dot"] == 16 * n and b["cg_update"] == 48 * n
    assert abs(b["scatter"] - 0.986e9) < 1e6   # 12 N_L + 8 N_G
    assert abs(b["gather"] - 1.139e9) < 1e6    # 12 N_L + 12 N_G + 4


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "8",
                          "--warmup", "1", "--log2n", "18", "--mesh", "3,6"], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["workload"] and d["config"]["n"] == 1 << 18
    assert "n=2^18" in d["cpu_baseline"]["sample"]


def test_roofline_kernel_names_are_the_kernels_the_ops_launch():
    """Each op's kernel named in the bench line (roofline.kernel) is a
    __global__ kernel of the library, and the one-op-per-kernel mapping
    matches the launcher each op calls (BS3: the split norm, BS6: the
    pipelined gather)."""
    import re
    src = ""
    csrc = os.path.join(ROOT, "paper_2009_10917_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            src += open(os.path.join(csrc, f)).read()
    kernels = set(re.findall(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s+)?(\w+)", src))
    assert set(bench.KERNEL_OF) == set(bench.OPS)
    for op, k in bench.KERNEL_OF.items():
        assert k in kernels, (op, k)
    assert bench.KERNEL_OF["norm"] == "k_norm_split" and bench.KERNEL_OF["gather"] == "k_gather_async"
