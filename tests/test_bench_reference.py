"""The reference arm's study modes on CPU: the oracle over a full (small) product and over a small
batched workload, each printing one JSON line with its cpu_baseline description."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_full_product():
    rec = _run("--size", "96", "--moduli", "14", "--ref-block", "96", "--steps", "1",
               "--warmup", "0")
    assert rec["impl"] == "reference" and rec["value"] > 0
    assert rec["config"]["sample"] == "full"
    assert rec["config"]["workload"] == "square FP64 GEMM m=n=k=96, phi=1.0, N=14 moduli"
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["steps"] == 1 and rec["warmup"] == 0   # a full product needs no warm-up


def test_reference_sampled_block_keeps_warmup():
    rec = _run("--size", "256", "--moduli", "8", "--ref-block", "32", "--steps", "1",
               "--warmup", "0")
    assert rec["config"]["sample"] == "32x32 block"
    assert rec["warmup"] == 3   # raised to the contract's minimum


def test_reference_batched():
    rec = _run("--batched", "--batch", "3", "--steps", "1", "--warmup", "0")
    assert rec["mode"] == "batched" and rec["value"] > 0
    assert rec["config"]["n_per_item"] == 15
    assert rec["cpu_baseline"]["sample"] == "every problem, full"


def test_stage_rooflines():
    sys.path.insert(0, ROOT)
    import bench

    m = n = k = 1024
    N = 16
    st = {"scale": 1.0, "convert": 2.0, "residue_gemm": 10.0, "crt": 1.0}
    r = bench.stage_rooflines(m, n, k, N, 8, st, 1000.0)
    elems = 2 * m * k
    assert r["scale"]["algorithmic_bytes"] == elems * 8
    assert r["convert"]["algorithmic_bytes"] == elems * (8 + 2 * N)
    assert r["crt"]["algorithmic_bytes"] == m * n * (N + 8)
    assert abs(r["scale"]["achieved_gbs"] - elems * 8 / 1e-3 / 1e9) < 1e-6
    assert abs(r["crt"]["frac_of_hbm"] - m * n * (N + 8) / 1e-3 / 1e9 / 1000.0) < 1e-9
    assert "scale" not in bench.stage_rooflines(m, n, k, N, 8, st, 1000.0, "accurate")
