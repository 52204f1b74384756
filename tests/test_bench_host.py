"""bench.py's host-only parts (no GPU): the oracle timings it reports beside
the device numbers, and the JSON line of the reference arm (the oracle timed
on the host cores on a bounded sample of the workload)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_cpu_config_baselines_report_every_configuration():
    out = bench.cpu_config_baselines(target_s=0.2)
    for name in ("small_100kx10", "mixed_50Mx50_upcast", "svd_20Mx100", "grad_4Mx64"):
        e = out[name]
        assert "error" not in e, e
        assert e["value"] > 0 and e["unit"] == "rows/s" and e["cores"] == (os.cpu_count() or 1)
        assert e["kind"] == "oracle" and "rows" in e["sample"]
    assert out["small_100kx10"]["serial"]["cores"] == 1
    assert out["numpy_lapack_qr_8Mx25"]["value"] > 0
    assert out["memory_peak_mb"] > 0


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--workload", "small"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "rows/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_paper_context_restates_table_vi():
    """The paper's direct-TSQR job times (Sec. V-B, Table VI) reported as
    context: rows/s = rows / job seconds (e.g. 600,000,000 x 25 in 1,910 s)."""
    ctx = bench.PAPER_CONTEXT
    json.dumps(ctx)
    rows = {(r["m"], r["n"]): r for r in ctx["direct_tsqr"]}
    assert rows[(600_000_000, 25)]["job_s"] == 1910
    assert abs(rows[(600_000_000, 25)]["rows_s"] - 3.1414e5) < 1e2
    assert abs(rows[(4_000_000_000, 4)]["rows_s"] - 6.527e5) < 1e2
    assert len(rows) == 5 and "40 cores" in ctx["machine"]
