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


class _FakeEvent:
    def __init__(self, enable_timing=False):
        pass

    def record(self):
        pass

    def elapsed_time(self, other):
        return 2.0


class _FakeTensor:
    def __init__(self, a):
        self.a = a

    def to(self, dev):
        return self


class _FakeTorch:
    class cuda:
        Event = _FakeEvent

        @staticmethod
        def synchronize():
            pass

        @staticmethod
        def empty_cache():
            pass

    @staticmethod
    def from_numpy(a):
        return _FakeTensor(a)


class _FakeLib:
    """Stands in for the CUDA binding: Cholesky QR breaks down from kappa
    1e12 on, the way the method does (Sec. IV)."""
    STATUS = {6: "TSQR_ERR_NOT_SPD"}

    class TSQRError(RuntimeError):
        def __init__(self, status):
            super().__init__(status)
            self.status = status

    def _qr(self, A):
        return A, None

    def direct(self, A, check=True, prec="native"):
        return self._qr(A)

    def cholqr(self, A, refine=0, check=True):
        kappa = float(A.a[0, 0])
        if check and kappa >= 1e12:
            raise self.TSQRError(6)
        return self._qr(A)

    def indirect_refine(self, A, refine=1, check=True):
        return self._qr(A)

    def accuracy(self, Q, R=None, A=None):
        return {"orth_2": 1e-16, "orth_F": 1e-16, "res_F": 1e-16, "res_2": 1e-16}


def test_stability_sweep_table_shape(monkeypatch):
    """The bench's stability table (Sec. IV) run against stand-ins for torch
    and the binding: one row per kappa, every method with its accuracy, rate,
    algorithmic GB/s and HBM fraction, and a breakdown reported as a status."""
    import numpy as np
    monkeypatch.setattr(bench.ti, "conditioned", lambda m, n, kappa, seed: np.full((2, 2), kappa))
    out = bench.stability_sweep(_FakeLib(), _FakeTorch, "cpu", A15=None, steps=2, m=1000, n=25)
    assert list(out["by_kappa"]) == ["1e+00", "1e+04", "1e+08", "1e+12", "1e+15"]
    peak, _ = bench.load_peaks()
    for kappa, row in out["by_kappa"].items():
        assert set(row) == {"direct", "direct_native", "cholqr", "cholqr_ir", "indirect_ir"}
        for name, e in row.items():
            assert "error" not in e, (kappa, name, e)
            if name.startswith("cholqr") and float(kappa) >= 1e12:
                assert e["status"] == "TSQR_ERR_NOT_SPD"
                continue
            assert e["ms"] == 1.0 and abs(e["rows_s"] - 1e6) < 1e-6
            assert abs(e["hbm_frac"] - e["hbm_gbs_algorithmic"] / peak) < 1e-12


def test_guarded_extras_record_errors_instead_of_raising():
    def boom(x, y=0):
        raise MemoryError(f"out of memory {x} {y}")
    out = bench.guarded(_FakeTorch, boom, 3, y=4)
    assert out == {"error": "MemoryError: out of memory 3 4"}
    assert bench.guarded(_FakeTorch, lambda a, b: {"v": a + b}, 1, 2) == {"v": 3}
