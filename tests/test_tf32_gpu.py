"""Parity of the 3xTF32 tensor-core Step 3 (TSQR_PREC_TF32X3, FP32 data).

Step 1 and the tree are those of the FP32 form; the Step-3 product Y_i W_i
runs on the tensor cores (tcgen05, kind::tf32) with Y and W split into TF32
high and low parts (three products, binary32 accumulation).  Bars: the FP32
form's (||Q^TQ - I||_2 <= 1e-5, ||A - QR||_F/||A||_F <= 1e-5, R and Q within
10 n kappa 2^-23 of the FP64 oracle on the upcast input).  n > 64 takes the
wide form (the running coefficient in binary64 in the workspace, the A
operands in two K halves), with the same bars.
"""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -23


def _run(A, **kw):
    import paper_1301_1071_gb300 as T
    Q, R = T.direct(torch.tensor(A, device="cuda"), prec="tf32x3", **kw)
    torch.cuda.synchronize()
    return Q.double().cpu().numpy(), R.cpu().numpy()


@pytest.mark.parametrize("m,n,b,f", [
    (100_000, 10, 1000, 0),
    (4099, 25, 0, 0),          # ragged last block
    (700, 25, 0, 0),           # one block
    (3000, 7, 64, 2),          # deep binary tree
    (513, 1, 0, 0),            # n = 1
    (37, 37, 0, 0),            # square
    (20_000, 50, 0, 0),
    (60_000, 50, 2999, 0),     # blocks of several register tiles
    (12_000, 64, 0, 0),        # largest n of the streaming form (16-row staggered staging)
    (50_000, 32, 0, 0),        # n % 8 == 0: staggered staging
    (1_000_000, 32, 0, 0),     # 50+ chunks per CTA: the copy warp trails the row groups by several chunks
    (30_000, 16, 1500, 0),     # n % 8 == 0, small n, blocks of several tiles
    (40_000, 8, 0, 0),
    (30_000, 48, 2500, 0),
    (25_000, 56, 0, 0),        # three Y buffers per group
    (30_000, 12, 0, 0),        # n % 8 == 4: 16-byte rows, row-major staging
    (20_000, 60, 0, 0),
    (30_000, 33, 0, 0),        # odd n: chunks with unaligned edges
    (100_003, 10, 1000, 0),    # last block of 3 rows (< n)
    (3000, 100, 0, 0),         # the wide form (n > 64), one block
    (20_000, 65, 0, 0),        # smallest wide n
    (40_000, 77, 3000, 0),     # wide, blocks of several tiles, odd n
    (30_000, 80, 0, 0),        # K = n, the Q stage at stride n + 1 exceeds the two K halves
    (25_000, 96, 2000, 0),     # wide, several tiles
    (60_000, 100, 0, 0),       # the largest n
    (30_001, 100, 4099, 0),    # ragged last block and last tile
    (200_000, 100, 2000, 0),   # three cluster tree levels (100 -> 13 -> 2 -> 1 nodes)
])
def test_tf32x3_parity(m, n, b, f):
    A = ti.gaussian(m, n, 3000 + m + n).astype(np.float32)
    Q, R = _run(A, block_rows=b, fanout=f)
    A64 = A.astype(np.float64)
    Qo, Ro = oracle.householder_qr(A64)
    kappa = np.linalg.cond(A64)
    tol = 10 * n * kappa * EPS32
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Q - Qo)) <= max(tol, 10 * n * EPS32)
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A64, Q, R)
    assert e2 <= 1e-5 and rF <= 1e-5, (e2, rF)


def test_tf32x3_column_scaled():
    """The mixed-precision workload's spectrum (column factors 1..1e-4)."""
    A = ti.column_scaled(200_000, 50, 1e-4, ti.SEED_MIXED).astype(np.float32)
    Q, R = _run(A)
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A.astype(np.float64), Q, R)
    assert e2 <= 1e-5 and rF <= 1e-5, (e2, rF)


def test_tf32x3_matches_fp32_form():
    """Same Step 1 and tree: the two Step-3 products agree to FP32 rounding."""
    import paper_1301_1071_gb300 as T
    A = torch.tensor(ti.gaussian(50_000, 40, 31).astype(np.float32), device="cuda")
    Qt, Rt = T.direct(A, prec="tf32x3")
    Qn, Rn = T.direct(A)
    assert float((Rt - Rn).abs().max()) == 0.0  # Step 1 and the tree are shared
    assert float((Qt - Qn).abs().max()) <= 1e-5


def test_tf32x3_svd():
    import paper_1301_1071_gb300 as T
    A = ti.power_spectrum(50_000, 20, 9).astype(np.float32)
    U, S, V = T.svd(torch.tensor(A, device="cuda"), prec="tf32x3")
    _, So, _ = oracle.svd(A.astype(np.float64))
    assert np.max(np.abs(S.cpu().numpy() - So) / So[0]) <= 1e-5
    e2, _ = oracle.orth_error(U.double().cpu().numpy())
    assert e2 <= 1e-5


def test_tf32x3_rejected_for_f64():
    import paper_1301_1071_gb300 as T
    with pytest.raises(T.TSQRError):
        T.direct(torch.randn(1000, 8, dtype=torch.float64, device="cuda"), prec="tf32x3")


@pytest.mark.parametrize("n", [10, 50, 64, 77])
def test_auto_precision_parity(n):
    """TSQR_PREC_AUTO: binary32 data at n >= 20 runs the 3xTF32 Step 3, below
    it the binary32 FMA Step 3; the result is bit for bit that of the mode it
    resolves to, and within the FP32 bars of the oracle."""
    import paper_1301_1071_gb300 as T
    A_np = ti.gaussian(30_000, n, 3100 + n).astype(np.float32)
    A = torch.tensor(A_np, device="cuda")
    Qa, Ra = T.direct(A, prec="auto")
    Qx, Rx = T.direct(A, prec="tf32x3" if n >= 20 else "native")
    torch.cuda.synchronize()
    assert torch.equal(Qa, Qx) and torch.equal(Ra, Rx)
    A64 = A_np.astype(np.float64)
    Qo, Ro = oracle.householder_qr(A64)
    tol = 10 * n * np.linalg.cond(A64) * EPS32
    Q, R = Qa.double().cpu().numpy(), Ra.cpu().numpy()
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Q - Qo)) <= tol
    assert oracle.orth_error(Q)[0] <= 1e-5


@pytest.mark.parametrize("n,mode", [(30, "ozaki"), (50, "native")])
def test_auto_precision_f64(n, mode):
    """Binary64 data: AUTO is the Ozaki form at n <= 32 and binary64 above,
    bit for bit."""
    import paper_1301_1071_gb300 as T
    A = torch.tensor(ti.gaussian(20_000, n, 3200 + n), device="cuda")
    Qa, Ra = T.direct(A, prec="auto")
    Qx, Rx = T.direct(A, prec=mode)
    assert torch.equal(Qa, Qx) and torch.equal(Ra, Rx)


def test_tf32x3_wide_svd():
    """The SVD variant at n = 100 (the benchmark's SVD width) with U formed
    by the wide tensor-core Step 3."""
    import paper_1301_1071_gb300 as T
    A = ti.power_spectrum(60_000, 100, 19).astype(np.float32)
    U, S, V = T.svd(torch.tensor(A, device="cuda"), prec="tf32x3")
    _, So, _ = oracle.svd(A.astype(np.float64))
    assert np.max(np.abs(S.cpu().numpy() - So) / So[0]) <= 1e-5
    e2, _ = oracle.orth_error(U.double().cpu().numpy())
    assert e2 <= 1e-5


def test_tf32x3_wide_host_buffers_match_device():
    """tsqr_direct_host with the wide tensor-core Step 3 (the coefficient
    updated in place chunk by chunk) equals tsqr_direct bit for bit."""
    import paper_1301_1071_gb300 as T
    m, n, b = 200_000, 90, 2500
    A = torch.tensor(ti.gaussian(m, n, 33).astype(np.float32))
    Qh, Rh = T.direct_host(A.pin_memory(), block_rows=b, prec="tf32x3")
    Qd, Rd = T.direct(A.cuda(), block_rows=b, prec="tf32x3")
    torch.cuda.synchronize()
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())


def test_tf32x3_misaligned_q_rejected():
    """Q must start on a 16-byte boundary (the chunk stream's bulk copies and
    vector row accesses rely on it): a pointer 4 bytes past one is refused
    on the host with TSQR_ERR_ALIGN, before any launch."""
    import paper_1301_1071_gb300 as T
    m, n = 5000, 24
    A = torch.tensor(ti.gaussian(m, n, 64).astype(np.float32), device="cuda")
    Qm = torch.empty(m * n + 1, dtype=torch.float32, device="cuda")[1:].view(m, n)
    Rm = torch.empty(n, n, dtype=torch.float64, device="cuda")
    assert Qm.data_ptr() % 16 == 4
    with pytest.raises(T.TSQRError, match="ALIGN"):
        T.direct(A, prec="tf32x3", out=(Qm, Rm))


@pytest.mark.parametrize("n", [25, 64])
def test_tf32x3_host_buffers_match_device(n):
    """tsqr_direct_host with the n <= 64 chunk stream (the W chain and the
    stream per batch of blocks) equals tsqr_direct bit for bit."""
    import paper_1301_1071_gb300 as T
    m, b = 300_000, 3000
    A = torch.tensor(ti.gaussian(m, n, 35 + n).astype(np.float32))
    Qh, Rh = T.direct_host(A.pin_memory(), block_rows=b, prec="tf32x3")
    Qd, Rd = T.direct(A.cuda(), block_rows=b, prec="tf32x3")
    torch.cuda.synchronize()
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())
