"""Parity of the Ozaki-split tensor-core Step 3 (TSQR_PREC_OZAKI, FP64 data).

Step 1 and the Step-2 tree are the binary64 ones, so R is bit for bit that
of the native form; the Step-3 product Y_i W_i runs on the tensor cores as
an error-free split product (7 digits of 8 bits per row of Y and column of
W, exact binary32 accumulation of binary16 digit products, one rounding to
binary64).  Bars: the FP64 ones (||R - R_oracle||_F/||R||_F and |Q - Q_oracle|
element-wise <= 10 n kappa 2^-52, ||Q^TQ - I||_2 <= 1e-13 and
||A - QR||_F/||A||_F <= 1e-13 at every kappa up to 1e15).  Above n = 32 the
native binary64 Step 3 runs and the result equals the native one bit for bit.
"""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52


def _T():
    import paper_1301_1071_gb300 as T
    return T


def _check(A, Q, R, kappa):
    m, n = A.shape
    Qo, Ro = oracle.householder_qr(A)
    tol = 10 * n * kappa * EPS64
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    rerr = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    assert rerr <= tol, rerr
    qerr = np.max(np.abs(Q - Qo))
    assert qerr <= max(tol, 10 * n * EPS64), qerr
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A, Q, R)
    assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)


SHAPES = [
    # (m, n, block_rows, fanout)
    (100_000, 10, 1000, 0),    # the small workload: 100 blocks of 1,000 rows
    (4099, 25, 0, 0),          # ragged last block
    (700, 25, 0, 0),           # p = 1 (one block)
    (3000, 7, 64, 2),          # binary tree, several levels
    (2500, 13, 50, 3),         # odd n, fanout 3, ragged levels
    (513, 1, 0, 0),            # n = 1
    (32, 32, 0, 0),            # square, the largest n of the tensor-core form
    (20_000, 16, 0, 0),        # K = 16 operands
    (20_000, 17, 0, 0),        # K = 32 operands, 15 padded columns
    (203_457, 25, 5000, 0),    # blocks of several tiles, ragged last block of one tile
    (150_001, 10, 12_345, 0),  # last block of several tiles, last tile short
    (30_000, 32, 2500, 0),     # tiles whose rows are not a multiple of the 128-row chunk
    (1_000_003, 25, 0, 0),     # the default plan on a million rows
]


@pytest.mark.parametrize("m,n,b,f", SHAPES)
def test_ozaki_parity(m, n, b, f):
    T = _T()
    A = ti.gaussian(m, n, 6000 + n + m % 1000)
    Ad = torch.tensor(A, device="cuda")
    Q, R = T.direct(Ad, block_rows=b, fanout=f, prec="ozaki")
    Qn, Rn = T.direct(Ad, block_rows=b, fanout=f)
    torch.cuda.synchronize()
    assert torch.equal(R, Rn)  # Step 1 and the tree are the binary64 ones
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    _check(A, Qh, Rh, np.linalg.cond(A))
    # the two Step-3 products agree to binary64 rounding
    assert float((Q - Qn).abs().max()) <= 10 * n * EPS64


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8, 1e12, 1e15])
def test_ozaki_stability_sweep(kappa):
    """The stability sweep (Sec. IV): orthogonality and residual stay at the
    binary64 level at every kappa, like the native form."""
    T = _T()
    A = ti.conditioned(200_000, 25, kappa, 6100)
    Ad = torch.tensor(A, device="cuda")
    Q, R = T.direct(Ad, prec="ozaki")
    torch.cuda.synchronize()
    _check(A, Q.cpu().numpy(), R.cpu().numpy(), kappa)


def test_ozaki_wide_dynamic_range():
    """Column factors spanning 1 .. 1e-12 within each row: each row of Y is
    split against its own largest exponent, so small entries keep only the
    digits below it -- the error bound is normwise, which the FP64 bars
    are."""
    T = _T()
    A = ti.column_scaled(100_000, 20, 1e-12, 6200)
    Ad = torch.tensor(A, device="cuda")
    Q, R = T.direct(Ad, prec="ozaki")
    torch.cuda.synchronize()
    Qh = Q.cpu().numpy()
    e2, _ = oracle.orth_error(Qh)
    rF, _ = oracle.residual(A, Qh, R.cpu().numpy())
    assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)


@pytest.mark.parametrize("n", [33, 50])
def test_ozaki_above_32_is_native(n):
    T = _T()
    Ad = torch.tensor(ti.gaussian(20_000, n, 6300 + n), device="cuda")
    Q, R = T.direct(Ad, prec="ozaki")
    Qn, Rn = T.direct(Ad)
    assert torch.equal(Q, Qn) and torch.equal(R, Rn)


def test_ozaki_deterministic():
    T = _T()
    Ad = torch.tensor(ti.conditioned(300_000, 25, 1e12, 6400), device="cuda")
    Q1, R1 = T.direct(Ad, prec="ozaki")
    Q2, R2 = T.direct(Ad, prec="ozaki")
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


def test_ozaki_svd():
    """The SVD variant with U = Q U_R formed by the split product."""
    T = _T()
    m, n = 50_000, 20
    A = ti.power_spectrum(m, n, 6500)
    U, S, V = T.svd(torch.tensor(A, device="cuda"), prec="ozaki")
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    Uo, So, Vo = oracle.svd(A)
    assert np.max(np.abs(S - So) / So[0]) <= 10 * n * EPS64
    gap = np.min(np.abs(np.diff(So))) / So[0]
    tolv = 100 * n * EPS64 / gap
    assert np.max(np.abs(V - Vo)) <= tolv and np.max(np.abs(U - Uo)) <= tolv
    assert oracle.orth_error(U)[0] <= 1e-13


def test_ozaki_host_buffers_match_device():
    """tsqr_direct_host with the split product equals tsqr_direct's bit for
    bit on the same row blocks."""
    T = _T()
    m, n, b = 400_000, 25, 4000
    A = torch.tensor(ti.gaussian(m, n, 6600))
    Qh, Rh = T.direct_host(A.pin_memory(), block_rows=b, prec="ozaki")
    Qd, Rd = T.direct(A.cuda(), block_rows=b, prec="ozaki")
    torch.cuda.synchronize()
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())


def test_ozaki_rejected_for_f32():
    T = _T()
    with pytest.raises(T.TSQRError):
        T.direct(torch.randn(1000, 8, dtype=torch.float32, device="cuda"), prec="ozaki")
