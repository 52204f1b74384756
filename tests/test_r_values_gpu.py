"""Parity of the R-only and singular-value-only paths with the oracle.

* tsqr_r (Sec. II-B, the R-only TSQR reduction): R element-wise against the
  oracle's R over several row blocks, ragged last blocks, multi-level trees,
  n = 1 and square A, blocks of several register tiles, FP32 data and
  double-float compute; its R is the R of tsqr_direct computed the same way
  (same plan, same kernels without the Householder vectors), so the two must
  agree bit for bit.
* tsqr_svd_values (Sec. III-B, SVD paragraph: Steps 1-2 and the SVD of R):
  S and V against the oracle's SVD and against tsqr_svd's S and V; V may be
  omitted.
* The full 8,000,000 x 25 FP64 matrix of the stability sweep in the default
  plan: R against the oracle's R.

Bars as for tsqr_direct: FP64 ||R - R_o||_F / ||R_o||_F <= 10 n kappa 2^-52,
FP32 the same with 2^-23, double-float with 2^-48.
"""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23
EPSDF = 2.0 ** -48


def _T():
    import paper_1301_1071_gb300 as T
    return T


def _cuda(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _check_r(R, Ro, tol):
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    rerr = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    assert rerr <= tol, f"R error {rerr:.3e} > {tol:.3e}"


R_SHAPES = [
    # (m, n, block_rows, fanout, kappa)
    (100_000, 10, 1000, 0, 1.0),   # 100 blocks of 1,000 rows
    (4099, 25, 0, 0, 1e8),         # ragged last block
    (700, 25, 0, 0, 1.0),          # one block
    (3000, 7, 64, 2, 1e4),         # binary tree, several levels
    (2500, 13, 50, 3, 1.0),        # odd n, fanout 3, ragged levels
    (513, 1, 0, 0, 1.0),           # n = 1
    (37, 37, 0, 0, 1.0),           # square
    (60_000, 20, 7001, 0, 1e12),   # blocks of several register tiles
    (30_000, 100, 0, 0, 1e4),      # n = NMAX
    (60_000, 100, 1000, 0, 1e8),   # cluster tree nodes (8 triangles, one per CTA)
    (45_000, 90, 500, 6, 1.0),     # clusters of 6, ragged levels
]


@pytest.mark.parametrize("m,n,b,f,kappa", R_SHAPES)
def test_r_parity_f64(m, n, b, f, kappa):
    A = ti.conditioned(m, n, kappa, ti.SEED_SWEEP) if n > 1 else ti.gaussian(m, n, ti.SEED_SWEEP)
    T = _T()
    Ad = _cuda(A)
    R = T.r(Ad, block_rows=b, fanout=f)
    torch.cuda.synchronize()
    Ro = oracle.householder_r(A)
    kappa = max(kappa, float(np.linalg.cond(Ro)))  # realised condition (square A: not 1)
    _check_r(R.cpu().numpy(), Ro, 10 * n * kappa * EPS64)
    # the same plan and kernels as tsqr_direct, without Y, T and Q2
    _, Rd = T.direct(Ad, block_rows=b, fanout=f)
    assert torch.equal(R, Rd)


@pytest.mark.parametrize("m,n,b", [(50_000, 20, 0), (40_000, 64, 0), (30_001, 50, 9000)])
def test_r_parity_f32(m, n, b):
    A = ti.column_scaled(m, n, 1e-4, ti.SEED_MIXED).astype(np.float32)
    R = _T().r(_cuda(A, torch.float32), block_rows=b)
    Ro = oracle.householder_r(A.astype(np.float64))
    kappa = float(np.linalg.cond(Ro))
    _check_r(R.cpu().numpy(), Ro, 10 * n * kappa * EPS32)


@pytest.mark.parametrize("m,n", [(60_000, 25), (20_000, 64)])
def test_r_parity_df64(m, n):
    A = ti.conditioned(m, n, 1e8, ti.SEED_SWEEP)
    Ad = _cuda(A)
    R = _T().r(Ad, prec="df64")
    _check_r(R.cpu().numpy(), oracle.householder_r(A), 10 * n * 1e8 * EPSDF)
    _, Rd = _T().direct(Ad, prec="df64")
    assert torch.equal(R, Rd)


@pytest.mark.parametrize("m,n,seed", [(20_000, 10, 1), (5000, 25, 2), (4000, 50, 4), (60_000, 20, 5)])
def test_svd_values_parity(m, n, seed):
    A = ti.power_spectrum(m, n, seed)
    T = _T()
    Ad = _cuda(A)
    S, V = T.svd_values(Ad)
    S, V = S.cpu().numpy(), V.cpu().numpy()
    _, So, Vo = oracle.svd(A)
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(S - So) / So[0]) <= 10 * n * EPS64
    gap = np.min(np.abs(np.diff(So))) / So[0]
    assert np.max(np.abs(V - Vo)) <= 100 * n * EPS64 / gap
    # the same R and the same Jacobi method as tsqr_svd: identical S and V
    _, S2, V2 = T.svd(Ad)
    assert np.array_equal(S, S2.cpu().numpy()) and np.array_equal(V, V2.cpu().numpy())
    # S alone
    S3, none = T.svd_values(Ad, want_v=False)
    assert none is None and np.array_equal(S3.cpu().numpy(), S)


def test_svd_values_f32_storage():
    m, n = 50_000, 20
    A = ti.power_spectrum(m, n, 9).astype(np.float32)
    S, _ = _T().svd_values(_cuda(A, torch.float32))
    _, So, _ = oracle.svd(A.astype(np.float64))
    assert np.max(np.abs(S.cpu().numpy() - So) / So[0]) <= 1e-5


def test_r_argument_errors():
    T = _T()
    A = torch.randn(1000, 10, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TSQRError):
        T.r(A, block_rows=5)            # block shorter than n
    with pytest.raises(T.TSQRError):
        T.svd_values(A, prec="tf32x3")  # TF32X3 is for FP32 data
    lib = T.load()
    R = torch.empty(10, 10, dtype=torch.float64, device="cuda")
    st = lib.tsqr_r(T._ptr(A), 1000, 10, 10, T.F64, T._ptr(R), 10, None, 0, None, T._stream(A.device))
    assert st == 4  # TSQR_ERR_WORKSPACE
    st = lib.tsqr_r(T._ptr(A), 1000, 10, 10, T.F64, T._ptr(R), 9, None, 0, None, T._stream(A.device))
    assert st == 3  # TSQR_ERR_ALIGN


def test_r_fullsize_sweep_matrix():
    """8,000,000 x 25 FP64, kappa 1e15, default plan: R against the oracle."""
    m, n, kappa = 8_000_000, 25, 1e15
    A_np = ti.conditioned(m, n, kappa, ti.SEED_SWEEP)
    R = _T().r(torch.tensor(A_np, device="cuda")).cpu().numpy()
    _check_r(R, oracle.householder_r(A_np), 10 * n * kappa * EPS64)
