"""Parity of the CUDA direct TSQR (Sec. III-B, Alg. 2) with the CPU oracle.

Element-wise comparison of Q and R on seeded inputs that span several row
blocks, ragged last blocks, a single block (p = 1), multi-level trees (Alg. 2
recursion), odd n, n = 1 and square A, in binary64 and binary32.

FP64 bar (stated for the path): ||R - R_oracle||_F / ||R||_F <= 10 n kappa 2^-52,
||Q^T Q - I||_2 <= 1e-13, ||A - QR||_F / ||A||_F <= 1e-13; element-wise
|Q - Q_oracle| <= 10 n kappa 2^-52 (both are backward-stable Householder
factorisations of the same A, so they agree to O(n kappa eps)).
FP32 bar: ||Q^T Q - I||_2 <= 1e-5 for kappa <= 1e5, residual <= 1e-5; R and
Q within 10 n kappa 2^-23 of the FP64 oracle on the upcast input.
"""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23


def _tsqr():
    import paper_1301_1071_gb300 as T
    return T


def _run(A_np, dtype, **kw):
    T = _tsqr()
    A = torch.tensor(A_np, dtype=dtype, device="cuda")
    Q, R = T.direct(A, **kw)
    torch.cuda.synchronize()
    return Q.double().cpu().numpy(), R.cpu().numpy()


def _check(A_np, Q, R, kappa, dtype):
    m, n = A_np.shape
    A64 = np.asarray(A_np, dtype=np.float64)
    Qo, Ro = oracle.householder_qr(A64)
    eps = EPS64 if dtype == torch.float64 else EPS32
    tol = 10 * n * kappa * eps
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    rerr = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    assert rerr <= tol, f"R error {rerr:.3e} > {tol:.3e}"
    qerr = np.max(np.abs(Q - Qo))
    assert qerr <= max(tol, 10 * n * eps), f"Q element error {qerr:.3e}"
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A64, Q, R)
    if dtype == torch.float64:
        assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)
    else:
        assert e2 <= 1e-5 and rF <= 1e-5, (e2, rF)


SHAPES = [
    # (m, n, block_rows, fanout)
    (100_000, 10, 1000, 0),   # the small workload: 100 blocks of 1,000 rows
    (4099, 25, 0, 0),         # ragged last block
    (700, 25, 0, 0),          # p = 1 (one block)
    (3000, 7, 64, 2),         # binary tree, several levels
    (2500, 13, 50, 3),        # odd n, fanout 3, ragged levels
    (513, 1, 0, 0),           # n = 1
    (37, 37, 0, 0),           # square
    (20_000, 50, 0, 0),
    (12_000, 64, 0, 0),
    (3000, 100, 0, 0),
    # blocks taller than the register tile: in-CTA flat tree of tiles
    (203_457, 25, 5000, 0),   # 41 blocks, ragged last block of one tile
    (150_001, 10, 12_345, 0), # last block of several tiles, last tile short
    (60_000, 50, 2999, 0),
    (30_000, 100, 1500, 0),   # many tiles of few rows (binary64: 28 per tile)
    (30_000, 32, 2500, 0),    # carried R fills one 32-row register slice
    (50_000, 33, 3000, 0),    # carried R padded to two slices (rows 33..63 zero)
    (40_000, 64, 2000, 0),
    (30_000, 56, 0, 0),       # the wide register tile (8 columns per thread, 50 < n <= 64)
    (25_000, 51, 3000, 0),    # wide tile, padded columns, several tiles per block
    (40_000, 77, 2500, 0),    # 10 columns per thread (n > 64), padded, several tiles per block
    # n > 84: tree nodes of 8 triangles on a cluster of 8 CTAs (one triangle each)
    (60_000, 100, 1000, 0),   # 60 blocks: levels of 8, 1 nodes (ragged: 8 x 7 + 4)
    (60_000, 100, 1000, 5),   # fanout 5 on clusters of 5, ragged levels (12 -> 3 -> 1)
    (30_000, 100, 1500, 2),   # fanout 2: one CTA per node
    (45_000, 90, 500, 0),     # 90 blocks, three cluster levels, a node of 2 blocks
    (1_000_003, 25, 0, 0),    # default block height (two tiles per block)
]


@pytest.mark.parametrize("m,n,b,f", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_direct_parity_gaussian(m, n, b, f, dtype):
    A = ti.gaussian(m, n, 1000 + m + n)
    if dtype == torch.float32:
        A = A.astype(np.float32)
    Q, R = _run(A, dtype, block_rows=b, fanout=f)
    kappa = np.linalg.cond(np.asarray(A, dtype=np.float64))
    _check(A, Q, R, kappa, dtype)


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8, 1e12, 1e15])
def test_direct_parity_conditioned_f64(kappa):
    A = ti.conditioned(50_000, 25, kappa, ti.SEED_SWEEP)
    Q, R = _run(A, torch.float64)
    m, n = A.shape
    Qo, Ro = oracle.householder_qr(A)
    rerr = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    assert rerr <= 10 * n * kappa * EPS64
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A, Q, R)
    assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)


def test_direct_is_deterministic():
    A = torch.tensor(ti.gaussian(30_000, 25, 5), device="cuda")
    T = _tsqr()
    Q1, R1 = T.direct(A)
    Q2, R2 = T.direct(A)
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


def test_direct_zero_column():
    A = ti.gaussian(5000, 6, 77)
    A[:, 3] = 0.0
    Q, R = _run(A, torch.float64)
    assert R[3, 3] == 0.0
    rF, _ = oracle.residual(A, Q, R)
    assert rF <= 1e-14


def test_direct_rejects_bad_arguments():
    T = _tsqr()
    with pytest.raises(ValueError):
        T.direct(torch.zeros(3, 5, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        T.direct(torch.zeros(300, 101, dtype=torch.float64, device="cuda"))
    A = torch.randn(1000, 10, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TSQRError):
        T.direct(A, block_rows=5)          # block_rows < n
    with pytest.raises(T.TSQRError):
        T.direct(A, block_rows=-1)
    # a block taller than the matrix is one block (factored tile by tile)
    Q, R = T.direct(A, block_rows=10**7)
    Qd, Rd = T.direct(A)
    assert float((R - Rd).abs().max()) <= 1e-13 * float(Rd.abs().max())
