"""Full-size checks at the benchmark configurations (8,000,000 x 25 FP64, the
stability-sweep matrix), in the launch configuration bench.py times (the
planner's default block height).

The oracle cannot form Q at this size in a test's time, so the checks are the
properties that hold at any size plus the parts the oracle computes directly:
R from the oracle's R-only Householder QR (the same unique factor, Sec. II-A),
and, for kappa = 1 where Q = A R^{-1} is well conditioned, sampled rows of Q
against A_r R_oracle^{-1} computed one by one by the oracle's row solver.
"""
import os

import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, N = 8_000_000, 25
EPS64 = 2.0 ** -52


def _gram_orth_resid(A, Q, R):
    """||Q^T Q - I||_2 and ||A - QR||_F / ||A||_F from the library's
    compensated (Dot2) device sums: accurate at the 1e-15 level at any m,
    where plain binary64 sums over 8e6 rows err by ~sqrt(m) eps."""
    import paper_1301_1071_gb300 as T
    acc = T.accuracy(Q, R, A)
    return acc["orth_2"], acc["res_F"]


@pytest.mark.parametrize("kappa", [1.0, 1e15])
def test_fullsize_sweep_matrix(kappa):
    import paper_1301_1071_gb300 as T
    A_np = ti.conditioned(M, N, kappa, ti.SEED_SWEEP)
    A = torch.tensor(A_np, device="cuda")
    Q, R = T.direct(A)  # default plan, as timed by bench.py
    torch.cuda.synchronize()
    Rn = R.cpu().numpy()
    assert np.all(np.tril(Rn, -1) == 0.0) and np.all(np.diag(Rn) >= 0.0)
    e2, rF = _gram_orth_resid(A, Q, R)
    assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)
    Ro = oracle.householder_r(A_np)
    rerr = np.linalg.norm(Rn - Ro) / np.linalg.norm(Ro)
    assert rerr <= 10 * N * kappa * EPS64, rerr
    if kappa == 1.0:
        # sampled rows of Q, one by one, against A_r R_o^{-1}
        rng = np.random.default_rng(ti.SEED_SWEEP)
        rows = np.sort(rng.choice(M, size=2000, replace=False))
        Qo_rows = oracle.right_solve_upper(A_np[rows], Ro)
        assert np.max(np.abs(Q[torch.tensor(rows, device="cuda")].cpu().numpy() - Qo_rows)) <= 10 * N * EPS64


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-4)])
def test_fullsize_gradient_4Mx64(dtype, tol):
    """The differentiation workload at full size: 4,000,000 x 64 N(0,1), row
    blocks of 4,096, cotangents W_Q, W_R ~ N(0,1) with dR = triu(W_R).  The
    device forward (direct TSQR) + adjoint (tsqr_backward) against the
    oracle's adjoint formula evaluated on the oracle's own Q and R of the
    same (upcast) matrix; bars 1e-12 (FP64) and 1e-4 (FP32) relative in the
    Frobenius norm."""
    import paper_1301_1071_gb300 as T
    m, n = 4_000_000, 64
    A = ti.gaussian(m, n, ti.SEED_GRAD).astype(dtype)
    WQ = ti.gaussian(m, n, ti.SEED_GRAD + 2).astype(dtype)
    WR = ti.gaussian(n, n, ti.SEED_GRAD + 3)
    Ad = torch.tensor(A, device="cuda")
    Q, R = T.direct(Ad, block_rows=4096)
    dA = T.backward(Q, R, torch.tensor(WQ, device="cuda"), torch.tensor(WR, device="cuda")).double().cpu().numpy()
    del Q, Ad
    prev = oracle.num_threads()
    oracle.set_num_threads(os.cpu_count() or 1)
    try:
        Qo, Ro = oracle.householder_qr(A.astype(np.float64))
        dAo = oracle.qr_backward(Qo, Ro, WQ.astype(np.float64), np.triu(WR))
    finally:
        oracle.set_num_threads(prev)
    err = np.linalg.norm(dA - dAo) / np.linalg.norm(dAo)
    assert err <= tol, err
