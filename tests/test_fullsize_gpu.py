"""Full-size checks at the benchmark configuration (8,000,000 x 25 FP64, the
stability-sweep matrix), in the launch configuration bench.py times (the
planner's default block height).

The oracle cannot form Q at this size in a test's time, so the checks are the
properties that hold at any size plus the parts the oracle computes directly:
R from the oracle's R-only Householder QR (the same unique factor, Sec. II-A),
and, for kappa = 1 where Q = A R^{-1} is well conditioned, sampled rows of Q
against A_r R_oracle^{-1} computed one by one by the oracle's row solver.
"""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, N = 8_000_000, 25
EPS64 = 2.0 ** -52


def _gram_orth_resid(A, Q, R):
    """||Q^T Q - I||_2 and ||A - QR||_F / ||A||_F in binary64 on the device,
    accumulated in chunks of 2^20 rows."""
    n = Q.shape[1]
    G = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    num = den = 0.0
    for r0 in range(0, Q.shape[0], 1 << 20):
        q = Q[r0:r0 + (1 << 20)]
        a = A[r0:r0 + (1 << 20)]
        G += q.T @ q
        num += float(((a - q @ R) ** 2).sum())
        den += float((a ** 2).sum())
    G -= torch.eye(n, dtype=torch.float64, device="cuda")
    return float(torch.linalg.eigvalsh(G.cpu()).abs().max()), (num / den) ** 0.5


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
