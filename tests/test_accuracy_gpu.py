"""tsqr_accuracy: the accuracy metrics of Sec. I-B (||Q^T Q - I||_2,
||A - QR||_2/||R||_2, ||A - QR||_F/||A||_F) accumulated on the device with
compensated (Dot2) sums.  Checked against the oracle's checkers (Dot2 Grams
and long-double Jacobi eigenvalues) on the same inputs, on known answers,
and on a cancellation that plain binary64 sums cannot resolve."""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _T():
    import paper_1301_1071_gb300 as T
    return T


def _close(a, b, rel=1e-6, abs_=1e-30):
    return abs(a - b) <= rel * abs(b) + abs_


@pytest.mark.parametrize("m,n,kappa,seed", [(100_000, 10, 1.0, 1), (300_000, 25, 1e15, 2), (20_000, 100, 1e8, 3),
                                            (5, 1, 1.0, 4), (777, 37, 1e4, 5)])
def test_accuracy_matches_oracle_checkers(m, n, kappa, seed):
    A = ti.conditioned(m, n, kappa, 5000 + seed) if n > 1 else ti.gaussian(m, n, 5000 + seed)
    Q, R = oracle.householder_qr(A)
    Q = Q * (1.0 + 1e-12 * ti.gaussian(m, n, 5100 + seed))  # an orthogonality error well above rounding
    got = _T().accuracy(torch.tensor(Q, device="cuda"), torch.tensor(R, device="cuda"), torch.tensor(A, device="cuda"))
    e2, eF = oracle.orth_error(Q)
    rF, r2 = oracle.residual(A, Q, R)
    assert _close(got["orth_2"], e2) and _close(got["orth_F"], eF), (got, e2, eF)
    assert _close(got["res_F"], rF, 1e-5) and _close(got["res_2"], r2, 1e-5), (got, rF, r2)


def test_accuracy_known_answer():
    """Q = H (I + delta E) with exactly orthonormal H: Q^T Q - I = 2 delta E +
    delta^2 E^2, a diagonal of known eigenvalues."""
    n = 6
    h = np.array([[1.0]])
    for _ in range(3):
        h = np.block([[h, h], [h, -h]])
    H = np.tile(h[:, :n], (2048, 1)) / 128.0  # 16,384 x 6, exactly orthonormal columns
    E = np.diag([3.0, -1.0, 0.5, 0.0, 2.0, 1.0])
    delta = 1e-13
    Q = H @ (np.eye(n) + delta * E)
    got = _T().accuracy(torch.tensor(Q, device="cuda"))
    want = 2 * delta * 3.0 + delta ** 2 * 9.0
    assert abs(got["orth_2"] - want) <= 1e-3 * want, got
    assert _T().accuracy(torch.tensor(H, device="cuda"))["orth_2"] == 0.0  # every sum is exact


def test_accuracy_resolves_cancellation():
    """Entries of 1e16 that cancel, next to entries of 1: the Gram of the
    columns is exact only with compensated sums."""
    x = np.zeros((4096, 2))
    x[0::4, 0] = 1e16
    x[2::4, 0] = -1e16
    x[1::4, 0] = 1.0
    x[3::4, 0] = 1.0
    x[:, 1] = 1.0
    got = _T().accuracy(torch.tensor(x, device="cuda"))
    G = oracle.gram_dot2(x, x)
    E = G - np.eye(2)
    assert _close(got["orth_2"], float(np.max(np.abs(np.linalg.eigvalsh(E)))), 1e-12)


def test_accuracy_fp32_data():
    A = ti.gaussian(50_000, 20, 5200).astype(np.float32)
    Q, R = oracle.householder_qr(A.astype(np.float64))
    Q32 = Q.astype(np.float32)
    got = _T().accuracy(torch.tensor(Q32, device="cuda"), torch.tensor(R, device="cuda"),
                        torch.tensor(A, device="cuda"))
    e2, _ = oracle.orth_error(Q32.astype(np.float64))
    rF, r2 = oracle.residual(A.astype(np.float64), Q32.astype(np.float64), R)
    assert _close(got["orth_2"], e2) and _close(got["res_F"], rF, 1e-5) and _close(got["res_2"], r2, 1e-5)


def test_accuracy_on_a_slice_of_the_sweep_matrix():
    """The bench's checker against the oracle's on the first 1,000,000 rows
    of the 8,000,000 x 25 stability-sweep matrix at kappa 1e15, factored by
    direct TSQR on the device."""
    T = _T()
    A = ti.conditioned(8_000_000, 25, 1e15, ti.SEED_SWEEP, rows=1_000_000)
    Ad = torch.tensor(A, device="cuda")
    Q, R = T.direct(Ad)
    got = T.accuracy(Q, R, Ad)
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    e2, _ = oracle.orth_error(Qh)
    rF, r2 = oracle.residual(A, Qh, Rh)
    assert _close(got["orth_2"], e2) and _close(got["res_F"], rF, 1e-5) and _close(got["res_2"], r2, 1e-5)
    assert got["orth_2"] <= 1e-13 and got["res_F"] <= 1e-13
