"""Parity of the double-float (df64) compute mode of direct TSQR with the oracle.

FP64 data, Steps 1 and 3 in pair-of-binary32 arithmetic (unit roundoff
u = 2^-48), tree and n x n work in binary64.  Bars: ||Q^T Q - I||_2 <= 1e-13
and ||A - QR||_F / ||A||_F <= 1e-13 for kappa up to 1e15 (the FP64 path's
accuracy bars); ||R - R_oracle||_F / ||R||_F <= 10 n kappa 2^-48 and
element-wise |Q - Q_oracle| <= 10 n kappa 2^-48 (the FP64 bound with the
df64 unit roundoff).
"""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U48 = 2.0 ** -48


def _direct(A, **kw):
    import paper_1301_1071_gb300 as T
    Q, R = T.direct(torch.tensor(A, device="cuda"), prec="df64", **kw)
    return Q.cpu().numpy(), R.cpu().numpy()


@pytest.mark.parametrize("m,n,b,f", [(100_000, 10, 1000, 0), (4099, 25, 0, 0), (3000, 7, 64, 2),
                                     (20_000, 50, 0, 0), (3000, 100, 0, 0), (513, 1, 0, 0),
                                     (203_457, 25, 5000, 0), (60_000, 50, 2999, 0), (40_000, 60, 3000, 0)])
def test_df64_parity_gaussian(m, n, b, f):
    A = ti.gaussian(m, n, 2000 + m + n)
    Q, R = _direct(A, block_rows=b, fanout=f)
    Qo, Ro = oracle.householder_qr(A)
    kappa = np.linalg.cond(A)
    tol = 10 * n * kappa * U48
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Q - Qo)) <= tol
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A, Q, R)
    assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8, 1e12, 1e15])
def test_df64_stability_sweep(kappa):
    """The stability-sweep matrix (G diag(sigma) V^T, n = 25) at every kappa."""
    A = ti.conditioned(200_000, 25, kappa, ti.SEED_SWEEP)
    Q, R = _direct(A)
    Qo, Ro = oracle.householder_qr(A)
    r_err = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    assert r_err <= 10 * 25 * kappa * U48
    # the binary64 path's own bound (10 n kappa 2^-52) holds as well on this matrix
    assert r_err <= 10 * 25 * kappa * 2.0 ** -52, r_err
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A, Q, R)
    assert e2 <= 1e-13 and rF <= 1e-13, (kappa, e2, rF)


def test_df64_tiny_and_huge_scales():
    """Power-of-two block scaling keeps binary32 pairs in range."""
    A = ti.gaussian(20_000, 12, 91)
    for s in (1e-30, 1e30):
        Q, R = _direct(A * s)
        e2, _ = oracle.orth_error(Q)
        rF, _ = oracle.residual(A * s, Q, R)
        assert e2 <= 1e-13 and rF <= 1e-13, (s, e2, rF)


def test_df64_scale_grows_between_tiles():
    """Tiles of one block with magnitudes 2^60 apart: the running power-of-two
    scale rises at the large tile and the carried R is rescaled exactly."""
    A = ti.gaussian(40_000, 12, 93)
    A[3000:6000] *= 2.0 ** 60
    Q, R = _direct(A, block_rows=10_000)
    Qo, Ro = oracle.householder_qr(A)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 10 * 12 * kappa * U48
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A, Q, R)
    assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)


def test_df64_svd():
    import paper_1301_1071_gb300 as T
    A = ti.power_spectrum(30_000, 20, 92)
    U, S, V = T.svd(torch.tensor(A, device="cuda"), prec="df64")
    _, So, _ = oracle.svd(A)
    S = S.cpu().numpy()
    assert np.max(np.abs(S - So) / So[0]) <= 10 * 20 * U48
    e2, _ = oracle.orth_error(U.cpu().numpy())
    assert e2 <= 1e-13


def test_df64_rejected_for_f32():
    import paper_1301_1071_gb300 as T
    A = torch.randn(1000, 8, dtype=torch.float32, device="cuda")
    with pytest.raises(T.TSQRError):
        T.direct(A, prec="df64")
