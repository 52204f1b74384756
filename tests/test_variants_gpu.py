"""Parity of the CUDA SVD variant, comparators and adjoint with the oracle.

* SVD (Sec. III-B, SVD paragraph): S against the oracle's S and the
  generated sigma; U, V element-wise (same sign convention); U^T U = I.
* Cholesky QR and indirect TSQR + refinement (Sec. II): element-wise at
  kappa = 1 where they agree with the thin QR; status on breakdown; the
  qualitative loss of orthogonality with kappa (Sec. IV).
* Adjoint: element-wise against the oracle's dA; FP64 finite differences.
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


def _cuda(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


# ------------------------------------------------------------------ SVD ---

@pytest.mark.parametrize("m,n,seed", [(20_000, 10, 1), (5000, 25, 2), (3001, 16, 3), (4000, 50, 4),
                                      (30_000, 100, 5)])  # n = 100: tree nodes on clusters
def test_svd_parity_f64(m, n, seed):
    A = ti.power_spectrum(m, n, seed)
    U, S, V = _T().svd(_cuda(A))
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    Uo, So, Vo = oracle.svd(A)
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(S - So) / So[0]) <= 10 * n * EPS64
    # relative accuracy of each sigma within the generation interval
    sig = ti.sigma_power(n)
    ratio = S / sig
    assert np.all(ratio > 0.9) and np.all(ratio < 1.1)
    # singular vectors: separated spectrum -> element-wise with the same signs
    gap = np.min(np.abs(np.diff(So))) / So[0]
    tolv = 100 * n * EPS64 / gap
    assert np.max(np.abs(V - Vo)) <= tolv
    assert np.max(np.abs(U - Uo)) <= tolv
    e2, _ = oracle.orth_error(U)
    assert e2 <= 1e-13
    rF = np.linalg.norm((U * S) @ V.T - A) / np.linalg.norm(A)
    assert rF <= 1e-13


def test_svd_tiled_blocks():
    """SVD variant over blocks of several register tiles."""
    m, n = 60_000, 20
    A = ti.power_spectrum(m, n, 5)
    U, S, V = _T().svd(_cuda(A), block_rows=7001)
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    Uo, So, Vo = oracle.svd(A)
    assert np.max(np.abs(S - So) / So[0]) <= 10 * n * EPS64
    gap = np.min(np.abs(np.diff(So))) / So[0]
    tolv = 100 * n * EPS64 / gap
    assert np.max(np.abs(V - Vo)) <= tolv and np.max(np.abs(U - Uo)) <= tolv
    assert oracle.orth_error(U)[0] <= 1e-13


def test_svd_f32_storage():
    m, n = 50_000, 20
    A = ti.power_spectrum(m, n, 9).astype(np.float32)
    U, S, V = _T().svd(_cuda(A, torch.float32))
    _, So, Vo = oracle.svd(A.astype(np.float64))
    S = S.cpu().numpy()
    assert np.max(np.abs(S - So) / So[0]) <= 1e-5
    e2, _ = oracle.orth_error(U.double().cpu().numpy())
    assert e2 <= 1e-5


# --------------------------------------------------------- Cholesky QR ---

@pytest.mark.parametrize("refine", [0, 1])
def test_cholqr_parity_well_conditioned(refine):
    A = ti.conditioned(40_000, 25, 1.0, 11)
    Q, R = _T().cholqr(_cuda(A), refine=refine)
    st, Qo, Ro = oracle.cholqr(A, refine)
    assert st == 0
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-13
    assert np.max(np.abs(Q - Qo)) <= 1e-13
    e2, _ = oracle.orth_error(Q)
    assert e2 <= (1e-13 if refine else 1e-12)


def test_cholqr_breakdown_status():
    A = ti.gaussian(10_000, 8, 12)
    A[:, 5] = 0.0
    T = _T()
    with pytest.raises(T.TSQRError) as ei:
        T.cholqr(_cuda(A))
    assert ei.value.status == 6  # TSQR_ERR_NOT_SPD


def test_cholqr_loses_orthogonality():
    """Sec. IV: Cholesky QR fails once kappa^2 eps ~ 1 (kappa >= 1e8)."""
    A = ti.conditioned(40_000, 25, 1e6, 13)
    Q, _ = _T().cholqr(_cuda(A))
    assert oracle.orth_error(Q.cpu().numpy())[0] > 1e-8
    T = _T()
    B = ti.conditioned(40_000, 25, 1e12, 14)
    try:
        Q, _ = T.cholqr(_cuda(B))
        assert oracle.orth_error(Q.cpu().numpy())[0] > 1e-2
    except T.TSQRError as e:
        assert e.status == 6


# -------------------------------------------------- indirect + refinement ---

@pytest.mark.parametrize("refine", [0, 1])
def test_indirect_parity_well_conditioned(refine):
    A = ti.conditioned(40_000, 25, 1.0, 21)
    Q, R = _T().indirect_refine(_cuda(A), refine=refine)
    st, Qo, Ro = oracle.indirect_refine(A, refine)
    assert st == 0
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-13
    assert np.max(np.abs(Q - Qo)) <= 1e-13


def test_indirect_tiled_blocks():
    """R-only TSQR over blocks of several register tiles."""
    A = ti.conditioned(40_000, 25, 1.0, 24)
    Q, R = _T().indirect_refine(_cuda(A), refine=1, block_rows=9000)
    st, Qo, Ro = oracle.indirect_refine(A, 1)
    assert st == 0
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-13
    assert np.max(np.abs(Q - Qo)) <= 1e-13


def test_indirect_refinement_repairs_moderate_kappa():
    """Sec. IV: one refinement step restores orthogonality at kappa = 1e12."""
    A = ti.conditioned(40_000, 25, 1e12, 22)
    T = _T()
    Q0, _ = T.indirect_refine(_cuda(A), refine=0)
    Q1, R1 = T.indirect_refine(_cuda(A), refine=1)
    assert oracle.orth_error(Q0.cpu().numpy())[0] > 1e-8
    assert oracle.orth_error(Q1.cpu().numpy())[0] <= 1e-13
    rF, _ = oracle.residual(A, Q1.cpu().numpy(), R1.cpu().numpy())
    assert rF <= 1e-13


def test_indirect_f32():
    A = ti.column_scaled(30_000, 12, 1e-2, 23).astype(np.float32)
    Q, R = _T().indirect_refine(_cuda(A, torch.float32), refine=1)
    e2, _ = oracle.orth_error(Q.double().cpu().numpy())
    assert e2 <= 1e-5


# ------------------------------------------------------------- adjoint ---

@pytest.mark.parametrize("m,n", [(2000, 8), (30_000, 25), (9000, 64)])
def test_backward_parity_f64(m, n):
    A = ti.gaussian(m, n, 31)
    WQ = ti.gaussian(m, n, 32)
    WR = ti.gaussian(n, n, 33)
    Qo, Ro = oracle.householder_qr(A)
    dAo = oracle.qr_backward(Qo, Ro, WQ, np.triu(WR))
    dA = _T().backward(_cuda(Qo), _cuda(Ro), _cuda(WQ), _cuda(WR)).cpu().numpy()
    assert np.linalg.norm(dA - dAo) / np.linalg.norm(dAo) <= 1e-12
    assert np.max(np.abs(dA - dAo)) <= 1e-12 * np.max(np.abs(dAo)) * 10


def test_backward_null_cotangents():
    A = ti.gaussian(3000, 10, 34)
    Qo, Ro = oracle.householder_qr(A)
    WR = ti.gaussian(10, 10, 35)
    T = _T()
    dA = T.backward(_cuda(Qo), _cuda(Ro), None, _cuda(WR)).cpu().numpy()
    assert np.linalg.norm(dA - oracle.qr_backward(Qo, Ro, None, np.triu(WR))) <= 1e-12 * np.linalg.norm(dA)
    WQ = ti.gaussian(3000, 10, 36)
    dA = T.backward(_cuda(Qo), _cuda(Ro), _cuda(WQ), None).cpu().numpy()
    assert np.linalg.norm(dA - oracle.qr_backward(Qo, Ro, WQ, None)) <= 1e-12 * np.linalg.norm(dA)


def test_autograd_function_fd_2000x8():
    """FP64 central finite differences on the 2,000 x 8 instance."""
    T = _T()
    m, n = 2000, 8
    A = ti.gaussian(m, n, ti.SEED_GRAD)
    WQ = _cuda(ti.gaussian(m, n, ti.SEED_GRAD + 1))
    WR = _cuda(ti.gaussian(n, n, ti.SEED_GRAD + 2))
    At = _cuda(A).requires_grad_(True)
    Q, R = T.QRFunction.apply(At)
    L = (WQ * Q).sum() + (WR * torch.triu(R)).sum()
    L.backward()
    g = At.grad.cpu().numpy()

    def loss(Anp):
        Qh, Rh = T.direct(_cuda(Anp))
        return float((WQ * Qh).sum() + (WR * torch.triu(Rh)).sum())

    rng = np.random.default_rng(7)
    for _ in range(4):
        E = rng.standard_normal((m, n))
        h = 1e-6
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        an = float(np.sum(g * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_backward_f32():
    m, n = 20_000, 16
    A = ti.gaussian(m, n, 41).astype(np.float32)
    WQ = ti.gaussian(m, n, 42)
    WR = ti.gaussian(n, n, 43)
    Qo, Ro = oracle.householder_qr(A.astype(np.float64))
    dAo = oracle.qr_backward(Qo, Ro, WQ, np.triu(WR))
    dA = _T().backward(_cuda(Qo, torch.float32), _cuda(Ro), _cuda(WQ, torch.float32), _cuda(WR))
    dA = dA.double().cpu().numpy()
    assert np.linalg.norm(dA - dAo) / np.linalg.norm(dAo) <= 1e-4
