"""Pins for the CPU oracle (no GPU).

The oracle is pinned to facts other than itself: closed forms, exact
special cases, long-double brute force (MGS, Cholesky of A^T A), an
independent library (numpy/LAPACK QR, run not read), algebraic identities the
paper states (Sec. II-A uniqueness, Sec. II-B any-tree R, Sec. III-B block
structure), finite differences for the adjoint, and known-answer checker
inputs.  Each pin would catch a plausible slip in oracle.c (a dropped term, a
wrong sign or index, a transposed operand).
"""
import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

EPS = np.finfo(np.float64).eps


def _hadamard(k):
    h = np.array([[1.0]])
    for _ in range(k):
        h = np.block([[h, h], [h, -h]])
    return h


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- thin QR ---

def test_n1_closed_form():
    a = ti.gaussian(37, 1, 11)
    Q, R = oracle.householder_qr(a)
    nrm = np.sqrt(np.sum(a[:, 0] ** 2))
    assert abs(R[0, 0] - nrm) <= 4 * EPS * nrm
    assert _rel(Q[:, 0], a[:, 0] / nrm) <= 8 * EPS


@pytest.mark.parametrize("k,n", [(3, 3), (4, 5), (6, 7)])
def test_orthonormal_columns_give_identity_R(k, n):
    # normalised Hadamard columns are exactly orthonormal (entries +-2^-k/2 for even k)
    m = 2 ** k
    H = _hadamard(k)[:, :n] / np.sqrt(m)
    Q, R = oracle.householder_qr(H)
    assert np.max(np.abs(R - np.eye(n))) <= 16 * EPS
    assert np.max(np.abs(Q - H)) <= 16 * EPS


def test_identity_stack_and_permutation():
    n = 6
    A = np.vstack([np.eye(n), np.zeros((10, n))])
    perm = np.random.default_rng(3).permutation(A.shape[0])
    Q, R = oracle.householder_qr(A[perm])
    assert np.array_equal(R, np.eye(n)) or np.max(np.abs(R - np.eye(n))) <= 4 * EPS
    assert np.max(np.abs(Q - A[perm])) <= 4 * EPS


def test_diagonal_scaling():
    A = ti.gaussian(50, 7, 21)
    c = np.linspace(0.5, 4.0, 7)
    Q0, R0 = oracle.householder_qr(A)
    Q1, R1 = oracle.householder_qr(A * c[None, :])
    assert _rel(R1, R0 * c[None, :]) <= 64 * EPS
    assert _rel(Q1, Q0) <= 64 * EPS


def test_row_permutation():
    A = ti.gaussian(64, 9, 22)
    perm = np.random.default_rng(5).permutation(64)
    Q0, R0 = oracle.householder_qr(A)
    Q1, R1 = oracle.householder_qr(A[perm])
    assert _rel(R1, R0) <= 64 * EPS
    assert _rel(Q1, Q0[perm]) <= 64 * EPS


@pytest.mark.parametrize("m,n", [(12, 4), (30, 8), (9, 9)])
def test_uniqueness_against_long_double_cholesky(m, n):
    # Sec. II-A: R is the (unique) Cholesky factor of A^T A.
    A = ti.gaussian(m, n, 100 + n)
    _, R = oracle.householder_qr(A)
    Rc = oracle.chol_gram_ld(A)
    kappa = np.linalg.cond(A)
    assert _rel(R, Rc) <= 50 * n * kappa * EPS


@pytest.mark.parametrize("m,n", [(15, 5), (40, 12)])
def test_against_long_double_mgs(m, n):
    A = ti.gaussian(m, n, 200 + n)
    Q, R = oracle.householder_qr(A)
    Qm, Rm = oracle.mgs_ld(A)
    kappa = np.linalg.cond(A)
    assert _rel(R, Rm) <= 50 * n * kappa * EPS
    assert _rel(Q, Qm) <= 50 * n * kappa * EPS


def test_long_double_mgs_pin_stays_orthonormal_at_high_kappa():
    # The MGS pin re-orthogonalises every column once ("twice is enough"), so
    # its Q stays orthonormal to long-double rounding even at kappa 1e12,
    # where one Gram-Schmidt pass would lose ~kappa * 2^-64 ~ 1e-7.
    A = ti.conditioned(60, 12, 1e12, 205)
    Qm, Rm = oracle.mgs_ld(A)
    e2, _ = oracle.orth_error(Qm)
    assert e2 <= 1e-14
    rF, _ = oracle.residual(A, Qm, Rm)
    assert rF <= 1e-14


@pytest.mark.parametrize("m,n,kappa", [(200, 10, 1.0), (500, 25, 1e8), (300, 16, 1e15)])
def test_library_cross_check(m, n, kappa):
    # numpy's LAPACK QR, sign-normalised: an independent implementation.
    A = ti.conditioned(m, n, kappa, 300 + n)
    Q, R = oracle.householder_qr(A)
    Ql, Rl = np.linalg.qr(A)
    d = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    Ql, Rl = Ql * d[None, :], Rl * d[:, None]
    assert _rel(R, Rl) <= 10 * n * kappa * EPS
    # Q columns are well determined up to the conditioning of the trailing R
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 50 * n * EPS
    assert _rel(Q @ R, A) <= 50 * n * EPS


@pytest.mark.parametrize("m,n,kappa", [(1000, 25, 1.0), (1000, 25, 1e15), (333, 7, 1e4)])
def test_invariants(m, n, kappa):
    A = ti.conditioned(m, n, kappa, 400 + n)
    Q, R = oracle.householder_qr(A)
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    e2, eF = oracle.orth_error(Q)
    assert e2 <= 1e-14 and eF <= 1e-14
    rF, r2 = oracle.residual(A, Q, R)
    assert rF <= n * EPS and r2 <= n * EPS   # backward error O(n eps)


def test_zero_column_gives_zero_R_row():
    A = ti.gaussian(20, 4, 7)
    A[:, 2] = 0.0
    Q, R = oracle.householder_qr(A)
    assert R[2, 2] == 0.0
    assert _rel(Q @ R, A) <= 50 * EPS


def test_square_matrix():
    A = ti.gaussian(12, 12, 8)
    Q, R = oracle.householder_qr(A)
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) <= 100 * EPS
    assert _rel(Q @ R, A) <= 100 * EPS


def test_rejects_bad_shapes():
    with pytest.raises(oracle.OracleError):
        oracle.householder_qr(np.zeros((3, 5)))


# ------------------------------------------- three-step structure (Sec. III-B) --

def test_block_diagonal_identity_of_the_paper_example():
    """Sec. III-B example: A with 8n rows split over four map tasks.
    Step 1 QR of each A_i, Step 2 QR of the stacked R_i, Step 3
    Q_i = Q1_i Q2_i reproduces the one-shot thin QR (after the sign fix)."""
    n = 5
    A = ti.gaussian(8 * n, n, 31)
    blocks = np.split(A, 4)
    fac = [oracle.householder_qr(b) for b in blocks]
    S = np.vstack([r for _, r in fac])          # 4n x n stack of R_i
    Q2, Rt = oracle.householder_qr(S)           # Step 2
    Q = np.vstack([q1 @ Q2[i * n:(i + 1) * n] for i, (q1, _) in enumerate(fac)])  # Step 3
    Qo, Ro = oracle.householder_qr(A)
    assert _rel(Rt, Ro) <= 100 * EPS
    assert _rel(Q, Qo) <= 100 * EPS


def test_any_reduction_tree_gives_the_same_R():
    """Sec. II-B: any reduction tree computes the same R (binary vs flat)."""
    n = 6
    A = ti.gaussian(16 * n, n, 32)
    leaves = [oracle.householder_r(b) for b in np.split(A, 8)]
    flat = oracle.householder_r(np.vstack(leaves))
    lvl = leaves
    while len(lvl) > 1:
        lvl = [oracle.householder_r(np.vstack(lvl[i:i + 2])) for i in range(0, len(lvl), 2)]
    assert _rel(flat, lvl[0]) <= 100 * EPS
    assert _rel(flat, oracle.householder_r(A)) <= 100 * EPS


# ---------------------------------------------------------- comparators ---

def test_cholqr_known_factorisation():
    # A = Q0 R0 with Q0 exactly orthonormal: Cholesky QR returns (Q0, R0).
    n = 6
    Q0 = _hadamard(6)[:, :n] / 8.0
    R0 = np.triu(ti.gaussian(n, n, 41)) + 4.0 * np.eye(n)
    R0 *= np.where(np.diag(R0) < 0, -1.0, 1.0)[:, None]
    A = Q0 @ R0
    st, Q, R = oracle.cholqr(A)
    assert st == 0
    assert _rel(R, R0) <= 1e-13 and _rel(Q, Q0) <= 1e-13
    st, Q, R = oracle.cholqr(A, refine_steps=1)
    assert st == 0 and _rel(R, R0) <= 1e-13


def test_cholqr_breakdown_on_rank_deficiency():
    A = ti.gaussian(30, 4, 42)
    A[:, 3] = 0.0
    st, _, _ = oracle.cholqr(A)
    assert st == oracle.ERR_NOT_SPD


def test_cholqr_loses_orthogonality_with_kappa():
    """Sec. IV: the indirect methods' error scales with the condition number;
    Cholesky QR fails outright once kappa^2 exceeds 1/eps."""
    A = ti.conditioned(2000, 10, 1e6, 43)
    st, Q, _ = oracle.cholqr(A)
    assert st == 0
    assert oracle.orth_error(Q)[0] > 1e-8       # ~ kappa^2 eps
    st, Q, _ = oracle.cholqr(A, refine_steps=1)
    assert st == 0 and oracle.orth_error(Q)[0] < 1e-13
    B = ti.conditioned(2000, 10, 1e12, 44)
    st, Q, _ = oracle.cholqr(B)
    assert st == oracle.ERR_NOT_SPD or oracle.orth_error(Q)[0] > 1e-2


def test_indirect_refine_matches_and_degrades():
    A = ti.conditioned(1500, 8, 1.0, 45)
    st, Q, R = oracle.indirect_refine(A, 1)
    Qo, Ro = oracle.householder_qr(A)
    assert st == 0 and _rel(R, Ro) <= 1e-14 and _rel(Q, Qo) <= 1e-14
    B = ti.conditioned(1500, 8, 1e12, 46)
    st, Q0, _ = oracle.indirect_refine(B, 0)
    assert st == 0 and oracle.orth_error(Q0)[0] > 1e-8   # ~ kappa eps without refinement
    st, Q1, _ = oracle.indirect_refine(B, 1)
    assert st == 0 and oracle.orth_error(Q1)[0] < 1e-13  # one refinement step repairs it


@pytest.mark.parametrize("kappa,seed", [(1e6, 51), (1e10, 52)])
def test_refinement_combines_r2_times_r1(kappa, seed):
    """Iterative refinement (Sec. I; Sec. II-C) ends with Q = Q0 R2^{-1} and
    R = R2 R1, so Q R = Q0 R1 = A holds by construction whatever R2 is.  At
    kappa >= 1e6 the second factor R2 is far from I (||R2 - I|| ~ kappa eps
    for indirect TSQR, ~ kappa^2 eps for Cholesky QR), so a combine in the
    wrong order (R1 R2) leaves a residual and an R error of order
    ||R2 - I|| (1e-10 .. 1e-6 here), far above these bars."""
    A = ti.conditioned(2000, 10, kappa, seed)
    Ro = oracle.householder_r(A)
    st, Q0, R1 = oracle.indirect_refine(A, 0)
    assert st == 0
    R2 = oracle.householder_r(Q0)
    assert np.linalg.norm(R2 - np.eye(10)) > 1e-10        # the pin is not vacuous
    runs = [("indirect", oracle.indirect_refine(A, 1))]
    if kappa * kappa * EPS < 0.1:                          # Cholesky QR survives kappa = 1e6 only
        runs.append(("cholqr", oracle.cholqr(A, 1)))
    for name, (st, Q, R) in runs:
        assert st == 0, name
        rF, r2 = oracle.residual(A, Q, R)
        assert rF <= 10 * 10 * EPS and r2 <= 10 * 10 * EPS, (name, rF, r2)
        # the refined R is the unique R of A (Sec. II-A) to working accuracy
        assert _rel(R, Ro) <= 1e-12, (name, _rel(R, Ro))
        assert oracle.orth_error(Q)[0] <= 1e-13, name


def test_residual_two_norm_known_answer():
    """rel2 = ||A - QR||_2 / ||R||_2 (Sec. I-B) on a rank-one perturbation of
    known 2-norm: A = H diag(s) V^T has exactly orthonormal H (Hadamard
    columns), so ||R||_2 = ||A||_2 = s_max; its exact QR factors applied to
    A + delta u w^T (unit u, w) leave the residual delta u w^T, whose 2-norm
    is delta and whose Frobenius norm is delta as well."""
    n = 6
    H = _hadamard(7)[:, :n] / np.sqrt(128.0)
    s = np.array([4.0, 2.0, 1.0, 0.5, 0.25, 0.125])
    V = ti.random_orthogonal(n, 73)
    A = (H * s) @ V.T
    Q, R = oracle.householder_qr(A)
    u = ti.gaussian(128, 1, 74)[:, 0]
    u /= np.linalg.norm(u)
    w = ti.gaussian(n, 1, 75)[:, 0]
    w /= np.linalg.norm(w)
    delta = 1e-9
    Ap = A + delta * np.outer(u, w)
    rF, r2 = oracle.residual(Ap, Q, R)
    assert abs(r2 - delta / 4.0) <= 1e-5 * delta / 4.0, r2
    assert abs(rF - delta / np.linalg.norm(Ap)) <= 1e-5 * rF
    # a rank-one residual: 2-norm and Frobenius norm agree (a squared or
    # unsquared 2-norm would not)
    rF2, r22 = oracle.residual(A + 1e-7 * np.outer(u, w), Q, R)
    assert abs(r22 * 4.0 - 1e-7) <= 1e-5 * 1e-7


def test_upper_inverse():
    R = np.triu(ti.gaussian(6, 6, 49)) + 3 * np.eye(6)
    X = oracle.upper_inverse(R)
    assert np.all(np.tril(X, -1) == 0.0)
    assert np.max(np.abs(X @ R - np.eye(6))) <= 1e-14
    assert np.max(np.abs(R @ X - np.eye(6))) <= 1e-14


def test_right_solve_upper():
    R = np.triu(ti.gaussian(5, 5, 47)) + 3 * np.eye(5)
    X0 = ti.gaussian(9, 5, 48)
    B = X0 @ R
    assert _rel(oracle.right_solve_upper(B, R), X0) <= 1e-14


# ------------------------------------------------------------------ SVD ---

def test_svd_known_singular_values():
    """A = H diag(sigma) V^T with H exactly orthonormal: the singular values
    are sigma and the right vectors are V (up to sign)."""
    n, m = 8, 64
    H = _hadamard(6)[:, :n] / 8.0
    sigma = ti.log_spaced(n, 1.0, 1e-6)
    V = ti.random_orthogonal(n, 51)
    A = (H * sigma[None, :]) @ V.T
    U, S, Vo = oracle.svd(A)
    assert np.max(np.abs(S - sigma) / sigma) <= 1e-9  # relative, graded by 1/sigma_min
    assert np.max(np.abs(S[:3] - sigma[:3])) <= 1e-14
    assert np.max(np.abs(np.abs(np.sum(Vo * V, axis=0)) - 1.0)) <= 1e-12
    assert _rel((U * S[None, :]) @ Vo.T, A) <= 1e-14


def test_svd_diagonal_matrix():
    d = np.array([3.0, -7.0, 0.5, 2.0])
    A = np.vstack([np.diag(d), np.zeros((6, 4))])
    _, S, _ = oracle.svd(A)
    assert np.allclose(S, np.sort(np.abs(d))[::-1], rtol=0, atol=1e-15)


def test_svd_against_long_double_eigenvalues():
    A = ti.gaussian(40, 6, 52)
    _, S, _ = oracle.svd(A)
    ev = np.sort(oracle.sym_eig(A.T @ A))[::-1]
    assert np.max(np.abs(S - np.sqrt(ev)) / S) <= 1e-13


def test_jacobi_svd_properties():
    R = np.triu(ti.gaussian(7, 7, 53)) + np.eye(7)
    U, S, V = oracle.jacobi_svd_ld(R)
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(U.T @ U - np.eye(7))) <= 1e-14
    assert np.max(np.abs(V.T @ V - np.eye(7))) <= 1e-14
    assert _rel((U * S) @ V.T, R) <= 1e-14
    for j in range(7):  # sign convention: largest-|.| entry of v_j positive
        i = int(np.argmax(np.abs(V[:, j])))
        assert V[i, j] > 0


# -------------------------------------------------------------- adjoint ---

def _loss(A, WQ, WR):
    Q, R = oracle.householder_qr(A)
    return np.sum(WQ * Q) + np.sum(WR * np.triu(R))


def test_backward_finite_differences_full():
    m, n = 40, 5
    A = ti.gaussian(m, n, 61)
    WQ = ti.gaussian(m, n, 62)
    WR = ti.gaussian(n, n, 63)
    Q, R = oracle.householder_qr(A)
    G = oracle.qr_backward(Q, R, WQ, np.triu(WR))
    Gfd = np.zeros_like(A)
    for i in range(m):
        for j in range(n):
            h = 1e-6 * max(1.0, abs(A[i, j]))
            Ap = A.copy(); Ap[i, j] += h
            Am = A.copy(); Am[i, j] -= h
            Gfd[i, j] = (_loss(Ap, WQ, WR) - _loss(Am, WQ, WR)) / (2 * h)
    assert _rel(G, Gfd) <= 1e-6


def test_backward_directional_fd_2000x8():
    """The FD instance of the differentiation workload (2,000 x 8, FP64)."""
    m, n = 2000, 8
    A = ti.gaussian(m, n, ti.SEED_GRAD)
    WQ = ti.gaussian(m, n, ti.SEED_GRAD + 1)
    WR = ti.gaussian(n, n, ti.SEED_GRAD + 2)
    Q, R = oracle.householder_qr(A)
    G = oracle.qr_backward(Q, R, WQ, np.triu(WR))
    rng = np.random.default_rng(64)
    for _ in range(6):
        E = rng.standard_normal((m, n))
        h = 1e-6
        fd = (_loss(A + h * E, WQ, WR) - _loss(A - h * E, WQ, WR)) / (2 * h)
        an = np.sum(G * E)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_backward_n1_closed_form():
    a = ti.gaussian(25, 1, 65)[:, 0]
    wq = ti.gaussian(25, 1, 66)[:, 0]
    wr = 0.7
    nrm = np.sqrt(a @ a)
    q = a / nrm
    expect = (wq - q * (q @ wq)) / nrm + wr * q
    G = oracle.qr_backward(q[:, None], np.array([[nrm]]), wq[:, None], np.array([[wr]]))
    assert _rel(G[:, 0], expect) <= 1e-14


def test_backward_against_torch_autograd():
    torch = pytest.importorskip("torch")
    m, n = 30, 6
    A = ti.gaussian(m, n, 67)
    WQ = ti.gaussian(m, n, 68)
    WR = ti.gaussian(n, n, 69)
    At = torch.tensor(A, requires_grad=True)
    Qt, Rt = torch.linalg.qr(At)
    d = torch.sign(torch.diagonal(Rt)).detach()
    d[d == 0] = 1.0
    Qt, Rt = Qt * d[None, :], Rt * d[:, None]
    L = (torch.tensor(WQ) * Qt).sum() + (torch.tensor(WR) * torch.triu(Rt)).sum()
    L.backward()
    Q, R = oracle.householder_qr(A)
    G = oracle.qr_backward(Q, R, WQ, np.triu(WR))
    assert _rel(G, At.grad.numpy()) <= 1e-12


def test_backward_zero_cotangents():
    A = ti.gaussian(20, 4, 70)
    Q, R = oracle.householder_qr(A)
    assert np.all(oracle.qr_backward(Q, R, None, None) == 0.0)


# ------------------------------------------------------------- checkers ---

def test_orth_error_known_answer():
    n = 6
    H = _hadamard(7)[:, :n] / np.sqrt(128.0)
    E = np.diag([3.0, -1.0, 0.5, 0.0, 2.0, 1.0])
    delta = 1e-11
    Q = H @ (np.eye(n) + delta * E)      # Q^TQ - I = 2 delta E + delta^2 E^2
    e2, eF = oracle.orth_error(Q)
    expect2 = 2 * delta * 3.0 + delta ** 2 * 9.0
    assert abs(e2 - expect2) <= 1e-4 * expect2
    expectF = np.linalg.norm(2 * delta * np.diag(E) + delta ** 2 * np.diag(E) ** 2)
    assert abs(eF - expectF) <= 1e-4 * expectF
    e2h, _ = oracle.orth_error(H)
    assert e2h <= 4 * EPS


def test_orth_error_known_answer_off_diagonal():
    # A symmetric perturbation with off-diagonal entries: Q = H (I + delta S)
    # gives Q^TQ - I = 2 delta S + delta^2 S^2 exactly (H^T H = I), so both the
    # 2-norm and the Frobenius norm (every off-diagonal entry counted twice)
    # have closed forms.
    n = 5
    H = _hadamard(6)[:, :n] / 8.0
    S = np.array([[0.0, 1.0, 0.0, 0.0, 2.0],
                  [1.0, 0.0, -1.0, 0.0, 0.0],
                  [0.0, -1.0, 0.0, 0.5, 0.0],
                  [0.0, 0.0, 0.5, 0.0, 0.0],
                  [2.0, 0.0, 0.0, 0.0, 0.0]])
    delta = 1e-10
    Q = H @ (np.eye(n) + delta * S)
    E = 2 * delta * S + delta ** 2 * (S @ S)
    e2, eF = oracle.orth_error(Q)
    expect2 = np.max(np.abs(np.linalg.eigvalsh(E)))
    expectF = np.sqrt(np.sum(E * E))
    assert abs(e2 - expect2) <= 1e-4 * expect2
    assert abs(eF - expectF) <= 1e-4 * expectF


def test_residual_known_answer():
    A = ti.gaussian(300, 5, 71)
    Q, R = oracle.householder_qr(A)
    F = ti.gaussian(300, 5, 72)
    rF, _ = oracle.residual(A + 1e-9 * F, Q, R)
    expect = 1e-9 * np.linalg.norm(F) / np.linalg.norm(A + 1e-9 * F)
    assert abs(rF - expect) <= 1e-3 * expect


def test_gram_dot2_cancellation():
    # x^T y with massive cancellation: plain FP64 loses everything, Dot2 doesn't
    x = np.array([[1e16], [1.0], [-1e16], [1.0]])
    y = np.ones((4, 1))
    assert oracle.gram_dot2(x, y)[0, 0] == 2.0


def test_gram_dot2_keeps_the_product_rounding_error():
    # a = 1 + 2^-30: a*a = 1 + 2^-29 + 2^-60 rounds to 1 + 2^-29 in binary64,
    # so a*a - 1*(1 + 2^-29) is exactly 2^-60 but plain FP64 gives 0.  Dot2
    # recovers the product's rounding error with an FMA (TwoProduct).
    a = 1.0 + 2.0 ** -30
    x = np.array([[a], [-1.0]])
    y = np.array([[a], [1.0 + 2.0 ** -29]])
    assert float(x[0, 0] * y[0, 0] + x[1, 0] * y[1, 0]) == 0.0
    assert oracle.gram_dot2(x, y)[0, 0] == 2.0 ** -60


@pytest.mark.parametrize("n", [37, 64, 100])
def test_orth_error_converges_at_large_n(n):
    # exactly orthonormal Hadamard columns: the checker must converge and give ~0
    H = _hadamard(8)[:, :n] / 16.0
    e2, eF = oracle.orth_error(H)
    assert e2 <= 4 * EPS and eF <= 4 * EPS
    A = ti.gaussian(3000, n, 80 + n)
    Q, R = oracle.householder_qr(A)
    e2, _ = oracle.orth_error(Q)
    assert e2 <= 1e-14
    rF, r2 = oracle.residual(A, Q, R)
    assert rF <= n * EPS and r2 <= n * EPS


def test_sym_eig_closed_form():
    S = np.array([[2.0, 1.0], [1.0, 2.0]])
    assert np.allclose(oracle.sym_eig(S), [1.0, 3.0], atol=1e-15)


# ------------------------------------------------------ input generators ---

def test_generators_are_seeded_and_shaped():
    a = ti.conditioned(100, 5, 1e4, 9)
    b = ti.conditioned(100, 5, 1e4, 9)
    assert a.shape == (100, 5) and np.array_equal(a, b)
    V = ti.random_orthogonal(7, 3)
    assert np.max(np.abs(V.T @ V - np.eye(7))) <= 1e-14
    s = ti.sigma_conditioned(5, 1e4)
    assert s[0] == 1.0 and abs(s[-1] - 1e-4) <= 1e-18


def test_parallel_oracle_is_bit_identical_to_serial():
    """The all-core oracle (the timed CPU baseline) runs only loops over
    independent columns or rows in parallel, each iteration doing the serial
    loop's operations: the results are the same bits at 1 and 4 threads."""
    A = ti.conditioned(150_000, 12, 1e8, 91)
    WQ = ti.gaussian(150_000, 12, 92)
    WR = np.triu(ti.gaussian(12, 12, 93))
    out = {}
    prev = oracle.num_threads()
    try:
        for t in (1, 4):
            oracle.set_num_threads(t)
            Q, R = oracle.householder_qr(A)
            dA = oracle.qr_backward(Q, R, WQ, WR)
            out[t] = (Q, R, dA)
    finally:
        oracle.set_num_threads(prev)
    for a, b in zip(out[1], out[4]):
        assert np.array_equal(a, b)
