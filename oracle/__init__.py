"""CPU oracle for direct TSQR -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_1301_1071_gb300``) and never imports it.

Paper: Benson, Gleich, Demmel, "Direct QR factorizations for tall-and-skinny
matrices in MapReduce architectures" (arXiv:1301.1071).

Every routine lives in ``oracle.c`` (plain C, IEEE binary64, long double in
the pins); this module only compiles it with gcc and marshals numpy arrays.

* ``householder_qr``     -- thin QR A = QR, diag(R) >= 0 (Sec. I; Sec. III-A
                            textbook Householder).  Direct TSQR reaches this
                            factorisation exactly in exact arithmetic
                            (Sec. III-B), so it is the direct-TSQR oracle.
* ``householder_r``      -- R only (indirect TSQR output, Sec. II-B).
* ``cholqr``             -- Cholesky QR with refinement (Sec. II-A, II-C).
* ``indirect_refine``    -- indirect TSQR + refinement (Sec. II-B, II-C).
* ``svd``                -- A = (Q U_R) S V^T (Sec. III-B, SVD paragraph).
* ``qr_backward``        -- adjoint dA of the thin QR (not in the paper).
* pins: ``mgs_ld``, ``chol_gram_ld``, ``jacobi_svd_ld``, ``sym_eig``.
* checkers: ``orth_error`` (||Q^TQ-I||_2, _F), ``residual`` (||A-QR||_F/||A||_F,
  ||A-QR||_2/||R||_2), ``gram_dot2``.

Every function is pinned to something other than itself (tests/test_oracle.py;
no function here is "parity unpinned"):

* ``householder_qr`` / ``householder_r``: the n = 1 closed form; exactly
  orthonormal columns give Q = A, R = I; diagonal scaling and row
  permutation; uniqueness against the long-double Cholesky factor of A^T A
  (Sec. II-A); long-double MGS; numpy's LAPACK QR run as a library; the
  block identity of the paper's 4-block example (Sec. III-B); the any-tree R
  of Sec. II-B; a zero column; square A.
* ``cholqr``: a known factorisation A = Q0 R0; breakdown on rank deficiency;
  loss of orthogonality with kappa and its repair by refinement (Sec. IV).
* ``indirect_refine``: agreement at kappa = 1, loss without refinement; the
  combine R = R2 R1 at kappa 1e6 and 1e10, where the swapped order fails.
* ``svd``: known singular values (Hadamard x diag x V), a diagonal matrix,
  long-double eigenvalues of A^T A, the sign and ordering conventions.
* ``qr_backward``: full and directional central finite differences at
  2,000 x 8, the n = 1 closed form, torch-CPU autograd, zero cotangents.
* ``orth_error`` / ``residual`` / ``gram_dot2`` / ``sym_eig``: known answers
  (Q = H (I + delta E) with diagonal and off-diagonal E; a rank-one residual
  of known 2-norm; Dot2 cancellation and a product's rounding error; the
  2 x 2 closed form); the pin ``mgs_ld`` is checked for its own
  orthogonality and residual at kappa 1e12.
* the OpenMP loops: bit-identical to the serial oracle at 1 and 4 threads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOT_SPD, ERR_SINGULAR, ERR_NOCONV = 0, 1, 6, 7, 10


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (no fused multiply-add
    contraction, so that x86 and Arm give the same bits)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    sigs = {
        "oracle_householder_qr": [P, I64, I64, P, P],
        "oracle_householder_r": [P, I64, I64, P],
        "oracle_right_solve_upper": [P, I64, I64, P, P],
        "oracle_upper_inverse": [P, I64, P],
        "oracle_cholqr": [P, I64, I64, ctypes.c_int, P, P],
        "oracle_indirect_refine": [P, I64, I64, ctypes.c_int, P, P],
        "oracle_qr_backward": [P, P, P, P, I64, I64, P],
        "oracle_sym_eig": [P, I64, P],
        "oracle_mgs_ld": [P, I64, I64, P, P],
        "oracle_chol_gram_ld": [P, I64, I64, P],
        "oracle_jacobi_svd_ld": [P, I64, P, P, P],
        "oracle_svd": [P, I64, I64, P, P, P],
        "oracle_orth_error": [P, I64, I64, P, P],
        "oracle_residual": [P, P, P, I64, I64, P, P],
        "oracle_gram_dot2": [P, P, I64, I64, P],
        "oracle_num_threads": [],
        "oracle_set_num_threads": [ctypes.c_int],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(st, what)


def householder_qr(A):
    """Thin QR (Sec. I), unblocked FP64 Householder (Sec. III-A), diag(R) >= 0."""
    A = _f64(A)
    m, n = A.shape
    Q = np.empty((m, n)); R = np.empty((n, n))
    _check(_load().oracle_householder_qr(_p(A), m, n, _p(Q), _p(R)), "householder_qr")
    return Q, R


def householder_r(A):
    """R factor only, diag(R) >= 0 (indirect TSQR output, Sec. II-B)."""
    A = _f64(A)
    m, n = A.shape
    R = np.empty((n, n))
    _check(_load().oracle_householder_r(_p(A), m, n, _p(R)), "householder_r")
    return R


def right_solve_upper(B, R):
    """X = B R^{-1} row by row (Sec. II-C)."""
    B = _f64(B); R = _f64(R)
    m, n = B.shape
    X = np.empty((m, n))
    _check(_load().oracle_right_solve_upper(_p(B), m, n, _p(R), _p(X)), "right_solve_upper")
    return X


def upper_inverse(R):
    """R^{-1} of an upper-triangular R by back substitution (Sec. II-C)."""
    R = _f64(R)
    n = R.shape[0]
    X = np.empty((n, n))
    _check(_load().oracle_upper_inverse(_p(R), n, _p(X)), "upper_inverse")
    return X


def cholqr(A, refine_steps: int = 0):
    """Cholesky QR (Sec. II-A) with refine_steps repeats on the computed Q.
    Returns (status, Q, R); status 6 = Cholesky breakdown."""
    A = _f64(A)
    m, n = A.shape
    Q = np.full((m, n), np.nan); R = np.full((n, n), np.nan)
    st = _load().oracle_cholqr(_p(A), m, n, int(refine_steps), _p(Q), _p(R))
    if st == ERR_ARG:
        raise OracleError(st, "cholqr")
    return st, Q, R


def indirect_refine(A, refine_steps: int = 1):
    """Indirect TSQR + refinement (Sec. II-B, II-C). Returns (status, Q, R)."""
    A = _f64(A)
    m, n = A.shape
    Q = np.full((m, n), np.nan); R = np.full((n, n), np.nan)
    st = _load().oracle_indirect_refine(_p(A), m, n, int(refine_steps), _p(Q), _p(R))
    if st == ERR_ARG:
        raise OracleError(st, "indirect_refine")
    return st, Q, R


def qr_backward(Q, R, dQ=None, dR=None):
    """dA = (dQ + Q copyltu(M)) R^{-T}, M = R dR^T - dQ^T Q."""
    Q = _f64(Q); R = _f64(R)
    m, n = Q.shape
    dQ = None if dQ is None else _f64(dQ)
    dR = None if dR is None else _f64(dR)
    dA = np.empty((m, n))
    _check(_load().oracle_qr_backward(_p(Q), _p(R), _p(dQ), _p(dR), m, n, _p(dA)), "qr_backward")
    return dA


def sym_eig(S):
    """Eigenvalues of a symmetric matrix (long-double cyclic Jacobi), ascending."""
    S = _f64(S)
    n = S.shape[0]
    ev = np.empty(n)
    _check(_load().oracle_sym_eig(_p(S), n, _p(ev)), "sym_eig")
    return np.sort(ev)


def mgs_ld(A):
    """Long-double MGS with re-orthogonalisation (pin)."""
    A = _f64(A)
    m, n = A.shape
    Q = np.empty((m, n)); R = np.empty((n, n))
    _check(_load().oracle_mgs_ld(_p(A), m, n, _p(Q), _p(R)), "mgs_ld")
    return Q, R


def chol_gram_ld(A):
    """Long-double Cholesky factor of A^T A (pin, Sec. II-A uniqueness)."""
    A = _f64(A)
    m, n = A.shape
    R = np.empty((n, n))
    _check(_load().oracle_chol_gram_ld(_p(A), m, n, _p(R)), "chol_gram_ld")
    return R


def jacobi_svd_ld(R):
    """One-sided Jacobi SVD of a square matrix in long double."""
    R = _f64(R)
    n = R.shape[0]
    U = np.empty((n, n)); S = np.empty(n); V = np.empty((n, n))
    _check(_load().oracle_jacobi_svd_ld(_p(R), n, _p(U), _p(S), _p(V)), "jacobi_svd_ld")
    return U, S, V


def svd(A):
    """SVD via thin QR + SVD of R (Sec. III-B): A = U diag(S) V^T."""
    A = _f64(A)
    m, n = A.shape
    U = np.empty((m, n)); S = np.empty(n); V = np.empty((n, n))
    _check(_load().oracle_svd(_p(A), m, n, _p(U), _p(S), _p(V)), "svd")
    return U, S, V


def orth_error(Q):
    """(||Q^T Q - I||_2, ||Q^T Q - I||_F) with Dot2 accumulation."""
    Q = _f64(Q)
    m, n = Q.shape
    e2 = ctypes.c_double(); eF = ctypes.c_double()
    _check(_load().oracle_orth_error(_p(Q), m, n, ctypes.byref(e2), ctypes.byref(eF)), "orth_error")
    return e2.value, eF.value


def residual(A, Q, R):
    """(||A-QR||_F/||A||_F, ||A-QR||_2/||R||_2) with Dot2 residual entries."""
    A = _f64(A); Q = _f64(Q); R = _f64(R)
    m, n = A.shape
    rF = ctypes.c_double(); r2 = ctypes.c_double()
    _check(_load().oracle_residual(_p(A), _p(Q), _p(R), m, n, ctypes.byref(rF), ctypes.byref(r2)),
           "residual")
    return rF.value, r2.value


def gram_dot2(X, Y):
    """X^T Y with Dot2 accumulation."""
    X = _f64(X); Y = _f64(Y)
    m, n = X.shape
    G = np.empty((n, n))
    _check(_load().oracle_gram_dot2(_p(X), _p(Y), m, n, _p(G)), "gram_dot2")
    return G


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(t: int) -> None:
    """Threads of the oracle's parallel loops (independent columns or rows;
    the results are the same bits for every thread count)."""
    _check(_load().oracle_set_num_threads(int(t)), "set_num_threads")
