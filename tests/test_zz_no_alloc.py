"""tsqr_direct_static: direct TSQR on the library's fixed device scratch.

For callers that cannot allocate device memory (a host framework that owns
all device memory, a latency-critical caller that cannot pay for the device
synchronisation of cudaMalloc/cudaFree, plain C code without an allocator).
Called through the C-ABI and compared with tsqr_direct (which takes a
caller-allocated workspace) on two calls in a row: the second call reuses the
same scratch, which still holds the first call's contents.  Collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import tsqr_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52
STATIC_BYTES = 16 * 1024 * 1024


def _static_call(lib, A, Q, R, opts):
    m, n = A.shape
    return lib.tsqr_direct_static(ctypes.c_void_p(A.data_ptr()), m, n, n, 0, ctypes.c_void_p(Q.data_ptr()), n,
                                  ctypes.c_void_p(R.data_ptr()), n, ctypes.byref(opts),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("m,n,b", [(100_000, 10, 1000), (300_000, 25, 0)])
def test_static_matches_direct_on_two_calls(m, n, b):
    """Two calls in a row on different matrices: the second reuses the scratch
    the first left behind.  tsqr_direct_static runs the plan and kernels of
    tsqr_direct on the same input (only the workspace address differs, and
    no reduction in the path depends on it), so Q and R must be identical
    bit for bit; both are also compared element-wise with the oracle."""
    import paper_1301_1071_gb300 as T
    lib = T.load()
    A1_np = ti.gaussian(m, n, 4000 + n)
    A2_np = ti.conditioned(m, n, 1e12, 4100 + n)
    assert T.workspace_size(T.OP_DIRECT, m, n, torch.float64, b) <= STATIC_BYTES
    opts = T.Opts()
    opts.block_rows = b
    opts.sync = 1  # the device status is returned by the call itself
    for A_np, kappa in ((A1_np, np.linalg.cond(A1_np)), (A2_np, 1e12)):
        A = torch.tensor(A_np, device="cuda")
        Qs = torch.empty_like(A)
        Rs = torch.empty(n, n, dtype=torch.float64, device="cuda")
        assert _static_call(lib, A, Qs, Rs, opts) == 0
        Qd, Rd = T.direct(A, block_rows=b)  # caller-allocated workspace
        torch.cuda.synchronize()
        assert torch.equal(Qs, Qd) and torch.equal(Rs, Rd)
        Qo, Ro = oracle.householder_qr(A_np)
        tol = 10 * n * kappa * EPS64
        Qh, Rh = Qs.cpu().numpy(), Rs.cpu().numpy()
        assert np.linalg.norm(Rh - Ro) / np.linalg.norm(Ro) <= tol
        assert np.max(np.abs(Qh - Qo)) <= max(tol, 10 * n * EPS64)
        e2, _ = oracle.orth_error(Qh)
        assert e2 <= 1e-13


def test_static_rejects_problems_beyond_its_scratch():
    import paper_1301_1071_gb300 as T
    lib = T.load()
    m, n = 2_000_000, 25  # needs more than 16 MiB of workspace
    assert T.workspace_size(T.OP_DIRECT, m, n, torch.float64) > STATIC_BYTES
    A = torch.zeros(m, n, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(A)
    R = torch.empty(n, n, dtype=torch.float64, device="cuda")
    opts = T.Opts()
    assert _static_call(lib, A, Q, R, opts) == 4  # TSQR_ERR_WORKSPACE, before any launch
