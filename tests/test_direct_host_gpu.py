"""tsqr_direct_host: direct TSQR from and to host memory with the copies
overlapped (chunks of row blocks).  The chunking only changes where each
launch starts, so with the same row blocks the result is bitwise that of
tsqr_direct; with its own default blocks it meets the oracle bars of the
direct path (Sec. III-B)."""
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


@pytest.mark.parametrize("m,n,b,dtype,prec", [
    (3_000_000, 25, 2000, torch.float64, "native"),   # 1,500 blocks: 4 chunks of whole waves
    (1_300_001, 10, 1000, torch.float64, "native"),   # ragged last block and chunk
    (2_500_000, 50, 2000, torch.float32, "native"),
    (2_500_000, 50, 2000, torch.float32, "tf32x3"),
    (2_000_000, 25, 4000, torch.float64, "df64"),
    (1_500_000, 100, 2000, torch.float32, "tf32x3"),  # 750 blocks: tree nodes on clusters of 8 CTAs
])
def test_host_matches_device_path_bitwise(m, n, b, dtype, prec):
    T = _T()
    A = torch.from_numpy(ti.gaussian(m, n, 4000 + n)).to(dtype).pin_memory()
    Qh, Rh = T.direct_host(A, block_rows=b, prec=prec)
    Qd, Rd = T.direct(A.cuda(), block_rows=b, prec=prec)
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())


def test_host_default_plan_meets_the_oracle():
    """2,000,000 x 25 FP64 (400 MB: three copy chunks of the host plan's own
    row blocks) at kappa 1e12."""
    T = _T()
    A_np = ti.conditioned(2_000_000, 25, 1e12, ti.SEED_SWEEP)
    Qh, Rh = T.direct_host(torch.from_numpy(A_np).pin_memory())
    Q, R = Qh.numpy(), Rh.numpy()
    Qo, Ro = oracle.householder_qr(A_np)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 10 * 25 * 1e12 * EPS64
    e2, _ = oracle.orth_error(Q)
    rF, _ = oracle.residual(A_np, Q, R)
    assert e2 <= 1e-13 and rF <= 1e-13, (e2, rF)


def test_host_pageable_and_single_block():
    """Pageable host memory (copies serialised, same result) and a matrix of
    one row block (one chunk)."""
    T = _T()
    A = torch.from_numpy(ti.gaussian(700, 25, 8))
    Qh, Rh = T.direct_host(A)
    Qd, Rd = T.direct(A.cuda())
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())
    A2 = torch.from_numpy(ti.gaussian(400_000, 12, 9))
    Qh2, Rh2 = T.direct_host(A2, block_rows=1000)
    Qd2, Rd2 = T.direct(A2.cuda(), block_rows=1000)
    assert torch.equal(Qh2, Qd2.cpu()) and torch.equal(Rh2, Rd2.cpu())


def test_host_rejects_bad_arguments():
    T = _T()
    with pytest.raises(ValueError):
        T.direct_host(torch.zeros(10, 3, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        T.direct_host(torch.zeros(3, 5, dtype=torch.float64))
    with pytest.raises(T.TSQRError):
        T.direct_host(torch.zeros(1000, 10, dtype=torch.float64), block_rows=5)
