"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/tsqr.h declares; host-side planning checks need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsqr.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1301_1071_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["tsqr_direct", "tsqr_svd", "cholqr", "tsqr_indirect_refine", "tsqr_backward",
                 "tsqr_workspace_size", "tsqr_status_string", "tsqr_read_status"]:
        assert want in names, want


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"missing export {name}"


def test_status_strings(lib):
    lib.tsqr_status_string.restype = ctypes.c_char_p
    assert lib.tsqr_status_string(0) == b"TSQR_OK"
    assert b"NOT_SPD" in lib.tsqr_status_string(6)
    assert b"unknown" in lib.tsqr_status_string(99)


class Opts(ctypes.Structure):
    _fields_ = [("block_rows", ctypes.c_int64), ("tree_fanout", ctypes.c_int32),
                ("sync", ctypes.c_int32), ("stage_events", ctypes.POINTER(ctypes.c_void_p)),
                ("prec", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _ws(lib, op, m, n, dtype, block_rows=0, fanout=0):
    f = lib.tsqr_workspace_size
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Opts),
                  ctypes.POINTER(ctypes.c_size_t)]
    f.restype = ctypes.c_int
    o = Opts(block_rows, fanout, 0, None, 0, 0)
    out = ctypes.c_size_t(0)
    st = f(op, m, n, dtype, ctypes.byref(o), ctypes.byref(out))
    return st, out.value


def test_workspace_size_host_only(lib):
    st, b = _ws(lib, 0, 8_000_000, 25, 0)
    assert st == 0
    # one binary64 R and T block per row block dominates: well under the data size
    assert 0 < b < 8_000_000 * 25 * 8 // 4
    st2, b2 = _ws(lib, 0, 100_000, 10, 0, block_rows=1000)
    assert st2 == 0 and b2 >= 100 * 2 * 10 * 10 * 8


def test_workspace_tiled_blocks(lib):
    """Blocks taller than the register tile are accepted: one R per block and
    one T per tile (lower bound with 640-row tiles, then 614-row tiles; the
    default binary64 tile at n = 25 is smaller, so it needs more)."""
    st, b = _ws(lib, 0, 200_000, 25, 0, block_rows=5000)
    assert st == 0
    p, kt = 40, 1 + -(-(5000 - 640) // 614)
    assert b >= (p + p * kt) * 25 * 25 * 8


@pytest.mark.parametrize("m,n,dt,b,f,want", [
    (10, 20, 0, 0, 0, 2),       # m < n
    (100, 0, 0, 0, 0, 2),       # n < 1
    (1000, 101, 0, 0, 0, 2),    # n > NMAX
    (1000, 10, 0, 5, 0, 2),     # block_rows < n
    (1000, 10, 0, 0, 1, 1),     # fanout 1
    (1000, 10, 7, 0, 0, 1),     # bad dtype
])
def test_workspace_size_rejects(lib, m, n, dt, b, f, want):
    st, _ = _ws(lib, 0, m, n, dt, b, f)
    assert st == want


@pytest.mark.parametrize("dt", [0, 1])
def test_plans_for_every_n(lib, dt):
    """Every op has a plan (tile choice, tree, workspace) for n = 1 .. NMAX."""
    for n in range(1, 101):
        for op in range(8):
            st, b = _ws(lib, op, 300_000, n, dt)
            assert st == 0 and b > 0, (op, n, st)


def _launches(lib, op, m, n, dt, block_rows=0):
    f = lib.tsqr_launch_count
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Opts),
                  ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int
    o = Opts(block_rows, 0, 0, None, 0, 0)
    out = ctypes.c_int32(0)
    assert f(op, m, n, dt, ctypes.byref(o), 0, ctypes.byref(out)) == 0
    return out.value


def test_host_path_plan(lib):
    """tsqr_direct_host (op 5): one copy chunk for a small problem (the same
    launches as tsqr_direct); a 1.6 GB matrix is split into several chunks
    of whole waves, each chunk adding a Step-1, T and Step-3 launch."""
    assert _launches(lib, 5, 100_000, 10, 0, block_rows=1000) == _launches(lib, 0, 100_000, 10, 0, block_rows=1000)
    big_host, big_dev = _launches(lib, 5, 8_000_000, 25, 0), _launches(lib, 0, 8_000_000, 25, 0)
    assert big_host >= big_dev + 3 * 3
    st, b = _ws(lib, 5, 8_000_000, 25, 0)
    assert st == 0 and 0 < b < 8_000_000 * 25 * 8 // 4


def test_r_only_plans(lib):
    """tsqr_r (op 6) launches one local QR per tree level and the sign fix;
    tsqr_svd_values (op 7) adds the Jacobi SVD; both take the workspace of
    tsqr_direct (op 0)."""
    for m, n, b in [(100_000, 10, 1000), (8_000_000, 25, 0), (3000, 7, 64)]:
        direct = _launches(lib, 0, m, n, 0, block_rows=b)
        levels = (direct - 1) // 3
        assert _launches(lib, 6, m, n, 0, block_rows=b) == levels + 1
        assert _launches(lib, 7, m, n, 0, block_rows=b) == levels + 2
        assert _ws(lib, 6, m, n, 0, block_rows=b) == _ws(lib, 0, m, n, 0, block_rows=b)
    assert _ws(lib, 9, 1000, 10, 0)[0] == 1  # unknown op


def _r_fn(lib):
    f = lib.tsqr_r
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(Opts), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _sv_fn(lib):
    f = lib.tsqr_svd_values
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(Opts),
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


# Stand-in addresses: every case below is rejected by the host-side checks
# before any launch, so nothing is ever read or written through them.  Where
# a GPU is visible these tests are skipped: a check that stopped rejecting a
# case would otherwise launch kernels on those addresses.
_P16 = 1 << 20        # 16-byte aligned
_P8 = (1 << 20) + 8   # not 16-byte aligned


def _gpu_visible():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


stand_in_addresses = pytest.mark.skipif(_gpu_visible(), reason="stand-in device addresses: host-only test")


@pytest.mark.parametrize("args,want", [
    (dict(A=None), 1),                    # NULL A
    (dict(R=None), 1),                    # NULL R
    (dict(dtype=7), 1),                   # unknown dtype
    (dict(n=101), 2),                     # n > NMAX
    (dict(m=5), 2),                       # m < n
    (dict(lda=11), 3),                    # lda != n
    (dict(A=_P8), 3),                     # A not 16-byte aligned
    (dict(ldr=9), 3),                     # ldr != n
    (dict(R=_P8), 3),                     # R not 16-byte aligned
    (dict(work=None), 4),                 # no workspace
    (dict(work_bytes=64), 4),             # workspace too small
    (dict(prec=2), 1),                    # TF32X3 on FP64 data
])
@stand_in_addresses
def test_r_only_rejects_before_any_launch(lib, args, want):
    """tsqr_r's argument, shape, alignment and workspace errors (Sec. II-B
    R-only TSQR) are returned synchronously, before any launch."""
    a = dict(A=_P16, m=1000, n=10, lda=10, dtype=0, R=_P16, ldr=10, work=_P16, work_bytes=1 << 30, prec=0)
    a.update(args)
    if "lda" not in args and "n" in args:
        a["lda"] = a["n"]
        a["ldr"] = a["n"]
    o = Opts(0, 0, 0, None, a["prec"], 0)
    st = _r_fn(lib)(a["A"], a["m"], a["n"], a["lda"], a["dtype"], a["R"], a["ldr"], a["work"], a["work_bytes"],
                    ctypes.byref(o), None)
    assert st == want


@pytest.mark.parametrize("args,want", [
    (dict(S=None), 1),                    # NULL S
    (dict(ldv=9), 3),                     # V given with ldv != n
    (dict(S=_P8), 3),                     # S not 16-byte aligned
    (dict(V=_P8), 3),                     # V given, not 16-byte aligned
    (dict(n=0), 2),                       # n < 1
    (dict(work=None), 4),                 # no workspace
])
@stand_in_addresses
def test_svd_values_rejects_before_any_launch(lib, args, want):
    """tsqr_svd_values (Sec. III-B, singular values only) checks its
    arguments before any launch; V may be NULL (only S wanted)."""
    a = dict(A=_P16, m=1000, n=10, lda=10, S=_P16, V=_P16, ldv=10, work=_P16, work_bytes=1 << 30)
    a.update(args)
    if "n" in args:
        a["lda"] = a["ldv"] = a["n"]
    o = Opts(0, 0, 0, None, 0, 0)
    st = _sv_fn(lib)(a["A"], a["m"], a["n"], a["lda"], 0, a["S"], a["V"], a["ldv"], a["work"], a["work_bytes"],
                     ctypes.byref(o), None)
    assert st == want


class PlanInfo(ctypes.Structure):
    _fields_ = [("block_rows", ctypes.c_int64), ("blocks", ctypes.c_int64), ("tiles_per_block", ctypes.c_int32),
                ("tree_levels", ctypes.c_int32), ("tree_fanout", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("step3_tensor", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _plan(lib, op, m, n, dt, block_rows=0, fanout=0, prec=0):
    f = lib.tsqr_plan_query
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Opts),
                  ctypes.POINTER(PlanInfo)]
    f.restype = ctypes.c_int
    o = Opts(block_rows, fanout, 0, None, prec, 0)
    info = PlanInfo()
    st = f(op, m, n, dt, ctypes.byref(o), ctypes.byref(info))
    return st, info


def test_plan_query_partition_and_tree(lib):
    """The row-block partition of Sec. III-B's example shape and the Alg. 2
    tree: 100,000 x 10 in blocks of 1,000 gives 100 R factors; with 10 of
    them per node the tree has two levels (100 -> 10 -> 1)."""
    st, info = _plan(lib, 0, 100_000, 10, 0, block_rows=1000, fanout=10)
    assert st == 0
    assert (info.block_rows, info.blocks) == (1000, 100) and info.tiles_per_block >= 1
    assert info.tree_fanout == 10 and info.tree_levels == 2
    # one block: no tree
    st, info = _plan(lib, 0, 900, 10, 0, block_rows=1000)
    assert st == 0 and info.blocks == 1 and info.tree_levels == 0
    # levels agree with the launch count (3 launches per level + sign fix)
    for m, n, b in [(8_000_000, 25, 0), (50_000_000, 50, 1024), (50_000_000, 50, 8192)]:
        st, info = _plan(lib, 0, m, n, 1 if n == 50 else 0, block_rows=b)
        assert st == 0
        assert _launches_dt(lib, 0, m, n, 1 if n == 50 else 0, b) == 3 * (info.tree_levels + 1) + 1
        assert info.blocks == -(-m // info.block_rows)


def _launches_dt(lib, op, m, n, dt, block_rows):
    f = lib.tsqr_launch_count
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Opts),
                  ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int
    o = Opts(block_rows, 0, 0, None, 0, 0)
    out = ctypes.c_int32(0)
    assert f(op, m, n, dt, ctypes.byref(o), 0, ctypes.byref(out)) == 0
    return out.value


@pytest.mark.parametrize("dt,n,want_prec,want_tc", [
    (1, 10, 0, 0),   # binary32 below n = 20: native binary32 Step 3
    (1, 50, 2, 1),   # binary32 from n = 20: 3xTF32 Step 3 on the tensor cores (the chunk stream)
    (1, 64, 2, 1),
    (1, 100, 2, 1),  # ... up to n = 100 (the wide form)
    (0, 64, 0, 0),   # binary64 data above n = 32: native binary64
    (0, 25, 4, 1),   # binary64 data at n <= 32: the Ozaki form
])
def test_auto_precision_plan(lib, dt, n, want_prec, want_tc):
    """TSQR_PREC_AUTO resolves to 3xTF32 for binary32 data at n >= 20 (where
    it is the faster Step 3; the split-precision products are asked for from
    n = 64), to the
    Ozaki form for binary64 data at n <= 32, and to the data's own arithmetic
    otherwise."""
    st, info = _plan(lib, 0, 1_000_000, n, dt, prec=3)
    assert st == 0
    assert info.prec == want_prec and info.step3_tensor == want_tc
    # the explicit modes are reported as given
    st, info = _plan(lib, 0, 1_000_000, n, dt, prec=0)
    assert st == 0 and info.prec == 0 and info.step3_tensor == 0
    # R only: no Step 3, so never on the tensor cores
    st, info = _plan(lib, 6, 1_000_000, n, dt, prec=3)
    assert st == 0 and info.step3_tensor == 0


def test_plan_query_rejects(lib):
    assert _plan(lib, 0, 10, 20, 0)[0] == 2          # m < n
    assert _plan(lib, 9, 1000, 10, 0)[0] == 1        # unknown op
    assert _plan(lib, 0, 1000, 10, 0, prec=5)[0] == 1  # unknown precision mode
    assert _plan(lib, 0, 1000, 10, 1, prec=4)[0] == 1  # OZAKI on binary32 data
    assert _plan(lib, 0, 1000, 10, 0, prec=2)[0] == 1  # TF32X3 on binary64 data


@pytest.mark.parametrize("n,want_tc", [(10, 1), (25, 1), (32, 1), (33, 0), (64, 0)])
def test_ozaki_plan(lib, n, want_tc):
    """TSQR_PREC_OZAKI: binary64 data; Step 3 on the tensor cores for n <= 32
    (the exact-accumulation bound of the split), the binary64 FMA Step 3
    above; the row blocks and tree are those of the native plan."""
    st, info = _plan(lib, 0, 1_000_000, n, 0, prec=4)
    assert st == 0 and info.prec == 4 and info.step3_tensor == want_tc
    st, nat = _plan(lib, 0, 1_000_000, n, 0, prec=0)
    assert st == 0
    assert (info.block_rows, info.blocks, info.tree_levels) == (nat.block_rows, nat.blocks, nat.tree_levels)


def test_ozaki_launches_include_the_tensor_core_gram(lib):
    """In the Ozaki form Step 1 leaves out its Gram dot products and one more
    launch forms the T factors' Gram entries on the tensor cores (n <= 32
    with a one-row-group Step-1 tile, as at 8,000,000 x 25)."""
    f = lib.tsqr_launch_count
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Opts),
                  ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int

    def count(prec, n):
        o = Opts(0, 0, 0, None, prec, 0)
        out = ctypes.c_int32(0)
        assert f(0, 8_000_000, n, 0, ctypes.byref(o), 0, ctypes.byref(out)) == 0
        return out.value

    assert count(4, 25) == count(0, 25) + 1
    assert count(4, 50) == count(0, 50)  # above n = 32: the native binary64 form


@pytest.mark.parametrize("dt", [0, 1])
def test_cluster_tree_fanin(lib, dt):
    """Tree nodes too large for one CTA's shared memory (n > 84 at four
    triangles) are factored over a cluster of one CTA per triangle: the
    default fan-in there is 8 (20,000,000 x 100: 4 tree levels, where two
    triangles per node gave 10), any fan-in 2..8 is accepted, and 9 (no
    single-CTA node, no portable cluster) is rejected."""
    st, info = _plan(lib, 0, 20_000_000, 100, dt)
    assert st == 0 and info.tree_fanout == 8
    assert info.tree_levels == len(_tree_levels(info.blocks, 8))
    for f in (2, 5, 8):
        st, info = _plan(lib, 0, 2_000_000, 100, dt, block_rows=2000, fanout=f)
        assert st == 0 and info.tree_fanout == f
        assert info.tree_levels == len(_tree_levels(info.blocks, f))
    assert _plan(lib, 0, 2_000_000, 100, dt, block_rows=2000, fanout=9)[0] == 2  # TSQR_ERR_SHAPE
    # below the cluster range the single-CTA node keeps its larger fan-in
    st, info = _plan(lib, 0, 8_000_000, 25, dt)
    assert st == 0 and info.tree_fanout == 25


def _tree_levels(p, f):
    """Node counts of the Alg. 2 tree over p blocks with fan-in f."""
    out = []
    while p > 1:
        p = -(-p // f)
        out.append(p)
    return out


@pytest.mark.parametrize("m", [2**62, 2**63 - 1, 2**61 // 25 + 1])
def test_unrepresentable_sizes_rejected(lib, m):
    """A problem whose m x n x 8 bytes int64 cannot hold is a shape error for
    every op (no workspace size that wrapped around)."""
    for op in range(9):
        for dt in (0, 1):
            st, _ = _ws(lib, op, m, 25, dt)
            assert st == 2, (op, dt)
    st, _ = _plan(lib, 0, m, 25, 0)
    assert st == 2


def test_plan_and_workspace_invariants_over_sizes(lib):
    """Over sizes from tiny to far beyond any device (m up to 2^50 rows),
    explicit and automatic block heights and fan-ins: the row blocks cover
    the m rows, the tree ends in one R, and the workspace of every op that
    stacks R factors holds at least one binary64 n x n R per row block."""
    for m in [1, 99, 100, 101, 10**6, 2**31 + 5, 10**12, 2**50]:
        for n in [1, 7, 25, 100]:
            for b in [0, n, 1000, 2**40]:
                for f in [0, 2, 3, 2**20]:
                    for dt in (0, 1):
                        st, info = _plan(lib, 0, m, n, dt, block_rows=b, fanout=f)
                        if st != 0:
                            assert st in (2,), (m, n, b, f, dt, st)
                            continue
                        assert info.blocks >= 1 and info.blocks * info.block_rows >= m
                        assert (info.blocks - 1) * info.block_rows < m
                        assert (info.tree_levels == 0) == (info.blocks == 1)
                        # Alg. 2: each level merges tree_fanout R factors per node
                        levels, nodes = 0, info.blocks
                        while nodes > 1:
                            nodes = -(-nodes // info.tree_fanout)
                            levels += 1
                        assert info.tree_levels == levels, (m, n, b, f, dt)
                        if f:
                            assert info.blocks == 1 or info.tree_fanout == f
                        for op in (0, 1, 3, 6, 7):
                            s2, w = _ws(lib, op, m, n, dt, b, f)
                            assert s2 == 0 and w >= info.blocks * n * n * 8, (op, m, n, b, f, dt)


def test_binding_rejects_caller_buffers_of_the_wrong_shape_dtype_or_device():
    """The library can check neither the size nor the device of a buffer it is
    given a pointer to, so the binding refuses mis-sized, mistyped,
    non-contiguous or misplaced caller buffers before any call (host-only)."""
    import torch
    import paper_1301_1071_gb300 as T
    cpu = torch.device("cpu")
    ok = torch.empty(30, 4, dtype=torch.float64)
    assert T._check_buf(ok, (30, 4), torch.float64, cpu, "Q") is ok
    with pytest.raises(ValueError, match="must be"):
        T._check_buf(torch.empty(29, 4, dtype=torch.float64), (30, 4), torch.float64, cpu, "Q")
    with pytest.raises(ValueError, match="must be"):
        T._check_buf(torch.empty(30, 4, dtype=torch.float32), (30, 4), torch.float64, cpu, "Q")
    with pytest.raises(ValueError, match="contiguous"):
        T._check_buf(torch.empty(4, 30, dtype=torch.float64).t(), (30, 4), torch.float64, cpu, "Q")
    with pytest.raises(ValueError, match="on cuda"):
        T._check_buf(ok, (30, 4), torch.float64, torch.device("cuda", 0), "Q")
    with pytest.raises(TypeError):
        T._check_buf(ok.numpy(), (30, 4), torch.float64, cpu, "Q")
    # a workspace that is not on the call's device is refused, not used
    with pytest.raises(ValueError, match="work"):
        T._workspace(T.OP_DIRECT, 1000, 10, torch.float64, torch.device("cuda", 0), 0, 0,
                     torch.empty(1 << 20, dtype=torch.uint8))
    # work_bytes counts bytes, whatever the workspace tensor's dtype
    assert T._nbytes(torch.empty(10, dtype=torch.float64)) == 80
    # no CPU path: the accuracy checker refuses a host Q
    with pytest.raises(ValueError, match="CUDA"):
        T.accuracy(torch.empty(30, 4, dtype=torch.float64))


@pytest.mark.parametrize("n", [1, 25, 100])
def test_int64_limit_in_blocks_of_n_rows_rejected(lib, n):
    """A whose bytes int64 just holds, in row blocks of n rows: its R and T
    stacks alone would pass size_t, and its blocks gridDim.x; a shape error
    for every op that stacks R factors, not a wrapped size."""
    m = (2**63 - 1) // 8 // n
    for op in (0, 1, 3, 6, 7):
        st, _ = _ws(lib, op, m, n, 0, block_rows=n)
        assert st == 2, op


def test_grid_and_block_height_limits(lib):
    """The kernels launch one CTA per row block (per T slot in the T build)
    and take a block's height as int: more than 2^31 - 1 blocks or T slots,
    or a block taller than 2^31 - 1 rows, is a shape error rather than a
    truncated launch; below each limit the problem plans."""
    lim = 2**31 - 1
    n = 25
    assert _ws(lib, 0, (lim + 1) * n, n, 0, block_rows=n)[0] == 2   # 2^31 row blocks
    st, w = _ws(lib, 0, 2**30 * n, n, 0, block_rows=n)               # 2^30 row blocks
    assert st == 0 and w >= 2 * 2**30 * n * n * 8
    # double-float, n = 1: blocks of up to 2^20 register tiles of 4,096 rows
    # reach past 2^31 rows (a 2^33-row A is 64 GB)
    assert _plan(lib, 0, 2**33, 1, 0, block_rows=2**31 + 2**20, prec=1)[0] == 2
    st, info = _plan(lib, 0, 2**33, 1, 0, block_rows=lim, prec=1)
    assert st == 0 and info.block_rows == lim and info.tiles_per_block > 1
    # binary64, n = 25: tall blocks whose T slots (one per tile) pass 2^31 - 1
    st, info = _plan(lib, 0, 2**29, 25, 0, block_rows=2**28)
    kt = info.tiles_per_block
    assert st == 0 and info.blocks == 2 and kt > 1
    assert _plan(lib, 0, (lim // kt + 1) * 2**28, 25, 0, block_rows=2**28)[0] == 2
    assert _plan(lib, 0, (lim // kt) * 2**28, 25, 0, block_rows=2**28)[0] == 0


def test_reserved_option_field_must_be_zero(lib):
    f = lib.tsqr_workspace_size
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Opts),
                  ctypes.POINTER(ctypes.c_size_t)]
    f.restype = ctypes.c_int
    out = ctypes.c_size_t(0)
    assert f(0, 1000, 10, 0, ctypes.byref(Opts(0, 0, 0, None, 0, 1)), ctypes.byref(out)) == 1
    assert f(0, 1000, 10, 0, ctypes.byref(Opts(0, 0, 0, None, -1, 0)), ctypes.byref(out)) == 1  # prec < 0
    assert f(0, 1000, 10, 0, ctypes.byref(Opts(0, 0, 0, None, 0, 0)), ctypes.byref(out)) == 0


@pytest.mark.parametrize("dt,esz,precs", [(0, 8, (0, 1, 3, 4)), (1, 4, (0, 2, 3))])
def test_default_blocks_start_on_16_byte_boundaries(lib, dt, esz, precs):
    """The planner's own block heights keep every row block (and, with its
    tile heights, every register tile) starting on a 16-byte boundary, so
    that Step 1 and Step 3 stage them by bulk copies rather than the plain
    loads they fall back to for an unaligned start."""
    for n in range(1, 101):
        for m in (100_000, 1_000_003, 8_000_000, 50_000_000):
            for prec in precs:
                st, info = _plan(lib, 0, m, n, dt, prec=prec)
                if st == 0 and info.blocks > 1:
                    assert (info.block_rows * n * esz) % 16 == 0, (n, m, prec, info.block_rows)


@stand_in_addresses
def test_invalid_arguments_never_reach_a_launch(lib):
    """Seeded random argument combinations for tsqr_direct and tsqr_r: with
    no GPU, a call whose host checks pass ends in a failed launch
    (TSQR_ERR_CUDA), so every combination with an invalid argument must be
    refused with its own code before that point."""
    import random
    P, I64, I32, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
    fd = lib.tsqr_direct
    fd.argtypes = [P, I64, I64, I64, I32, P, I64, P, I64, P, SZ, ctypes.POINTER(Opts), P]
    fd.restype = ctypes.c_int
    fr = _r_fn(lib)
    rng = random.Random(1301107106)
    for _ in range(3000):
        ptrs = [rng.choice([_P16, _P16, _P16, None, _P8]) for _ in range(4)]  # A, Q (or R), R, work
        n = rng.choice([1, 10, 25, 100, 0, 101])
        m = rng.choice([n, 1000, 10**6, 5, 0, 2**62])
        ld = rng.choice([n, n, n + 1])
        dt = rng.choice([0, 1, 1, 7])
        wb = rng.choice([1 << 40, 1 << 40, 64])
        br, fo = rng.choice([0, 0, 5, 1000]), rng.choice([0, 0, 1, 2])
        prec, res = rng.choice([0, 0, 1, 2, 3, 4, 5]), rng.choice([0, 0, 0, 1])
        o = Opts(br, fo, 0, None, prec, res)
        A, Q, R, W = ptrs
        rest = (1 <= n <= 100 and n <= m <= 2**60 // max(n, 1) and ld == n and dt in (0, 1) and wb > 64
                and res == 0 and 0 <= prec <= 4 and fo != 1 and (br == 0 or br >= n))
        valid_r = rest and A == R == W == _P16   # tsqr_r takes no Q
        valid_d = valid_r and Q == _P16
        st_d = fd(A, m, n, ld, dt, Q, ld, R, ld, W, wb, ctypes.byref(o), None)
        st_r = fr(A, m, n, ld, dt, R, ld, W, wb, ctypes.byref(o), None)
        case = (ptrs, n, m, ld, dt, wb, br, fo, prec, res)
        assert valid_d or st_d != 5, case
        assert valid_r or st_r != 5, case
