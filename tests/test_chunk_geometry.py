"""The Step-3 chunk sequence of the streaming tensor-core kernels
(csrc/chunks.cuh) checked on the host: a small C++ harness
(tests/host/chunk_cover.cpp) compiles the header with g++ and walks the
sequence as the kernel's CTAs do (Sec. III-B Step 3: every row of every
block Q_i = Q1_i Q2_i is formed once).  For ragged last blocks, one-tile and
many-tile blocks, last tiles of one row and grids from 1 to 304 CTAs, every
row is visited exactly once and every chunk stays inside its tile, block and
T slot.  No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1301_1071_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "host", "chunk_cover.cpp")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("chunks") / "chunk_cover")
    subprocess.run([gxx, "-std=c++17", "-O2", "-Wall", "-I", CSRC, "-o", exe, SRC], check=True)
    return exe


def _run(exe, cases):
    txt = "".join(f"{m} {n} {b} {B} {bt} {g}\n" for m, n, b, B, bt, g in cases)
    r = subprocess.run([exe], input=txt, capture_output=True, text=True, timeout=600)
    lines = r.stdout.split("\n")
    assert r.returncode == 0, next((l for l in lines if l.startswith("FAIL")), r.stdout[-400:])
    assert sum(l.startswith("ok") for l in lines) == len(cases)


# (m, n, b, B, bt, grid): B = a register tile's rows, bt = rows per further tile
EDGE = [
    (1, 1, 1, 32, 31, 1),              # one row
    (37, 37, 37, 64, 24, 4),           # square A, one block, more CTAs than chunks
    (1000, 25, 1000, 640, 614, 3),     # one block of two tiles
    (100_000, 10, 1000, 1024, 1012, 152),  # 100 blocks of one tile
    (100_003, 10, 1000, 1024, 1012, 152),  # ragged last block (3 rows)
    (30_000, 16, 1500, 1024, 1008, 7),
    (60_000, 50, 2999, 512, 460, 152),     # many tiles, ragged tiles and blocks
    (200_000, 64, 2000, 384, 320, 304),
    (129, 1, 129, 128, 127, 2),         # last tile of one row
    (4097, 8, 4097, 256, 248, 152),     # one tall block of 17 tiles
    (1_000_003, 32, 0, 1024, 992, 152),  # b = 0 stands for the planner's 6,600-row blocks below
]


def test_chunk_sequence_edge_cases(harness):
    cases = [c if c[2] else (c[0], c[1], 6600, c[3], c[4], c[5]) for c in EDGE]
    _run(harness, cases)


def test_chunk_sequence_random_geometries(harness):
    rng = np.random.default_rng(1301107199)
    cases = []
    for _ in range(300):
        n = int(rng.integers(1, 65))
        B = int(32 * rng.integers(max(1, (n + 31) // 32), 65))
        bt = int(rng.integers(1, B - n + 1)) if B > n else 1
        m = int(rng.integers(n, 60_000))
        b = int(rng.integers(n, m + 1)) if rng.random() < 0.7 else m
        g = int(rng.choice([1, 2, 3, 7, 64, 152, 304]))
        cases.append((m, n, b, B, bt, g))
    _run(harness, cases)
