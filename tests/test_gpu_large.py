"""GPU parity at full problem sizes, through the C-ABI.

* Single folds of n = 4000 and 6000 (uniform and GC-rich, q swept 4..10):
  the whole D table against the CPU oracle (Eq. 1), element by element.
* Large folds, n = 8000, 16384 and 32768 (uniform, GC-rich and the
  structured segment + reverse-complement variant): the whole table against
  the CPU oracle's, through digests the oracle wrote once
  (oracle/make_digests.py, stored in tests/golden/digest_*.txt): the SHA-256
  of the row-major int16 table, the CRC-32 of every row and D(0, n-1).  A
  mismatch names the rows that differ.
* The split task queues (tile-only CTAs), with and without column mode,
  forced on at sizes the oracle finishes quickly, so those paths are
  compared element by element too; and every work split run repeatedly on
  the same inputs, tables against the oracle each time.
"""
import hashlib

import numpy as np
import pytest

import oracle
from oracle.make_digests import digest_path, read_digest, table_digests
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu

def _full_equal(D, ref):
    bad = np.argwhere(D.astype(np.int32) != ref)
    assert bad.size == 0, f"first mismatch at {bad[0].tolist()}: gpu={D[tuple(bad[0])]} ref={ref[tuple(bad[0])]}"


def _digest_check(D, seq, variant, seed, what, mask=oracle.MASK6):
    """The whole table D (n*n int16) against the oracle's digest of the same input."""
    n = len(seq)
    ref = read_digest(digest_path(n, variant, mask))
    assert (ref["n"], ref["variant"], ref["seed"], ref["mask"]) == (n, variant, seed, mask)
    assert ref["seq_sha256"] == hashlib.sha256(seq.encode()).hexdigest(), "the input generator changed"
    assert int(D[0, n - 1]) == ref["score"], f"{what}: D(0,n-1) = {int(D[0, n - 1])}, oracle {ref['score']}"
    sha, crcs = table_digests(D)
    if sha != ref["table_sha256"]:
        bad = [i for i, (x, y) in enumerate(zip(crcs, ref["row_crc32"])) if x != y]
        pytest.fail(f"{what}: table differs from the oracle's in {len(bad)} rows, first {bad[:8]}")


def _fold_table(method, q, seq):
    f = fold.Folder(q=q, method=method)
    try:
        mp, D = f.score(seq, want_D=True)
        assert mp == int(D[0, len(seq) - 1])
        return D
    finally:
        f.close()


# (n, tile CTAs, column mode): 700 bases are 22 tile columns, 2000 bases 63 (q = 8), so one tile
# CTA (8 warps) cannot hold every column and three can; column mode off keeps the tile-task queue
SPLITS = [(700, 1, -1), (700, 3, 0), (700, 3, -1), (2000, 8, 0), (2000, 8, -1), (2000, 30, -1), (1500, 6, 8), (1500, 12, 4), (2000, 33, 2)]


@pytest.mark.parametrize("method", ["two_vector", "plain"])
@pytest.mark.parametrize("n,near,cols", SPLITS)
def test_split_queues_full_table(method, n, near, cols):
    f = fold.Folder(q=8, method=method)
    try:
        f.option(fold.FOLD_OPT_NEAR_CTAS, near)
        f.option(fold.FOLD_OPT_COLUMNS, cols)
        seq = synth.uniform(n, 4242 + n + near)
        mp, D = f.score(seq, want_D=True)
        ref = oracle.nussinov(seq)
        assert mp == int(ref[0, n - 1])
        _full_equal(D, ref)
    finally:
        f.close()


@pytest.mark.parametrize("q", [2, 3, 4, 6, 10])
def test_column_mode_all_q(q):
    """Column mode with every tile width (T = 30 for q = 3, 6, 10) and group count."""
    f = fold.Folder(q=q)
    try:
        n = 37 * f.tile + 11   # 38 tile columns
        f.option(fold.FOLD_OPT_NEAR_CTAS, (37 + 1 + 7) // 8)
        for kind in ["uniform", "structured"]:
            seq = synth.variant(kind, n, 500 + q)
            ref = oracle.nussinov(seq)
            # 8 columns per CTA (shared-memory handoffs) and 1 (every left neighbour through its flag)
            for cpc in [8, 1]:
                f.option(fold.FOLD_OPT_COLUMNS, cpc)
                mp, D = f.score(seq, want_D=True)
                assert mp == int(ref[0, n - 1])
                _full_equal(D, ref)
    finally:
        f.close()


@pytest.mark.slow
def test_config2_n4000_gc_rich_q_sweep():
    seq = synth.gc_rich(4000, 4000)
    ref = oracle.nussinov(seq)
    for q in range(4, 11):
        f = fold.Folder(q=q)
        try:
            mp, D = f.score(seq, want_D=True)
            assert mp == int(ref[0, 3999]), f"q={q}"
            _full_equal(D, ref)
        finally:
            f.close()
    f = fold.Folder(q=8, method="plain")
    try:
        _full_equal(f.score(seq, want_D=True)[1], ref)
    finally:
        f.close()


@pytest.mark.slow
def test_config2_n6000_full_table():
    """The benchmark's single-fold workload, whole table, both kernels."""
    seq = synth.uniform(6000, 1307 + 1)
    ref = oracle.nussinov(seq)
    for method in ["two_vector", "plain"]:
        f = fold.Folder(q=8, method=method)
        try:
            mp, D = f.score(seq, want_D=True)
            assert mp == int(ref[0, 5999])
            _full_equal(D, ref)
        finally:
            f.close()


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["uniform", "gc_rich"])
def test_config2_n8000_full_table(kind):
    seq = synth.variant(kind, 8000, 8000)
    _digest_check(_fold_table("plain", 8, seq), seq, kind, 8000, "plain")
    for q in [4, 8, 10]:
        _digest_check(_fold_table("two_vector", q, seq), seq, kind, 8000, f"two-vector q={q}")


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["uniform", "structured"])
def test_config3_n16384_full_table(kind):
    seq = synth.variant(kind, 16384, 16384)
    _digest_check(_fold_table("plain", 8, seq), seq, kind, 16384, "plain")
    _digest_check(_fold_table("two_vector", 8, seq), seq, kind, 16384, "two-vector q=8")


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["structured", "uniform"])
def test_config3_n32768_full_table(kind):
    seq = synth.variant(kind, 32768, 32768)
    f = fold.Folder(q=8)
    try:
        mp, D = f.score(seq, want_D=True)
        _digest_check(D, seq, kind, 32768, "two-vector q=8")
        # the score alone (no table copy) agrees with the table
        assert f.score(seq) == mp == int(D[0, -1])
    finally:
        f.close()
    del D
    _digest_check(_fold_table("plain", 8, seq), seq, kind, 32768, "plain")


def test_layouts_full_tables_repeated():
    # every work split (automatic, which is column mode at this size, one shared queue, tile-only
    # CTAs), each fold run twice: the tables must equal the oracle's every time.  The chunks'
    # merges are bulk reductions whose ordering against the chunk counters rests on async-proxy
    # fences; a missing fence would show as an occasional stale partial maximum.
    for seed in range(4):
        s = synth.variant(["uniform", "gc_rich", "structured"][seed % 3], 2500, 4000 + seed)
        ref = oracle.nussinov(s)
        for near, cols in ((-1, -1), (0, -1), (24, 0)):
            f = fold.Folder(q=8)
            try:
                f.option(fold.FOLD_OPT_NEAR_CTAS, near)
                f.option(fold.FOLD_OPT_COLUMNS, cols)
                for _ in range(2):
                    mp, D = f.score(s, want_D=True)
                    assert mp == ref[0, -1]
                    assert np.array_equal(D.astype(np.int32), ref)
            finally:
                f.close()


def test_column_mode_joining_with_short_wait_bound():
    """n = 16384 in column mode with 8 columns per tile CTA, the tile CTAs joining the chunk workers,
    and a 10 ms bound on every device wait: the first tile CTA's idle warps wait for its last column
    about as long as the whole fold (~24 ms) and must leave quietly, not fail the fold; the table
    equals the oracle's digest."""
    seq = synth.variant("uniform", 16384, 16384)
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_COLUMNS, 8)
        f.option(fold.FOLD_OPT_COL_JOIN, 1)
        f.option(fold.FOLD_OPT_TIMEOUT_MS, 10)
        mp, D = f.score(seq, want_D=True)
        _digest_check(D, seq, "uniform", 16384, "two-vector, column mode, joining")
    finally:
        f.close()
