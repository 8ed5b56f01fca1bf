"""GPU parity at full problem sizes, through the C-ABI.

* Single folds of n = 4000 and 6000 (uniform and GC-rich, q swept 4..10):
  the whole D table against the CPU oracle (Eq. 1), element by element.
* Large folds, n = 8000, 16384 and 32768 (uniform and the structured
  segment + reverse-complement variant), where the cubic oracle takes too
  long for the whole table:
    - sampled cells against the oracle: D(i,j) depends only on s_i..s_j, so
      the oracle's score of that substring is the expected value;
    - the unit-step invariants of Lemma 1 over the whole table
      (0 <= D(i,j+1) - D(i,j) <= 1 and 0 <= D(i-1,j) - D(i,j) <= 1);
    - Eq. 1 re-evaluated from the returned table at sampled cells, including
      the answer cell (0, n-1);
    - the plain kernel's table equals the two-vector kernel's.
* The split task queues (tile-only CTAs), with and without column mode,
  forced on at sizes the oracle finishes quickly, so those paths are
  compared element by element too; and every work split run repeatedly on
  the same inputs, tables against the oracle each time.
"""
import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu

BASE = {"A": 0, "C": 1, "G": 2, "U": 3}


def _full_equal(D, ref):
    bad = np.argwhere(D.astype(np.int32) != ref)
    assert bad.size == 0, f"first mismatch at {bad[0].tolist()}: gpu={D[tuple(bad[0])]} ref={ref[tuple(bad[0])]}"


def _check_invariants(D, block=4096):
    """Lemma 1 over the whole table (lower triangle and diagonal are zero)."""
    n = D.shape[0]
    assert not np.any(np.diagonal(D))
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        rows = D[r0:r1]
        assert not np.any(np.tril(rows, r0 - 1)), "nonzero entry below the diagonal"
        dh = np.diff(rows, axis=1)
        assert dh.min() >= 0 and dh.max() <= 1, f"row step outside {{0,1}} in rows {r0}..{r1}"
        if r0 > 0:
            dv = D[r0 - 1:r1 - 1].astype(np.int16) - rows
            assert dv.min() >= 0 and dv.max() <= 1, f"column step outside {{0,1}} in rows {r0}..{r1}"
        else:
            dv = rows[:-1] - rows[1:]
            assert dv.min() >= 0 and dv.max() <= 1


def _eq1_at(D, codes, mask, i, j):
    """Eq. 1 evaluated at (i, j) from the returned table itself."""
    inner = int(D[i + 1, j - 1]) if i + 1 <= j - 1 else 0
    best = ((mask >> (4 * int(codes[i]) + int(codes[j]))) & 1) + inner
    split = D[i, i:j].astype(np.int32) + D[i + 1:j + 1, j].astype(np.int32)
    return max(best, int(split.max()))


def _sample_cells(n, count, max_span, rng):
    cells = []
    for _ in range(count):
        span = int(rng.integers(1, max_span))
        i = int(rng.integers(0, n - span))
        cells.append((i, i + span))
    return cells


def _large_checks(f, seq, mask, rng, D_other=None):
    n = len(seq)
    mp, D = f.score(seq, want_D=True)
    assert mp == int(D[0, n - 1])
    _check_invariants(D)
    codes = np.array([BASE[c] for c in seq], dtype=np.int64)
    # Eq. 1 at sampled cells of every span, the answer cell and the last row/column
    picks = [(0, n - 1), (0, n // 2), (n // 2, n - 1), (n - 2, n - 1)]
    picks += [(int(a), int(a) + int(b)) for a, b in zip(rng.integers(0, n // 2, 200), rng.integers(1, n // 2, 200))]
    for i, j in picks:
        assert int(D[i, j]) == _eq1_at(D, codes, mask, i, j), f"Eq. 1 fails at ({i},{j})"
    # short spans against the oracle on the substring
    for i, j in _sample_cells(n, 40, 500, rng):
        assert int(D[i, j]) == oracle.score(seq[i:j + 1], mask), f"cell ({i},{j})"
    if D_other is not None:
        assert np.array_equal(D, D_other)
    return D


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
def test_config2_n8000_sampled(kind):
    seq = synth.variant(kind, 8000, 8000)
    rng = np.random.default_rng(8000)
    fp = fold.Folder(q=8, method="plain")
    try:
        Dp = fp.score(seq, want_D=True)[1]
    finally:
        fp.close()
    for q in [4, 8, 10]:
        f = fold.Folder(q=q)
        try:
            _large_checks(f, seq, oracle.MASK6, rng, D_other=Dp)
        finally:
            f.close()


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["uniform", "structured"])
def test_config3_n16384_sampled(kind):
    seq = synth.variant(kind, 16384, 16384)
    rng = np.random.default_rng(16384)
    fp = fold.Folder(q=8, method="plain")
    try:
        Dp = fp.score(seq, want_D=True)[1]
    finally:
        fp.close()
    f = fold.Folder(q=8)
    try:
        _large_checks(f, seq, oracle.MASK6, rng, D_other=Dp)
    finally:
        f.close()


@pytest.mark.slow
def test_config3_n32768_structured_sampled():
    seq = synth.structured(32768, 32768)
    rng = np.random.default_rng(32768)
    f = fold.Folder(q=8)
    try:
        D = _large_checks(f, seq, oracle.MASK6, rng)
        # the score alone (no table copy) agrees with the table
        assert f.score(seq) == int(D[0, -1])
    finally:
        f.close()


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
