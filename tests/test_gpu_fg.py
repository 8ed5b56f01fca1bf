"""GPU parity of Section 3.2's FG algorithm (FOLD_METHOD_FG: Algorithm 1's
groups with a table per row and group, built when the group completes)
against the FG oracle and the Eq. 1 oracle: full D tables bit-exact across q,
ragged lengths, pair sets and input variants, and the structure traced on its
table.  All calls go through the C-ABI."""
import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def folders():
    cache = {}

    def get(q, mask=oracle.MASK6):
        key = (q, mask)
        if key not in cache:
            cache[key] = fold.Folder(q=q, pair_mask=mask, method="fg")
        return cache[key]

    yield get
    for f in cache.values():
        f.close()


def _check(f, seq, q, mask):
    n = len(seq)
    mp, D = f.score(seq, want_D=True)
    if n == 0:
        assert mp == 0
        return
    ref = oracle.fg(seq, q, mask)
    bad = np.argwhere(D.astype(np.int32) != ref)
    assert bad.size == 0, f"q={q} n={n} first mismatch at {bad[0].tolist()}"
    assert mp == int(ref[0, n - 1])


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_full_tables_ragged(folders, q):
    f = folders(q)
    for n in sorted({0, 1, 2, 3, q - 1, q, q + 1, 2 * q - 1, 2 * q, 2 * q + 1, 33, 100, 257}):
        _check(f, synth.uniform(n, 41 * q + n), q, oracle.MASK6)


@pytest.mark.parametrize("mask", [oracle.MASK6, oracle.MASK4])
@pytest.mark.parametrize("kind", ["uniform", "gc_rich", "structured"])
def test_variants_and_masks(folders, mask, kind):
    _check(folders(3, mask), synth.variant(kind, 640, 56), 3, mask)


def test_n2000_equals_eq1(folders):
    for q in (3, 8):
        seq = synth.uniform(2000, 1400 + q)
        mp, D = folders(q).score(seq, want_D=True)
        assert np.array_equal(D.astype(np.int32), oracle.nussinov(seq))


def test_structure_and_refusals(folders):
    f = folders(3)
    seq = synth.structured(700, 23)
    mp, partner, db = f.structure(seq)
    assert mp == oracle.score(seq)
    assert np.array_equal(partner, oracle.traceback(seq))
    with pytest.raises(fold.FoldError) as ei:
        f.batch(["GGGAAAUCC"])
    assert ei.value.code == fold.FOLD_EINVAL
    with pytest.raises(fold.FoldError) as ei:
        fold.fold_serve_start(f.ctx, 1 << 28, 4)
    assert ei.value.code == fold.FOLD_EINVAL
