"""GPU parity of Section 4's organisation (FOLD_METHOD_SLIDING: one warp per
column, groups of q splits relative to i, difference vectors at every cell)
against the oracle of the same algorithm and the Eq. 1 oracle: full D tables
bit-exact across q, ragged lengths, pair sets and input variants; the
structure traced on its table; and the entry points that refuse the method.
All calls go through the C-ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def folders():
    cache = {}

    def get(q, mask=oracle.MASK6):
        key = (q, mask)
        if key not in cache:
            cache[key] = fold.Folder(q=q, pair_mask=mask, method="sliding")
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
    ref = oracle.two_vector_sliding(seq, q, mask)
    bad = np.argwhere(D.astype(np.int32) != ref)
    assert bad.size == 0, f"q={q} n={n} first mismatch at {bad[0].tolist()}"
    assert mp == int(ref[0, n - 1])


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_full_tables_ragged(folders, q):
    f = folders(q)
    for n in sorted({0, 1, 2, 3, q - 1, q, q + 1, 2 * q, 31, 32, 33, 100, 257}):
        _check(f, synth.uniform(n, 31 * q + n), q, oracle.MASK6)


@pytest.mark.parametrize("mask", [oracle.MASK6, oracle.MASK4])
@pytest.mark.parametrize("kind", ["uniform", "gc_rich", "structured"])
def test_variants_and_masks(folders, mask, kind):
    _check(folders(8, mask), synth.variant(kind, 640, 55), 8, mask)


def test_n3000_equals_eq1(folders):
    """Several thousand columns in flight, more than one per resident warp at q = 10."""
    for q in (8, 10):
        seq = synth.uniform(3000, 1308 + q)
        mp, D = folders(q).score(seq, want_D=True)
        assert np.array_equal(D.astype(np.int32), oracle.nussinov(seq))


def test_device_path_and_structure(folders):
    f = folders(8)
    seq = synth.structured(900, 21)
    n = len(seq)
    codes = torch.from_numpy(fold.encode_codes(seq)).cuda()
    ws = torch.empty(f.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    f.score_dev(codes, ws, out)
    torch.cuda.synchronize()
    assert int(out.item()) == oracle.score(seq)
    # the table is D plus two n*n vector tables
    assert f.workspace_bytes(n) >= 10 * n * n
    mp, partner, db = f.structure(seq)
    assert mp == oracle.score(seq)
    assert np.array_equal(partner, oracle.traceback(seq))


def test_entry_points_that_refuse_the_method(folders):
    f = folders(8)
    with pytest.raises(fold.FoldError) as ei:
        f.batch(["GGGAAAUCC", "ACGU"])
    assert ei.value.code == fold.FOLD_EINVAL
    with pytest.raises(fold.FoldError) as ei:
        fold.fold_serve_start(f.ctx, 1 << 28, 4)
    assert ei.value.code == fold.FOLD_EINVAL
    with pytest.raises(fold.FoldError) as ei:
        f.tune(500)
    assert ei.value.code == fold.FOLD_EINVAL
    # switching back and forth keeps both methods exact
    g = fold.Folder(q=8)
    try:
        seq = synth.uniform(500, 9)
        a = g.score(seq)
        g.set_method("sliding")
        b = g.score(seq)
        g.set_method("two_vector")
        c = g.score(seq)
        assert a == b == c == oracle.score(seq)
    finally:
        g.close()
