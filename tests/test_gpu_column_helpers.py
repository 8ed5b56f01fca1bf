"""Column mode with a helper warp per tile column (FOLD_OPT_COL_HELPERS), through the C-ABI: the
column warp computes only the rows of each tile while its helper loads the tile's inputs, does the
late middle blocks' lookups (Eq. 3) and the chunk merge, and publishes each finished tile.  Every
table must equal the oracle's (Eq. 1) element by element, for every q and tile width, with one,
two and four columns per tile CTA, with the partially memoised R, and fold after fold."""
import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


def _fold(f, seq, near, cpc, helpers):
    f.option(fold.FOLD_OPT_NEAR_CTAS, near)
    f.option(fold.FOLD_OPT_COLUMNS, cpc)
    f.option(fold.FOLD_OPT_COL_HELPERS, helpers)
    return f.score(seq, want_D=True)


@pytest.mark.parametrize("q", range(2, 11))
def test_helpers_every_q(q):
    f = fold.Folder(q=q)
    try:
        T = f.tile
        n = 37 * T + 11                     # 38 tile columns and a ragged last one
        for kind in ["uniform", "structured"]:
            seq = synth.variant(kind, n, 600 + q)
            ref = oracle.nussinov(seq)
            for cpc in [4, 1]:
                mp, D = _fold(f, seq, (38 + cpc - 1) // cpc, cpc, 1)
                assert mp == int(ref[0, n - 1])
                assert np.array_equal(D.astype(np.int32), ref), (q, kind, cpc)
    finally:
        f.close()


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 65, 700, 2501])
def test_helpers_sizes_and_repeats(n):
    seq = synth.gc_rich(n, 900 + n)
    ref = oracle.nussinov(seq)
    f = fold.Folder(q=8)
    try:
        NT = (n + 31) // 32
        for cpc in [2, 4]:
            for _ in range(2):
                mp, D = _fold(f, seq, max(1, (NT + cpc - 1) // cpc), cpc, 1)
                assert mp == (int(ref[0, n - 1]) if n else 0)
                assert np.array_equal(D.astype(np.int32), ref), (n, cpc)
    finally:
        f.close()


def test_helpers_memoised_r():
    seq = synth.uniform(2400, 77)
    ref = oracle.nussinov(seq)
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_R_MEMO, 1)
        mp, D = _fold(f, seq, 19, 4, 1)
        assert np.array_equal(D.astype(np.int32), ref)
    finally:
        f.close()


def test_helpers_off_and_on_agree_at_6000():
    """The benchmark's fold with and without helpers (automatic layout otherwise)."""
    seq = synth.uniform(6000, 1307 + 1)
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_COL_HELPERS, 0)
        mp0, D0 = f.score(seq, want_D=True)
        f.option(fold.FOLD_OPT_COL_HELPERS, 1)
        mp1, D1 = f.score(seq, want_D=True)
        assert mp0 == mp1 and np.array_equal(D0, D1)
    finally:
        f.close()


def test_helper_option_range():
    f = fold.Folder(q=8)
    try:
        for v in (-1, 0, 1):
            f.option(fold.FOLD_OPT_COL_HELPERS, v)
            assert f.option(fold.FOLD_OPT_COL_HELPERS) == v
        with pytest.raises(fold.FoldError):
            f.option(fold.FOLD_OPT_COL_HELPERS, 2)
    finally:
        f.close()


@pytest.mark.parametrize("join", [0, 1])
@pytest.mark.parametrize("helpers", [0, 1])
def test_finished_columns_join_chunks(join, helpers):
    """Tile CTAs whose columns are all finished take chunk tasks (FOLD_OPT_COL_JOIN), with and without
    helpers, 2 and 4 columns per tile CTA and the plain kernel: every table equals the oracle's."""
    n = 61 * 32 + 9
    seq = synth.structured(n, 4400 + join)
    ref = oracle.nussinov(seq)
    for method in ["two_vector", "plain"]:
        f = fold.Folder(q=8, method=method)
        try:
            f.option(fold.FOLD_OPT_COL_JOIN, join)
            assert f.option(fold.FOLD_OPT_COL_JOIN) == join
            for cpc in [4, 2]:
                if method == "plain" and helpers:
                    continue
                mp, D = _fold(f, seq, (62 + cpc - 1) // cpc, cpc, helpers)
                assert mp == int(ref[0, n - 1])
                assert np.array_equal(D.astype(np.int32), ref), (method, cpc, helpers, join)
        finally:
            f.close()
