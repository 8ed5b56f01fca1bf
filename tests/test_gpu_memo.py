"""GPU parity of Section 3.2's partially memoised variant (FOLD_OPT_R_MEMO):
each CTA starts with an empty R and tabulates a row against every column
vector the first time one of its warps stages that horizontal vector.  The
results must equal the oracle exactly for every work split (column mode, tile
CTAs, one queue), batches and serving.  All calls go through the C-ABI."""
import time

import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


def _memo_folder(q, method="two_vector"):
    f = fold.Folder(q=q, method=method)
    f.option(fold.FOLD_OPT_R_MEMO, 1)
    assert f.option(fold.FOLD_OPT_R_MEMO) == 1
    return f


@pytest.mark.parametrize("q", [2, 3, 4, 6, 8, 9])
def test_memo_full_tables(q):
    f = _memo_folder(q)
    try:
        for n in sorted({1, 2, q + 1, 33, 257, 700}):
            seq = synth.uniform(n, 500 + 7 * q + n)
            mp, D = f.score(seq, want_D=True)
            assert np.array_equal(D.astype(np.int32), oracle.nussinov(seq)), (q, n)
    finally:
        f.close()


@pytest.mark.parametrize("near,cols", [(0, 0), (8, 0), (-1, 4), (-1, 8)])
def test_memo_every_work_split(near, cols):
    f = _memo_folder(8)
    try:
        f.option(fold.FOLD_OPT_NEAR_CTAS, near)
        f.option(fold.FOLD_OPT_COLUMNS, cols)
        seq = synth.variant("gc_rich", 2000, 91)
        mp, D = f.score(seq, want_D=True)
        assert np.array_equal(D.astype(np.int32), oracle.nussinov(seq))
    finally:
        f.close()


def test_memo_batch_serve_and_refusals():
    f = _memo_folder(8)
    try:
        seqs = [synth.variant(["uniform", "structured"][k % 2], 40 + 97 * k, 300 + k) for k in range(12)]
        assert list(f.batch(seqs)) == [oracle.score(s) for s in seqs]
        fold.fold_serve_start(f.ctx, 1 << 30, 16)
        with pytest.raises(fold.FoldError) as ei:
            f.option(fold.FOLD_OPT_R_MEMO, 0)
        assert ei.value.code == fold.FOLD_EAGAIN
        tickets = [fold.fold_serve_submit(f.ctx, s) for s in seqs[:6]]
        got, t0 = {}, time.time()
        while len(got) < len(tickets) and time.time() - t0 < 60:
            for t in tickets:
                if t not in got:
                    r = fold.fold_serve_poll(f.ctx, t)
                    if r is not None:
                        got[t] = r
            time.sleep(0.001)
        assert [got[t] for t in tickets] == [oracle.score(s) for s in seqs[:6]]
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()
    g = fold.Folder(q=10)
    try:
        with pytest.raises(fold.FoldError) as ei:
            g.option(fold.FOLD_OPT_R_MEMO, 1)
        assert ei.value.code == fold.FOLD_EINVAL
    finally:
        g.close()
    # the plain method has no table: the option leaves it exact
    p = _memo_folder(8, "plain")
    try:
        s = synth.uniform(900, 4)
        assert p.score(s) == oracle.score(s)
    finally:
        p.close()
