"""The autotuner on the GPU: it measures the single-fold settings (work split
and chunk size) and q, keeps the fastest per size bucket, and folds with
them; results stay exact (compared with the oracle).  All through the C-ABI."""
import os

import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


def test_tune_keeps_fastest_and_stays_exact():
    f = fold.Folder(q=8)
    try:
        r = f.tune(3000, reps=2)
        assert r["q"] == 8
        assert r["ms"] > 0 and r["default_ms"] > 0
        # the automatic choice is one of the candidates, so the winner is never slower
        assert r["ms"] <= r["default_ms"] * (1 + 1e-6)
        assert r["near_ctas"] >= -1 and -1 <= r["columns"] <= 8 and 0 <= r["kchunk"] <= 64
        for seed in (1, 2):
            seq = synth.uniform(3000 + seed, 700 + seed)   # same size bucket
            assert f.score(seq) == oracle.score(seq)
    finally:
        f.close()


def test_tune_save_load_roundtrip(tmp_path):
    path = str(tmp_path / "tune.txt")
    f = fold.Folder(q=8)
    try:
        f.tune(1200, reps=1)
        f.tune(2500, reps=1)
        fold.fold_tune_save(f.ctx, path)
    finally:
        f.close()
    lines = [ln for ln in open(path) if ln.startswith("fold-tune-v1 ")]
    assert len(lines) == 2 and all(" q=8 method=0 " in ln for ln in lines)
    g = fold.Folder(q=8)
    try:
        fold.fold_tune_load(g.ctx, path)
        seq = synth.gc_rich(2500, 31)
        mp, D = g.score(seq, want_D=True)
        assert mp == oracle.score(seq)
    finally:
        g.close()
    # another q finds no entry of its own
    h = fold.Folder(q=6)
    try:
        with pytest.raises(fold.FoldError) as ei:
            fold.fold_tune_load(h.ctx, path)
        assert ei.value.code == fold.FOLD_EINVAL
        # saving keeps the q=8 lines
        h.tune(1200, reps=1)
        fold.fold_tune_save(h.ctx, path)
        text = open(path).read()
        assert text.count(" q=8 method=0 ") == 2 and text.count(" q=6 method=0 ") == 1
    finally:
        h.close()


def test_tune_q_single_and_batch():
    r = fold.fold_tune_q([1500], q_min=6, q_max=9)
    assert 6 <= r["q"] <= 9 and r["ms"] > 0
    f = fold.Folder(q=r["q"])
    try:
        seq = synth.structured(1500, 77)
        assert f.score(seq) == oracle.score(seq)
    finally:
        f.close()
    lens = [100 + 50 * k for k in range(16)]
    rb = fold.fold_tune_q(lens, q_min=7, q_max=8)
    assert rb["q"] in (7, 8) and rb["ms"] > 0


def test_tune_refused_while_serving():
    f = fold.Folder(q=8)
    try:
        fold.fold_serve_start(f.ctx, 1 << 28, 4)
        with pytest.raises(fold.FoldError) as ei:
            f.tune(500)
        assert ei.value.code == fold.FOLD_EAGAIN
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()
