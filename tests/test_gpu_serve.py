"""Serving (continuous batching) on the GPU: requests that arrive while
others are in flight are admitted as memory frees up, share the persistent
launch (the serving ring, or slice launches with FOLD_OPT_SERVE_RING = 0) with
them, and every result equals the one the same sequence gives alone (exactly:
the work is integer).  All calls go through the C-ABI."""
import time

import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


def _drain(ctx, tickets, timeout=120.0, want_D=None):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            D = want_D.get(t) if want_D else None
            r = fold.fold_serve_poll(ctx, t, D)
            if r is not None:
                out[t] = r
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.001)
    return out


@pytest.mark.parametrize("ring", [1, 0])
def test_serve_mix_equals_alone(ring):
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_SERVE_RING, ring)
        kinds = ["uniform", "gc_rich", "structured"]
        lens = [0, 1, 2, 31, 32, 33, 100, 500, 1200, 64, 2500, 7, 300, 900]
        seqs = [synth.variant(kinds[k % 3], L, 900 + k) for k, L in enumerate(lens)]
        alone = [f.score(s, want_D=True) for s in seqs]
        fold.fold_serve_start(f.ctx, 8 << 30, 64)
        tickets = []
        tables = {}
        # staggered arrivals: some while others are already on the GPU
        for k, s in enumerate(seqs):
            t = fold.fold_serve_submit(f.ctx, s)
            tickets.append(t)
            if len(s):
                tables[t] = np.full((len(s), len(s)), -1, dtype=np.int16)
            if k % 4 == 3:
                time.sleep(0.002)
        res = _drain(f.ctx, tickets, want_D=tables)
        got = [res[t] for t in tickets]
        assert got == [a[0] for a in alone]
        assert got == [oracle.score(s) if len(s) else 0 for s in seqs]
        # every full table folded in the mix equals the one folded alone and the oracle's (Eq. 1)
        for t, s, (mp, D_alone) in zip(tickets, seqs, alone):
            if not len(s):
                continue
            assert np.array_equal(tables[t], D_alone), len(s)
            assert np.array_equal(tables[t].astype(np.int32), oracle.nussinov(s)), len(s)
        st = fold.fold_serve_stats(f.ctx)
        nonempty = sum(1 for s in seqs if len(s))
        assert st["admitted"] == st["finished"] == nonempty
        assert st["queued"] == 0 and st["inflight"] == 0
        assert st["slices"] >= 1 and st["tasks"] >= nonempty
        assert 0 < st["gpu_ms"] <= st["slice_ms"] and st["prep_ms"] >= 0
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()


def test_serve_long_request_cap():
    # requests of at least 20 tile columns (n >= 609) are long and at most one of them is in flight:
    # the others wait in arrival order while the short ones pass them; every answer as the oracle's
    f = fold.Folder(q=8)
    try:
        assert f.option(fold.FOLD_OPT_SERVE_LONG_TILES) == 160 and f.option(fold.FOLD_OPT_SERVE_LONG_CAP) == 2
        for opt, bad in ((fold.FOLD_OPT_SERVE_LONG_TILES, 0), (fold.FOLD_OPT_SERVE_LONG_CAP, -1)):
            with pytest.raises(fold.FoldError) as ei:
                f.option(opt, bad)
            assert ei.value.code == fold.FOLD_EINVAL
        f.option(fold.FOLD_OPT_SERVE_LONG_TILES, 20)
        f.option(fold.FOLD_OPT_SERVE_LONG_CAP, 1)
        kinds = ["uniform", "gc_rich", "structured"]
        lens = [900, 40, 1300, 75, 650, 120, 1100, 33, 700, 260, 610, 9]
        seqs = [synth.variant(kinds[k % 3], L, 5100 + k) for k, L in enumerate(lens)]
        fold.fold_serve_start(f.ctx, 8 << 30, 64)
        with pytest.raises(fold.FoldError) as ei:
            f.option(fold.FOLD_OPT_SERVE_LONG_CAP, 3)   # fixed while serving
        assert ei.value.code == fold.FOLD_EAGAIN
        tickets = [fold.fold_serve_submit(f.ctx, s) for s in seqs]
        res = _drain(f.ctx, tickets)
        assert [res[t] for t in tickets] == [oracle.score(s) for s in seqs]
        st = fold.fold_serve_stats(f.ctx)
        assert st["admitted"] == st["finished"] == len(seqs)
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()


def test_serve_lone_requests_fold_in_one_launch():
    # each request arrives to an idle server: up to 8192 long it folds in one launch with the single
    # fold's work split (stats "solo"), longer ones slice by slice; scores and tables as alone
    f = fold.Folder(q=8)
    try:
        seqs = [synth.uniform(2, 51), synth.gc_rich(33, 52), synth.structured(700, 53), synth.uniform(3000, 54),
                synth.uniform(8192, 55), synth.gc_rich(9000, 56)]
        alone = [f.score(s) for s in seqs]
        fold.fold_serve_start(f.ctx, 8 << 30, 64)
        for k, s in enumerate(seqs):
            t = fold.fold_serve_submit(f.ctx, s)
            D = np.zeros((len(s), len(s)), dtype=np.int16) if len(s) <= 700 else None
            r = _drain(f.ctx, [t], want_D={t: D} if D is not None else None)[t]
            assert r == alone[k]
            if D is not None:
                ref = oracle.nussinov(s)
                assert r == ref[0, len(s) - 1]
                assert np.array_equal(D.astype(np.int32), ref)
        st = fold.fold_serve_stats(f.ctx)
        assert st["solo"] == 5
        assert st["admitted"] == st["finished"] == len(seqs)
        assert st["slices"] > st["solo"]   # the 9000-long one took the ring launch (or slice launches)
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()


@pytest.mark.parametrize("ring", [1, 0])
def test_serve_wait_any_reports_each_finished_request_once(ring):
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_SERVE_RING, ring)
        fold.fold_serve_start(f.ctx, 8 << 30, 64)
        assert fold.fold_serve_wait_any(f.ctx, 20) is None   # nothing submitted: times out
        seqs = [synth.uniform(n, 70 + n) for n in (0, 5, 64, 400, 1500, 3000, 200)]
        tickets = [fold.fold_serve_submit(f.ctx, s) for s in seqs]
        got = {}
        while len(got) < len(seqs):
            t = fold.fold_serve_wait_any(f.ctx, 5000)
            assert t is not None and t in tickets and t not in got
            got[t] = fold.fold_serve_poll(f.ctx, t)
        assert [got[t] for t in tickets] == [oracle.score(s) if len(s) else 0 for s in seqs]
        # a ticket collected by poll before wait_any reports it is skipped
        t = fold.fold_serve_submit(f.ctx, synth.uniform(300, 9))
        while fold.fold_serve_poll(f.ctx, t) is None:
            time.sleep(0.001)
        assert fold.fold_serve_wait_any(f.ctx, 20) is None
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()


@pytest.mark.parametrize("ring", [1, 0])
def test_serve_budget_admission_and_tables(ring):
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_SERVE_RING, ring)
        one = f.workspace_bytes(800)
        # room for about three 800-base requests at a time
        fold.fold_serve_start(f.ctx, int(3.5 * one), 16)
        seqs = [synth.uniform(800, 40 + k) for k in range(10)]
        tickets = [fold.fold_serve_submit(f.ctx, s) for s in seqs]
        Ds = {t: np.zeros((800, 800), dtype=np.int16) for t in tickets[:3]}
        res = _drain(f.ctx, tickets, want_D=Ds)
        for t, s in zip(tickets, seqs):
            assert res[t] == oracle.score(s)
        for t, s in zip(tickets[:3], seqs[:3]):
            assert np.array_equal(Ds[t].astype(np.int32), oracle.nussinov(s))
        # a request that can never fit the budget is refused, not queued forever
        with pytest.raises(fold.FoldError) as ei:
            fold.fold_serve_submit(f.ctx, synth.uniform(4000, 1))
        assert ei.value.code == fold.FOLD_EAGAIN
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()


def test_serve_poll_unknown_ticket_and_restart():
    f = fold.Folder(q=8)
    try:
        fold.fold_serve_start(f.ctx, 1 << 28, 4)
        with pytest.raises(fold.FoldError) as ei:
            fold.fold_serve_poll(f.ctx, 123456)
        assert ei.value.code == fold.FOLD_EINVAL
        t = fold.fold_serve_submit(f.ctx, "GGGAAAUCC")
        assert _drain(f.ctx, [t])[t] == 3
        fold.fold_serve_stop(f.ctx)
        fold.fold_serve_start(f.ctx, 1 << 28, 4)
        t = fold.fold_serve_submit(f.ctx, "ACUGACUG")
        assert _drain(f.ctx, [t])[t] == 3
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()


def test_serve_warm_then_mixed_lengths():
    """Task lists built ahead (for every length up to 3000) give the same results as lists built
    at first use; lengths past the warmed range still work."""
    f = fold.Folder(q=8)
    try:
        with pytest.raises(fold.FoldError) as ei:
            fold.fold_serve_warm(f.ctx, -1)
        assert ei.value.code == fold.FOLD_EINVAL
        fold.fold_serve_warm(f.ctx, 3000)
        fold.fold_serve_start(f.ctx, 4 << 30, 32)
        lens = [40, 999, 2048, 3000, 3100, 17, 1500]
        seqs = [synth.variant(["uniform", "gc_rich", "structured"][k % 3], L, 4200 + k) for k, L in enumerate(lens)]
        tickets = [fold.fold_serve_submit(f.ctx, s) for s in seqs]
        res = _drain(f.ctx, tickets)
        assert [res[t] for t in tickets] == [oracle.score(s) for s in seqs]
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()


def test_serve_ring_restarts_and_option_while_serving():
    """The ring launch stops whenever nothing is in flight and starts again with the next requests;
    bursts separated by idle gaps, each mixing short and long requests, all equal the oracle."""
    f = fold.Folder(q=8)
    try:
        fold.fold_serve_start(f.ctx, 4 << 30, 64)
        with pytest.raises(fold.FoldError) as ei:   # fixed while serving
            f.option(fold.FOLD_OPT_SERVE_RING, 0)
        assert ei.value.code == fold.FOLD_EAGAIN
        for burst in range(3):
            seqs = [synth.variant(["uniform", "structured"][k % 2], L, 7000 + 10 * burst + k)
                    for k, L in enumerate([2500, 30, 600, 1, 1200, 90])]
            tickets = [fold.fold_serve_submit(f.ctx, x) for x in seqs]
            res = _drain(f.ctx, tickets)
            assert [res[t] for t in tickets] == [oracle.score(x) if len(x) else 0 for x in seqs]
            time.sleep(0.05)   # idle: the launch ends
        st = fold.fold_serve_stats(f.ctx)
        assert st["inflight"] == 0 and st["queued"] == 0
    finally:
        fold.fold_serve_stop(f.ctx)
        f.close()
