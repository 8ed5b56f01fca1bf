"""GPU parity: every D table and score from the CUDA library equals the CPU
oracle exactly (integer work, bit-exact), for the two-vector kernel and the
plain comparison kernel, across q, ragged lengths, pair sets and input
variants.  All calls go through the C-ABI (paper_1307_7820_b300.fold)."""
import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu

MASKS = [oracle.MASK6, oracle.MASK4]


@pytest.fixture(scope="module")
def folders():
    cache = {}

    def get(q, method="two_vector", mask=oracle.MASK6):
        key = (q, method, mask)
        if key not in cache:
            cache[key] = fold.Folder(q=q, pair_mask=mask, method=method)
        return cache[key]

    yield get
    for f in cache.values():
        f.close()


def _full_check(f, seq, mask):
    mp, D = f.score(seq, want_D=True)
    ref = oracle.nussinov(seq, mask)
    n = len(seq)
    assert mp == (int(ref[0, n - 1]) if n else 0)
    if n:
        bad = np.argwhere(D.astype(np.int32) != ref)
        assert bad.size == 0, f"n={n} first mismatch at {bad[0].tolist()}: gpu={D[tuple(bad[0])]} ref={ref[tuple(bad[0])]}"


@pytest.mark.parametrize("q", list(range(2, 11)))
def test_rtable_matches_oracle(folders, q):
    assert np.array_equal(folders(q).rtable(), oracle.rtable(q))


@pytest.mark.parametrize("method", ["two_vector", "plain"])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 8, 9, 31, 32, 33, 63, 64, 65, 96, 127, 129, 200, 257])
def test_small_full_tables_q8(folders, method, n):
    seq = synth.uniform(n, 1000 + n)
    _full_check(folders(8, method), seq, oracle.MASK6)


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6, 7, 9, 10])
def test_full_tables_all_q(folders, q):
    f = folders(q)
    T = f.tile
    for n in sorted({1, q - 1, q, q + 1, T - 1, T, T + 1, 3 * T + 5, 333}):
        _full_check(f, synth.uniform(n, 77 * q + n), oracle.MASK6)


@pytest.mark.parametrize("method", ["two_vector", "plain"])
def test_config1_n1000(folders, method):
    """The n = 1000 workload: uniform ACGU, 6-pair set, q = 8, full D bit-exact."""
    seq = synth.uniform(1000, synth.SEED_BASE)
    _full_check(folders(8, method), seq, oracle.MASK6)


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("kind", ["gc_rich", "structured"])
def test_variants_and_masks(folders, mask, kind):
    for method in ("two_vector", "plain"):
        f = folders(8, method, mask)
        _full_check(f, synth.variant(kind, 700, 31), mask)


def test_asymmetric_mask(folders):
    m = oracle.mask_from_pairs(["AU", "CG", "GU"])
    f = folders(8, "two_vector", m)
    _full_check(f, synth.uniform(300, 5), m)


def test_lowercase_and_invalid(folders):
    f = folders(8)
    s = synth.uniform(120, 9)
    assert f.score(s.lower()) == f.score(s)
    with pytest.raises(fold.FoldError) as ei:
        f.score(s[:50] + "T" + s[51:])
    assert ei.value.code == fold.FOLD_EINVAL


@pytest.mark.parametrize("method", ["two_vector", "plain"])
def test_n2000_full(folders, method):
    seq = synth.gc_rich(2000, 2)
    _full_check(folders(8, method), seq, oracle.MASK6)


def test_batch_matches_single(folders):
    f = folders(8)
    T = f.tile
    lens = [0, 1, 2, 7, 8, 9, T - 1, T, T + 1, 100, 333, 64, 1000, 5, 250]
    seqs = [synth.uniform(L, 500 + k) for k, L in enumerate(lens)]
    res, Ds = f.batch(seqs, want_D=True)
    for s, r, D in zip(seqs, res, Ds):
        ref = oracle.nussinov(s)
        n = len(s)
        assert r == (ref[0, n - 1] if n else 0)
        if n:
            assert np.array_equal(D.astype(np.int32), ref)


def test_batch_threaded_encode_case_and_invalid(folders):
    # over 2 MB of bases: the host encodes the batch on several threads
    f = folders(8)
    seqs = synth.batch(900, 2000, 3000, 77)
    mixed = [s.lower() if k % 3 == 0 else s for k, s in enumerate(seqs)]
    r1 = f.batch(seqs)
    assert np.array_equal(f.batch(mixed), r1)
    k = int(np.argmin([len(s) for s in seqs]))
    assert r1[k] == oracle.score(seqs[k])
    for k in (1, 450, 899):
        assert r1[k] == f.score(seqs[k])
    bad = list(seqs)
    bad[600] = bad[600][:10] + "T" + bad[600][11:]
    with pytest.raises(fold.FoldError) as ei:
        f.batch(bad)
    assert ei.value.code == fold.FOLD_EINVAL
    assert np.array_equal(f.batch(seqs), r1)   # the context is still usable


def test_batch_gather_and_host_lists_agree(folders):
    # the task list gathered on the device from the context's template copies (default) and the one
    # built on the host; new length mixes each call, so the device store grows and is reused
    f = folders(8)
    try:
        for seed in (1, 2, 3):
            seqs = synth.batch(300, 20 + 100 * seed, 800 * seed, 900 + seed)
            f.option(fold.FOLD_OPT_BATCH_GATHER, 1)
            a = f.batch(seqs)
            f.option(fold.FOLD_OPT_BATCH_GATHER, 0)
            b = f.batch(seqs)
            assert np.array_equal(a, b)
            for k in np.argsort([len(x) for x in seqs])[:3]:
                assert a[k] == oracle.score(seqs[k])
    finally:
        f.option(fold.FOLD_OPT_BATCH_GATHER, 1)
    assert f.option(fold.FOLD_OPT_BATCH_GATHER) == 1


def test_batch_many_short(folders):
    f = folders(8)
    seqs = synth.batch(300, 20, 300, 4242)
    res = f.batch(seqs)
    want = np.array([oracle.score(s) for s in seqs])
    assert np.array_equal(res, want)


def test_device_path_torch(folders):
    torch = pytest.importorskip("torch")
    f = folders(8)
    seq = synth.uniform(777, 12)
    n = len(seq)
    codes = torch.from_numpy(fold.encode_codes(seq)).cuda()
    ws = torch.empty(f.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    D = torch.empty((n, n), dtype=torch.int16, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())   # inputs were written on the default stream
    f.score_dev(codes, ws, out, D, stream=s.cuda_stream)
    s.synchronize()
    ref = oracle.nussinov(seq)
    assert int(out.item()) == ref[0, n - 1]
    assert np.array_equal(D.cpu().numpy().astype(np.int32), ref)
    # run twice on the same workspace (reuse must not leak state)
    f.score_dev(codes, ws, out, None, stream=s.cuda_stream)
    s.synchronize()
    assert int(out.item()) == ref[0, n - 1]


def test_timeout_reports_status_and_context_survives():
    """Fault injected on the host: the task of tile (0,1) is left out of the
    schedule, so the tiles that depend on it wait on a flag nothing sets.  The
    bounded waits expire, the call returns FOLD_ETIMEOUT, and the context still
    folds correctly afterwards."""
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_TIMEOUT_MS, 200)
        f.option(fold.FOLD_OPT_TEST_DROP_TASK, 1)
        seq = synth.uniform(300, 3)
        with pytest.raises(fold.FoldError) as ei:
            f.score(seq)
        assert ei.value.code == fold.FOLD_ETIMEOUT
        f.option(fold.FOLD_OPT_TEST_DROP_TASK, 0)
        assert f.score(seq) == oracle.score(seq)
    finally:
        f.close()


def test_launch_counter(folders):
    f = folders(8)
    before = f.launches
    f.score(synth.uniform(100, 1))
    assert f.launches > before
