"""Host logic of the persistent kernel's task list (no GPU): every middle
block of every tile is merged exactly once (by a single-tile chunk or a strip
chunk), each tile's chunk count matches, and every task waits only on tasks
placed before it -- the property that makes the ordered list deadlock-free."""
import pytest

from paper_1307_7820_b300 import build as fbuild
from paper_1307_7820_b300 import fold


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fbuild.build()
    fold.lib()


@pytest.mark.parametrize("method", [fold.FOLD_METHOD_TWO_VECTOR, fold.FOLD_METHOD_PLAIN])
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 100, 129, 160, 161, 257, 300, 777, 1000, 2049, 3000, 6000])
def test_schedule_valid_q8(n, method):
    assert fold.fold_schedule_check(n, 8, method, 0) == 0


@pytest.mark.parametrize("q", list(range(2, 11)))
def test_schedule_valid_all_q(q):
    for n in (5, 90, 333, 1200):
        assert fold.fold_schedule_check(n, q, fold.FOLD_METHOD_TWO_VECTOR, 0) == 0


@pytest.mark.parametrize("kchunk", [1, 2, 3, 5, 64])
def test_schedule_valid_chunk_sizes(kchunk):
    for n in (400, 1500):
        assert fold.fold_schedule_check(n, 8, fold.FOLD_METHOD_TWO_VECTOR, kchunk) == 0
        assert fold.fold_schedule_check(n, 8, fold.FOLD_METHOD_PLAIN, kchunk) == 0


@pytest.mark.parametrize("method", [fold.FOLD_METHOD_TWO_VECTOR, fold.FOLD_METHOD_PLAIN])
def test_batch_list_valid(method):
    # fold_batch's interleaved list (longest sequence first within a step): each sequence's tasks in
    # its own list's order, every distinct size's list valid
    from paper_1307_7820_b300 import synth
    lens = [len(s) for s in synth.batch(300, 1, 3000, 31)] + [0, 1, 32, 33, 3000, 3000]
    assert fold.fold_batch_schedule_check(lens, 8, method, 0) == 0
    assert fold.fold_batch_schedule_check(lens[:7], 8, method, 3) == 0
    assert fold.fold_batch_schedule_check([], 8, method, 0) == 0
    assert fold.fold_batch_schedule_check([65536], 8, method, 0) == -fold.FOLD_EINVAL


def test_schedule_check_rejects_bad_arguments():
    assert fold.fold_schedule_check(-1, 8, 0, 0) == -fold.FOLD_EINVAL
    assert fold.fold_schedule_check(100, 11, 0, 0) == -fold.FOLD_EINVAL
    assert fold.fold_schedule_check(100, 8, 7, 0) == -fold.FOLD_EINVAL
