"""The per-task trace (FOLD_OPT_TRACE) through the C-ABI: one record per tile
of the tile grid, chunks only for tiles with middle blocks, times in order
within each record, workers and SMs inside the launch, and a traced fold
still scores as the oracle."""
import pytest
import torch

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", [(0, 0), (-1, 4), (-1, -1)])
def test_trace_records(layout):
    near_ctas, columns = layout
    n = 1900
    seq = synth.uniform(n, 77)
    f = fold.Folder(q=8)
    try:
        f.option(fold.FOLD_OPT_NEAR_CTAS, near_ctas)
        f.option(fold.FOLD_OPT_COLUMNS, columns)
        f.option(fold.FOLD_OPT_TRACE, 1)
        assert f.score(seq) == oracle.score(seq)
        tr = fold.fold_trace_copy(f.ctx)
        f.option(fold.FOLD_OPT_TRACE, 0)
    finally:
        f.close()
    T = 32
    NT = (n + T - 1) // T
    tiles = tr[tr["type"] == 0]
    got = sorted(zip(tiles["I"].tolist(), tiles["J"].tolist()))
    assert got == [(i, j) for i in range(NT) for j in range(i, NT)]
    chunks = tr[tr["type"] != 0]
    assert ((chunks["J"] - chunks["I"]) >= 4).all()   # middle blocks I+2 .. J-2
    assert (tr["t_start"] <= tr["t_end"]).all()
    assert (tiles["t_deps"] <= tiles["t_end"]).all()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ((tr["sm"] >= 0) & (tr["sm"] < sms)).all()
    assert (tr["worker"] >= 0).all() and (tr["reserved"] == 0).all()
    # a worker (one warp) runs on one SM for the whole launch
    by_worker = {}
    for w, s in zip(tr["worker"].tolist(), tr["sm"].tolist()):
        assert by_worker.setdefault(w, s) == s
