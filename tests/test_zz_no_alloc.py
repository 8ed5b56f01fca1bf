"""The allocation-free entry point (fold_score_static), for callers that
cannot call cudaMalloc when they fold: it must give exactly what the
workspace entry point (fold_score_dev) gives, call after call, although all
its calls reuse one fixed device array.  This file is collected last so that
a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


def test_static_entry_point_matches_workspace_entry_point():
    torch = pytest.importorskip("torch")
    f = fold.Folder(q=8)
    try:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        # two calls in a row; the second reuses the scratch the first one left behind
        for k, n in enumerate([1000, 777]):
            seq = synth.uniform(n, 4100 + k)
            codes = torch.from_numpy(fold.encode_codes(seq)).cuda()
            ws = torch.empty(f.workspace_bytes(n), dtype=torch.uint8, device="cuda")
            out_ws = torch.zeros(1, dtype=torch.int32, device="cuda")
            out_st = torch.zeros(1, dtype=torch.int32, device="cuda")
            D_ws = torch.empty((n, n), dtype=torch.int16, device="cuda")
            D_st = torch.full((n, n), -1, dtype=torch.int16, device="cuda")
            torch.cuda.synchronize()
            f.score_dev(codes, ws, out_ws, D_ws, stream=s.cuda_stream)
            fold.fold_score_static(codes.data_ptr(), n, fold.FOLD_PAIRS_DEFAULT, out_st.data_ptr(),
                                   D_st.data_ptr(), s.cuda_stream)
            s.synchronize()
            assert int(out_st.item()) == int(out_ws.item()) > 0
            assert torch.equal(D_st, D_ws)
    finally:
        f.close()


def test_static_entry_point_rejects_n_above_its_limit():
    torch = pytest.importorskip("torch")
    n = fold.FOLD_STATIC_MAX_N + 1
    codes = torch.zeros(n, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(fold.FoldError) as ei:
        fold.fold_score_static(codes.data_ptr(), n, fold.FOLD_PAIRS_DEFAULT, out.data_ptr())
    assert ei.value.code == fold.FOLD_EINVAL
