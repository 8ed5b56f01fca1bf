"""The allocation-free entry point (fold_score_static), for callers that
cannot call cudaMalloc when they fold (a framework whose allocator owns all
device memory, a service that allocates only at start-up, a plugin called
where allocation is not allowed).  All its calls reuse one fixed device array
inside the library, so each call must clear what the previous one left: the
tests make calls back to back on that array and check every table against the
CPU oracle (Eq. 1) and against the workspace entry point (fold_score_dev).
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu

MASKS = [(fold.FOLD_PAIRS_DEFAULT, oracle.MASK6), (fold.FOLD_PAIRS_PAPER, oracle.MASK4)]


def _static(torch, codes, n, mask, stream):
    out = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    D = torch.full((max(n, 1), max(n, 1)), -1, dtype=torch.int16, device="cuda")
    fold.fold_score_static(codes.data_ptr() if n else 0, n, mask, out.data_ptr(), D.data_ptr() if n else 0,
                           stream.cuda_stream)
    return out, D


@pytest.mark.parametrize("mask,omask", MASKS)
def test_static_entry_point_matches_oracle_and_workspace_entry_point(mask, omask):
    torch = pytest.importorskip("torch")
    f = fold.Folder(q=8, pair_mask=mask)
    try:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        # calls in a row on the one scratch array: the largest size, sizes below, at and just past one
        # 32-base tile, the empty and the one-base sequence, then the largest size again
        sizes = [fold.FOLD_STATIC_MAX_N, 33, 0, 31, 1, 1000, fold.FOLD_STATIC_MAX_N]
        for k, n in enumerate(sizes):
            seq = synth.variant(["uniform", "gc_rich", "structured"][k % 3], n, 4100 + k)
            codes = torch.from_numpy(fold.encode_codes(seq)).cuda() if n else None
            out_st, D_st = _static(torch, codes, n, mask, s)
            s.synchronize()
            ref = oracle.nussinov(seq, omask)
            want = int(ref[0, n - 1]) if n else 0
            assert int(out_st.item()) == want, f"n={n}"
            if n == 0:
                continue
            assert np.array_equal(D_st.cpu().numpy().astype(np.int32), ref), f"n={n}"
            # the workspace entry point on the same input gives the same table
            ws = torch.empty(f.workspace_bytes(n), dtype=torch.uint8, device="cuda")
            out_ws = torch.zeros(1, dtype=torch.int32, device="cuda")
            D_ws = torch.empty((n, n), dtype=torch.int16, device="cuda")
            torch.cuda.synchronize()
            f.score_dev(codes, ws, out_ws, D_ws, stream=s.cuda_stream)
            s.synchronize()
            assert int(out_ws.item()) == want
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
