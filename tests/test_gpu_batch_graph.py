"""A batch planned once and folded from device buffers (fold_batch_plan_create + fold_batch_dev),
recorded into a CUDA graph by stream capture and replayed on new inputs: every replay folds what
the captured code buffer then holds, and every score and table equals the oracle's (Eq. 1).  All
calls go through the C-ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu

LENS = [0, 1, 2, 31, 32, 33, 100, 700, 1500, 64, 257, 3]


def _seqs(seed):
    kinds = ["uniform", "gc_rich", "structured"]
    return [synth.variant(kinds[k % 3], L, seed + k) for k, L in enumerate(LENS)]


@pytest.mark.parametrize("method", ["two_vector", "plain"])
def test_batch_plan_capture_and_replay(method):
    f = fold.Folder(q=8, method=method)
    bp = fold.BatchPlan(f.ctx, LENS)
    try:
        count = len(LENS)
        codes = torch.zeros(max(1, bp.codes_bytes), dtype=torch.uint8, device="cuda")
        ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
        outs = torch.zeros(count, dtype=torch.int32, device="cuda")
        tabs = {k: torch.zeros((LENS[k], LENS[k]), dtype=torch.int16, device="cuda") for k in (3, 7, 8) }
        seqs = _seqs(300)
        codes[:bp.codes_bytes].copy_(torch.from_numpy(bp.encode(seqs)))
        # uncaptured: scores as fold_batch and the oracle
        bp.fold_dev(codes.data_ptr(), ws.data_ptr(), ws.numel(), outs.data_ptr())
        torch.cuda.synchronize()
        want = [oracle.score(s) if len(s) else 0 for s in seqs]
        assert outs.tolist() == want
        assert f.batch(seqs).tolist() == want
        # captured once, replayed on two sets of inputs
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            st = torch.cuda.current_stream().cuda_stream
            bp.fold_dev(codes.data_ptr(), ws.data_ptr(), ws.numel(), outs.data_ptr(), stream=st)
            for k, D in tabs.items():
                bp.table_dev(ws.data_ptr(), k, D.data_ptr(), stream=st)
        for seed in (500, 700):
            seqs = _seqs(seed)
            codes[:bp.codes_bytes].copy_(torch.from_numpy(bp.encode(seqs)))
            outs.fill_(-7)
            g.replay()
            torch.cuda.synchronize()
            assert outs.tolist() == [oracle.score(s) if len(s) else 0 for s in seqs]
            for k, D in tabs.items():
                assert np.array_equal(D.cpu().numpy().astype(np.int32), oracle.nussinov(seqs[k])), (seed, k)
    finally:
        bp.close()
        f.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")   # the refused call recorded nothing
def test_batch_plan_refusals():
    f = fold.Folder(q=8)
    bp = fold.BatchPlan(f.ctx, [100, 200])
    try:
        codes = torch.zeros(300, dtype=torch.uint8, device="cuda")
        ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
        outs = torch.zeros(2, dtype=torch.int32, device="cuda")
        with pytest.raises(fold.FoldError) as ei:   # workspace too small
            bp.fold_dev(codes.data_ptr(), ws.data_ptr(), 256, outs.data_ptr())
        assert ei.value.code == fold.FOLD_ENOMEM
        f.option(fold.FOLD_OPT_TIMING, 1)           # timing is refused under capture
        g = torch.cuda.CUDAGraph()
        with pytest.raises(fold.FoldError) as ei:
            with torch.cuda.graph(g):
                bp.fold_dev(codes.data_ptr(), ws.data_ptr(), ws.numel(), outs.data_ptr(),
                            stream=torch.cuda.current_stream().cuda_stream)
        assert ei.value.code == fold.FOLD_EINVAL
        f.option(fold.FOLD_OPT_TIMING, 0)
        f.set_method("plain")                        # planned for the two-vector method
        with pytest.raises(fold.FoldError) as ei:
            bp.fold_dev(codes.data_ptr(), ws.data_ptr(), ws.numel(), outs.data_ptr())
        assert ei.value.code == fold.FOLD_EINVAL
    finally:
        bp.close()
        f.close()
