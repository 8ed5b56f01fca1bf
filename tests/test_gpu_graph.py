"""Single folds recorded into a CUDA graph by stream capture (torch.cuda.graph)
and replayed: every replay folds what the captured code buffers hold at that
time, exactly as the oracle; capture refuses what cannot be recorded.  All
calls go through the C-ABI."""
import pytest
import torch

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["two_vector", "plain", "sliding"])
def test_capture_and_replay(method):
    f = fold.Folder(q=8, method=method)
    try:
        n, count = 1400 if method != "sliding" else 400, 4
        seqs = [synth.variant(["uniform", "gc_rich", "structured"][k % 3], n, 60 + k) for k in range(count)]
        codes = [torch.from_numpy(fold.encode_codes(s)).cuda() for s in seqs]
        ws = torch.empty(f.workspace_bytes(n), dtype=torch.uint8, device="cuda")
        outs = torch.zeros(count, dtype=torch.int32, device="cuda")
        # one uncaptured fold of this length builds and caches its task list
        f.score_dev(codes[0], ws, outs[0:1])
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            s = torch.cuda.current_stream().cuda_stream
            for k in range(count):
                f.score_dev(codes[k], ws, outs[k:k + 1], stream=s)
        outs.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert outs.tolist() == [oracle.score(x) for x in seqs]
        # new inputs in the same buffers, same graph
        seqs2 = [synth.uniform(n, 900 + k) for k in range(count)]
        for k in range(count):
            codes[k].copy_(torch.from_numpy(fold.encode_codes(seqs2[k])))
        g.replay()
        torch.cuda.synchronize()
        assert outs.tolist() == [oracle.score(x) for x in seqs2]
    finally:
        f.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")   # the refused calls recorded nothing
def test_capture_refuses_uncached_length_and_timing():
    f = fold.Folder(q=8)
    try:
        codes = torch.from_numpy(fold.encode_codes(synth.uniform(777, 3))).cuda()
        ws = torch.empty(f.workspace_bytes(777), dtype=torch.uint8, device="cuda")
        out = torch.zeros(1, dtype=torch.int32, device="cuda")
        g = torch.cuda.CUDAGraph()
        with pytest.raises(fold.FoldError) as ei:
            with torch.cuda.graph(g):
                f.score_dev(codes, ws, out, stream=torch.cuda.current_stream().cuda_stream)
        assert ei.value.code == fold.FOLD_EINVAL
        f.score_dev(codes, ws, out)   # cached now; timing still refused under capture
        torch.cuda.synchronize()
        f.option(fold.FOLD_OPT_TIMING, 1)
        g2 = torch.cuda.CUDAGraph()
        with pytest.raises(fold.FoldError) as ei:
            with torch.cuda.graph(g2):
                f.score_dev(codes, ws, out, stream=torch.cuda.current_stream().cuda_stream)
        assert ei.value.code == fold.FOLD_EINVAL
    finally:
        f.close()
