"""GPU traceback (fold_structure / fold_structure_dev) against the oracle's
traceback: both re-evaluate the argmax of Eq. 1 with the same order of
preference on the same (bit-exact) table, so the structures must be identical;
at large n, where the oracle's table takes too long, the oracle's traceback
runs on the GPU's own table and the structure is checked for validity and for
holding D(0,n-1) pairs.  All through the C-ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_7820_b300 import fold, synth

pytestmark = pytest.mark.gpu

CODE = {"A": 0, "C": 1, "G": 2, "U": 3}


def _valid_pairs(seq, partner, mask):
    stack, pairs = [], 0
    for k, p in enumerate(partner):
        p = int(p)
        if p < 0:
            continue
        assert int(partner[p]) == k
        if p > k:
            assert (mask >> (4 * CODE[seq[k]] + CODE[seq[p]])) & 1
            stack.append(p)
            pairs += 1
        else:
            assert stack and stack[-1] == k
            stack.pop()
    assert not stack
    return pairs


@pytest.mark.parametrize("method", ["two_vector", "plain"])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 33, 200, 700, 1500])
def test_structure_equals_oracle(method, n):
    f = fold.Folder(q=8, method=method)
    try:
        seq = synth.variant(["uniform", "gc_rich", "structured"][n % 3], n, 3100 + n)
        mp, partner, db = f.structure(seq)
        want = oracle.traceback(seq)
        assert np.array_equal(partner, want)
        assert db == oracle.dot_bracket(want)
        assert mp == (oracle.score(seq) if n else 0)
    finally:
        f.close()


@pytest.mark.parametrize("q,mask", [(4, oracle.MASK6), (10, oracle.MASK4), (8, oracle.MASK4)])
def test_structure_other_q_and_masks(q, mask):
    f = fold.Folder(q=q, pair_mask=mask)
    try:
        for n in (95, 611):
            seq = synth.uniform(n, 77 + n + q)
            mp, partner, _ = f.structure(seq)
            assert np.array_equal(partner, oracle.traceback(seq, mask))
    finally:
        f.close()


@pytest.mark.parametrize("n", [6000, 16384])
def test_structure_large(n):
    """Column mode at n = 6000, one shared queue at 16384: the trace of the GPU's table equals the
    oracle's trace of that same table, is valid and holds D(0,n-1) pairs."""
    f = fold.Folder(q=8)
    try:
        seq = synth.structured(n, n + 5) if n > 8000 else synth.uniform(n, n + 5)
        mp, partner, db = f.structure(seq)
        mp2, D = f.score(seq, want_D=True)
        assert mp == mp2
        assert np.array_equal(partner, oracle.traceback(seq, D=D.astype(np.int32)))
        assert _valid_pairs(seq, partner, oracle.MASK6) == mp
        assert db.count("(") == mp == db.count(")")
    finally:
        f.close()


def test_structure_device_path():
    f = fold.Folder(q=8)
    try:
        seq = synth.gc_rich(900, 12)
        n = len(seq)
        codes = torch.from_numpy(fold.encode_codes(seq)).cuda()
        ws = torch.empty(fold.fold_structure_workspace_bytes(f.ctx, n), dtype=torch.uint8, device="cuda")
        out = torch.zeros(1, dtype=torch.int32, device="cuda")
        partner = torch.empty(n, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        fold.fold_structure_dev(f.ctx, codes.data_ptr(), n, ws.data_ptr(), ws.numel(), out.data_ptr(),
                                partner.data_ptr(), s.cuda_stream)
        s.synchronize()
        assert int(out.item()) == oracle.score(seq)
        assert np.array_equal(partner.cpu().numpy(), oracle.traceback(seq))
        # a workspace that is too small is refused before anything is enqueued
        with pytest.raises(fold.FoldError) as ei:
            fold.fold_structure_dev(f.ctx, codes.data_ptr(), n, ws.data_ptr(), f.workspace_bytes(n), out.data_ptr(),
                                    partner.data_ptr(), s.cuda_stream)
        assert ei.value.code == fold.FOLD_ENOMEM
    finally:
        f.close()
