"""The multi-threaded CPU two-vector baseline (Section 3.1, Algorithm 1 on a tiled wavefront)
equals the oracle's Eq. 1 table element by element, for every q it accepts, on 1 and several
threads, at sizes spanning several of its tiles with a ragged tail; its lookup count equals
Algorithm 1's."""
import numpy as np
import pytest

import baseline
import oracle
from paper_1307_7820_b300 import synth


@pytest.mark.parametrize("q", range(2, 11))
def test_matches_oracle_every_q(q):
    for k, (kind, n) in enumerate([("uniform", 1), ("uniform", 2), ("gc_rich", q + 1), ("structured", 97),
                                   ("uniform", 2 * 96 + 37), ("structured", 301)]):
        s = synth.variant(kind, n, 70 + 10 * q + k)
        ref = oracle.nussinov(s)
        for threads in (1, 4):
            mp, D, nl, used = baseline.fold(s, q=q, threads=threads, want_D=True)
            assert mp == (int(ref[0, n - 1]) if n else 0)
            assert np.array_equal(D.astype(np.int32), ref), (q, kind, n, threads)
            assert used == threads or n < 2
        if n >= 2:
            assert nl == oracle.two_vector(s, q, return_lookups=True)[1]


def test_paper_pair_set_and_score_only():
    s = synth.uniform(500, 9)
    ref = oracle.nussinov(s, oracle.MASK4)
    mp, D, _, _ = baseline.fold(s, q=8, mask=oracle.MASK4, want_D=True)
    assert np.array_equal(D.astype(np.int32), ref)
    assert baseline.fold(s, q=8, mask=oracle.MASK4)[0] == int(ref[0, -1])
    assert baseline.fold("", q=8)[0] == 0
