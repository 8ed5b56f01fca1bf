"""Pins for the oracle of Section 4's two-vector algorithm with difference
vectors at every cell and groups relative to i (no GPU).

It is checked against things other than itself: brute force over matchings
(no DP), the Eq. 1 oracle (a different algorithm, itself pinned to brute
force), the hand-worked fixtures in tests/golden/, and the number of table
lookups the reading of Section 4's loops implies (floor((j-i)/q) per cell).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_seq(rng, n):
    return "".join(rng.choice(list("ACGU"), size=n))


def _lookups(n, q):
    # one lookup per full group relative to i: floor((j - i)/q) for every cell i < j
    return sum((j - i) // q for i in range(n) for j in range(i + 1, n))


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_sliding_vs_brute(q):
    rng = np.random.default_rng(700 + q)
    for _ in range(120):
        n = int(rng.integers(1, 15))
        s = _rand_seq(rng, n)
        for mask in (oracle.MASK6, oracle.MASK4):
            D = oracle.two_vector_sliding(s, q, mask)
            assert D[0, n - 1] == oracle.brute(s, mask), (s, q)


@pytest.mark.parametrize("q", list(range(1, 11)))
def test_sliding_equals_nussinov_and_counts(q):
    rng = np.random.default_rng(800 + q)
    for n in [0, 1, 2, q - 1, q, q + 1, 2 * q + 3, 61, 150]:
        if n < 0:
            continue
        for mask in (oracle.MASK6, oracle.MASK4):
            s = _rand_seq(rng, n)
            D, nl = oracle.two_vector_sliding(s, q, mask, return_lookups=True)
            assert np.array_equal(D, oracle.nussinov(s, mask)), (q, n)
            assert nl == _lookups(n, q)


def test_sliding_structured_gc_and_long():
    for kind in ["gc_rich", "structured"]:
        s = synth.variant(kind, 300, 4343)
        for q in (4, 8, 10):
            assert np.array_equal(oracle.two_vector_sliding(s, q), oracle.nussinov(s))
    s = synth.uniform(700, synth.SEED_BASE + 11)
    assert np.array_equal(oracle.two_vector_sliding(s, 8), oracle.nussinov(s))


def test_sliding_hand_examples():
    with open(os.path.join(GOLD, "hand_examples.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 12
    for seq, s6, s4 in rows:
        n = len(seq)
        for q in (2, 3, 8):
            assert oracle.two_vector_sliding(seq, q, oracle.MASK6)[0, n - 1] == int(s6), (seq, q)
            assert oracle.two_vector_sliding(seq, q, oracle.MASK4)[0, n - 1] == int(s4), (seq, q)


def test_sliding_makes_more_lookups_than_aligned_groups():
    """Relative groups fit one more group into many cells than absolute ones
    (Section 4 trades that for equal work per process)."""
    s = synth.uniform(200, 5)
    for q in (4, 8):
        _, nl_rel = oracle.two_vector_sliding(s, q, return_lookups=True)
        _, nl_abs = oracle.two_vector(s, q, return_lookups=True)
        assert nl_rel > nl_abs


def test_metrics_relative_lookup_count():
    """The closed form bench.py reports for Section 4's organisation equals the lookups the
    oracle of that algorithm makes."""
    from paper_1307_7820_b300 import metrics
    rng = np.random.default_rng(9)
    for n, q in [(0, 8), (1, 8), (17, 4), (100, 8), (257, 8), (300, 9), (129, 3)]:
        _, nl = oracle.two_vector_sliding(_rand_seq(rng, n), q, return_lookups=True)
        assert metrics.lookups_relative(n, q) == nl == _lookups(n, q)
