"""Pins for the oracle of Section 3.2's FG algorithm (no GPU): brute force
over matchings, the Eq. 1 oracle (a different algorithm, pinned to brute
force), the hand-worked fixtures, and the two counts the algorithm's
structure fixes: one lookup per full group of every cell (Algorithm 1's groups)
and one table per complete (row, group)."""
import os

import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_seq(rng, n):
    return "".join(rng.choice(list("ACGU"), size=n))


def _lookups(n, q):
    # cell (i,j) uses group g iff g*q >= i and g*q + q <= j
    return sum(1 for i in range(n) for j in range(i + 1, n) for g in range(n // q + 1) if g * q >= i and g * q + q <= j)


def _tables(n, q):
    # row i's group g is complete when D(i, g*q+q-1) exists, for rows i <= g*q
    return sum(1 for i in range(n) for g in range(n // q + 1) if g * q >= i and g * q + q - 1 <= n - 1)


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_fg_vs_brute(q):
    rng = np.random.default_rng(900 + q)
    for _ in range(100):
        n = int(rng.integers(1, 15))
        s = _rand_seq(rng, n)
        for mask in (oracle.MASK6, oracle.MASK4):
            assert oracle.fg(s, q, mask)[0, n - 1] == oracle.brute(s, mask), (s, q)


@pytest.mark.parametrize("q", list(range(1, 11)))
def test_fg_equals_nussinov_and_counts(q):
    rng = np.random.default_rng(950 + q)
    for n in [0, 1, 2, q - 1, q, q + 1, 2 * q + 3, 61, 130]:
        if n < 0:
            continue
        s = _rand_seq(rng, n)
        D, nl, nt = oracle.fg(s, q, return_counts=True)
        assert np.array_equal(D, oracle.nussinov(s)), (q, n)
        assert nl == _lookups(n, q)
        assert nt == _tables(n, q)


def test_fg_variants_and_hand_examples():
    for kind in ["gc_rich", "structured"]:
        s = synth.variant(kind, 300, 4545)
        for q in (3, 8):
            assert np.array_equal(oracle.fg(s, q), oracle.nussinov(s))
    with open(os.path.join(GOLD, "hand_examples.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for seq, s6, s4 in rows:
        n = len(seq)
        assert oracle.fg(seq, 3, oracle.MASK6)[0, n - 1] == int(s6), seq
        assert oracle.fg(seq, 3, oracle.MASK4)[0, n - 1] == int(s4), seq


def test_fg_same_lookups_as_algorithm1():
    """FG and the two-vector method take the same group terms; FG's extra work is the
    tables it builds (one per complete row group)."""
    s = synth.uniform(200, 8)
    for q in (3, 8):
        _, nl_fg, nt = oracle.fg(s, q, return_counts=True)
        _, nl_tv = oracle.two_vector(s, q, return_lookups=True)
        assert nl_fg == nl_tv and nt > 0


def test_metrics_fg_table_count():
    from paper_1307_7820_b300 import metrics
    rng = np.random.default_rng(4)
    for n, q in [(0, 3), (1, 3), (17, 4), (100, 3), (131, 8)]:
        _, _, nt = oracle.fg(_rand_seq(rng, n), q, return_counts=True)
        assert metrics.fg_tables(n, q) == nt == _tables(n, q)
