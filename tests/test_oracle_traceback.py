"""Pins of the oracle's traceback (Section 2: the argmax of Eq. 1 re-evaluated
at each visited cell).  The structure must be valid (every base in at most one
pair, pairs allowed by the mask, no two pairs crossing), hold D(0,n-1) pairs
(checked against brute force for tiny inputs, which shares nothing with the
DP), and follow the stated order of preference on hand-derived examples
(tests/golden/hand_structures.txt)."""
import os
import random

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
BASES = "ACGU"


def _valid(seq, partner, mask):
    n = len(seq)
    code = {"A": 0, "C": 1, "G": 2, "U": 3}
    assert len(partner) == n
    stack = []
    pairs = 0
    for k in range(n):
        p = int(partner[k])
        if p < 0:
            continue
        assert 0 <= p < n and p != k and int(partner[p]) == k, f"partner not symmetric at {k}"
        if p > k:
            x, y = code[seq[k]], code[seq[p]]
            assert (mask >> (4 * x + y)) & 1, f"pair ({k},{p}) {seq[k]}{seq[p]} not allowed"
            stack.append(p)
            pairs += 1
        else:
            assert stack and stack[-1] == k, f"pairs cross at {k}"
            stack.pop()
    assert not stack
    return pairs


def test_hand_structures():
    for line in open(os.path.join(HERE, "golden", "hand_structures.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        seq, want = line.split()
        p = oracle.traceback(seq)
        assert oracle.dot_bracket(p) == want, seq
        assert _valid(seq, p, oracle.MASK6) == oracle.score(seq)


@pytest.mark.parametrize("mask", [oracle.MASK6, oracle.MASK4])
def test_tiny_against_brute_force(mask):
    rng = random.Random(99)
    for _ in range(300):
        n = rng.randint(0, 13)
        seq = "".join(rng.choice(BASES) for _ in range(n))
        p = oracle.traceback(seq, mask)
        assert _valid(seq, p, mask) == oracle.brute(seq, mask), seq


def test_random_sizes_hold_the_optimum():
    rng = random.Random(7)
    for _ in range(40):
        n = rng.randint(20, 300)
        seq = "".join(rng.choice(BASES) for _ in range(n))
        D = oracle.nussinov(seq)
        p = oracle.traceback(seq, D=D)
        assert _valid(seq, p, oracle.MASK6) == int(D[0, n - 1])


def test_edges_and_inconsistent_table():
    assert oracle.traceback("").size == 0
    assert list(oracle.traceback("A")) == [-1]
    assert list(oracle.traceback("AA")) == [-1, -1]
    seq = "GGGAAAUCC"
    D = oracle.nussinov(seq)
    D[0, 8] += 5   # no argmax can reach this value
    with pytest.raises(ValueError):
        oracle.traceback(seq, D=D)
