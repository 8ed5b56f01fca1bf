"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: exhaustive brute
force over matchings (no DP), hand-worked fixtures (tests/golden/), closed
forms, and the invariants of Lemma 1.  Algorithm 1 (serial two-vector) and
the R table are pinned to Eq. 1 through these.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1307_7820_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MASKS = {"6": oracle.MASK6, "4": oracle.MASK4}


def _rand_seq(rng, n):
    return "".join(rng.choice(list("ACGU"), size=n))


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("mask", [oracle.MASK6, oracle.MASK4])
def test_exhaustive_small_vs_brute(mask):
    """Every string of length <= 6: D(0,n-1) equals the brute-force optimum."""
    for n in range(0, 7):
        for tup in itertools.product("ACGU", repeat=n):
            s = "".join(tup)
            assert oracle.score(s, mask) == oracle.brute(s, mask), s


@pytest.mark.parametrize("mask", [oracle.MASK6, oracle.MASK4])
def test_random_full_tables_vs_brute(mask):
    """Random n <= 12: every entry D(i,j) equals brute force on s[i..j]."""
    rng = np.random.default_rng(11)
    for trial in range(14):
        n = int(rng.integers(2, 13))
        s = _rand_seq(rng, n)
        D = oracle.nussinov(s, mask)
        for i in range(n):
            for j in range(n):
                want = oracle.brute(s[i:j + 1], mask) if j > i else 0
                assert D[i, j] == want, (s, i, j)


def test_random_length8_vs_brute():
    rng = np.random.default_rng(5)
    for _ in range(1500):
        s = _rand_seq(rng, 8)
        assert oracle.score(s) == oracle.brute(s), s


# ---------------------------------------------------------------- golden files
def _hand_examples():
    rows = []
    with open(os.path.join(GOLD, "hand_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                seq, s6, s4 = line.split()
                rows.append((seq, int(s6), int(s4)))
    return rows


def test_hand_examples():
    rows = _hand_examples()
    assert len(rows) >= 12
    for seq, s6, s4 in rows:
        assert oracle.score(seq, oracle.MASK6) == s6, seq
        assert oracle.score(seq, oracle.MASK4) == s4, seq
        # the fixture itself is also brute-force checked
        assert oracle.brute(seq, oracle.MASK6) == s6, seq
        assert oracle.brute(seq, oracle.MASK4) == s4, seq


def test_hand_rows():
    with open(os.path.join(GOLD, "hand_rows.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            seq, mk, row = parts[0], parts[1], int(parts[2])
            vals = [int(x) for x in parts[3:]]
            D = oracle.nussinov(seq, MASKS[mk])
            assert list(D[row]) == vals, (seq, row)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("m", [1, 2, 5, 17, 60])
def test_closed_form_AmUm(m):
    s = "A" * m + "U" * m
    assert oracle.score(s, oracle.MASK6) == m
    assert oracle.score(s, oracle.MASK4) == m


def test_closed_form_revcomp_hairpin():
    """s + revcomp(s) folds into |s| nested Watson-Crick pairs: the maximum n/2."""
    for k, L in enumerate([1, 3, 10, 41, 150]):
        s = synth.uniform(L, 99 + k)
        t = s + synth.revcomp(s)
        assert oracle.score(t, oracle.MASK6) == L
        assert oracle.score(t, oracle.MASK4) == L


def test_closed_form_no_pairable_letters():
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(1, 120))
        s = "".join(rng.choice(list("AC"), size=n))   # A-C never pairs
        assert oracle.score(s, oracle.MASK6) == 0
        s = "".join(rng.choice(list("GU"), size=n))   # G-U only with the wobble pair
        assert oracle.score(s, oracle.MASK4) == 0


def test_alternating_wobble():
    for m in [1, 4, 33]:
        assert oracle.score("GU" * m, oracle.MASK6) == m
        assert oracle.score("GU" * m, oracle.MASK4) == 0


# ---------------------------------------------------------------- invariants
def _check_invariants(s, D, mask):
    n = len(s)
    if n < 2:
        assert np.all(D == 0)
        return
    up = np.triu(np.ones((n, n), dtype=bool))
    # Lemma 1: along a row left->right steps are 0 or 1 ...
    dr = np.diff(D, axis=1)
    assert dr.min() >= 0 and dr.max() <= 1
    # ... and up a column (decreasing i) steps are 0 or 1
    dc = D[:-1, :] - D[1:, :]
    assert dc.min() >= 0 and dc.max() <= 1
    # at most one pair per two bases
    ii, jj = np.nonzero(up)
    assert np.all(D[ii, jj] <= (jj - ii + 1) // 2)
    assert np.all(D[~up] == 0)
    # superadditivity: D(i,j) >= D(i,k-1) + D(k,j)
    for i in range(0, n, max(1, n // 7)):
        for j in range(i + 1, n, max(1, n // 7)):
            ks = np.arange(i + 1, j + 1)
            assert D[i, j] >= (D[i, ks - 1] + D[ks, j]).max()
    if mask == oracle.MASK4:
        c = {b: s.count(b) for b in "ACGU"}
        assert D[0, n - 1] <= min(c["A"], c["U"]) + min(c["C"], c["G"])


@pytest.mark.parametrize("mask", [oracle.MASK6, oracle.MASK4])
def test_invariants_random(mask):
    rng = np.random.default_rng(7)
    for n in [1, 2, 3, 9, 33, 100, 257]:
        for kind in ["uniform", "gc_rich", "structured"]:
            s = synth.variant(kind, n, int(rng.integers(1 << 30)))
            _check_invariants(s, oracle.nussinov(s, mask), mask)


def test_reversal_symmetry():
    """For a symmetric pair set, reading the sequence backwards mirrors the table."""
    rng = np.random.default_rng(8)
    for n in [5, 40, 131]:
        s = _rand_seq(rng, n)
        D = oracle.nussinov(s)
        Dr = oracle.nussinov(s[::-1])
        # D_rev(i,j) = D(n-1-j, n-1-i)
        assert np.array_equal(Dr, D[::-1, ::-1].T)


def test_mask_asymmetry_is_ordered():
    """b(x,y) uses the base at the smaller index first: 'AU' only, not 'UA'."""
    m = oracle.mask_from_pairs(["AU"])
    assert oracle.score("AU", m) == 1
    assert oracle.score("UA", m) == 0
    assert oracle.brute("UAAU", m) == oracle.score("UAAU", m) == 1


# ---------------------------------------------------------------- R table
@pytest.mark.parametrize("q", list(range(1, 11)))
def test_rtable_identities(q):
    R = oracle.rtable(q)
    nv = 1 << (q - 1)
    T = R.reshape(nv, nv)   # T[h, c]
    assert T.min() >= 0 and T.max() <= q - 1
    assert np.all(T[0, :] == 0)                       # R(0, c) = 0
    pop = np.array([bin(h).count("1") for h in range(nv)])
    assert np.array_equal(T[:, 0], pop)               # R(h, 0) = popcount(h)
    assert np.all(np.diag(T) == 0)                    # R(h, h) = 0
    # R(h, c) >= R(h, c | x): more vertical decrements never help
    if nv > 1:
        c = np.arange(nv)
        assert np.all(T[:, c] >= T[:, c | 1])


@pytest.mark.parametrize("q", [2, 3, 5, 8])
def test_rtable_equals_dp_group_max(q):
    """Eq. 2 == Eq. 3: for every group of q consecutive splits inside a real
    table, the plain max over the splits equals base values plus R."""
    R = oracle.rtable(q)
    rng = np.random.default_rng(q)
    for trial in range(3):
        s = _rand_seq(rng, 70)
        D = oracle.nussinov(s)
        n = len(s)
        for i in range(0, n, 3):
            for l in range(i, n - q, 2):
                for j in range(l + q, n, 5):
                    plain = max(D[i, l + k] + D[l + 1 + k, j] for k in range(q))
                    h = sum(int(D[i, l + p] - D[i, l + p - 1]) << (p - 1) for p in range(1, q))
                    c = sum(int(D[l + p, j] - D[l + p + 1, j]) << (p - 1) for p in range(1, q))
                    assert plain == D[i, l] + D[l + 1, j] + R[(h << (q - 1)) | c]


def test_rtable_max_index_smallest_argmax():
    q = 6
    R, Ri = oracle.rtable(q, with_index=True)
    nv = 1 << (q - 1)
    for h in range(0, nv, 3):
        for c in range(0, nv, 5):
            pref = [0]
            for p in range(1, q):
                pref.append(pref[-1] + ((h >> (p - 1)) & 1) - ((c >> (p - 1)) & 1))
            idx = (h << (q - 1)) | c
            assert R[idx] == max(pref)
            assert Ri[idx] == pref.index(max(pref))


# ---------------------------------------------------------------- Algorithm 1
def lookup_count(n, q):
    """Number of full groups summed over all cells: sum_{i<j} #{g : gq >= i, gq+q <= j}."""
    tot = 0
    for i in range(n):
        g0 = -(-i // q)
        for g in range(g0, n):
            first_j = g * q + q
            if first_j > n - 1:
                break
            tot += n - first_j
    return tot


@pytest.mark.parametrize("q", list(range(1, 11)))
def test_two_vector_equals_nussinov(q):
    rng = np.random.default_rng(100 + q)
    for n in [0, 1, 2, q - 1, q, q + 1, 2 * q + 3, 61, 150]:
        if n < 0:
            continue
        for mask in (oracle.MASK6, oracle.MASK4):
            s = _rand_seq(rng, n)
            D1 = oracle.nussinov(s, mask)
            D2, nl = oracle.two_vector(s, q, mask, return_lookups=True)
            assert np.array_equal(D1, D2), (q, n)
            assert nl == lookup_count(n, q)


def test_two_vector_n1000_q8():
    s = synth.uniform(1000, synth.SEED_BASE)
    assert np.array_equal(oracle.nussinov(s), oracle.two_vector(s, 8))


def test_two_vector_structured_and_gc():
    for kind in ["gc_rich", "structured"]:
        s = synth.variant(kind, 400, 4242)
        for q in (4, 7, 9):
            assert np.array_equal(oracle.nussinov(s), oracle.two_vector(s, q))


def test_metrics_lookup_count_matches_algorithm1():
    """The closed-form lookup count used by the roofline equals the number of
    table lookups Algorithm 1 actually makes."""
    from paper_1307_7820_b300 import metrics
    rng = np.random.default_rng(2)
    for n, q in [(0, 8), (1, 8), (17, 4), (100, 8), (257, 8), (300, 9), (129, 3)]:
        s = _rand_seq(rng, n)
        _, nl = oracle.two_vector(s, q, return_lookups=True)
        assert metrics.lookups(n, q) == nl == lookup_count(n, q)
        assert metrics.splits(n) == sum(j - i for i in range(n) for j in range(i + 1, n))
        assert metrics.residual_splits(n, q) >= 0
