"""Algorithmic work counts and roofline arithmetic for the fold.

These are counts of the method's own work, independent of how the kernels
organise it:

* cells(n)          = n(n-1)/2 table entries above the diagonal (Section 2);
* splits(n)         = sum over cells of (j - i) split points of Eq. 1;
* lookups(n, q)     = sum over cells of the number of full groups (Section 3.1:
                      group g serves cell (i,j) iff g*q >= i and g*q + q <= j),
                      i.e. the R-table lookups the two-vector method makes;
* hbm_bytes(n)      = 8 bytes per cell: each int16 entry is written to the
                      row-major and the column-major copy and read back at
                      least once from each.

The lookup roofline of a B300: one conflict-free shared-memory wavefront
(32 lanes, one lookup each) per SM per clock, i.e. n_sm * 32 * f_sm lookups/s.
"""
from __future__ import annotations


def cells(n: int) -> int:
    return n * (n - 1) // 2


def splits(n: int) -> int:
    # sum_{d=1}^{n-1} (n - d) * d
    return sum((n - d) * d for d in range(1, n))


def lookups_relative(n: int, q: int) -> int:
    """Table lookups of Section 4's organisation: floor((j-i)/q) groups relative to i for every
    cell, i.e. the sum over diagonals d of (n - d) * floor(d / q)."""
    return sum((n - d) * (d // q) for d in range(1, n))


def fg_tables(n: int, q: int) -> int:
    """Row-group tables the FG algorithm builds: row i's group g is complete (and tabulated) when
    D(i, g*q+q-1) exists, for every row i <= g*q."""
    return sum(g * q + 1 for g in range(n // q + 1) if g * q + q - 1 <= n - 1)


def lookups(n: int, q: int) -> int:
    """Number of full groups summed over all cells.

    Group g is full for cell (i, j) iff i <= g*q and j >= g*q + q, so it is
    counted (g*q + 1) * (n - g*q - q) times (rows 0..g*q, columns g*q+q..n-1).
    """
    tot = 0
    g = 0
    while g * q + q <= n - 1:
        tot += (g * q + 1) * (n - g * q - q)
        g += 1
    return tot


def residual_splits(n: int, q: int) -> int:
    """Splits evaluated directly by the two-vector method (outside full groups)."""
    return splits(n) - q * lookups(n, q)


def hbm_bytes(n: int) -> int:
    return 8 * cells(n)


def lookup_peak(n_sm: int, sm_mhz: float) -> float:
    """Conflict-free shared-memory lookup rate of the whole GPU (lookups/s)."""
    return n_sm * 32 * sm_mhz * 1e6
