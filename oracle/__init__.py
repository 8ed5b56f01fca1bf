"""CPU oracle for the Nussinov DP and the two-vector method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  The GPU
library under ``paper_1307_7820_b300/`` never imports it, and the two share no
code: this package has its own base encoder and its own C source
(``oracle.c``), built with gcc into ``liboracle.so`` by :func:`build`.

Functions (each cites the passage of the paper it follows; see ``oracle.c``):

* :func:`nussinov`      -- Section 2, Eq. 1, cubic, full table.
* :func:`brute`         -- Section 2 problem statement, exhaustive matchings.
* :func:`rtable`        -- Section 3.1 preprocessing routine over all vector pairs.
* :func:`two_vector`    -- Section 3.1, Algorithm 1 (serial two-vector).
* :func:`two_vector_sliding` -- Section 4, the parallel two-vector algorithm with
  difference vectors at every cell and groups relative to i.
* :func:`fg`            -- Section 3.2, the FG algorithm (a table per row and group).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against brute force, hand-worked fixtures in ``tests/golden/``, closed forms
and the invariants of Lemma 1; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Section 2: complementary bases pair.  Codes A=0, C=1, G=2, U=3; bit (4x+y).
_CODE = {"A": 0, "C": 1, "G": 2, "U": 3, "a": 0, "c": 1, "g": 2, "u": 3}


def mask_from_pairs(pairs) -> int:
    """Pair mask with bit (4x+y) set for every ordered pair 'XY' in ``pairs``."""
    m = 0
    for p in pairs:
        m |= 1 << (4 * _CODE[p[0]] + _CODE[p[1]])
    return m


#: Watson-Crick plus wobble pairs, both orders (the default of this project).
MASK6 = mask_from_pairs(["AU", "UA", "CG", "GC", "GU", "UG"])
#: The pair set the paper names (A-U and C-G), both orders.
MASK4 = mask_from_pairs(["AU", "UA", "CG", "GC"])


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so (no GPU code involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_nussinov.argtypes = [u8p, ctypes.c_int, ctypes.c_uint16, i32p]
        lib.oracle_nussinov.restype = ctypes.c_int
        lib.oracle_nussinov_score.argtypes = [u8p, ctypes.c_int, ctypes.c_uint16]
        lib.oracle_nussinov_score.restype = ctypes.c_int
        lib.oracle_brute.argtypes = [u8p, ctypes.c_int, ctypes.c_uint16]
        lib.oracle_brute.restype = ctypes.c_int
        lib.oracle_rtable.argtypes = [ctypes.c_int, u8p, u8p]
        lib.oracle_rtable.restype = ctypes.c_long
        lib.oracle_two_vector.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16, i32p, i64p]
        lib.oracle_two_vector.restype = ctypes.c_int
        lib.oracle_two_vector_sliding.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16, i32p, i64p]
        lib.oracle_two_vector_sliding.restype = ctypes.c_int
        lib.oracle_fg.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16, i32p, i64p, i64p]
        lib.oracle_fg.restype = ctypes.c_int
        lib.oracle_traceback.argtypes = [u8p, ctypes.c_int, ctypes.c_uint16, i32p, i32p]
        lib.oracle_traceback.restype = ctypes.c_int
        _lib = lib
    return _lib


def encode(seq: str) -> np.ndarray:
    """Map a string over {A,C,G,U} (either case) to codes 0..3; anything else raises."""
    try:
        return np.fromiter((_CODE[ch] for ch in seq), dtype=np.uint8, count=len(seq))
    except KeyError as e:  # pragma: no cover - message path
        raise ValueError(f"invalid base {e.args[0]!r}") from None


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def nussinov(seq: str, mask: int = MASK6) -> np.ndarray:
    """Full n*n table of Eq. 1 (int32, row-major, zero below the diagonal)."""
    lib = _load()
    c = encode(seq)
    n = len(c)
    D = np.zeros((n, n), dtype=np.int32)
    if n:
        rc = lib.oracle_nussinov(_u8(c), n, mask, D.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc != 0:
            raise MemoryError("oracle_nussinov failed")
    return D


def score(seq: str, mask: int = MASK6) -> int:
    """D(0, n-1) of Eq. 1 (0 for n <= 1)."""
    lib = _load()
    c = encode(seq)
    s = lib.oracle_nussinov_score(_u8(c), len(c), mask) if len(c) > 1 else 0
    if s < 0:
        raise MemoryError("oracle_nussinov_score failed")
    return int(s)


def traceback(seq: str, mask: int = MASK6, D: np.ndarray | None = None) -> np.ndarray:
    """Partner of each base (-1 unpaired) of one optimal structure: the argmax of Eq. 1 taken
    at each visited cell in a fixed order of preference (unpaired, pair, smallest split)."""
    lib = _load()
    c = encode(seq)
    n = len(c)
    if D is None:
        D = nussinov(seq, mask)
    D = np.ascontiguousarray(D, dtype=np.int32)
    partner = np.full(n, -1, dtype=np.int32)
    if n:
        rc = lib.oracle_traceback(_u8(c), n, mask, D.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  partner.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc < 0:
            raise ValueError("the table admits no argmax: not a table of Eq. 1")
    return partner


def dot_bracket(partner: np.ndarray) -> str:
    """'(' / ')' for the smaller / larger index of each pair, '.' for unpaired bases."""
    return "".join("." if p < 0 else ("(" if p > k else ")") for k, p in enumerate(partner))


def brute(seq: str, mask: int = MASK6) -> int:
    """Largest non-crossing matching by enumeration (tiny inputs only)."""
    lib = _load()
    c = encode(seq)
    if len(c) > 24:
        raise ValueError("brute force is for tiny inputs")
    return int(lib.oracle_brute(_u8(c), len(c), mask))


def rtable(q: int, with_index: bool = False):
    """R table, index (h << (q-1)) | c, as uint8 of length 4**(q-1)."""
    lib = _load()
    n = 1 << (2 * (q - 1))
    R = np.zeros(n, dtype=np.uint8)
    Ri = np.zeros(n, dtype=np.uint8)
    lib.oracle_rtable(q, _u8(R), _u8(Ri))
    return (R, Ri) if with_index else R


def two_vector(seq: str, q: int, mask: int = MASK6, return_lookups: bool = False):
    """Full table by Algorithm 1 (int32); optionally the number of R lookups made."""
    lib = _load()
    c = encode(seq)
    n = len(c)
    D = np.zeros((n, n), dtype=np.int32)
    nl = ctypes.c_int64(0)
    if n:
        rc = lib.oracle_two_vector(_u8(c), n, q, mask, D.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ctypes.byref(nl))
        if rc != 0:
            raise MemoryError("oracle_two_vector failed")
    return (D, int(nl.value)) if return_lookups else D


def two_vector_sliding(seq: str, q: int, mask: int = MASK6, return_lookups: bool = False):
    """Full table by Section 4's two-vector algorithm with per-cell difference vectors (int32);
    optionally the number of R lookups made."""
    lib = _load()
    c = encode(seq)
    n = len(c)
    D = np.zeros((n, n), dtype=np.int32)
    nl = ctypes.c_int64(0)
    if n:
        rc = lib.oracle_two_vector_sliding(_u8(c), n, q, mask, D.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           ctypes.byref(nl))
        if rc != 0:
            raise MemoryError("oracle_two_vector_sliding failed")
    return (D, int(nl.value)) if return_lookups else D


def fg(seq: str, q: int, mask: int = MASK6, return_counts: bool = False):
    """Full table by the FG algorithm (int32); optionally (lookups, row-group tables built)."""
    lib = _load()
    c = encode(seq)
    n = len(c)
    D = np.zeros((n, n), dtype=np.int32)
    nl, nt = ctypes.c_int64(0), ctypes.c_int64(0)
    if n:
        rc = lib.oracle_fg(_u8(c), n, q, mask, D.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(nl),
                           ctypes.byref(nt))
        if rc != 0:
            raise MemoryError("oracle_fg failed")
    return (D, int(nl.value), int(nt.value)) if return_counts else D
