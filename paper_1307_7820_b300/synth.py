"""Seeded synthetic RNA inputs.

This module is the only code that both the CPU oracle side (``oracle/``,
tests) and the GPU side (bench, serving driver) use.  It draws random
sequences and arrival times and holds none of the folding arithmetic.

The paper's own inputs (mouse non-coding RNA and substrings of real RNA,
Section 6) are not available here; its third workload, random strings over
{A, C, G, U}, is what these generators produce, plus the variants the
workloads below need.  Every generator takes an explicit integer seed and uses
numpy's PCG64 bit generator, so a (generator, seed, size) triple always
yields the same input.

Workloads (seed = 1307 + workload index, sequence index mixed in for batches):

* uniform i.i.d. bases, P(A)=P(C)=P(G)=P(U)=1/4;
* GC-rich: P(G)=P(C)=0.3, P(A)=P(U)=0.2;
* structured: concatenated segments, each a uniform string of length
  L ~ U{20..200} followed by its reverse complement (A<->U, C<->G, reversed),
  truncated to n -- forces deep nested pairings;
* batches: lengths round(exp(U(ln lo, ln hi))) (log-uniform), uniform bases;
* serving: Poisson arrivals (exponential gaps) at a given rate, log-uniform
  lengths, 80% uniform / 10% GC-rich / 10% structured.
"""
from __future__ import annotations

import numpy as np

BASES = np.array(list("ACGU"))
_COMP = str.maketrans("ACGU", "UGCA")

SEED_BASE = 1307


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(n: int, seed: int) -> str:
    """n i.i.d. uniform bases."""
    if n <= 0:
        return ""
    return "".join(BASES[rng(seed).integers(0, 4, size=n)])


def gc_rich(n: int, seed: int) -> str:
    """n i.i.d. bases with P(G)=P(C)=0.3 and P(A)=P(U)=0.2."""
    if n <= 0:
        return ""
    return "".join(rng(seed).choice(BASES, size=n, p=[0.2, 0.3, 0.3, 0.2]))


def revcomp(s: str) -> str:
    return s.translate(_COMP)[::-1]


def structured(n: int, seed: int, lo: int = 20, hi: int = 200) -> str:
    """Segments s_k + revcomp(s_k) with |s_k| ~ U{lo..hi}, truncated to n."""
    g = rng(seed)
    parts = []
    total = 0
    while total < n:
        L = int(g.integers(lo, hi + 1))
        s = "".join(BASES[g.integers(0, 4, size=L)])
        parts.append(s)
        parts.append(revcomp(s))
        total += 2 * L
    return "".join(parts)[:n]


def variant(kind: str, n: int, seed: int) -> str:
    if kind == "uniform":
        return uniform(n, seed)
    if kind in ("gc", "gc_rich"):
        return gc_rich(n, seed)
    if kind == "structured":
        return structured(n, seed)
    raise ValueError(f"unknown variant {kind!r}")


def log_uniform_lengths(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """round(exp(U(ln lo, ln hi))) as int32."""
    g = rng(seed)
    x = np.exp(g.uniform(np.log(lo), np.log(hi), size=count))
    return np.clip(np.rint(x), lo, hi).astype(np.int32)


def batch(count: int, lo: int, hi: int, seed: int) -> list[str]:
    """``count`` uniform sequences with log-uniform lengths in [lo, hi]."""
    lens = log_uniform_lengths(count, lo, hi, seed)
    return [uniform(int(L), seed * 1_000_003 + k) for k, L in enumerate(lens)]


def serve_requests(rate: float, count: int, lo: int, hi: int, seed: int):
    """Poisson arrivals: list of (arrival_time_s, sequence, kind)."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    lens = log_uniform_lengths(count, lo, hi, seed + 17)
    kinds = g.choice(["uniform", "gc_rich", "structured"], size=count, p=[0.8, 0.1, 0.1])
    out = []
    for k in range(count):
        out.append((float(t[k]), variant(str(kinds[k]), int(lens[k]), seed * 7919 + k), str(kinds[k])))
    return out
