"""Write digests of whole oracle tables for the large single folds -- TEST INFRASTRUCTURE ONLY.

At n = 8000, 16384 and 32768 the cubic oracle (Section 2, Eq. 1) takes from a
minute to a few hours on one core, too long to run inside a test.  This script
runs it once per (variant, n, seed, pair mask) and stores what a GPU test needs
to check a whole table bit for bit:

* D(0, n-1), the answer;
* the SHA-256 of the row-major int16 table (n*n entries, zero below the
  diagonal, little-endian), i.e. exactly the bytes ``fold_score`` writes;
* the CRC-32 of every row's n int16 entries, so that a mismatch names its rows;
* the SHA-256 of the input string, so that a change in the generator shows up
  as such and not as a wrong table.

It calls only the oracle (``oracle.nussinov``) and the seeded input generator
(``synth``), which holds no folding arithmetic.  Usage, from the repository
root::

    python -m oracle.make_digests --variant structured --n 32768 --seed 32768

writes ``tests/golden/digest_n32768_structured.txt``.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time
import zlib

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
from paper_1307_7820_b300 import synth  # noqa: E402  (input generator only)

GOLDEN = os.path.join(_ROOT, "tests", "golden")
ROWS_PER_LINE = 8


def digest_path(n: int, variant: str, mask: int = oracle.MASK6) -> str:
    tag = "" if mask == oracle.MASK6 else f"_m{mask:04x}"
    return os.path.join(GOLDEN, f"digest_n{n}_{variant}{tag}.txt")


def table_digests(D16: np.ndarray):
    """(SHA-256 hex of the whole table, list of per-row CRC-32) of an int16 n*n table."""
    D16 = np.ascontiguousarray(D16, dtype="<i2")
    sha = hashlib.sha256(memoryview(D16).cast("B")).hexdigest()
    crcs = [zlib.crc32(memoryview(D16[i]).cast("B")) for i in range(D16.shape[0])]
    return sha, crcs


def write_digest(variant: str, n: int, seed: int, mask: int = oracle.MASK6) -> str:
    seq = synth.variant(variant, n, seed)
    t0 = time.time()
    D = oracle.nussinov(seq, mask)
    secs = time.time() - t0
    assert int(D.max()) <= n // 2 < 32768
    D16 = D.astype("<i2")
    del D
    sha, crcs = table_digests(D16)
    path = digest_path(n, variant, mask)
    lines = [
        "# Whole-table digest of the Nussinov recurrence (Section 2, Eq. 1), computed by the CPU oracle",
        "# (oracle.nussinov) through oracle/make_digests.py; no value here comes from the GPU library.",
        f"# oracle time {secs:.0f} s on one core",
        f"variant {variant}",
        f"n {n}",
        f"seed {seed}",
        f"mask 0x{mask:04x}",
        f"seq_sha256 {hashlib.sha256(seq.encode()).hexdigest()}",
        f"score {int(D16[0, n - 1]) if n else 0}",
        f"table_sha256 {sha}",
        f"row_crc32 {n}",
    ]
    for r in range(0, n, ROWS_PER_LINE):
        lines.append(" ".join(f"{c:08x}" for c in crcs[r:r + ROWS_PER_LINE]))
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    os.replace(tmp, path)
    return path


def read_digest(path: str) -> dict:
    """Parse a digest file into {variant, n, seed, mask, seq_sha256, score, table_sha256, row_crc32}."""
    out: dict = {}
    crcs: list[int] = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if "row_crc32" in out:
                crcs.extend(int(x, 16) for x in line.split())
            elif key in ("n", "seed", "score"):
                out[key] = int(rest)
            elif key == "mask":
                out[key] = int(rest, 16)
            elif key == "row_crc32":
                out[key] = int(rest)
            else:
                out[key] = rest
    if len(crcs) != out.get("row_crc32", -1):
        raise ValueError(f"{path}: expected {out.get('row_crc32')} row checksums, found {len(crcs)}")
    out["row_crc32"] = crcs
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--variant", required=True, choices=["uniform", "gc_rich", "structured"])
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--seed", type=int, required=True)
    ap.add_argument("--mask", type=lambda s: int(s, 0), default=oracle.MASK6)
    a = ap.parse_args(argv)
    print(write_digest(a.variant, a.n, a.seed, a.mask))


if __name__ == "__main__":
    main()
