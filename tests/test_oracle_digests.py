"""The whole-table digests the oracle wrote for the large single folds (oracle/make_digests.py):
the format reads back what was written, and every committed digest still describes the input the
generator draws today, with the shape Eq. 1 fixes (last row all zero, D(0,n-1) <= n/2)."""
import glob
import hashlib
import os
import zlib

import numpy as np

import oracle
from oracle import make_digests as md
from paper_1307_7820_b300 import synth


def test_digest_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(md, "GOLDEN", str(tmp_path))
    path = md.write_digest("structured", 150, 77)
    d = md.read_digest(path)
    seq = synth.structured(150, 77)
    D = oracle.nussinov(seq).astype("<i2")
    assert d["n"] == 150 and d["seed"] == 77 and d["variant"] == "structured" and d["mask"] == oracle.MASK6
    assert d["score"] == int(D[0, -1])
    assert d["table_sha256"] == hashlib.sha256(D.tobytes()).hexdigest()
    assert d["row_crc32"] == [zlib.crc32(D[i].tobytes()) for i in range(150)]
    # a single changed entry changes the table hash and exactly that row's checksum
    D2 = D.copy()
    D2[40, 90] += 1
    sha2, crc2 = md.table_digests(D2)
    assert sha2 != d["table_sha256"]
    assert [i for i in range(150) if crc2[i] != d["row_crc32"][i]] == [40]


def test_committed_digests_match_todays_inputs():
    files = sorted(glob.glob(os.path.join(md.GOLDEN, "digest_n*.txt")))
    assert files, "no committed digests"
    for path in files:
        d = md.read_digest(path)
        n = d["n"]
        assert os.path.basename(path) == os.path.basename(md.digest_path(n, d["variant"], d["mask"]))
        seq = synth.variant(d["variant"], n, d["seed"])
        assert d["seq_sha256"] == hashlib.sha256(seq.encode()).hexdigest(), path
        assert len(d["row_crc32"]) == n
        assert 0 < d["score"] <= n // 2
        # row n-1 of the table is all zero (D(i,j) = 0 for i >= j)
        assert d["row_crc32"][n - 1] == zlib.crc32(np.zeros(n, dtype="<i2").tobytes())
