"""C-ABI checks that need no GPU: the library loads and exports every symbol
include/fold.h declares; status strings; argument validation paths that
return before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1307_7820_b300 import build as fbuild
from paper_1307_7820_b300 import fold

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fold.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fold_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    fbuild.build()
    return fold.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert sorted(fold.ABI_SYMBOLS) == names


def test_option_and_status_constants_match_the_header():
    # every FOLD_OPT_* / FOLD_* enumerator and #define of include/fold.h has the same value in the binding
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "fold.h")).read(), flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", src, flags=re.S):
        nxt = 0
        for item in [x.strip() for x in body.split(",") if x.strip()]:
            name, _, val = item.partition("=")
            nxt = int(val.strip(), 0) if val.strip() else nxt
            consts[name.strip()] = nxt
            nxt += 1
    for name, val in re.findall(r"#define\s+(FOLD_[A-Z0-9_]+)\s+(0x[0-9A-Fa-f]+|\d+)", src):
        consts[name] = int(val, 0)
    opts = [k for k in consts if k.startswith("FOLD_OPT_")]
    assert len(opts) >= 21
    for name, val in consts.items():
        assert getattr(fold, name) == val, name


def test_strerror_all_codes(L):
    for code in range(7):
        s = fold.fold_strerror(code)
        assert s and s != "unknown status"
    assert fold.fold_strerror(99) == "unknown status"


def test_null_and_range_arguments(L):
    # all of these are rejected on the host before any device work
    assert L.fold_init(3, 0x5A48, 0, None) == fold.FOLD_EINVAL
    h = ctypes.c_void_p()
    assert L.fold_init(11, 0x5A48, 0, ctypes.byref(h)) == fold.FOLD_EINVAL
    assert L.fold_init(1, 0x5A48, 0, ctypes.byref(h)) == fold.FOLD_EINVAL
    assert L.fold_init(8, 0x5A48, -1, ctypes.byref(h)) == fold.FOLD_EINVAL
    assert L.fold_score(None, b"AU", 2, None, None) == fold.FOLD_EINVAL
    assert L.fold_set_option(None, fold.FOLD_OPT_METHOD, 0) == fold.FOLD_EINVAL
    assert L.fold_workspace_bytes(None, 10) == -fold.FOLD_EINVAL
    assert L.fold_batch(None, 1, None, None, None, None) == fold.FOLD_EINVAL
    r = fold.TuneResult()
    assert L.fold_tune(None, 100, 3, ctypes.byref(r)) == fold.FOLD_EINVAL
    lens = (ctypes.c_int32 * 1)(100)
    assert L.fold_tune_q(0, 0x5A48, 0, lens, 1, 9, 8, ctypes.byref(r)) == fold.FOLD_EINVAL   # empty q range
    assert L.fold_tune_q(0, 0x5A48, 0, lens, 1, 1, 8, ctypes.byref(r)) == fold.FOLD_EINVAL   # q below 2
    assert L.fold_tune_q(0, 0x5A48, 2, lens, 1, 8, 8, ctypes.byref(r)) == fold.FOLD_EINVAL   # unknown method
    assert L.fold_tune_q(0, 0x5A48, 0, lens, 0, 8, 8, ctypes.byref(r)) == fold.FOLD_EINVAL   # no lengths
    assert L.fold_tune_save(None, b"/tmp/x") == fold.FOLD_EINVAL
    assert L.fold_tune_load(None, b"/tmp/x") == fold.FOLD_EINVAL
    st = fold.ServeStats()
    assert L.fold_serve_stats_get(None, ctypes.byref(st)) == fold.FOLD_EINVAL
    assert L.fold_serve_warm(None, 100) == fold.FOLD_EINVAL


def test_pair_mask_constants():
    import oracle
    assert fold.FOLD_PAIRS_DEFAULT == oracle.MASK6
    assert fold.FOLD_PAIRS_PAPER == oracle.MASK4


def test_encode_is_the_section2_alphabet(L):
    """fold_encode (host only) maps A, C, G, U in either case to 0..3 and rejects anything else."""
    import numpy as np
    c = fold.encode_codes("ACGUacguGGGAAAUCC")
    assert c.tolist() == [0, 1, 2, 3, 0, 1, 2, 3, 2, 2, 2, 0, 0, 0, 3, 1, 1]
    assert fold.encode_codes("").size == 0
    for bad in ["ACGT", "AC GU", "N", "acgu\x00", "ACGU\u00e9"]:
        with pytest.raises(fold.FoldError) as ei:
            fold.encode_codes(bad)
        assert ei.value.code == fold.FOLD_EINVAL
    out = np.zeros(4, dtype=np.uint8)
    assert L.fold_encode(None, 4, out.ctypes.data) == fold.FOLD_EINVAL
    assert L.fold_encode(b"ACGU", -1, out.ctypes.data) == fold.FOLD_EINVAL
    assert L.fold_encode(b"ACGU", 4, None) == fold.FOLD_EINVAL
