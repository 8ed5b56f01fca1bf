"""Multi-threaded CPU two-vector folding (Section 3.1, Algorithm 1 on a tiled wavefront) -- the
host-core baseline reported beside the GPU kernels.

It is an independent C implementation (``cpu_two_vector.c``, built with gcc and OpenMP into
``libcpu_two_vector.so`` by :func:`build`): it shares no code with the GPU library or with the CPU
oracle, and neither of them uses it.  ``tests/`` checks it against the oracle; ``bench.py`` times it
on the host cores.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_two_vector.c")
_LIB = os.path.join(_HERE, "libcpu_two_vector.so")
_lib = None

_LUT = np.full(256, 255, dtype=np.uint8)
for _ch, _v in zip(b"ACGUacgu", (0, 1, 2, 3, 0, 1, 2, 3)):
    _LUT[_ch] = _v


def build(force: bool = False) -> str:
    """Compile cpu_two_vector.c with gcc -O3 -fopenmp (portable x86-64 code, no -march=native)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.cpu_two_vector.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint16, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
        lib.cpu_two_vector.restype = ctypes.c_int
        _lib = lib
    return _lib


def fold(seq: str, q: int = 8, mask: int = 0x5A48, threads: int = 0, want_D: bool = False):
    """(D(0,n-1), table or None, lookups, threads used) of one fold on ``threads`` host threads (0 = all)."""
    lib = _load()
    c = _LUT[np.frombuffer(seq.encode("ascii"), dtype=np.uint8)]
    if c.size and c.max() == 255:
        raise ValueError("invalid base letter")
    n = int(c.size)
    D = np.zeros((n, n), dtype=np.int16) if want_D else None
    nl = ctypes.c_int64(0)
    used = ctypes.c_int(0)
    rc = lib.cpu_two_vector(c.ctypes.data if n else None, n, q, mask, threads,
                            D.ctypes.data if (want_D and n) else None, ctypes.byref(nl), ctypes.byref(used))
    if rc < 0:
        raise ValueError(f"cpu_two_vector failed ({rc})")
    return rc, D, int(nl.value), int(used.value)
