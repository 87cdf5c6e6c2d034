"""CPU oracle for perm(A) mod 3 over F3 (arXiv 2407.20205).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2407_20205_gb300``) never does.  The oracle shares no code with the
CUDA path.

The arithmetic lives in ``perm_f3_oracle.c`` (plain C, exact integers); this
module compiles it with gcc and exposes it through ctypes:

* ``perm_bruteforce(A)``      -- Eq. (1), the n! definition (n <= 11).
* ``ryser_range(A, a, b)``    -- Eq. (2) over column subsets, Gray indices a..b
                                 (inclusive); returns the (+1, -1) term counts.
* ``perm_mod3(A)``            -- Eq. (2) over all 2^n subsets, times (-1)^n.
* ``ryser_range_par``         -- Sec. 3.1 block split over OpenMP threads.
* ``perm_batch``              -- many matrices, OpenMP over matrices.
* ``count_exhaustive(n)``     -- Table 2: perm over all 3^{n^2} matrices.

Entries are uint8 in {0,1,2} (2 == -1 mod 3); results are in {0,1,2}.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "perm_f3_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_perm_f3.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle_perm_f3.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-Wall", "-Wextra", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.oracle_perm_bruteforce.argtypes = [u8p, ctypes.c_int]
            L.oracle_perm_bruteforce.restype = ctypes.c_int
            L.oracle_perm_bruteforce_int.argtypes = [u8p, ctypes.c_int]
            L.oracle_perm_bruteforce_int.restype = ctypes.c_longlong
            L.oracle_ryser_range.argtypes = [u8p, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_uint64, u64p, u64p]
            L.oracle_ryser_range.restype = ctypes.c_int
            L.oracle_perm_mod3.argtypes = [u8p, ctypes.c_int]
            L.oracle_perm_mod3.restype = ctypes.c_int
            L.oracle_ryser_range_par.argtypes = [u8p, ctypes.c_int, ctypes.c_uint64,
                                                 ctypes.c_uint64, ctypes.c_int,
                                                 ctypes.c_int, u64p, u64p]
            L.oracle_ryser_range_par.restype = ctypes.c_int
            L.oracle_perm_batch.argtypes = [u8p, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.c_int64, u8p, ctypes.c_int]
            L.oracle_perm_batch.restype = ctypes.c_int
            L.oracle_count_exhaustive.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
            L.oracle_count_exhaustive.restype = ctypes.c_int
            L.oracle_max_threads.argtypes = []
            L.oracle_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _mat(A) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(np.asarray(A, dtype=np.uint8))
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a, a.shape[0]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _check(rc: int) -> int:
    if rc < 0:
        raise ValueError(f"oracle rejected its arguments (code {rc})")
    return rc


def perm_bruteforce(A) -> int:
    a, n = _mat(A)
    return _check(lib().oracle_perm_bruteforce(_ptr(a), n))


def perm_bruteforce_int(A) -> int:
    a, n = _mat(A)
    if n > 11:
        raise ValueError("n <= 11")
    return int(lib().oracle_perm_bruteforce_int(_ptr(a), n))


def ryser_range(A, first: int, last: int) -> tuple[int, int]:
    a, n = _mat(A)
    p, m = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().oracle_ryser_range(_ptr(a), n, first, last,
                                    ctypes.byref(p), ctypes.byref(m)))
    return p.value, m.value


def ryser_range_par(A, first: int, last: int, nparts: int = 0,
                    nthreads: int = 0) -> tuple[int, int]:
    a, n = _mat(A)
    if nparts <= 0:
        nparts = 4 * max(1, max_threads() if nthreads <= 0 else nthreads)
    p, m = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().oracle_ryser_range_par(_ptr(a), n, first, last, nparts, nthreads,
                                        ctypes.byref(p), ctypes.byref(m)))
    return p.value, m.value


def counts(A, nthreads: int = 0) -> tuple[int, int]:
    """(+1, -1) Ryser term counts over all 2^n Gray indices."""
    a, n = _mat(A)
    if n == 0:
        raise ValueError("n >= 1")
    last = (1 << n) - 1
    if n <= 16:
        return ryser_range(a, 0, last)
    return ryser_range_par(a, 0, last, nthreads=nthreads)


def perm_from_counts(n: int, plus: int, minus: int) -> int:
    """(-1)^n (plus - minus) mod 3, in {0,1,2}."""
    d = plus - minus
    if n & 1:
        d = -d
    return d % 3


def perm_mod3(A, nthreads: int = 0) -> int:
    a, n = _mat(A)
    if n == 0:
        return 1
    if n <= 16:
        return _check(lib().oracle_perm_mod3(_ptr(a), n))
    p, m = counts(a, nthreads=nthreads)
    return perm_from_counts(n, p, m)


def perm_batch(mats, nthreads: int = 0) -> np.ndarray:
    """perm mod 3 of a list of square uint8 matrices."""
    mats = [np.ascontiguousarray(np.asarray(x, dtype=np.uint8)) for x in mats]
    ns = np.array([x.shape[0] for x in mats], dtype=np.int32)
    flat = (np.concatenate([x.ravel() for x in mats]) if mats
            else np.zeros(1, np.uint8))
    if flat.size == 0:
        flat = np.zeros(1, np.uint8)
    out = np.zeros(max(1, len(mats)), dtype=np.uint8)
    _check(lib().oracle_perm_batch(_ptr(flat), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   len(mats), _ptr(out), nthreads))
    return out[:len(mats)]


def count_exhaustive(n: int, nthreads: int = 0) -> tuple[int, int, int]:
    c = (ctypes.c_uint64 * 3)()
    _check(lib().oracle_count_exhaustive(n, nthreads, c))
    return int(c[0]), int(c[1]), int(c[2])


def max_threads() -> int:
    return int(lib().oracle_max_threads())
