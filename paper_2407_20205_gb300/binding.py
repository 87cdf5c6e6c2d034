"""Thin ctypes binding over libperm_f3.so (include/perm_f3.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host buffers are numpy arrays (or anything numpy can view); device
buffers are raw pointers (int) or CUDA tensors (their ``data_ptr()``), and
streams are raw ``cudaStream_t`` handles (int) or ``torch.cuda.Stream``.

Importing this module loads the library and raises ImportError when it has
not been built (``python -c "import __graft_entry__ as g; g.build()"``): there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libperm_f3.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(paper_2407_20205_gb300.build.build())")

_lib = ctypes.CDLL(LIB_PATH)

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p

PF3_OK = 0
PF3_PENDING = 1
PF3_EINVAL = -1
PF3_EDOMAIN = -2
PF3_ECUDA = -3
PF3_ENOMEM = -4
PF3_ETIMEDOUT = -5
PF3_ECANCELED = -6
PF3_EBUSY = -7
PF3_ETOOBIG = -8
MAX_N = 64
NOALLOC_MAX_CTAS = 1024


def _sig(name, restype, argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = argtypes
    return f


_lib_strerror = _sig("pf3_strerror", ctypes.c_char_p, [ctypes.c_int])
_lib_version = _sig("pf3_version", ctypes.c_char_p, [])
_lib_perm = _sig("perm_f3", ctypes.c_int, [_u8p, ctypes.c_int])
_lib_counts = _sig("perm_f3_counts", ctypes.c_int, [_u8p, ctypes.c_int, _u64p, _u64p])
_lib_range = _sig("perm_f3_range_counts", ctypes.c_int,
                  [_u8p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p])
_lib_range_async = _sig("perm_f3_range_counts_async", ctypes.c_int,
                        [_vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _vp, _vp])
_lib_range_noalloc = _sig("perm_f3_range_counts_noalloc", ctypes.c_int,
                          [_vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _vp, ctypes.c_int, _vp])
_lib_batch = _sig("perm_f3_batch", ctypes.c_int, [_u8p, _i32p, ctypes.c_int64, _u8p, _u64p])
_lib_batch_async = _sig("perm_f3_batch_async", ctypes.c_int,
                        [_vp, _i32p, ctypes.c_int64, _vp, _vp, _vp])
_lib_step_table = _sig("pf3_step_table", ctypes.c_int, [_u32p])
_lib_pack = _sig("pf3_pack", ctypes.c_int, [_u8p, ctypes.c_int, _u64p, _u64p])
_lib_intpipe = _sig("pf3_intpipe_bench", ctypes.c_int,
                    [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp])
_lib_devinfo = _sig("pf3_device_info", ctypes.c_int, [_ip, _ip])
_lib_vcount = _sig("pf3_variant_count", ctypes.c_int, [ctypes.c_int])
_lib_setv = _sig("pf3_set_variant", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int])
_lib_getv = _sig("pf3_get_variant", ctypes.c_int, [ctypes.c_int, ctypes.c_int])
_lib_vinfo = _sig("pf3_variant_info", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _ip, _ip, _ip])
_lib_split = _sig("pf3_set_batch_split", ctypes.c_int, [ctypes.c_int, ctypes.c_int])
_lib_vthreads = _sig("pf3_variant_threads", ctypes.c_int, [ctypes.c_int, ctypes.c_int])
_lib_autotune = _sig("pf3_autotune", ctypes.c_int, [_dp, _dp])
_lib_autotune_ex = _sig("pf3_autotune_ex", ctypes.c_int, [_dp, _dp, _dp, _dp, _dp])
_lib_set_btune = _sig("pf3_set_batch_tuning", ctypes.c_int, [ctypes.c_int] * 4)
_lib_get_btune = _sig("pf3_get_batch_tuning", ctypes.c_int, [_ip] * 4)


class PlanItem(ctypes.Structure):
    _fields_ = [("mat", ctypes.c_int64), ("n", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("first_block", ctypes.c_uint64), ("num_blocks", ctypes.c_uint64), ("block_log2", ctypes.c_int32),
                ("cls", ctypes.c_int32)]


_lib_plan = _sig("pf3_batch_plan", ctypes.c_int,
                 [ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, _ip, _ip, ctypes.POINTER(PlanItem), ctypes.c_int64,
                  ctypes.POINTER(ctypes.c_int64), _ip])


class PF3Error(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


def strerror(code: int) -> str:
    return _lib_strerror(code).decode()


def version() -> str:
    return _lib_version().decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise PF3Error(rc, what)
    return rc


def _host_u8(A):
    a = np.ascontiguousarray(np.asarray(A), dtype=np.uint8)
    return a, a.ctypes.data_as(_u8p)


def _square(A):
    a, p = _host_u8(A)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a, p, a.shape[0]


def _dev_ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError("device pointer expected (int or CUDA tensor)")


def _stream_ptr(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError("stream expected (int handle or torch.cuda.Stream)")


# ------------------------------------------------------------ one matrix

def perm_f3(A) -> int:
    """perm(A) mod 3 in {0,1,2} for a square {0,1,2} matrix (host)."""
    a, p, n = _square(A)
    if n == 0:
        return _check(_lib_perm(None, 0), "perm_f3")
    return _check(_lib_perm(p, n), "perm_f3")


_lib_from_counts = _sig("pf3_perm_from_counts", ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64])


def perm_from_counts(n: int, plus: int, minus: int) -> int:
    """perm mod 3 in {0,1,2} from exact (plus, minus) term counts of an n x n
    matrix (the library's final map; counts are unsigned 64-bit)."""
    return _check(_lib_from_counts(n, plus, minus), "pf3_perm_from_counts")


def perm_f3_counts(A) -> tuple[int, int]:
    """(plus, minus) Ryser term counts over all 2^n Gray indices."""
    a, p, n = _square(A)
    P, M = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib_counts(p if n else None, n, ctypes.byref(P), ctypes.byref(M)), "perm_f3_counts")
    return P.value, M.value


def perm_f3_range_counts(A, first: int, last: int) -> tuple[int, int]:
    """(plus, minus) over the Gray indices first..last inclusive."""
    a, p, n = _square(A)
    P, M = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib_range(p, n, first, last, ctypes.byref(P), ctypes.byref(M)), "perm_f3_range_counts")
    return P.value, M.value


def perm_f3_range_counts_async(dA, n: int, first: int, last: int, d_out, stream=None) -> None:
    """Device form: dA (n*n bytes) and d_out (3 x uint64) on the device."""
    _check(_lib_range_async(_dev_ptr(dA), n, first, last, _dev_ptr(d_out), _stream_ptr(stream)),
           "perm_f3_range_counts_async")


def perm_f3_range_counts_noalloc(dA, n: int, first: int, last: int, d_out, ctas: int = 0,
                                 stream=None) -> None:
    """Same as perm_f3_range_counts_async, but the library allocates nothing:
    its scratch is a fixed array inside the library (for callers whose memory
    manager forbids foreign device allocations, or that cannot afford the
    device-wide synchronisation cudaMalloc may cause).  The first call on a
    device looks up that array; calls that overlap on the GPU race."""
    _check(_lib_range_noalloc(_dev_ptr(dA), n, first, last, _dev_ptr(d_out), ctas, _stream_ptr(stream)),
           "perm_f3_range_counts_noalloc")


# ------------------------------------------------------------ batches

def pack_batch(mats):
    """Back-to-back bytes and sizes of a list of square matrices."""
    mats = [np.ascontiguousarray(np.asarray(m), dtype=np.uint8) for m in mats]
    ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    flat = np.concatenate([m.ravel() for m in mats]) if mats else np.zeros(0, np.uint8)
    return flat, ns


def perm_f3_batch(mats=None, *, flat=None, ns=None, with_hist: bool = False):
    """perm mod 3 of many matrices: a list of matrices, or (flat, ns)."""
    if mats is not None:
        flat, ns = pack_batch(mats)
    flat = np.ascontiguousarray(flat, dtype=np.uint8)
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    count = int(ns.shape[0])
    res = np.zeros(max(count, 1), dtype=np.uint8)
    hist = np.zeros(3, dtype=np.uint64)
    fp = flat.ctypes.data_as(_u8p) if flat.size else None
    _check(_lib_batch(fp, ns.ctypes.data_as(_i32p), count, res.ctypes.data_as(_u8p),
                      hist.ctypes.data_as(_u64p)), "perm_f3_batch")
    return (res[:count], hist) if with_hist else res[:count]


def perm_f3_batch_async(dAs, ns, d_results, d_hist, stream=None) -> None:
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    _check(_lib_batch_async(_dev_ptr(dAs), ns.ctypes.data_as(_i32p), int(ns.shape[0]),
                            _dev_ptr(d_results), _dev_ptr(d_hist), _stream_ptr(stream)),
           "perm_f3_batch_async")


# ------------------------------------------------------------ Table 2

_lib_zcount = _sig("pf3_count_exhaustive", ctypes.c_int, [ctypes.c_int, _u64p])


def count_exhaustive(n: int) -> tuple[int, int, int]:
    """(#perm=0, #perm=1, #perm=2) over all 3^(n^2) matrices, n <= 5."""
    c = (ctypes.c_uint64 * 3)()
    _check(_lib_zcount(n, c), "pf3_count_exhaustive")
    return int(c[0]), int(c[1]), int(c[2])


# ------------------------------------------------------------ long runs

_lib_longrun = _sig("pf3_longrun", ctypes.c_int,
                    [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.c_double, _u64p, _u64p, _u64p, _ip,
                     _ip])
LONGRUN_MAX_CHUNK_LOG2 = 44
_lib_longrun_cancel = _sig("pf3_longrun_cancel", None, [ctypes.c_int])


def longrun(A, chunk_log2: int = 42, checkpoint: str | None = None, max_seconds: float = 0.0) -> dict:
    """Walk all 2^n Gray indices in launches of 2^chunk_log2, checkpointing
    after each; returns counts, progress and the return code (PF3_OK,
    PF3_ETIMEDOUT or PF3_ECANCELED leave a resumable checkpoint)."""
    a, p, n = _square(A)
    P, M, nxt, fin, res_ = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int(), ctypes.c_int(-1)
    rc = _lib_longrun(p, n, chunk_log2, checkpoint.encode() if checkpoint else None, max_seconds,
                      ctypes.byref(P), ctypes.byref(M), ctypes.byref(nxt), ctypes.byref(fin), ctypes.byref(res_))
    if rc < 0 and rc not in (PF3_ETIMEDOUT, PF3_ECANCELED):
        raise PF3Error(rc, "pf3_longrun")
    res = {"rc": rc, "plus": P.value, "minus": M.value, "next_index": nxt.value, "finished": bool(fin.value)}
    if fin.value:
        res["perm"] = int(res_.value)
    return res


def longrun_cancel(on: bool = True) -> None:
    _lib_longrun_cancel(1 if on else 0)


# ------------------------------------------------------------ serving

class PF3Config(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int32), ("queue_depth", ctypes.c_int32), ("chunk_log2", ctypes.c_int32),
                ("launch_items", ctypes.c_int32), ("max_admit", ctypes.c_int32), ("small_work_log2", ctypes.c_int32),
                ("launch_budget", ctypes.c_uint64), ("class_max_cols", ctypes.c_int32)]


_lib_cfg_default = _sig("pf3_config_default", None, [ctypes.POINTER(PF3Config)])
_lib_create = _sig("pf3_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PF3Config)])
_lib_destroy = _sig("pf3_destroy", None, [ctypes.c_void_p])
_lib_submit = _sig("perm_f3_submit", ctypes.c_int64, [ctypes.c_void_p, _u8p, ctypes.c_int])
_lib_poll = _sig("perm_f3_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _u8p])
_lib_wait = _sig("perm_f3_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _u8p, ctypes.c_int64])
_lib_times = _sig("pf3_job_times", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _u64p, _u64p])
_lib_stats = _sig("pf3_serve_stats", ctypes.c_int, [ctypes.c_void_p, _u64p, _u64p, _u64p])
_lib_now = _sig("pf3_now_ns", ctypes.c_uint64, [])
_lib_cancel = _sig("pf3_cancel_queued", ctypes.c_int, [ctypes.c_void_p])


class ServeItem(ctypes.Structure):
    _fields_ = [("request", ctypes.c_int64), ("launch", ctypes.c_int32), ("cls", ctypes.c_int32),
                ("first_block", ctypes.c_uint64), ("num_blocks", ctypes.c_uint64), ("block_log2", ctypes.c_int32),
                ("last", ctypes.c_int32)]


_lib_serve_plan = _sig("pf3_serve_plan", ctypes.c_int,
                       [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                        ctypes.POINTER(PF3Config), _ip, ctypes.c_int, ctypes.POINTER(ServeItem), ctypes.c_int64,
                        ctypes.POINTER(ctypes.c_int64)])


def serve_plan(ns, ms=None, launches: int = 1, U=(9, 9), **cfg_overrides) -> list[dict]:
    """The serving loop's work items for requests of sizes ns (columns ms),
    computed on the host (no device needed): one dict per item in issue order."""
    cfg = config_default()
    for k, v in cfg_overrides.items():
        setattr(cfg, k, v)
    nsa = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
    msa = None if ms is None else np.ascontiguousarray(np.asarray(ms, dtype=np.int32))
    p_ns = nsa.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p_ms = None if msa is None else msa.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    Ua = (ctypes.c_int * 2)(*U)
    num = ctypes.c_int64()
    _check(_lib_serve_plan(p_ns, p_ms, len(nsa), ctypes.byref(cfg), Ua, launches, None, 0, ctypes.byref(num)),
           "pf3_serve_plan")
    buf = (ServeItem * max(1, num.value))()
    _check(_lib_serve_plan(p_ns, p_ms, len(nsa), ctypes.byref(cfg), Ua, launches, buf, num.value, ctypes.byref(num)),
           "pf3_serve_plan")
    return [{f: getattr(x, f) for f, _ in ServeItem._fields_} for x in buf[:num.value]]


def config_default() -> PF3Config:
    c = PF3Config()
    _lib_cfg_default(ctypes.byref(c))
    return c


def now_ns() -> int:
    return int(_lib_now())


class ServeContext:
    """pf3_create / perm_f3_submit / perm_f3_poll / perm_f3_wait."""

    def __init__(self, **overrides):
        cfg = config_default()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self._h = ctypes.c_void_p()
        _check(_lib_create(ctypes.byref(self._h), ctypes.byref(cfg)), "pf3_create")
        self.config = cfg

    def close(self):
        if self._h:
            _lib_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, A) -> int:
        a, p, n = _square(A)
        return _check(int(_lib_submit(self._h, p if n else None, n)), "perm_f3_submit")

    def try_submit(self, A) -> int:
        """Like submit, but returns the negative code (e.g. PF3_EBUSY) instead of raising."""
        a, p, n = _square(A)
        return int(_lib_submit(self._h, p if n else None, n))

    def poll(self, ticket: int):
        r = ctypes.c_uint8()
        rc = _lib_poll(self._h, ticket, ctypes.byref(r))
        if rc == PF3_PENDING:
            return None
        _check(rc, "perm_f3_poll")
        return int(r.value)

    def wait(self, ticket: int, timeout_us: int = -1) -> int:
        r = ctypes.c_uint8()
        _check(_lib_wait(self._h, ticket, ctypes.byref(r), timeout_us), "perm_f3_wait")
        return int(r.value)

    def wait_code(self, ticket: int, timeout_us: int = -1) -> int:
        r = ctypes.c_uint8()
        return int(_lib_wait(self._h, ticket, ctypes.byref(r), timeout_us))

    def times(self, ticket: int) -> tuple[int, int]:
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib_times(self._h, ticket, ctypes.byref(a), ctypes.byref(b)), "pf3_job_times")
        return int(a.value), int(b.value)

    def cancel_queued(self) -> int:
        return _check(_lib_cancel(self._h), "pf3_cancel_queued")

    def stats(self) -> dict:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "pf3_serve_stats")
        return {"launches": a.value, "items": b.value, "jobs_done": c.value}


# ------------------------------------------------------------ bipedal vectors

OP_ADD, OP_SUB, OP_MUL, OP_DIV = 0, 1, 2, 3
VEC_MAX_N = 1 << 24
_lib_vecop = _sig("pf3_vec_op", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _u64p, _u64p, _u64p,
                                               _u64p, _u64p, _u64p])
_lib_unpack = _sig("pf3_vec_unpack", ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _u64p, _u64p, _u8p])
_lib_vpack = _sig("pf3_vec_pack", ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _u8p, _u64p, _u64p])


def vec_words(n: int) -> int:
    """64-bit words per plane of one vector of length n."""
    return (n + 63) // 64


def _u64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    return a, a.ctypes.data_as(_u64p)


def _vec_count(n: int, a: np.ndarray) -> int:
    w = vec_words(n)
    if a.size % w:
        raise ValueError(f"a length-{n} vector takes {w} words per plane")
    return a.size // w


def vec_op(op: int, n: int, m1, s1, m2, s2):
    """Elementwise bipedal add/sub/mul/div of arrays of vectors (Theorem 2.1).
    Each plane is uint64[count * ceil(n / 64)] (or [count, ceil(n / 64)]);
    the results have the shape of m1."""
    (m1, p1), (s1, q1), (m2, p2), (s2, q2) = _u64(m1), _u64(s1), _u64(m2), _u64(s2)
    count = _vec_count(n, m1)
    if not (m1.size == s1.size == m2.size == s2.size):
        raise ValueError("planes of different sizes")
    m3 = np.zeros(m1.shape, np.uint64)
    s3 = np.zeros(m1.shape, np.uint64)
    _check(_lib_vecop(op, n, count, p1, q1, p2, q2, m3.ctypes.data_as(_u64p), s3.ctypes.data_as(_u64p)),
           "pf3_vec_op")
    return m3, s3


def vec_unpack(n: int, mag, sgn) -> np.ndarray:
    """psi: uint8[count, n] entries in {0,1,2}."""
    (m, p), (s, q) = _u64(mag), _u64(sgn)
    count = _vec_count(n, m)
    out = np.zeros((count, n), np.uint8)
    _check(_lib_unpack(n, count, p, q, out.ctypes.data_as(_u8p)), "pf3_vec_unpack")
    return out


def vec_pack(X) -> tuple[np.ndarray, np.ndarray]:
    """phi: uint8[count, n] entries in {0,1,2} to planes uint64[count, ceil(n / 64)]."""
    x = np.ascontiguousarray(np.asarray(X), dtype=np.uint8)
    if x.ndim != 2:
        raise ValueError("[count, n] expected")
    count, n = x.shape
    mag = np.zeros((count, vec_words(n)), np.uint64)
    sgn = np.zeros((count, vec_words(n)), np.uint64)
    _check(_lib_vpack(n, count, x.ctypes.data_as(_u8p), mag.ctypes.data_as(_u64p), sgn.ctypes.data_as(_u64p)),
           "pf3_vec_pack")
    return mag, sgn


# ------------------------------------------------------------ diagnostics

_lib_colmerge = _sig("pf3_column_merge", ctypes.c_int, [_u8p, ctypes.c_int, _u8p, _ip, _ip])


_lib_class_counts = _sig("pf3_class_counts", ctypes.c_int, [_u8p, ctypes.c_int, _u64p, _u64p])
_lib_set_class_limit = _sig("pf3_set_class_limit", ctypes.c_int, [ctypes.c_int])
_lib_get_class_limit = _sig("pf3_get_class_limit", ctypes.c_int, [])
CLASS_MAX_COLS = 8


def class_counts(A):
    """(plus, minus) of A counted by column-sum vector on the device, or None
    when A's columns merge into more than CLASS_MAX_COLS columns."""
    a, p, n = _square(A)
    P, M = ctypes.c_uint64(), ctypes.c_uint64()
    rc = _check(_lib_class_counts(p, n, ctypes.byref(P), ctypes.byref(M)), "pf3_class_counts")
    return (P.value, M.value) if rc == 1 else None


def set_class_limit(max_cols: int) -> None:
    """Widest merged matrix perm_f3, perm_f3_counts and a fresh long run count
    by column-sum vector (0: walk every matrix)."""
    _check(_lib_set_class_limit(max_cols), "pf3_set_class_limit")


def get_class_limit() -> int:
    return _check(_lib_get_class_limit(), "pf3_get_class_limit")


def column_merge(A):
    """The column merge the host-pointer single-matrix calls apply: (B, negate)
    with B the n x m matrix walked instead of A, or None when A is walked as
    it is (host only, no device)."""
    a, p, n = _square(A)
    B = np.zeros(n * 32, np.uint8)
    m, neg = ctypes.c_int(), ctypes.c_int()
    rc = _check(_lib_colmerge(p, n, B.ctypes.data_as(_u8p), ctypes.byref(m), ctypes.byref(neg)),
                "pf3_column_merge")
    if rc == 0:
        return None
    return B[:n * m.value].reshape(n, m.value).copy(), bool(neg.value)


def step_table() -> np.ndarray:
    """uint32[4, 3, 2, 2]: (mag', sgn') for state, constant c, direction."""
    out = np.zeros(48, dtype=np.uint32)
    _check(_lib_step_table(out.ctypes.data_as(_u32p)), "pf3_step_table")
    return out.reshape(4, 3, 2, 2)


def pack(A) -> tuple[np.ndarray, np.ndarray]:
    a, p, n = _square(A)
    mag = np.zeros(n, dtype=np.uint64)
    sgn = np.zeros(n, dtype=np.uint64)
    _check(_lib_pack(p, n, mag.ctypes.data_as(_u64p), sgn.ctypes.data_as(_u64p)), "pf3_pack")
    return mag, sgn


INTPIPE_KINDS = {"lop3": 0, "imad": 1, "iadd": 2, "lop3_imad": 3, "step": 4, "popc": 5, "max_imad": 6,
                 "lop3x2_max": 7, "probe": 8, "step_imad": 9, "lop3x2_iadd": 10, "probe_inv": 11,
                 "probe_ones": 12, "probe_and": 13}


def intpipe_bench(kind, ctas_per_sm: int = 4, threads: int = 256, iters: int = 4096) -> dict:
    k = INTPIPE_KINDS[kind] if isinstance(kind, str) else int(kind)
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib_intpipe(k, ctas_per_sm, threads, iters, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "pf3_intpipe_bench")
    return {"inst_per_clk_per_sm": a.value, "inst_per_s": b.value, "sm_mhz": c.value}


def device_info() -> dict:
    sm, dev = ctypes.c_int(), ctypes.c_int()
    _check(_lib_devinfo(ctypes.byref(sm), ctypes.byref(dev)), "pf3_device_info")
    return {"sm_count": sm.value, "device": dev.value}


# ------------------------------------------------------------ tuning

SINGLE, BATCH, SINGLE_SHORT, SINGLE_MERGED = 0, 1, 2, 3


def variant_count(which: int) -> int:
    return _check(_lib_vcount(which), "pf3_variant_count")


def set_variant(which: int, W: int, v: int) -> None:
    _check(_lib_setv(which, W, v), "pf3_set_variant")


def get_variant(which: int, W: int) -> int:
    return _check(_lib_getv(which, W), "pf3_get_variant")


def variant_info(which: int, v: int) -> dict:
    U, G, mc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib_vinfo(which, v, ctypes.byref(U), ctypes.byref(G), ctypes.byref(mc)), "pf3_variant_info")
    return {"U": U.value, "G": G.value, "min_ctas": mc.value,
            "threads": _check(_lib_vthreads(which, v), "pf3_variant_threads")}


def set_batch_split(cutoff: int, chunk_log2: int) -> None:
    _check(_lib_split(cutoff, chunk_log2), "pf3_set_batch_split")


TINY_MAX_N = 16
SPLIT_CANDIDATES = (1, 2, 4, 8, 16)


def set_batch_tuning(tiny_cutoff: int, split_cutoff: int, chunk_log2: int, items_per_warp: int) -> None:
    _check(_lib_set_btune(tiny_cutoff, split_cutoff, chunk_log2, items_per_warp), "pf3_set_batch_tuning")


def get_batch_tuning() -> dict:
    v = [ctypes.c_int() for _ in range(4)]
    _check(_lib_get_btune(*[ctypes.byref(x) for x in v]), "pf3_get_batch_tuning")
    return dict(zip(("tiny_cutoff", "split_cutoff", "chunk_log2", "items_per_warp"), (x.value for x in v)))


_lib_range_plan = _sig("pf3_range_plan", ctypes.c_int,
                       [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u64p, _u64p,
                        _u64p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)])
RANGE_PLAN_FIELDS = ("has_head", "head_first", "head_last", "has_tail", "tail_first", "tail_last", "mid_B0",
                     "mid_NB", "dynamic", "U", "threads", "nchunks")


def range_plan(n: int, first: int, last: int, variant: int = 0, grid: int = 304) -> dict:
    """The single-matrix launch plan of Gray indices [first, last], computed on
    the host (no device needed); chunks as (first block, blocks) relative to
    mid_B0 when the launch hands out guided chunks."""
    info = (ctypes.c_uint64 * 12)()
    num = ctypes.c_int64()
    _check(_lib_range_plan(n, first, last, variant, grid, info, None, None, 0, ctypes.byref(num)),
           "pf3_range_plan")
    cf = (ctypes.c_uint64 * max(1, num.value))()
    cl = (ctypes.c_uint64 * max(1, num.value))()
    _check(_lib_range_plan(n, first, last, variant, grid, info, cf, cl, num.value, ctypes.byref(num)),
           "pf3_range_plan")
    out = dict(zip(RANGE_PLAN_FIELDS, (int(x) for x in info)))
    out["chunks"] = list(zip((int(x) for x in cf[:num.value]), (int(x) for x in cl[:num.value])))
    return out


PLAN_KINDS = ("whole", "piece", "packed", "lane")


def batch_plan(ns, tiny_cutoff: int = 10, split_cutoff: int = 28, chunk_log2: int = 0, items_per_warp: int = 8,
               variant=(0, 0), warps=(2432, 2432)) -> dict:
    """The batch planner's work items for sizes `ns`, computed on the host
    (no device needed): launch order per class, as perm_f3_batch would run
    them."""
    nsa = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
    p = nsa.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    va = (ctypes.c_int * 2)(*variant)
    wa = (ctypes.c_int * 2)(*warps)
    num = ctypes.c_int64()
    cl = (ctypes.c_int * 2)()
    args = (p, len(nsa), tiny_cutoff, split_cutoff, chunk_log2, items_per_warp, va, wa)
    _check(_lib_plan(*args, None, 0, ctypes.byref(num), cl), "pf3_batch_plan")
    buf = (PlanItem * max(1, num.value))()
    _check(_lib_plan(*args, buf, num.value, ctypes.byref(num), cl), "pf3_batch_plan")
    items = [{"mat": x.mat, "n": x.n, "kind": PLAN_KINDS[x.kind], "first_block": x.first_block,
              "num_blocks": x.num_blocks, "block_log2": x.block_log2, "cls": x.cls} for x in buf[:num.value]]
    return {"items": items, "chunk_log2": [cl[0], cl[1]]}


def autotune() -> dict:
    """Variant timings per W, the packed and warp walk times per n (packing
    cutoff), the split-granularity timings, and the choices made."""
    ns, nb = variant_count(SINGLE), variant_count(BATCH)
    a = (ctypes.c_double * (2 * ns))()
    a2 = (ctypes.c_double * (2 * ns))()
    b = (ctypes.c_double * (2 * nb))()
    pk = (ctypes.c_double * (2 * (TINY_MAX_N + 1)))()
    sp = (ctypes.c_double * len(SPLIT_CANDIDATES))()
    _check(_lib_autotune_ex(a, a2, b, pk, sp), "pf3_autotune_ex")
    pk = list(pk)
    return {"single_ms": {1: list(a)[:ns], 2: list(a)[ns:]},
            "single_short_ms": {1: list(a2)[:ns], 2: list(a2)[ns:]},
            "single_short_variant": {W: get_variant(SINGLE_SHORT, W) for W in (1, 2)},
            "single_merged_variant": get_variant(SINGLE_MERGED, 1),
            "batch_ms": {1: list(b)[:nb], 2: list(b)[nb:]},
            "pack_ms": {n: [pk[n], pk[TINY_MAX_N + 1 + n]] for n in range(TINY_MAX_N + 1) if pk[n] > 0},
            "split_ms": dict(zip(SPLIT_CANDIDATES, list(sp))),
            "single_variant": {W: get_variant(SINGLE, W) for W in (1, 2)},
            "batch_variant": {W: get_variant(BATCH, W) for W in (1, 2)},
            "batch_tuning": get_batch_tuning()}


def exported_symbols() -> list[str]:
    return [n for n in ("pf3_strerror", "pf3_version", "perm_f3", "perm_f3_counts",
                        "perm_f3_range_counts", "perm_f3_range_counts_async", "perm_f3_batch",
                        "perm_f3_batch_async", "pf3_step_table", "pf3_pack", "pf3_intpipe_bench",
                        "pf3_device_info", "pf3_variant_count", "pf3_set_variant", "pf3_get_variant",
                        "pf3_set_batch_split", "pf3_autotune", "perm_f3_range_counts_noalloc",
                        "pf3_config_default", "pf3_create", "pf3_destroy", "perm_f3_submit", "perm_f3_poll",
                        "perm_f3_wait", "pf3_job_times", "pf3_serve_stats", "pf3_now_ns",
                        "pf3_cancel_queued", "pf3_longrun", "pf3_longrun_cancel",
                        "pf3_count_exhaustive", "pf3_variant_info", "pf3_vec_op",
                        "pf3_vec_unpack", "pf3_set_batch_tuning", "pf3_get_batch_tuning",
                        "pf3_autotune_ex", "pf3_batch_plan", "pf3_variant_threads",
                        "pf3_range_plan", "pf3_perm_from_counts", "pf3_vec_pack",
                        "pf3_column_merge", "pf3_serve_plan", "pf3_class_counts", "pf3_set_class_limit",
                        "pf3_get_class_limit")
            if hasattr(_lib, n)]
