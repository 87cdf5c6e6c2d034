"""Seeded synthetic inputs: random matrices over F3 in {0,1,2} (2 == -1).

This module is shared by the tests, the benchmark and the oracle checks.  It
holds no arithmetic of the permanent method: it only draws matrices.

Generator: splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; the 64-bit finaliser constants of Vigna's
public reference version).  Matrix ``k`` of a stream with seed ``seed`` starts
from the state ``seed xor ((k + 1) * 0x9E3779B97F4A7C15 mod 2^64)`` and draws
successive outputs from there.

* uniform entries: each 64-bit output gives 32 two-bit fields, least
  significant first; the field value 3 is rejected, so the entries are exactly
  uniform on {0,1,2} -- the paper draws its timing and Monte Carlo matrices
  uniformly from {-1,0,1} (Sec. 3, Sec. 4);
* sparse entries (the serving mix): output x, rejected when
  x >= floor(2^64/5)*5; x mod 5 in {0,1,2} -> 0, 3 -> 1, 4 -> 2, so that
  P(0) = 0.6, P(1) = P(2) = 0.2.

Known-answer families (permuted identities, J_n, block-diagonal products under
monomial transforms) are built from the same streams.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1
_LIMIT5 = ((1 << 64) // 5) * 5

# seeds of the five workloads (n = 20; n = 36 and 40; batch n = 24; serving
# mix; n = 48)
SEED_N20 = 20
SEED_N36 = 36
SEED_N40 = 40
SEED_BATCH24 = 24
SEED_SERVE = 4
SEED_N48 = 48


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_states(seed: int, ks) -> np.ndarray:
    ks = np.asarray(ks, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return np.uint64(seed & _MASK64) ^ ((ks + np.uint64(1)) * GOLDEN)


def draw(states: np.ndarray, count: int) -> tuple[np.ndarray, np.ndarray]:
    """``count`` successive splitmix64 outputs for every state.

    Returns (outputs[len(states), count], advanced states)."""
    st = states.astype(np.uint64).copy()
    out = np.empty((st.shape[0], count), dtype=np.uint64)
    with np.errstate(over="ignore"):
        for c in range(count):
            st += GOLDEN
            out[:, c] = _mix(st.copy())
    return out, st


def _splitmix_scalar(state: int) -> tuple[int, int]:
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31), state


class Stream:
    """Scalar splitmix64 stream (for per-job choices)."""

    def __init__(self, seed: int, k: int):
        self.state = (seed ^ (((k + 1) * 0x9E3779B97F4A7C15) & _MASK64)) & _MASK64

    def next(self) -> int:
        x, self.state = _splitmix_scalar(self.state)
        return x

    def below(self, m: int) -> int:
        """uniform integer in [0, m) by rejection"""
        lim = ((1 << 64) // m) * m
        while True:
            x = self.next()
            if x < lim:
                return x % m

    def uniform01(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))


def _first_valid(fields: np.ndarray, valid: np.ndarray, need: int):
    ok = valid.sum(axis=1) >= need
    order = np.argsort(~valid, axis=1, kind="stable")[:, :need]
    return np.take_along_axis(fields, order, axis=1), ok


def uniform_matrices(seed: int, n: int, count: int, start: int = 0,
                     chunk: int = 8192) -> np.ndarray:
    """Matrices start..start+count-1 of the stream `seed`, uniform in {0,1,2}.

    Returns uint8[count, n, n]."""
    need = n * n
    out = np.empty((count, n, n), dtype=np.uint8)
    if need == 0 or count == 0:
        return out
    shifts = (np.arange(32, dtype=np.uint64) * np.uint64(2))
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        ks = np.arange(start + c0, start + c1, dtype=np.uint64)
        words = -(-need * 11 // 240) + 8  # ~1.1 * need / 24 outputs, plus slack
        todo = np.arange(c1 - c0)
        while todo.size:
            outs, _ = draw(stream_states(seed, ks[todo]), words)
            fields = ((outs[:, :, None] >> shifts) & np.uint64(3)).astype(np.uint8)
            fields = fields.reshape(todo.size, -1)
            sel, ok = _first_valid(fields, fields != 3, need)
            out[c0 + todo[ok]] = sel[ok].reshape(-1, n, n)
            todo = todo[~ok]
            words *= 2
    return out


def uniform_matrix(seed: int, n: int, k: int = 0) -> np.ndarray:
    return uniform_matrices(seed, n, 1, start=k)[0]


def sparse_matrix_from_stream(st: Stream, n: int) -> np.ndarray:
    vals = np.empty(n * n, dtype=np.uint8)
    lut = (0, 0, 0, 1, 2)
    i = 0
    while i < n * n:
        x = st.next()
        if x >= _LIMIT5:
            continue
        vals[i] = lut[x % 5]
        i += 1
    return vals.reshape(n, n)


def uniform_matrix_from_stream(st: Stream, n: int) -> np.ndarray:
    vals = np.empty(n * n, dtype=np.uint8)
    i = 0
    while i < n * n:
        x = st.next()
        for f in range(32):
            v = (x >> (2 * f)) & 3
            if v == 3:
                continue
            vals[i] = v
            i += 1
            if i == n * n:
                break
    return vals.reshape(n, n)


def random_permutation(st: Stream, n: int) -> np.ndarray:
    """Fisher-Yates shuffle of 0..n-1."""
    p = np.arange(n)
    for i in range(n - 1, 0, -1):
        j = st.below(i + 1)
        p[i], p[j] = p[j], p[i]
    return p


def monomial(st: Stream, n: int) -> np.ndarray:
    """A permutation matrix with every nonzero entry drawn from {1,2}."""
    p = random_permutation(st, n)
    M = np.zeros((n, n), dtype=np.uint8)
    for i in range(n):
        M[i, p[i]] = 1 + st.below(2)
    return M


def f3_matmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Matrix product over F3 of {0,1,2} matrices (used only to build inputs)."""
    return ((X.astype(np.int64) @ Y.astype(np.int64)) % 3).astype(np.uint8)


def ones_matrix(n: int) -> np.ndarray:
    return np.ones((n, n), dtype=np.uint8)


def block_diag(*blocks) -> np.ndarray:
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n), dtype=np.uint8)
    o = 0
    for b in blocks:
        k = b.shape[0]
        M[o:o + k, o:o + k] = b
        o += k
    return M


def serve_job(seed: int, j: int, nmin: int = 12, nmax: int = 40):
    """Job j of the serving mix: (n, kind, matrix, parts).

    kind is 'uniform' (80%), 'sparse' (15%) or one of the known-answer kinds
    'perm_identity', 'ones', 'blockdiag' (5%, split evenly).  For the
    known-answer kinds, ``parts`` holds the pieces the matrix was built from
    (so a test can compute its permanent from closed forms)."""
    st = Stream(seed, j)
    n = nmin + st.below(nmax - nmin + 1)
    u = st.below(1000)
    if u < 800:
        return n, "uniform", uniform_matrix_from_stream(st, n), None
    if u < 950:
        return n, "sparse", sparse_matrix_from_stream(st, n), None
    kind = ("perm_identity", "ones", "blockdiag")[st.below(3)]
    if kind == "perm_identity":
        M = monomial(st, n)
        return n, kind, M, {"monomial": M}
    if kind == "ones":
        return n, kind, ones_matrix(n), None
    # blockdiag: P1 * blockdiag(B1, ..., Bk) * P2, blocks of size <= 12
    sizes = []
    left = n
    while left > 0:
        s = 1 + st.below(min(12, left))
        sizes.append(s)
        left -= s
    blocks = [uniform_matrix_from_stream(st, s) for s in sizes]
    P1 = monomial(st, n)
    P2 = monomial(st, n)
    M = f3_matmul(f3_matmul(P1, block_diag(*blocks)), P2)
    return n, kind, M, {"blocks": blocks, "P1": P1, "P2": P2}


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    st = Stream(seed ^ 0x5EED, 0)
    t = 0.0
    out = np.empty(count, dtype=np.float64)
    for i in range(count):
        u = st.uniform01()
        t += -np.log1p(-u) / rate_per_s
        out[i] = t
    return out


def pooled_columns(seed: int, n: int, low_pool: int, high_pool: int | None) -> np.ndarray:
    """An n x n matrix whose columns 0..31 are each a random nonzero multiple
    (1 or 2) of one of `low_pool` random column vectors, and whose columns
    32..n-1 are drawn the same way from `high_pool` vectors (uniform entries
    when high_pool is None).  A row subset's column sums then take few
    distinct values on each 32-column word, so the share of subsets whose
    first 32 sums are all nonzero is about (2/3)^low_pool instead of
    (2/3)^32: a small pool makes most subsets pass that test.  Drawn from the
    splitmix64 stream (seed, 0)."""
    st = Stream(seed, 0)
    A = np.zeros((n, n), dtype=np.uint8)

    def fill(cols, pool):
        if not cols:
            return
        if pool is None:
            A[:, cols] = uniform_matrix_from_stream(st, n)[:, :len(cols)]
            return
        vecs = uniform_matrix_from_stream(st, max(n, pool))[:pool, :n]
        for c in cols:
            k = st.below(pool)
            A[:, c] = (vecs[k].astype(np.int64) * (1 + st.below(2)) % 3).astype(np.uint8)

    fill(list(range(min(32, n))), low_pool)
    fill(list(range(32, n)), high_pool)
    return A
