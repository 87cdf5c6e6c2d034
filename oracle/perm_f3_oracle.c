/*
 * perm_f3_oracle.c -- plain, slow CPU oracle for perm(A) mod 3, A in F3^{n x n}.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * Arithmetic: entries are read as {0,1,2} and centred to {0,1,-1} (2 == -1 in
 * F3).  Everything is exact integer arithmetic; there is no floating point.
 *
 * What each routine follows (Scheinerman, "Fast computation of permanents
 * over F3 via F2 arithmetic", arXiv 2407.20205):
 *   oracle_perm_bruteforce  -- Eq. (1): sum over all n! permutations of the
 *                              product a_{1,s(1)} ... a_{n,s(n)}.
 *   oracle_ryser_range      -- Eq. (2) (Ryser), summed over the COLUMN subsets
 *                              S exactly as Eq. (2) is written, visited in the
 *                              reflected binary Gray code order of Sec. 3
 *                              (footnote: step i flips bit tz(i); Sec. 3.1
 *                              footnote: state i is i xor (i >> 1)).  Each row
 *                              sum is kept centred in {-1,0,1} after every
 *                              update (the cmod3 variant of Sec. 3), so the
 *                              product never overflows.  The sign (-1)^{|S|}
 *                              is taken from the popcount of the subset.
 *   oracle_perm_mod3        -- Eq. (2) over the whole range, times (-1)^n,
 *                              reduced mod 3 into {0,1,2}.
 *   oracle_ryser_range_par  -- Sec. 3.1: contiguous blocks of Gray indices,
 *                              each started from its own directly computed
 *                              subset sum, partial counts added.
 *   oracle_count_exhaustive -- Sec. 4, Table 2: perm over all 3^{n^2} matrices.
 *
 * Conventions where the paper is silent: perm of the 0 x 0 matrix is 1 (the
 * empty product); results are returned in {0,1,2} with -1 -> 2.
 *
 * Counts: for a Gray index i with subset S_i, the Ryser term is
 * (-1)^{|S_i|} * prod_rows (sum_{j in S_i} a_rj)  in {-1,0,1} (mod 3, centred).
 * "plus" counts the indices whose term is +1, "minus" those whose term is -1.
 * perm(A) = (-1)^n (plus - minus)  (mod 3).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAXN 64

/* centred residue of x modulo 3, in {-1,0,1} (the paper's cmod3) */
static int cmod3(long long x)
{
    long long a = ((x % 3) + 3) % 3;
    return a == 2 ? -1 : (int)a;
}

/* entry e in {0,1,2} as a centred F3 value */
static int centred(uint8_t e)
{
    return e == 2 ? -1 : (int)e;
}

/* map a centred residue to {0,1,2} */
static int to012(long long x)
{
    return (int)(((x % 3) + 3) % 3);
}

static int popcount64(uint64_t x)
{
    int c = 0;
    while (x) { c += (int)(x & 1u); x >>= 1; }
    return c;
}

static int trailing_zeros64(uint64_t x) /* x != 0 */
{
    int t = 0;
    while (!(x & 1u)) { x >>= 1; ++t; }
    return t;
}

/* 0 on success, -2 if an entry is outside {0,1,2} */
static int check_entries(const uint8_t* A, int n)
{
    for (long k = 0; k < (long)n * n; ++k)
        if (A[k] > 2) return -2;
    return 0;
}

/* ------------------------------------------------------------------ Eq. (1) */

static long long bf_rec(const uint8_t* A, int n, int row, int* used)
{
    if (row == n) return 1;
    long long total = 0;
    for (int col = 0; col < n; ++col) {
        if (used[col]) continue;
        int a = centred(A[row * n + col]);
        if (a == 0) continue;
        used[col] = 1;
        total += a * bf_rec(A, n, row + 1, used);
        used[col] = 0;
    }
    return total;
}

/* perm(A) mod 3 by the definition, Eq. (1).  n <= 11.  Returns {0,1,2} or <0. */
int oracle_perm_bruteforce(const uint8_t* A, int n)
{
    if (n < 0 || n > 11) return -1;
    if (n == 0) return 1;
    if (!A) return -1;
    if (check_entries(A, n)) return -2;
    int used[11] = {0};
    return to012(bf_rec(A, n, 0, used));
}

/* Exact integer permanent by Eq. (1) (no reduction), for tests that need the
 * integer value.  Entries centred.  n <= 11. */
long long oracle_perm_bruteforce_int(const uint8_t* A, int n)
{
    if (n == 0) return 1;
    int used[11] = {0};
    return bf_rec(A, n, 0, used);
}

/* ------------------------------------------------------------------ Eq. (2) */

/* Ryser terms for the Gray indices first..last (inclusive) of the column-subset
 * walk.  n in 1..64, first <= last < 2^n.  Returns 0, or <0 on bad arguments. */
int oracle_ryser_range(const uint8_t* A, int n, uint64_t first, uint64_t last,
                       uint64_t* plus, uint64_t* minus)
{
    if (!A || !plus || !minus || n < 1 || n > ORACLE_MAXN || first > last) return -1;
    if (n < 64 && last >= ((uint64_t)1 << n)) return -1;
    if (check_entries(A, n)) return -2;

    int a[ORACLE_MAXN][ORACLE_MAXN];
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < n; ++j) a[r][j] = centred(A[r * n + j]);

    /* row sums over the column subset S = gray(first), computed directly */
    uint64_t g = first ^ (first >> 1);
    int rowsum[ORACLE_MAXN];
    for (int r = 0; r < n; ++r) {
        long long acc = 0;
        for (int j = 0; j < n; ++j)
            if ((g >> j) & 1u) acc += a[r][j];
        rowsum[r] = cmod3(acc);
    }

    uint64_t p = 0, m = 0;
    uint64_t i = first;
    for (;;) {
        /* term for subset g = gray(i) */
        int prod = 1;
        for (int r = 0; r < n && prod != 0; ++r) prod *= rowsum[r];
        if (prod != 0) {
            int sign = (popcount64(g) & 1) ? -1 : 1;
            if (sign * prod > 0) ++p; else ++m;
        }
        if (i == last) break;
        ++i;
        /* next Gray state: flip column t = tz(i) */
        int t = trailing_zeros64(i);
        uint64_t gnext = g ^ ((uint64_t)1 << t);
        int entering = (int)((gnext >> t) & 1u); /* column t joins S */
        for (int r = 0; r < n; ++r)
            rowsum[r] = cmod3((long long)rowsum[r] + (entering ? a[r][t] : -a[r][t]));
        g = gnext;
    }
    *plus = p;
    *minus = m;
    return 0;
}

/* perm(A) mod 3 by Eq. (2).  Returns {0,1,2}, or <0. */
int oracle_perm_mod3(const uint8_t* A, int n)
{
    if (n < 0 || n > ORACLE_MAXN) return -1;
    if (n == 0) return 1;
    uint64_t last = (n == 64) ? ~(uint64_t)0 : (((uint64_t)1 << n) - 1);
    uint64_t p, m;
    int rc = oracle_ryser_range(A, n, 0, last, &p, &m);
    if (rc) return rc;
    long long d = (long long)(p % 3) - (long long)(m % 3);
    if (n & 1) d = -d;
    return to012(d);
}

/* Sec. 3.1: the same sum split into nparts contiguous blocks of Gray indices,
 * run on up to nthreads OpenMP threads (nthreads <= 0: all). */
int oracle_ryser_range_par(const uint8_t* A, int n, uint64_t first, uint64_t last,
                           int nparts, int nthreads, uint64_t* plus, uint64_t* minus)
{
    if (!A || !plus || !minus || n < 1 || n > ORACLE_MAXN || first > last || nparts < 1)
        return -1;
    if (n < 64 && last >= ((uint64_t)1 << n)) return -1;
    if (check_entries(A, n)) return -2;
    uint64_t span_m1 = last - first; /* number of indices minus one */
    if ((uint64_t)nparts - 1 > span_m1) nparts = (int)(span_m1 + 1);
    /* part k covers [first + k*q + min(k,r), ...) with span = nparts*q + r */
    uint64_t q = span_m1 / (uint64_t)nparts, r = span_m1 % (uint64_t)nparts;
    /* span = span_m1 + 1 = nparts*q + r + 1 ; distribute the extra r+1 */
    uint64_t extra = r + 1; /* parts 0..extra-1 get q+1 indices, others q */
    uint64_t sp = 0, sm = 0;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : sp, sm) reduction(| : bad)
#endif
    for (int k = 0; k < nparts; ++k) {
        uint64_t uk = (uint64_t)k;
        uint64_t lo = first + uk * q + (uk < extra ? uk : extra);
        uint64_t cnt = q + (uk < extra ? 1 : 0);
        if (cnt == 0) continue;
        uint64_t hi = lo + (cnt - 1);
        uint64_t p, m;
        if (oracle_ryser_range(A, n, lo, hi, &p, &m)) { bad |= 1; continue; }
        sp += p;
        sm += m;
    }
    if (bad) return -1;
    *plus = sp;
    *minus = sm;
    return 0;
}

/* perm mod 3 of `count` matrices back to back (matrix k has size ns[k]),
 * matrices distributed over OpenMP threads.  Returns 0 or <0. */
int oracle_perm_batch(const uint8_t* As, const int32_t* ns, int64_t count,
                      uint8_t* results, int nthreads)
{
    if (count < 0 || (count > 0 && (!As || !ns || !results))) return -1;
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(count + 1));
    if (!off) return -4;
    off[0] = 0;
    for (int64_t k = 0; k < count; ++k) {
        if (ns[k] < 0 || ns[k] > ORACLE_MAXN) { free(off); return -1; }
        off[k + 1] = off[k] + (int64_t)ns[k] * ns[k];
    }
    int bad = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : bad)
#endif
    for (int64_t k = 0; k < count; ++k) {
        int r = oracle_perm_mod3(As + off[k], ns[k]);
        if (r < 0) bad |= 1; else results[k] = (uint8_t)r;
    }
    free(off);
    return bad ? -1 : 0;
}

/* Table 2: over all 3^{n^2} matrices (n <= 4), count how many have perm equal
 * to 0, 1 and 2 (mod 3).  counts[0..2]. */
int oracle_count_exhaustive(int n, int nthreads, uint64_t* counts)
{
    if (n < 1 || n > 4 || !counts) return -1;
    int cells = n * n;
    uint64_t total = 1;
    for (int k = 0; k < cells; ++k) total *= 3;
    uint64_t c0 = 0, c1 = 0, c2 = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static, 65536) num_threads(nthreads) reduction(+ : c0, c1, c2)
#endif
    for (int64_t idx = 0; idx < (int64_t)total; ++idx) {
        uint8_t A[16];
        uint64_t x = (uint64_t)idx;
        for (int k = 0; k < cells; ++k) { A[k] = (uint8_t)(x % 3); x /= 3; }
        int r = oracle_perm_mod3(A, n);
        if (r == 0) ++c0; else if (r == 1) ++c1; else ++c2;
    }
    counts[0] = c0;
    counts[1] = c1;
    counts[2] = c2;
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
