// pf3_device.cuh -- device building blocks of the bit-sliced Gray-code Ryser
// walk for perm(A) mod 3, A in F3^{n x n}, n <= 64 (arXiv 2407.20205).
//
// Representation (Sec. 2, the "bipedal" pair): an F3 vector of length n is a
// pair of bit vectors (mag, sgn); column j is bit j (least significant first;
// the paper's appendix packs most significant first, which only permutes the
// columns and leaves the permanent unchanged).  phi: 0 -> (0,0), 1 -> (1,0),
// -1 -> (1,1); (0,1) is a second representation of 0 (Definition 2.1).
// Each plane is held as W 32-bit words (W = 1 for up to 32 columns, 2 for up
// to 64).  The walk functions below take the number of columns as `n`: it only
// places the padding; the rows come from the row table (a matrix of n rows
// may be walked with fewer columns, see pf3_capi.cu's column merge).
//
// Row step (Sec. 2, Theorem 2.1 and the addition truth table, Table 1):
// adding a row r, or subtracting it, adds a per-column constant c in F3 to the
// running subset sum.  Instead of Theorem 2.1's six two-input gates we use
// three three-input gates (one LOP3 each) and two per-row masks, chosen by an
// exhaustive search over the zero-representation freedom the paper describes
// (Sec. 2, discussion of Table 1):
//     K1 = [c == 0],  K2 = [c == 1]
//     g    = ~K1 & (sgn ^ K2)
//     mag' = K1 ? mag : (~mag | g)
//     sgn' = ~(mag ^ sgn ^ g)
// Subtracting row r adds -r, whose masks are K1 = [r == 0], K2 = [r == -1]:
// K1 is shared by both directions, only K2 differs (k2p / k2m below).
// Columns j >= n are padding: they start as (1,0), i.e. the constant 1, and
// every row holds 0 there, so they stay (1,0) and neither change the product
// nor its sign.  The zero test of Sec. 3 ("mag == mask") then becomes
// "every mag word is all ones".
//
// Gray order (Sec. 3, footnote on the reflected binary code): index i has
// subset gray(i) = i ^ (i >> 1); step i flips row t = tz(i), and the row is
// subtracted when bit t+1 of i is 1 (the bit is being cleared), added
// otherwise.  The sign (-1)^{|S|} of Eq. (2) is (-1)^(i & 1) because each
// step changes |S| by one.  The product of a subset sum with no zero entry is
// (-1)^{popcount(sgn)} (Sec. 3, footnote on poppar).
#pragma once
#include <cstdint>

namespace pf3 {

constexpr int kMaxN = 64;

template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

// LUT immediates: F(0xF0, 0xCC, 0xAA) for inputs (a, b, c)
constexpr int kLutG = 0x12;    // g    = ~b & (a ^ c)        a=sgn, b=K1, c=K2
constexpr int kLutMag = 0xE3;  // mag' = b ? a : (~a | c)    a=mag, b=K1, c=g
constexpr int kLutSgn = 0x69;  // sgn' = ~(a ^ b ^ c)        a=mag, b=sgn, c=g
constexpr int kLutMagInv = (~kLutMag) & 0xFF;  // ~mag', same inputs as kLutMag

// add the per-column constant described by (k1, k2) to one word of the state
__device__ __forceinline__ void add_word(uint32_t& m, uint32_t& s, uint32_t k1, uint32_t k2)
{
    const uint32_t g = lop3<kLutG>(s, k1, k2);
    const uint32_t mn = lop3<kLutMag>(m, k1, g);
    const uint32_t sn = lop3<kLutSgn>(m, s, g);
    m = mn;
    s = sn;
}

template <int W>
struct State {
    uint32_t m[W];
    uint32_t s[W];
};

template <int W>
__device__ __forceinline__ void add_masks(State<W>& st, const uint32_t (&k1)[W], const uint32_t (&k2)[W])
{
#pragma unroll
    for (int w = 0; w < W; ++w) add_word(st.m[w], st.s[w], k1[w], k2[w]);
}

// Row tables in shared memory: for direction d (0 = add, 1 = subtract) and
// row r, the W words of K1 followed by the W words of K2(d).
template <int W>
struct RowEntry {
    uint32_t k1[W];
    uint32_t k2[W];
};

template <int W>
struct RowTable {
    RowEntry<W> e[2][kMaxN];
};

// masks of one row from its packed mag/sgn words (K1 = ~mag, K2+ = mag & ~sgn,
// K2- = mag & sgn); padding columns (mag = 0) get K1 = 1, K2 = 0.
__device__ __forceinline__ void row_masks(uint32_t mag, uint32_t sgn, uint32_t& k1, uint32_t& k2p,
                                          uint32_t& k2m)
{
    k1 = ~mag;
    k2p = mag & ~sgn;
    k2m = mag & sgn;
}

// initial state: the zero vector on the n real columns, the constant 1 on padding
template <int W>
__device__ __forceinline__ State<W> initial_state(int n)
{
    State<W> st;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int lo = 32 * w;
        uint32_t real;
        if (n >= lo + 32) real = 0xFFFFFFFFu;
        else if (n <= lo) real = 0u;
        else real = (1u << (n - lo)) - 1u;
        st.m[w] = ~real;
        st.s[w] = 0u;
    }
    return st;
}

template <int W>
__device__ __forceinline__ void add_row(State<W>& st, const RowTable<W>& tab, int dir, int r)
{
    const RowEntry<W>& e = tab.e[dir][r];
    uint32_t k1[W], k2[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        k1[w] = e.k1[w];
        k2[w] = e.k2[w];
    }
    add_masks<W>(st, k1, k2);
}

// state for Gray index i: the subset sum of the rows in gray(i), from scratch
// (Sec. 3.1: each block of consecutive Gray states starts from a direct jump)
template <int W>
__device__ __forceinline__ State<W> seed_state(const RowTable<W>& tab, int n, uint64_t i)
{
    State<W> st = initial_state<W>(n);
    uint64_t g = i ^ (i >> 1);
    while (g) {
        const int r = __ffsll((long long)g) - 1;
        add_row<W>(st, tab, 0, r);
        g &= g - 1;
    }
    return st;
}

// the low word (columns 0..31) of seed_state: all the grouped walk carries
template <int W>
__device__ __forceinline__ void seed_low(const RowTable<W>& tab, int n, uint64_t i, uint32_t& m, uint32_t& sg)
{
    const State<W> init = initial_state<W>(n);
    m = init.m[0];
    sg = init.s[0];
    uint64_t g = i ^ (i >> 1);
    while (g) {
        const int r = __ffsll((long long)g) - 1;
        const RowEntry<W>& e = tab.e[0][r];
        add_word(m, sg, e.k1[0], e.k2[0]);
        g &= g - 1;
    }
}

template <int W>
__device__ __forceinline__ bool all_ones(const State<W>& st)
{
    bool ok = true;
#pragma unroll
    for (int w = 0; w < W; ++w) ok = ok && (st.m[w] == 0xFFFFFFFFu);
    return ok;
}

// sign of a nonzero product times (-1)^{|S|}: 0 -> +1, 1 -> -1
template <int W>
__device__ __forceinline__ uint32_t term_parity(const State<W>& st, uint64_t i)
{
    uint32_t c = (uint32_t)i;
#pragma unroll
    for (int w = 0; w < W; ++w) c += __popc(st.s[w]);
    return c & 1u;
}

struct Counts {
    unsigned long long plus;
    unsigned long long minus;
};

// Generic walk of Gray indices [first, last] (inclusive), every step looked up
// in the row table.  Used for small n, ragged range ends and rare-path replays.
template <int W>
__device__ __noinline__ void walk_generic(const RowTable<W>& tab, int n, uint64_t first, uint64_t last,
                                          Counts& c)
{
    State<W> st = seed_state<W>(tab, n, first);
    uint64_t i = first;
    for (;;) {
        if (all_ones<W>(st)) {
            if (term_parity<W>(st, i)) ++c.minus;
            else ++c.plus;
        }
        if (i == last) break;
        ++i;
        const int t = __ffsll((long long)i) - 1;
        const int dir = (int)((i >> (t + 1)) & 1u);
        add_row<W>(st, tab, dir, t);
    }
}

// ---------------------------------------------------------------------------
// Grouped walk.  The Gray indices are cut into groups of 2^G consecutive
// indices (group k = indices k*2^G .. k*2^G + 2^G - 1).  Only one state per
// group (the "base") is carried in full (all W words of mag and sgn); the
// other 2^G - 1 states of the group are evaluated as "probes" that compute
// only the low mag word (two LOP3) for the zero test of Sec. 3.  A probe whose
// low 32 columns are all nonzero marks the group; marked groups are replayed
// exactly (all words, sign from the popcount of sgn) from the saved base.
//
// Index facts used (reflected binary code, gray(i) = i ^ (i >> 1)):
//  * inside group k the bits >= G of gray(i) are gray(k), and the low G bits
//    are gray(j) ^ ((k & 1) << (G-1)) for i = k*2^G + j;
//  * so the base of an even group is its first state (j = 0) and the base of
//    an odd group its last state (j = 2^G - 1): in both cases the base's low G
//    bits are 0, and the group's 2^G states are exactly base + (sum of the
//    rows in s) for the 2^G subsets s of rows 0..G-1, all ADDED;
//  * consecutive bases differ in one row only: row t = G + tz(k+1), the flip
//    at index (k+1)*2^G, subtracted iff bit t+1 of that index is set.
// Groups are unrolled 2^(U-G) at a time ("block" of 2^U indices); inside a
// block every row, sign and mask is a compile-time choice except the flip of
// row U-1 in the middle of the block (sign = parity of the block index) and
// the flip into the next block (row U + tz(B+1), from the row table).
// ---------------------------------------------------------------------------

__host__ __device__ constexpr int ctz_const(int x)
{
    return (x & 1) ? 0 : 1 + ctz_const(x >> 1);
}

// masks (K1 = [c == 0], K2 = [c == 1]) of the per-column constant
// c = sum of the rows in `rows`
template <int W>
__device__ __forceinline__ void subset_masks(const RowTable<W>& tab, uint64_t rows, uint32_t (&k1)[W],
                                             uint32_t (&k2)[W])
{
    State<W> c;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        c.m[w] = 0u;
        c.s[w] = 0u;
    }
    while (rows) {
        add_row<W>(c, tab, 0, __ffsll((long long)rows) - 1);
        rows &= rows - 1;
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        k1[w] = ~c.m[w];
        k2[w] = c.m[w] & ~c.s[w];
    }
}

// Per-thread registers of the grouped walk.  The walk itself only needs the
// LOW word of every state (the zero test looks at columns 0..31; columns are
// independent, so the low word evolves on its own): probe masks for the
// 2^G - 1 nonzero subsets s of rows 0..G-1 (slot s - 1) and the masks of rows
// G..U-1 for the in-block base steps, all low word only.  Marked groups are
// replayed exactly with every word.
template <int G, int U>
struct GroupRows {
    static constexpr int kProbes = (1 << G) - 1;
    static constexpr int kRows = U - G;
    uint32_t pk1[kProbes];
    uint32_t pk2[kProbes];
    uint32_t rk1[kRows];
    uint32_t rk2p[kRows];
    uint32_t rk2m[kRows];
};

template <int W, int G, int U>
__device__ __forceinline__ void load_group_rows(GroupRows<G, U>& R, const RowTable<W>& tab)
{
#pragma unroll
    for (int sub = 1; sub < (1 << G); ++sub) {
        uint32_t k1[W], k2[W];
        subset_masks<W>(tab, (uint64_t)sub, k1, k2);
        R.pk1[sub - 1] = k1[0];
        R.pk2[sub - 1] = k2[0];
    }
#pragma unroll
    for (int t = G; t < U; ++t) {
        R.rk1[t - G] = tab.e[0][t].k1[0];
        R.rk2p[t - G] = tab.e[0][t].k2[0];
        R.rk2m[t - G] = tab.e[1][t].k2[0];
    }
}

// Exact terms of group k (indices i0 .. i0 + 2^G - 1, i0 = k * 2^G): its first
// state is re-seeded from scratch (all words), then the group is walked.
template <int W, int G>
__device__ __noinline__ void replay_group(const RowTable<W>& tab, int n, uint64_t i0, Counts& c)
{
    State<W> st = seed_state<W>(tab, n, i0);
    for (uint32_t j = 0; j < (1u << G); ++j) {
        const uint64_t i = i0 + j;
        if (j) {
            const int t = __ffs((int)j) - 1;
            const int dir = (int)((i >> (t + 1)) & 1u);
            add_row<W>(st, tab, dir, t);
        }
        if (all_ones<W>(st)) {
            if (term_parity<W>(st, i)) ++c.minus;
            else ++c.plus;
        }
    }
}

// Per-warp queue of marked groups awaiting exact replay (shared memory).
// Lanes push as they find marks; the whole warp drains the queue together,
// one group per lane, so a rare replay does not stall 31 idle lanes.
constexpr int kQueueCap = 64;
// Queued marks at a block's end at which a warp leaves the low-word walk for
// the dense walk: at least 129 of the block's 32 x 2^(U-G) groups marked
// (a quarter for U - G = 4), where replaying them one by one costs more.
constexpr unsigned kDenseSwitch = 160;
// Groups the dense walk evaluates side by side (a divisor of every variant's
// 2^(U-G) groups per block).
constexpr int kDenseH = 4;

// A warp's queue slot.  Once a warp switches to the dense walk its queue is
// empty, so the same bytes hold the dense walk's subset masks: for each
// nonzero subset s of rows 0..G-1, (K1, K2) of word 0 and (K1, K2) of word 1
// of the constant sum_{r in s} row_r.
template <int G>
struct WarpQueue {
    union {
        unsigned long long i0[kQueueCap];
        uint4 dk[(1 << G) - 1];
    };
    unsigned count;
    unsigned pad;
};

template <int W, int G>
__device__ __noinline__ void queue_push(WarpQueue<G>& q, const RowTable<W>& tab, int n, uint64_t i0, Counts* c)
{
    const unsigned slot = atomicAdd(&q.count, 1u);
    if (slot < (unsigned)kQueueCap) q.i0[slot] = i0;
    else replay_group<W, G>(tab, n, i0, *c);  // queue full: replay in place
}

// all 32 lanes: replay the queued groups and empty the queue (out of line:
// it is rare, and kept inline it took instruction-cache room from the walk)
template <int W, int G>
__device__ __noinline__ void queue_drain(WarpQueue<G>& q, const RowTable<W>& tab, int n, int lane, Counts& c)
{
    __syncwarp();
    const unsigned cnt = *(volatile unsigned*)&q.count;
    if (cnt == 0) return;
    const unsigned lim = cnt < (unsigned)kQueueCap ? cnt : (unsigned)kQueueCap;
    for (unsigned e = lane; e < lim; e += 32) replay_group<W, G>(tab, n, q.i0[e], c);
    __syncwarp();
    if (lane == 0) q.count = 0;
    __syncwarp();
}

// all 32 lanes: the dense walk's subset masks into the warp's queue slot, in
// Gray order of the subsets
template <int W, int G>
__device__ __noinline__ void build_dense_masks(WarpQueue<G>& q, const RowTable<W>& tab, int lane)
{
    // entry t - 1 holds subset gray(t) = t ^ (t >> 1), t = 1 .. 2^G - 1: in
    // this order |s| is odd exactly for odd t
    for (int j = lane; j < (1 << G) - 1; j += 32) {
        uint32_t k1[W], k2[W];
        const uint32_t t = (uint32_t)j + 1u;
        subset_masks<W>(tab, (uint64_t)(t ^ (t >> 1)), k1, k2);
        q.dk[j] = make_uint4(k1[0], k2[0], W > 1 ? k1[W - 1] : 0u, W > 1 ? k2[W - 1] : 0u);
    }
    __syncwarp();
}

// Integer multiply-add, d = a * b + c (low or high 32 bits of the product).
// On this GPU it issues to the multiply-add pipe, not to the ALU pipe that
// the bitwise gates saturate; a multiplier the compiler cannot see as a
// constant keeps it there (a literal 1 would be turned into an ALU add).
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// The dense walk's states "base h + the rows of one subset s" for the H bases
// of a batch, given the subset's masks k (K1, K2 of word 0 and of the last
// word); ODD = |s| is odd (it flips the sign).  See walk_dense.
template <int W, int H, bool ODD>
__device__ __forceinline__ void dense_states(const State<W> (&b)[H], const uint32_t (&be)[H], const uint4 k,
                                             uint32_t one, uint32_t half, uint32_t& cnt, uint32_t& sum_p,
                                             uint32_t& sum_h)
{
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const uint32_t g0 = lop3<kLutG>(b[h].s[0], k.x, k.y);
        uint32_t z = lop3<kLutMagInv>(b[h].m[0], k.x, g0);
        const uint32_t bsub = ODD ? (be[h] ^ 1u) : be[h];
        uint32_t x;
        if (W > 1) {
            const uint32_t g1 = lop3<kLutG>(b[h].s[W - 1], k.z, k.w);
            z |= lop3<kLutMagInv>(b[h].m[W - 1], k.z, g1);
            x = lop3<0x96>(bsub, g0, g1);  // a ^ b ^ c
        } else {
            x = bsub ^ g0;
        }
        const uint32_t p = __popc(x);
        if (z == 0u) {
            cnt = mad_lo(one, one, cnt);
            sum_p = mad_lo(p, one, sum_p);
            sum_h = mad_hi(p, half, sum_h);
        }
    }
}

// 16-byte shared-memory load that the compiler may not move out of a loop:
// the dense walk reads its 2^G - 1 subset masks from shared memory once per
// group, and hoisted into registers they would not fit.
__device__ __forceinline__ uint4 lds128(const uint4* p)
{
    uint4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// Exact walk of Gray blocks [B0, B0 + len) for matrices whose terms are often
// nonzero (the low-word test would mark most groups, and replaying them one
// by one costs far more): group K's 2^G states are its base state plus each
// subset s of rows 0..G-1, every one evaluated in full (all words) from the
// base and the subset masks, with the exact sign.  The base of an even group
// is its first index and of an odd group its last, so |S| is even exactly
// for even K, and consecutive bases differ in row G + tz(K+1), subtracted
// iff bit tz(K+1)+1 of K+1 is set (the Gray flip at index (K+1)·2^G).
//
// Per state the walk computes, for each word, the gate g and the inverted
// mag word (two LOP3) and tests every column nonzero (one LOP3 writing a
// predicate).  The sign needs no sgn word: the new sgn is ~(mag ^ sgn ^ g)
// per word, so the XOR of the new sgn words equals (mag0 ^ sgn0 ^ mag1 ^
// sgn1) ^ g0 ^ g1 -- a base constant and the two gates, one LOP3 -- and the
// parity of its popcount is the parity of the number of -1 entries (Sec. 3's
// poppar).  The (-1)^{|S|} factor, kpar + |s|, is folded into the base
// constant by flipping its bit 0; the subsets are visited in Gray order, so
// |s| alternates between odd and even from one to the next.  The +1 / -1 tallies are kept on the
// multiply-add pipe: with p the popcount, sum(p) - 2 sum(p >> 1) counts the
// odd ones, and mad.hi(p, 2^31) is p >> 1; 32-bit tallies are moved into the
// 64-bit counts every 16 batches of kDenseH groups.
template <int W, int G, int U>
__device__ __noinline__ void walk_dense(const RowTable<W>& tab, const uint4* dk, int n, uint64_t B0, uint64_t len,
                                        Counts* c)
{
    // groups are taken kDenseH at a time: each subset mask is read once and
    // applied to kDenseH bases held in registers, which gives the schedulers
    // kDenseH independent chains (the popcount and the shared-memory load
    // have long latencies) per mask
    constexpr int H = kDenseH;
    static_assert(((1 << (U - G)) % H) == 0, "a block holds a whole number of group batches");
    if (!len) return;
    const uint32_t one = (uint32_t)(n > 0);  // 1 at run time, opaque to the compiler
    const uint32_t half = one << 31;
    State<W> cur = seed_state<W>(tab, n, B0 << U);
    uint64_t K = B0 << (U - G);
    const uint64_t K_end = (B0 + len) << (U - G);  // K_end - K is a multiple of H
    unsigned long long plus = 0, minus = 0;
    uint32_t cnt = 0, sum_p = 0, sum_h = 0;  // nonzero states, sum of p, sum of p >> 1
    uint32_t batches = 0;
    for (;;) {
        State<W> b[H];
        uint32_t be[H];
        b[0] = cur;
#pragma unroll
        for (int h = 1; h < H; ++h) {
            b[h] = b[h - 1];
            const uint64_t Kh = K + (uint64_t)h;
            const int zt = __ffsll((long long)Kh) - 1;
            add_row<W>(b[h], tab, (int)((Kh >> (zt + 1)) & 1u), G + zt);
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const uint32_t kpar = (uint32_t)(K + (uint64_t)h) & 1u;
            uint32_t bw = b[h].m[0] ^ b[h].s[0];
            uint32_t zb = ~b[h].m[0];
            uint32_t xb = b[h].s[0] ^ kpar;
            if (W > 1) {
                bw ^= b[h].m[W - 1] ^ b[h].s[W - 1];
                zb |= ~b[h].m[W - 1];
                xb ^= b[h].s[W - 1];
            }
            be[h] = bw ^ kpar;
            // the base state itself (s = {})
            const uint32_t p = __popc(xb);
            if (zb == 0u) {
                cnt = mad_lo(one, one, cnt);
                sum_p = mad_lo(p, one, sum_p);
                sum_h = mad_hi(p, half, sum_h);
            }
        }
        // the masks are in Gray order of the subsets (build_dense_masks), so
        // |s| is odd at odd t: a loop over pairs (t, t + 1) keeps each
        // sign a compile-time choice with a short loop body
#pragma unroll 1
        for (int t = 1; t + 1 < (1 << G); t += 2) {
            dense_states<W, H, true>(b, be, lds128(dk + (t - 1)), one, half, cnt, sum_p, sum_h);
            dense_states<W, H, false>(b, be, lds128(dk + t), one, half, cnt, sum_p, sum_h);
        }
        dense_states<W, H, true>(b, be, lds128(dk + ((1 << G) - 2)), one, half, cnt, sum_p, sum_h);
        K += H;
        // at most 16 batches x H x 2^G states x 33 in sum_p between flushes
        if (++batches == 16 || K == K_end) {
            const uint32_t odd = sum_p - 2u * sum_h;
            minus += odd;
            plus += cnt - odd;
            cnt = sum_p = sum_h = 0;
            batches = 0;
        }
        if (K == K_end) break;
        cur = b[H - 1];
        const int zt = __ffsll((long long)K) - 1;
        add_row<W>(cur, tab, (int)((K >> (zt + 1)) & 1u), G + zt);
    }
    c->plus += plus;
    c->minus += minus;
}

template <int W, int G, int U, int GI>
struct GroupSteps {
    static __device__ __forceinline__ void run(uint32_t& m, uint32_t& sg, const GroupRows<G, U>& R, uint32_t kmid2,
                                               uint64_t ibase, WarpQueue<G>& q, const RowTable<W>& tab, int n,
                                               Counts& c)
    {
        GroupSteps<W, G, U, GI - 1>::run(m, sg, R, kmid2, ibase, q, tab, n, c);
        constexpr int g = GI - 1;  // group inside the block
        bool hit = (m == 0xFFFFFFFFu);
#pragma unroll
        for (int sub = 1; sub < (1 << G); ++sub) {
            // the probe's mag word is produced inverted and tested against
            // zero: on GB300 this form issues fewer ALU instructions than a
            // test of the plain word against all ones (measured)
            const uint32_t gq = lop3<kLutG>(sg, R.pk1[sub - 1], R.pk2[sub - 1]);
            const uint32_t nmq = lop3<kLutMagInv>(m, R.pk1[sub - 1], gq);
            hit |= (nmq == 0u);
        }
        if (hit) queue_push<W, G>(q, tab, n, ibase + ((uint64_t)g << G), &c);
        if (g + 1 < (1 << (U - G))) {
            constexpr int t = G + ctz_const(g + 1);
            constexpr int dir = ((g + 1) >> (t + 1 - G)) & 1;
            const uint32_t k2 = (t == U - 1) ? kmid2 : (dir ? R.rk2m[t - G] : R.rk2p[t - G]);
            add_word(m, sg, R.rk1[t - G], k2);
        }
    }
};

template <int W, int G, int U>
struct GroupSteps<W, G, U, 0> {
    static __device__ __forceinline__ void run(uint32_t&, uint32_t&, const GroupRows<G, U>&, uint32_t, uint64_t,
                                               WarpQueue<G>&, const RowTable<W>&, int, Counts&)
    {
    }
};

// Walk blocks [B0, B0 + len) of 2^U indices.  `trip` (>= len) must be the
// same in all 32 lanes of the warp: lanes with len < trip idle through the
// extra iterations so that the warp drains its queue together.  Returns the
// number of blocks walked; when it is below len the warp has switched to the
// dense walk (its masks are in q.dk) and the caller walks the rest with
// walk_dense.
template <int W, int G, int U>
__device__ __forceinline__ uint64_t walk_groups(const RowTable<W>& tab, const GroupRows<G, U>& R, int n,
                                                uint64_t B0, uint64_t len, uint64_t trip, WarpQueue<G>& q, int lane,
                                                Counts& c)
{
    uint32_t m = 0, sg = 0;  // low word of the base state
    if (len) seed_low<W>(tab, n, B0 << U, m, sg);
    for (uint64_t it = 0; it < trip; ++it) {
        if (it < len) {
            const uint64_t B = B0 + it;
            // row U-1 flips mid-block: subtracted in odd blocks
            const uint32_t kmid2 = (B & 1u) ? R.rk2m[U - 1 - G] : R.rk2p[U - 1 - G];
            GroupSteps<W, G, U, (1 << (U - G))>::run(m, sg, R, kmid2, B << U, q, tab, n, c);
            if (it + 1 < len) {
                // the flip into block B+1 (the block's last group is odd, its
                // base already sits at the block's last index)
                const uint64_t nb = B + 1;
                const int z = __ffsll((long long)nb) - 1;
                const RowEntry<W>& e = tab.e[(int)((nb >> (z + 1)) & 1u)][U + z];
                add_word(m, sg, e.k1[0], e.k2[0]);
            }
        }
        __syncwarp();
        const unsigned cnt = *(volatile unsigned*)&q.count;
        if (__builtin_expect(cnt >= 32u, 0)) {
            // the queue is drained whenever it holds 32 at a block's end, so
            // a count of kDenseSwitch means that this block alone marked at
            // least kDenseSwitch - 31 groups: finish the walked groups
            // exactly, then walk the rest densely
            queue_drain<W, G>(q, tab, n, lane, c);
            if (cnt >= kDenseSwitch) {
                build_dense_masks<W, G>(q, tab, lane);
                return it + 1 < len ? it + 1 : len;
            }
        }
    }
    queue_drain<W, G>(q, tab, n, lane, c);
    return len;
}

// balanced split of `total` items over `parts`: part k gets [start, start+len)
__device__ __forceinline__ void split_range(uint64_t total, uint64_t parts, uint64_t k, uint64_t& start,
                                            uint64_t& len)
{
    const uint64_t q = total / parts, r = total % parts;
    start = k * q + (k < r ? k : r);
    len = q + (k < r ? 1 : 0);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

}  // namespace pf3

namespace pf3 {

// Pack row r of the rows x cols matrix A (row-major, entries {0,1,2}, 2 == -1)
// into bit planes with one warp: lane l reads column l (and 32 + l).
// Implements phi of Sec. 2 column by column.  `bad` is set in the lanes that
// saw an entry above 2.
__device__ __forceinline__ void pack_row_warp(const uint8_t* A, int rows, int cols, int r, int lane,
                                              uint32_t (&mag)[2], uint32_t (&sgn)[2], bool& bad)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int col = 32 * h + lane;
        uint32_t a = 0;
        if (r < rows && col < cols) a = A[(size_t)r * cols + col];
        bad |= (a > 2u);
        mag[h] = __ballot_sync(0xFFFFFFFFu, a == 1u || a == 2u);
        sgn[h] = __ballot_sync(0xFFFFFFFFu, a == 2u);
    }
}

// Build the row table of the rows x cols matrix A with the warps
// [warp0, warp0 + nwarps) of the calling group; every row r >= rows is the
// identity (adds 0).
template <int W>
__device__ __forceinline__ bool build_row_table(RowTable<W>& tab, const uint8_t* A, int rows, int cols, int warp,
                                                int nwarps, int lane)
{
    bool bad = false;
    for (int r = warp; r < kMaxN; r += nwarps) {
        uint32_t mag[2], sgn[2];
        pack_row_warp(A, rows, cols, r, lane, mag, sgn, bad);
        if (lane < W) {
            uint32_t k1, k2p, k2m;
            row_masks(mag[lane], sgn[lane], k1, k2p, k2m);
            tab.e[0][r].k1[lane] = k1;
            tab.e[0][r].k2[lane] = k2p;
            tab.e[1][r].k1[lane] = k1;
            tab.e[1][r].k2[lane] = k2m;
        }
    }
    return bad;
}

}  // namespace pf3
