// pf3_internal.h -- host-side declarations shared by the library's translation
// units (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace pf3 {

// The final map of Eq. (2): perm(A) = (-1)^n (plus - minus) mod 3, in
// {0,1,2}, from the exact counts of +1 and -1 terms (the closing cmod3 of
// Sec. 3).  Each count is reduced mod 3 on its own, so no signed difference
// of two 64-bit counts is ever formed (both may exceed 2^63 at n = 64).  One
// definition for the kernels' epilogues and the host entry point
// pf3_perm_from_counts.
__host__ __device__ inline uint32_t perm_from_counts(int n, unsigned long long plus, unsigned long long minus)
{
    int d = (int)(plus % 3ull) - (int)(minus % 3ull);
    if (n & 1) d = -d;
    return (uint32_t)((d + 3) % 3);
}

// A compiled variant of a walk kernel: probe groups of 2^G Gray indices,
// unrolled blocks of 2^U indices, the minimum resident CTAs per SM it was
// compiled for (its register budget) and its CTA size.
struct KernelVariant {
    int U;
    int G;
    int min_ctas;
    int threads;
};
constexpr int kMaxVariants = 16;
// Single-matrix launches of fewer Gray indices than this form their own size
// class for variant selection (their fixed costs decide, not the walk's rate).
constexpr uint64_t kShortLaunch = 1ull << 28;
constexpr int kNumSingleVariants = 9;
constexpr KernelVariant kSingleVariants[kNumSingleVariants] = {
    {9, 5, 2, 256}, {9, 4, 2, 256}, {8, 4, 2, 256}, {10, 5, 2, 256}, {8, 5, 2, 256},
    {9, 5, 3, 256}, {9, 5, 1, 256}, {9, 5, 4, 128}, {9, 6, 1, 384}};
constexpr int kNumBatchVariants = 6;
constexpr KernelVariant kBatchVariants[kNumBatchVariants] = {{9, 5, 4, 128}, {9, 4, 4, 128}, {8, 4, 4, 128},
                                                             {9, 5, 2, 128}, {10, 5, 2, 128}, {8, 5, 4, 128}};
static_assert(kNumSingleVariants <= kMaxVariants && kNumBatchVariants <= kMaxVariants, "variant tables");

// One range job for the single-matrix kernel; all indices are Gray indices.
struct SingleArgs {
    const uint8_t* A;        // device, n rows x m columns, row-major {0,1,2}
    int n;                   // rows: the Gray range is [0, 2^n) and the sign (-1)^n
    int m;                   // columns (n unless the host merged equal columns)
    int has_head;            // generic walk of [head_first, head_last]
    int has_tail;            // generic walk of [tail_first, tail_last]
    uint64_t head_first, head_last;
    uint64_t tail_first, tail_last;
    uint64_t mid_B0;         // aligned blocks [mid_B0, mid_B0 + mid_NB)
    uint64_t mid_NB;
    // The middle blocks are handed to warps in chunks through an atomic
    // cursor, in guided phases: phase j is per_phase chunks of len0 >> j
    // blocks (while that is at least tail_len), then chunks of tail_len
    // blocks cover the rest up to mid_NB; nchunks in all.  Each phase takes
    // about half of what is left, so warps that run ahead take more and all
    // finish together.  Set by launch_single from the grid size.
    // With dynamic == 0 each thread walks one contiguous share of the middle
    // blocks instead and the cursor is not used.
    uint64_t len0, tail_len;
    unsigned per_phase, nchunks;
    int dynamic;
    unsigned long long* partials;  // device scratch, 2 per CTA
    unsigned int* ticket;          // device scratch, 0 between launches
    unsigned int* err;             // device scratch, 0 between launches
    unsigned int* cursor;          // device scratch, 0 between launches
    unsigned long long* out;       // device: plus, minus, result (~0 on bad entry)
};

// Chunk k < nchunks of the middle blocks, relative to mid_B0 (Sec. 3.1's
// blocks of consecutive Gray states, handed to warps in guided phases): phase
// j is per_phase chunks of len0 >> j blocks (rounded down to a multiple of 32)
// while that is at least tail_len, then chunks of tail_len blocks up to
// mid_NB.  One definition for the kernel, which calls it for the chunk index
// it took from the cursor, and for the host planner that lists the chunks; at
// most one turn of the loop per guided phase (the length halves each turn).
__host__ __device__ inline void chunk_range(const SingleArgs& a, unsigned k, uint64_t& start, uint64_t& len)
{
    uint64_t s = 0, L = a.len0;
    while (L >= a.tail_len) {
        if (k < a.per_phase) {
            start = s + (uint64_t)k * L;
            const uint64_t left = a.mid_NB - start;
            len = left < L ? left : L;
            return;
        }
        s += (uint64_t)a.per_phase * L;
        k -= a.per_phase;
        L = (L >> 1) & ~31ull;
    }
    start = s + (uint64_t)k * a.tail_len;
    const uint64_t left = a.mid_NB - start;
    len = left < a.tail_len ? left : a.tail_len;
}

// split [first, last] into a ragged head, aligned middle blocks of 2^U
// indices and a ragged tail (sets a.n = a.m = n)
void plan_range(int n, uint64_t first, uint64_t last, int U, SingleArgs& a);

// split the middle blocks into the chunks warps take from the cursor, for
// `grid` CTAs of `threads` threads
void plan_chunks(SingleArgs& a, int grid, int threads);

// launch variant `v` of the single-matrix walk (W = 1 for m <= 32 columns, else 2);
// plans the chunks for `grid` CTAs
cudaError_t launch_single(const SingleArgs& a, int v, int grid, cudaStream_t stream);

// CTAs of variant v to launch for this plan given the device (one resident
// wave at most)
int single_grid_for(const SingleArgs& a, int v, int sm_count, int max_ctas_per_sm);

// resident CTAs per SM of variant v of the single-matrix kernel for W
int single_max_ctas_per_sm(int W, int v);

// device debug helpers
cudaError_t launch_step_table(uint32_t* out, cudaStream_t stream);
cudaError_t launch_pack(const uint8_t* A, int n, unsigned long long* out_mag, unsigned long long* out_sgn,
                        unsigned int* err, cudaStream_t stream);

// integer pipe microbenchmark
cudaError_t launch_intpipe(int kind, int grid, int threads, int iters, uint32_t* sink,
                           unsigned long long* cycles, cudaStream_t stream);

}  // namespace pf3
