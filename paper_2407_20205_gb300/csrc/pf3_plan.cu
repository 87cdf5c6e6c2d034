// pf3_plan.cu -- the single-matrix launch plan on the host alone: how a Gray
// range is cut into a ragged head, aligned blocks of 2^U indices and a ragged
// tail (Sec. 3.1's blocks of consecutive Gray states), and how the blocks are
// handed to warps.  Diagnostic only; no device is touched.  The plan comes
// from the same host functions a launch uses (plan_range, plan_chunks), and
// each chunk from the same chunk_range the kernel calls.
#include <cstring>

#include "perm_f3.h"
#include "pf3_internal.h"

using namespace pf3;

extern "C" int pf3_range_plan(int n, uint64_t first, uint64_t last, int variant, int grid, uint64_t* info,
                              uint64_t* chunk_first, uint64_t* chunk_len, int64_t capacity, int64_t* num_chunks)
{
    if (n < 1 || n > PF3_MAX_N || first > last || (n < 64 && last >= (1ull << n))) return PF3_EINVAL;
    if (variant < 0 || variant >= kNumSingleVariants || grid < 1 || !info || !num_chunks || capacity < 0)
        return PF3_EINVAL;
    SingleArgs a;
    std::memset(&a, 0, sizeof(a));
    plan_range(n, first, last, kSingleVariants[variant].U, a);
    plan_chunks(a, grid, kSingleVariants[variant].threads);
    const uint64_t vals[12] = {(uint64_t)a.has_head, a.head_first, a.head_last, (uint64_t)a.has_tail,
                               a.tail_first, a.tail_last, a.mid_B0, a.mid_NB, (uint64_t)a.dynamic,
                               (uint64_t)kSingleVariants[variant].U, (uint64_t)kSingleVariants[variant].threads,
                               (uint64_t)a.nchunks};
    std::memcpy(info, vals, sizeof(vals));
    const int64_t count = a.dynamic ? (int64_t)a.nchunks : 0;
    *num_chunks = count;
    if (!chunk_first || !chunk_len) return PF3_OK;
    if (capacity < count) return PF3_ETOOBIG;
    for (int64_t k = 0; k < count; ++k) chunk_range(a, (unsigned)k, chunk_first[k], chunk_len[k]);
    return PF3_OK;
}
