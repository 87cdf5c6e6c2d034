// pf3_plan.cu -- the single-matrix launch plan on the host alone: how a Gray
// range is cut into a ragged head, aligned blocks of 2^U indices and a ragged
// tail (Sec. 3.1's blocks of consecutive Gray states), and how the blocks are
// handed to warps.  Diagnostic only; no device is touched.  The plan comes
// from the same host functions a launch uses (plan_range, plan_chunks); the
// chunk enumeration below restates the kernel's chunk mapping.
#include <cstring>

#include "perm_f3.h"
#include "pf3_internal.h"

using namespace pf3;

namespace {

// chunk k < nchunks of the middle blocks, relative to mid_B0: guided phases of
// per_phase chunks of len0 >> j blocks (rounded down to 32) while that is at
// least tail_len, then chunks of tail_len blocks up to mid_NB
void host_chunk(const SingleArgs& a, unsigned k, uint64_t& start, uint64_t& len)
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

}  // namespace

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
    for (int64_t k = 0; k < count; ++k) host_chunk(a, (unsigned)k, chunk_first[k], chunk_len[k]);
    return PF3_OK;
}
