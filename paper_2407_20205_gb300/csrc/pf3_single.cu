// pf3_single.cu -- one matrix, one launch: the Gray-code Ryser sum of Eq. (2)
// over a range of Gray indices, split across every thread of the grid.
//
// Sec. 3.1 of the paper splits the 2^n Gray states into blocks of consecutive
// states, each started by jumping to gray(start).  Here a block is 2^U
// consecutive indices (U picked by the autotuner); thread k of the grid walks a
// contiguous run of blocks, seeded once by a direct subset sum.  Each CTA
// packs the matrix into a shared-memory row table itself (no separate pack
// launch), the per-thread (+1, -1) term counts are reduced by warp shuffles
// and shared memory, and the last CTA to finish adds the per-CTA partials and
// maps the counts to perm mod 3.
#include <cuda_runtime.h>

#include "pf3_device.cuh"
#include "pf3_internal.h"

namespace pf3 {

namespace {

template <int W, int U, int G, int MINB>
__global__ void __launch_bounds__(kSingleThreads, MINB) single_kernel(SingleArgs a)
{
    __shared__ RowTable<W> tab;
    __shared__ WarpQueue queues[kSingleThreads / 32];
    __shared__ unsigned long long red[2][kSingleThreads / 32];
    __shared__ bool s_last;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (lane == 0) queues[warp].count = 0;
    const bool bad_local = build_row_table<W>(tab, a.A, a.n, warp, kSingleThreads / 32, lane);
    const bool bad = __syncthreads_or(bad_local) != 0;

    Counts c{0ull, 0ull};
    if (!bad) {
        const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
        const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (a.mid_NB) {
            GroupRows<G, U> R;
            load_group_rows<W, G, U>(R, tab);
            uint64_t s, len;
            split_range(a.mid_NB, T, tid, s, len);
            const uint64_t trip = __shfl_sync(0xFFFFFFFFu, len, 0);  // lane 0 holds the longest share
            walk_groups<W, G, U>(tab, R, a.n, a.mid_B0 + s, len, trip, queues[warp], lane, c);
        }
        if (a.has_head && tid == T - 1) walk_generic<W>(tab, a.n, a.head_first, a.head_last, c);
        if (a.has_tail && tid == (T > 1 ? T - 2 : 0)) walk_generic<W>(tab, a.n, a.tail_first, a.tail_last, c);
    }

    unsigned long long p = warp_sum(c.plus);
    unsigned long long m = warp_sum(c.minus);
    if (lane == 0) {
        red[0][warp] = p;
        red[1][warp] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p = 0;
        m = 0;
        for (int w = 0; w < kSingleThreads / 32; ++w) {
            p += red[0][w];
            m += red[1][w];
        }
        a.partials[2 * blockIdx.x] = p;
        a.partials[2 * blockIdx.x + 1] = m;
        if (bad) atomicOr(a.err, 1u);
        __threadfence();
        const unsigned t = atomicAdd(a.ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;

    // last CTA: sum the partials of every CTA
    __threadfence();
    p = 0;
    m = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        p += __ldcg(&a.partials[2 * b]);
        m += __ldcg(&a.partials[2 * b + 1]);
    }
    p = warp_sum(p);
    m = warp_sum(m);
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = p;
        red[1][warp] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p = 0;
        m = 0;
        for (int w = 0; w < kSingleThreads / 32; ++w) {
            p += red[0][w];
            m += red[1][w];
        }
        const unsigned e = atomicExch(a.err, 0u);
        a.out[0] = p;
        a.out[1] = m;
        a.out[2] = e ? ~0ull : (unsigned long long)perm_from_counts(a.n, p, m);
        *a.ticket = 0u;
        __threadfence();
    }
}

// every combination of a 2-bit state (mag, sgn), a constant c in {0,1,2} and
// a direction, through the same mask and step code as the walk:
// out[((state * 3 + c) * 2 + dir) * 2 + {0,1}] = (mag', sgn')
__global__ void step_table_kernel(uint32_t* out)
{
    const int idx = threadIdx.x;  // 0..23
    if (idx >= 24) return;
    const int dir = idx & 1;
    const int c = (idx >> 1) % 3;
    const int state = (idx >> 1) / 3;
    uint32_t m = (uint32_t)(state >> 1) & 1u, s = (uint32_t)state & 1u;
    // all 32 columns hold the same case; the row word encodes c by phi
    const uint32_t rmag = (c != 0) ? 0xFFFFFFFFu : 0u;
    const uint32_t rsgn = (c == 2) ? 0xFFFFFFFFu : 0u;
    uint32_t k1, k2p, k2m;
    row_masks(rmag, rsgn, k1, k2p, k2m);
    uint32_t mw = m ? 0xFFFFFFFFu : 0u, sw = s ? 0xFFFFFFFFu : 0u;
    add_word(mw, sw, k1, dir ? k2m : k2p);
    out[2 * idx] = mw & 1u;
    out[2 * idx + 1] = sw & 1u;
}

__global__ void pack_kernel(const uint8_t* A, int n, unsigned long long* out_mag, unsigned long long* out_sgn,
                            unsigned int* err)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    bool bad = false;
    for (int r = warp; r < n; r += blockDim.x / 32) {
        uint32_t mag[2], sgn[2];
        pack_row_warp(A, n, r, lane, mag, sgn, bad);
        if (lane == 0) {
            out_mag[r] = ((unsigned long long)mag[1] << 32) | mag[0];
            out_sgn[r] = ((unsigned long long)sgn[1] << 32) | sgn[0];
        }
    }
    if (bad) atomicOr(err, 1u);
}

template <int W>
const void* single_kernel_ptr(int v)
{
    switch (v) {
    case 0: return (const void*)single_kernel<W, kSingleVariants[0].U, kSingleVariants[0].G, kSingleVariants[0].min_ctas>;
    case 1: return (const void*)single_kernel<W, kSingleVariants[1].U, kSingleVariants[1].G, kSingleVariants[1].min_ctas>;
    case 2: return (const void*)single_kernel<W, kSingleVariants[2].U, kSingleVariants[2].G, kSingleVariants[2].min_ctas>;
    case 3: return (const void*)single_kernel<W, kSingleVariants[3].U, kSingleVariants[3].G, kSingleVariants[3].min_ctas>;
    case 4: return (const void*)single_kernel<W, kSingleVariants[4].U, kSingleVariants[4].G, kSingleVariants[4].min_ctas>;
    case 5: return (const void*)single_kernel<W, kSingleVariants[5].U, kSingleVariants[5].G, kSingleVariants[5].min_ctas>;
    default: return (const void*)single_kernel<W, kSingleVariants[6].U, kSingleVariants[6].G, kSingleVariants[6].min_ctas>;
    }
}

}  // namespace

void plan_range(int n, uint64_t first, uint64_t last, int U, SingleArgs& a)
{
    a.n = n;
    a.has_head = a.has_tail = 0;
    a.mid_B0 = a.mid_NB = 0;
    a.head_first = a.head_last = a.tail_first = a.tail_last = 0;
    const uint64_t bs = 1ull << U;
    // blocks fully inside [first, last]
    const uint64_t B_begin = (first >> U) + ((first & (bs - 1)) ? 1 : 0);
    const uint64_t B_end = (last >> U) + (((last & (bs - 1)) == bs - 1) ? 1 : 0);
    if (n < U + 1 || B_begin >= B_end) {
        a.has_head = 1;
        a.head_first = first;
        a.head_last = last;
        return;
    }
    a.mid_B0 = B_begin;
    a.mid_NB = B_end - B_begin;
    if (first < (B_begin << U)) {
        a.has_head = 1;
        a.head_first = first;
        a.head_last = (B_begin << U) - 1;
    }
    // B_end * 2^U - 1 <= last; a tail exists when last is not a block's end
    if (((last & (bs - 1)) != bs - 1)) {
        a.has_tail = 1;
        a.tail_first = B_end << U;
        a.tail_last = last;
    }
}

int single_max_ctas_per_sm(int W, int v)
{
    int ctas = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, W == 1 ? single_kernel_ptr<1>(v) : single_kernel_ptr<2>(v),
                                                  kSingleThreads, 0);
    return ctas > 0 ? ctas : 1;
}

int single_grid_for(const SingleArgs& a, int sm_count, int max_ctas_per_sm)
{
    const uint64_t wave = (uint64_t)sm_count * (uint64_t)max_ctas_per_sm;
    const uint64_t need = (a.mid_NB + kSingleThreads - 1) / kSingleThreads;
    uint64_t g = need < wave ? need : wave;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_single(const SingleArgs& a, int v, int grid, cudaStream_t stream)
{
    const void* fn = a.n <= 32 ? single_kernel_ptr<1>(v) : single_kernel_ptr<2>(v);
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSingleThreads), args, 0, stream);
}

cudaError_t launch_step_table(uint32_t* out, cudaStream_t stream)
{
    step_table_kernel<<<1, 32, 0, stream>>>(out);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t* A, int n, unsigned long long* out_mag, unsigned long long* out_sgn,
                        unsigned int* err, cudaStream_t stream)
{
    pack_kernel<<<1, 256, 0, stream>>>(A, n, out_mag, out_sgn, err);
    return cudaGetLastError();
}

}  // namespace pf3
