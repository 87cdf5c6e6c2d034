// pf3_single.cu -- one matrix, one launch: the Gray-code Ryser sum of Eq. (2)
// over a range of Gray indices, split across every thread of the grid.
//
// Sec. 3.1 of the paper splits the 2^n Gray states into blocks of consecutive
// states, each started by jumping to gray(start).  Here a block is 2^U
// consecutive indices (U picked by the autotuner).  In a short launch each
// thread walks one contiguous run of blocks, seeded once by a direct subset
// sum.  In a long one a warp takes chunks of consecutive blocks from an
// atomic cursor (each lane a contiguous run of the chunk); chunks are long at
// first and short at the end, so warps that the schedulers favour take more
// of them and the SMs' pipes stay full until the last chunk (with fixed
// shares about a quarter of the warps sat idle at the end).
// Each CTA packs the matrix into a shared-memory row table itself (no
// separate pack launch), the per-thread (+1, -1) term counts are reduced by
// warp shuffles and shared memory, and the last CTA to finish adds the
// per-CTA partials and maps the counts to perm mod 3.
#include <cuda_runtime.h>

#include "pf3_device.cuh"
#include "pf3_internal.h"

namespace pf3 {

namespace {

template <int W, int U, int G, int MINB, int THREADS>
__global__ void __launch_bounds__(THREADS, MINB) single_kernel(SingleArgs a)
{
    __shared__ RowTable<W> tab;
    __shared__ WarpQueue<G> queues[THREADS / 32];
    __shared__ unsigned long long red[2][THREADS / 32];
    __shared__ bool s_last;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (lane == 0) queues[warp].count = 0;
    const bool bad_local = build_row_table<W>(tab, a.A, a.n, a.m, warp, THREADS / 32, lane);
    const bool bad = __syncthreads_or(bad_local) != 0;

    Counts c{0ull, 0ull};
    if (!bad) {
        const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
        const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (a.mid_NB) {
            GroupRows<G, U> R;
            load_group_rows<W, G, U>(R, tab);
            if (!a.dynamic) {
                // one contiguous share of the blocks per thread
                uint64_t s, len;
                split_range(a.mid_NB, T, tid, s, len);
                const uint64_t trip = __shfl_sync(0xFFFFFFFFu, len, 0);  // lane 0 holds the longest share
                const uint64_t done =
                    walk_groups<W, G, U>(tab, R, a.m, a.mid_B0 + s, len, trip, queues[warp], lane, c);
                if (done < len) walk_dense<W, G, U>(tab, queues[warp].dk, a.m, a.mid_B0 + s + done, len - done, &c);
            } else {
                // the cursor only grows, and every chunk index at or past
                // nchunks ends the loop: at most nchunks + 1 turns per warp
                for (;;) {
                    unsigned k = 0;
                    if (lane == 0) k = atomicAdd(a.cursor, 1u);
                    k = __shfl_sync(0xFFFFFFFFu, k, 0);
                    if (k >= a.nchunks) break;
                    uint64_t cs, clen, s, len;
                    chunk_range(a, k, cs, clen);
                    split_range(clen, 32, (uint64_t)lane, s, len);
                    const uint64_t trip = __shfl_sync(0xFFFFFFFFu, len, 0);
                    const uint64_t done =
                        walk_groups<W, G, U>(tab, R, a.m, a.mid_B0 + cs + s, len, trip, queues[warp], lane, c);
                    if (done < len)
                        walk_dense<W, G, U>(tab, queues[warp].dk, a.m, a.mid_B0 + cs + s + done, len - done, &c);
                }
            }
        }
        if (a.has_head && tid == T - 1) walk_generic<W>(tab, a.m, a.head_first, a.head_last, c);
        if (a.has_tail && tid == (T > 1 ? T - 2 : 0)) walk_generic<W>(tab, a.m, a.tail_first, a.tail_last, c);
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
        for (int w = 0; w < THREADS / 32; ++w) {
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
        for (int w = 0; w < THREADS / 32; ++w) {
            p += red[0][w];
            m += red[1][w];
        }
        const unsigned e = atomicExch(a.err, 0u);
        a.out[0] = p;
        a.out[1] = m;
        a.out[2] = e ? ~0ull : (unsigned long long)perm_from_counts(a.n, p, m);
        // every CTA took its last chunk before its ticket
        *a.cursor = 0u;
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
        pack_row_warp(A, n, n, r, lane, mag, sgn, bad);
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
    case 0: return (const void*)single_kernel<W, kSingleVariants[0].U, kSingleVariants[0].G, kSingleVariants[0].min_ctas,
                                                   kSingleVariants[0].threads>;
    case 1: return (const void*)single_kernel<W, kSingleVariants[1].U, kSingleVariants[1].G, kSingleVariants[1].min_ctas,
                                                   kSingleVariants[1].threads>;
    case 2: return (const void*)single_kernel<W, kSingleVariants[2].U, kSingleVariants[2].G, kSingleVariants[2].min_ctas,
                                                   kSingleVariants[2].threads>;
    case 3: return (const void*)single_kernel<W, kSingleVariants[3].U, kSingleVariants[3].G, kSingleVariants[3].min_ctas,
                                                   kSingleVariants[3].threads>;
    case 4: return (const void*)single_kernel<W, kSingleVariants[4].U, kSingleVariants[4].G, kSingleVariants[4].min_ctas,
                                                   kSingleVariants[4].threads>;
    case 5: return (const void*)single_kernel<W, kSingleVariants[5].U, kSingleVariants[5].G, kSingleVariants[5].min_ctas,
                                                   kSingleVariants[5].threads>;
    case 6: return (const void*)single_kernel<W, kSingleVariants[6].U, kSingleVariants[6].G, kSingleVariants[6].min_ctas,
                                                   kSingleVariants[6].threads>;
    case 7: return (const void*)single_kernel<W, kSingleVariants[7].U, kSingleVariants[7].G, kSingleVariants[7].min_ctas,
                                                   kSingleVariants[7].threads>;
    default: return (const void*)single_kernel<W, kSingleVariants[8].U, kSingleVariants[8].G, kSingleVariants[8].min_ctas,
                                                   kSingleVariants[8].threads>;
    }
}

}  // namespace

void plan_range(int n, uint64_t first, uint64_t last, int U, SingleArgs& a)
{
    a.n = n;
    a.m = n;
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
                                                  kSingleVariants[v].threads, 0);
    return ctas > 0 ? ctas : 1;
}

int single_grid_for(const SingleArgs& a, int v, int sm_count, int max_ctas_per_sm)
{
    const uint64_t threads = (uint64_t)kSingleVariants[v].threads;
    const uint64_t wave = (uint64_t)sm_count * (uint64_t)max_ctas_per_sm;
    const uint64_t need = (a.mid_NB + threads - 1) / threads;
    uint64_t g = need < wave ? need : wave;
    if (g < 1) g = 1;
    return (int)g;
}

// Work split for `grid` CTAs of `threads` threads (P warps).  Below 512
// blocks per lane each thread walks one contiguous share (dynamic = 0): the
// finishing spread of a short launch costs less than re-seeding chunks would.
// Above, guided chunks, every length a multiple of 32 blocks so the lanes of
// a warp share a chunk evenly: phase j is 4P chunks of len0 >> j blocks
// (rounded down to 32), len0 = mid_NB / 8P, so each phase takes half of what
// is left and the phases cover at most mid_NB, while that length is at least
// 128 blocks; tail chunks of 128 blocks (4 per lane) cover the rest.
void plan_chunks(SingleArgs& a, int grid, int threads)
{
    const uint64_t P = (uint64_t)(grid > 0 ? grid : 1) * (uint64_t)(threads / 32);
    const uint64_t NB = a.mid_NB;
    if (NB < P * 32 * 512) {
        a.len0 = a.tail_len = 0;
        a.per_phase = a.nchunks = 0;
        a.dynamic = 0;
        return;
    }
    const uint64_t tl = 128;
    const uint64_t per = 4 * P;
    const uint64_t L0 = (NB / (8 * P)) & ~31ull;                // >= 2048
    uint64_t used = 0, chunks = 0;
    for (uint64_t L = L0; L >= tl; L = (L >> 1) & ~31ull) {
        used += per * L;
        chunks += per;
    }
    chunks += (NB - used + tl - 1) / tl;
    a.len0 = L0;
    a.tail_len = tl;
    a.per_phase = (unsigned)per;
    a.nchunks = (unsigned)chunks;
    a.dynamic = 1;
}

cudaError_t launch_single(const SingleArgs& args, int v, int grid, cudaStream_t stream)
{
    SingleArgs a = args;
    const int threads = kSingleVariants[v].threads;
    plan_chunks(a, grid, threads);
    const void* fn = a.m <= 32 ? single_kernel_ptr<1>(v) : single_kernel_ptr<2>(v);
    void* kargs[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), kargs, 0, stream);
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
