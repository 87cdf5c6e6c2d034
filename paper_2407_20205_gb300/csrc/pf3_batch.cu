// pf3_batch.cu -- many matrices of uneven n in one persistent launch per
// plane width (the Monte Carlo workload of Sec. 4: permanents of many random
// matrices).
//
// The host plans work items: up to 32 consecutive matrices of the same small
// n (n <= the packing cutoff, at most 16) form one item walked one matrix per
// lane; a larger matrix is one item walked by one warp (its 32 lanes split
// the 2^(n-U) Gray blocks) unless it is cut into items of consecutive Gray
// indices (Sec. 3.1's blocks of consecutive Gray states), whose counts meet
// in per-matrix accumulators; the warp that finishes a matrix's last item
// maps its counts to perm mod 3.  The item length is fixed or sized from the
// batch's total work so that every warp of the grid gets several items.
// Items are sorted largest first and handed out through an atomic cursor, so
// the grid stays full until the end.  Each warp packs its matrix into its own
// shared-memory row table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "perm_f3.h"
#include "pf3_batch.h"
#include "pf3_context.h"
#include "pf3_device.cuh"
#include "pf3_internal.h"

namespace pf3 {

namespace {

constexpr unsigned kBadBit = 0x80000000u;

// Per-lane row masks of one tiny matrix: [row][component][lane], component
// 0 = K1, 1 = K2 (add), 2 = K2 (subtract).
struct TinyTable {
    uint32_t k[kTinyMaxN][3][32];
};

// One lane: pack its n x n matrix (n <= kTinyMaxN) and walk all 2^n Gray
// indices with the row step of Sec. 2 (Theorem 2.1 semantics), full zero test
// and popcount sign at every index.  Returns perm mod 3, or 255 on a bad entry.
__device__ __forceinline__ int tiny_perm(TinyTable& T, const uint8_t* A, int n, int lane)
{
    bool bad = false;
    for (int r = 0; r < n; ++r) {
        uint32_t mag = 0, sgn = 0;
        for (int c = 0; c < n; ++c) {
            const uint32_t v = A[r * n + c];
            bad |= v > 2u;
            mag |= (uint32_t)(v == 1u || v == 2u) << c;
            sgn |= (uint32_t)(v == 2u) << c;
        }
        uint32_t k1, k2p, k2m;
        row_masks(mag, sgn, k1, k2p, k2m);
        T.k[r][0][lane] = k1;
        T.k[r][1][lane] = k2p;
        T.k[r][2][lane] = k2m;
    }
    if (bad) return 255;
    uint32_t m = ~((1u << n) - 1u), s = 0u;  // zero vector, padding columns = 1
    unsigned long long p = 0, q = 0;
    const uint32_t last = (1u << n) - 1u;
    for (uint32_t i = 1; i <= last; ++i) {
        const int t = __ffs((int)i) - 1;
        const int dir = (int)((i >> (t + 1)) & 1u);
        add_word(m, s, T.k[t][0][lane], T.k[t][1 + dir][lane]);
        if (m == 0xFFFFFFFFu) {
            if ((__popc(s) + i) & 1u) ++q;
            else ++p;
        }
    }
    return (int)perm_from_counts(n, p, q);
}

// COLS: the work items may carry a column count below n (serving merges equal
// columns at submit); the batch API's items are square and use the instance
// without it
template <int W, int U, int G, int MINB, bool COLS>
__global__ void __launch_bounds__(kBatchThreads, MINB) batch_kernel(BatchArgs a)
{
    __shared__ RowTable<W> tabs[kBatchThreads / 32];
    __shared__ WarpQueue<G> queues[kBatchThreads / 32];
    __shared__ TinyTable tiny[W == 1 ? kBatchThreads / 32 : 1];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    RowTable<W>& tab = tabs[warp];
    WarpQueue<G>& q = queues[warp];
    if (lane == 0) q.count = 0;
    __syncwarp();

    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(a.cursor, 1u);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= a.num_items) break;
        const WorkItem it = a.items[item];
        const int n = it.n;
        const uint8_t* A = a.As + it.offset;

        if (W == 1 && it.split == kTinyItem) {
            // a group of up to 32 small matrices: one per lane
            int r = -1;
            if ((unsigned long long)lane < it.NB) {
                r = (n == 0) ? 1 : tiny_perm(tiny[warp], A + (size_t)lane * n * n, n, lane);
                a.results[it.mat + lane] = (uint8_t)r;
            }
            if (a.hist) {
                for (int v = 0; v < 3; ++v) {
                    const unsigned cnt = __popc(__ballot_sync(0xFFFFFFFFu, r == v));
                    if (lane == 0 && cnt) atomicAdd(a.hist + v, (unsigned long long)cnt);
                }
            }
            __syncwarp();
            continue;
        }

        bool bad = false;
        const int cols = (COLS && it.cols) ? it.cols : n;  // the walk's column count (padding starts there)
        const int rows = n > U ? n : U;
        for (int r = 0; r < rows; ++r) {
            uint32_t mag[2], sgn[2];
            pack_row_warp(A, n, cols, r, lane, mag, sgn, bad);
            if (lane < W) {
                uint32_t k1, k2p, k2m;
                row_masks(mag[lane], sgn[lane], k1, k2p, k2m);
                tab.e[0][r].k1[lane] = k1;
                tab.e[0][r].k2[lane] = k2p;
                tab.e[1][r].k1[lane] = k1;
                tab.e[1][r].k2[lane] = k2m;
            }
        }
        bad = __any_sync(0xFFFFFFFFu, bad);
        __syncwarp();

        Counts c{0ull, 0ull};
        if (!bad && n > 0) {
            if (it.NB == 0) {
                // n <= U (serving items): one lane walks all 2^n indices
                if (lane == 0) walk_generic<W>(tab, cols, 0, (n == 64) ? ~0ull : ((1ull << n) - 1), c);
            } else {
                GroupRows<G, U> R;
                load_group_rows<W, G, U>(R, tab);
                uint64_t s, len;
                split_range(it.NB, 32, (uint64_t)lane, s, len);
                const uint64_t trip = __shfl_sync(0xFFFFFFFFu, len, 0);
                const uint64_t done = walk_groups<W, G, U>(tab, R, cols, it.B0 + s, len, trip, q, lane, c);
                if (done < len) walk_dense<W, G, U>(tab, q.dk, cols, it.B0 + s + done, len - done, &c);
            }
        }
        const unsigned long long p = warp_sum(c.plus);
        const unsigned long long m = warp_sum(c.minus);
        if (lane == 0) {
            int result = -1;
            if (it.split < 0) {
                result = bad ? 255 : (n == 0 ? 1 : (int)perm_from_counts(n, p, m));
            } else {
                unsigned long long* acc = a.acc + 2 * it.split;
                atomicAdd(acc, p);
                atomicAdd(acc + 1, m);
                if (bad) atomicOr(a.left + it.split, kBadBit);
                __threadfence();
                const unsigned before = atomicSub(a.left + it.split, 1u);
                if ((before & ~kBadBit) == 1u) {
                    __threadfence();
                    const unsigned long long P = __ldcg(acc), M = __ldcg(acc + 1);
                    result = (before & kBadBit) ? 255 : (int)perm_from_counts(n, P, M);
                }
            }
            if (result >= 0) {
                a.results[it.mat] = (uint8_t)result;
                if (result < 3 && a.hist) atomicAdd(a.hist + result, 1ull);
            }
        }
        __syncwarp();
    }
}

// one CTA per admitted job: matrix into its slot, counters reset
__global__ void slot_init_kernel(const SlotInit* inits, int count, const uint8_t* staging, uint8_t* mats,
                                 int slot_bytes, unsigned long long* acc, unsigned* left, uint8_t* results)
{
    const int k = blockIdx.x;
    if (k >= count) return;
    const SlotInit in = inits[k];
    const int nn = in.n * (in.cols ? (int)in.cols : in.n);
    uint8_t* dst = mats + (size_t)in.slot * slot_bytes;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) dst[i] = staging[in.src + i];
    if (threadIdx.x == 0) {
        acc[2 * in.slot] = 0ull;
        acc[2 * in.slot + 1] = 0ull;
        left[in.slot] = in.items;
        results[in.slot] = 0xFEu;
    }
}

template <int W, bool COLS>
const void* batch_kernel_ptr(int v)
{
    switch (v) {
    case 0: return (const void*)batch_kernel<W, kBatchVariants[0].U, kBatchVariants[0].G, kBatchVariants[0].min_ctas, COLS>;
    case 1: return (const void*)batch_kernel<W, kBatchVariants[1].U, kBatchVariants[1].G, kBatchVariants[1].min_ctas, COLS>;
    case 2: return (const void*)batch_kernel<W, kBatchVariants[2].U, kBatchVariants[2].G, kBatchVariants[2].min_ctas, COLS>;
    case 3: return (const void*)batch_kernel<W, kBatchVariants[3].U, kBatchVariants[3].G, kBatchVariants[3].min_ctas, COLS>;
    case 4: return (const void*)batch_kernel<W, kBatchVariants[4].U, kBatchVariants[4].G, kBatchVariants[4].min_ctas, COLS>;
    default: return (const void*)batch_kernel<W, kBatchVariants[5].U, kBatchVariants[5].G, kBatchVariants[5].min_ctas, COLS>;
    }
}

}  // namespace

int batch_max_ctas_per_sm(int W, int v)
{
    int ctas = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, W == 1 ? batch_kernel_ptr<1, false>(v) : batch_kernel_ptr<2, false>(v),
                                                  kBatchThreads, 0);
    return ctas > 0 ? ctas : 1;
}

cudaError_t launch_batch(int W, int v, const BatchArgs& a, int grid, cudaStream_t stream)
{
    const void* fn = W == 1 ? batch_kernel_ptr<1, false>(v) : batch_kernel_ptr<2, false>(v);
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBatchThreads), args, 0, stream);
}

const void* batch_kernel_fn(int W, int v) { return W == 1 ? batch_kernel_ptr<1, true>(v) : batch_kernel_ptr<2, true>(v); }

const void* slot_init_fn() { return (const void*)slot_init_kernel; }

cudaError_t launch_slot_init(const SlotInit* inits, int count, const uint8_t* staging, uint8_t* mats,
                             int slot_bytes, unsigned long long* acc, unsigned* left, uint8_t* results,
                             cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    slot_init_kernel<<<count, 128, 0, stream>>>(inits, count, staging, mats, slot_bytes, acc, left, results);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- planning

// Largest power-of-two exponent e with 2^e <= x (x >= 1), capped at 63.
static int floor_log2(double x)
{
    int e = 0;
    while (e < 63 && std::ldexp(1.0, e + 1) <= x) ++e;
    return e;
}

static WorkItem make_item(long long offset, int64_t mat, int n)
{
    WorkItem it;
    std::memset(&it, 0, sizeof(it));
    it.offset = offset;
    it.mat = (int)mat;
    it.n = n;
    it.split = -1;
    return it;
}

void plan_batch(const int32_t* ns, int64_t count, const BatchTuning& tune, const int warps[2], BatchPlan& plan)
{
    const int Ucls[2] = {kBatchVariants[tune.variant[0]].U, kBatchVariants[tune.variant[1]].U};
    const int tiny = std::min(tune.tiny_cutoff, kTinyMaxN);
    plan.items[0].clear();
    plan.items[1].clear();
    plan.split_items.clear();
    plan.num_split = 0;
    plan.total_bytes = 0;
    plan.chunk_log2[0] = plan.chunk_log2[1] = 0;
    std::vector<long long> offset((size_t)count);
    long long off = 0;
    for (int64_t k = 0; k < count; ++k) {
        offset[(size_t)k] = off;
        off += (long long)ns[k] * ns[k];
    }
    plan.total_bytes = off;

    // packed groups: runs of up to 32 consecutive matrices with one small n
    for (int64_t k = 0; k < count; ++k) {
        const int n = ns[k];
        if (n > tiny) continue;
        int64_t e = k + 1;
        while (e < count && e - k < 32 && ns[e] == n) ++e;
        WorkItem it = make_item(offset[(size_t)k], k, n);
        it.split = kTinyItem;
        it.NB = (unsigned long long)(e - k);
        plan.items[0].push_back(it);
        k = e - 1;
    }

    // the other matrices, per class, largest first (ties in matrix order)
    std::vector<int64_t> order[2];
    for (int64_t k = 0; k < count; ++k)
        if (ns[k] > tiny) order[ns[k] <= 32 ? 0 : 1].push_back(k);
    for (int cls = 0; cls < 2; ++cls) {
        std::vector<int64_t>& ord = order[cls];
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return ns[x] > ns[y]; });
        const int U = Ucls[cls];
        // work from each matrix to the end of the order (guided split)
        std::vector<double> rest(ord.size() + 1, 0.0);
        for (size_t q = ord.size(); q-- > 0;) rest[q] = rest[q + 1] + std::ldexp(1.0, ns[ord[q]]);
        const int lo = std::max(kMinChunkLog2, U + 5);
        const double div = (double)std::max(1, warps ? warps[cls] : 1) * (double)tune.items_per_warp;
        for (size_t q = 0; q < ord.size(); ++q) {
            const int64_t k = ord[q];
            const int n = ns[k];
            WorkItem it = make_item(offset[(size_t)k], k, n);
            if (n < U + 1) {
                it.NB = 0;  // generic walk by one lane
                plan.items[cls].push_back(it);
                continue;
            }
            const uint64_t NB = (n == 64) ? (1ull << (64 - U)) : (1ull << (n - U));
            // piece length: fixed, or the work left from here on over
            // (warps x items_per_warp), so pieces shrink toward the end
            int cl;
            if (tune.chunk_log2 > 0) cl = n > tune.cutoff ? tune.chunk_log2 : n;
            else cl = std::max(lo, floor_log2(rest[q] / div));
            if (q == 0) plan.chunk_log2[cls] = std::min(cl, n);
            if (cl >= n) {
                it.NB = NB;
                plan.items[cls].push_back(it);
                continue;
            }
            // at most 2^20 items per matrix keeps the item table small for n near 64
            cl = std::max(std::max(cl, U + 5), n - 20);
            const uint64_t per = 1ull << (cl - U);
            const uint64_t nitems = (NB + per - 1) / per;
            it.split = plan.num_split++;
            plan.split_items.push_back((unsigned)nitems);
            for (uint64_t b0 = 0; b0 < NB; b0 += per) {
                it.B0 = b0;
                it.NB = std::min<unsigned long long>(per, NB - b0);
                plan.items[cls].push_back(it);
            }
        }
    }
    // largest first (longest-processing-time order); ties keep plan order.
    // Cost = warp time in units of one Gray index of the grouped walk: a
    // packed lane walks each index about four times slower than the 32 lanes
    // of a warp walk theirs, so a packed item costs about 2^n x 128.
    for (int cls = 0; cls < 2; ++cls) {
        const int U = Ucls[cls];
        auto cost = [U](const WorkItem& x) -> unsigned long long {
            if (x.split == kTinyItem) return (1ull << x.n) << 7;
            if (x.NB == 0) return 1ull << x.n;
            return (unsigned long long)x.NB << U;
        };
        std::stable_sort(plan.items[cls].begin(), plan.items[cls].end(),
                         [&](const WorkItem& x, const WorkItem& y) { return cost(x) > cost(y); });
    }
}

void batch_warps(DeviceCtx* c, const BatchTuning& tune, int warps[2])
{
    for (int cls = 0; cls < 2; ++cls)
        warps[cls] = c->sm_count * batch_ctas(c, cls + 1, tune.variant[cls]) * (kBatchThreads / 32);
}

// grow-only device scratch for a plan
static int ensure_batch_scratch(DeviceCtx* c, size_t items, size_t splits, size_t bytes, size_t mats)
{
    BatchScratch& b = c->batch;
    cudaError_t e = cudaSuccess;
    if (items > b.items_cap) {
        cudaFree(b.d_items);
        cudaFreeHost(b.h_items);
        b.d_items = nullptr;
        b.h_items = nullptr;
        size_t cap = std::max(items, (size_t)1024);
        if ((e = cudaMalloc(&b.d_items, cap * sizeof(WorkItem))) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaMallocHost(&b.h_items, cap * sizeof(WorkItem))) != cudaSuccess) return cuda_rc(e);
        b.items_cap = cap;
    }
    if (splits + 1 > b.mats_cap || !b.d_cursor) {
        cudaFree(b.d_acc);
        cudaFree(b.d_left);
        cudaFree(b.d_cursor);
        size_t cap = std::max(splits + 1, (size_t)1024);
        if ((e = cudaMalloc(&b.d_acc, cap * 2 * sizeof(unsigned long long))) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaMalloc(&b.d_left, cap * sizeof(unsigned int))) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaMalloc(&b.d_cursor, 4 * sizeof(unsigned int))) != cudaSuccess) return cuda_rc(e);
        b.mats_cap = cap;
    }
    if (bytes > b.bytes_cap || mats > b.res_cap) {
        cudaFree(b.d_As);
        cudaFree(b.d_results);
        cudaFree(b.d_hist);
        b.d_As = nullptr;
        b.d_results = nullptr;
        b.d_hist = nullptr;
        size_t bcap = std::max(bytes, (size_t)4096), rcap = std::max(mats, (size_t)1024);
        if ((e = cudaMalloc(&b.d_As, bcap)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaMalloc(&b.d_results, rcap)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaMalloc(&b.d_hist, 4 * sizeof(unsigned long long))) != cudaSuccess) return cuda_rc(e);
        b.bytes_cap = bcap;
        b.res_cap = rcap;
    }
    return PF3_OK;
}

// device buffers one batch launch sequence works on
struct BatchBufs {
    const WorkItem* d_items;       // class W = 2 items first, then W = 1
    unsigned long long* d_acc;
    unsigned* d_left;
    unsigned* d_cursor;
    const void* h_items;           // pinned source of the item table
    const unsigned* h_left;        // source of the split item counts
};

// the launch sequence itself: upload the item table and split counters, reset
// cursors and histogram, one persistent grid per plane width (W = 2 first)
static int enqueue_batch_core(DeviceCtx* c, const BatchPlan& plan, const BatchBufs& bb, const uint8_t* dAs,
                              uint8_t* d_results, unsigned long long* d_hist, cudaStream_t stream)
{
    const size_t n0 = plan.items[0].size(), n1 = plan.items[1].size();
    cudaError_t e = cudaSuccess;
    if (n0 + n1)
        e = cudaMemcpyAsync((void*)bb.d_items, bb.h_items, (n0 + n1) * sizeof(WorkItem), cudaMemcpyHostToDevice,
                            stream);
    if (e == cudaSuccess && plan.num_split) {
        e = cudaMemsetAsync(bb.d_acc, 0, (size_t)plan.num_split * 2 * sizeof(unsigned long long), stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bb.d_left, bb.h_left, (size_t)plan.num_split * sizeof(unsigned int),
                                cudaMemcpyHostToDevice, stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(bb.d_cursor, 0, 4 * sizeof(unsigned int), stream);
    if (e == cudaSuccess && d_hist) e = cudaMemsetAsync(d_hist, 0, 3 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_rc(e);
    BatchArgs a;
    a.As = dAs;
    a.results = d_results;
    a.hist = d_hist;
    a.acc = bb.d_acc;
    a.left = bb.d_left;
    for (int cls = 1; cls >= 0; --cls) {
        const size_t cnt = plan.items[cls].size();
        if (!cnt) continue;
        a.items = bb.d_items + (cls == 1 ? 0 : n1);
        a.num_items = (unsigned)cnt;
        a.cursor = bb.d_cursor + cls;
        const int v = c->tune.variant[cls];
        const int per_sm = batch_ctas(c, cls + 1, v);
        int grid = c->sm_count * per_sm;
        const size_t ctas_needed = (cnt + kBatchThreads / 32 - 1) / (kBatchThreads / 32);
        if ((size_t)grid > ctas_needed) grid = (int)ctas_needed;
        if ((e = launch_batch(cls == 0 ? 1 : 2, v, a, grid, stream)) != cudaSuccess) return cuda_rc(e);
    }
    return PF3_OK;
}

// enqueue a planned batch on `stream` using the context's batch scratch
int enqueue_batch(DeviceCtx* c, const BatchPlan& plan, const uint8_t* dAs, uint8_t* d_results,
                  unsigned long long* d_hist, cudaStream_t stream)
{
    const size_t n0 = plan.items[0].size(), n1 = plan.items[1].size();
    BatchScratch& b = c->batch;
    int rc = ensure_batch_scratch(c, n0 + n1, (size_t)plan.num_split, 0, 0);
    if (rc) return rc;
    WorkItem* h = (WorkItem*)b.h_items;
    // the pinned mirror may still be read by an earlier upload on this stream
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_rc(e);
    if (n1) std::memcpy(h, plan.items[1].data(), n1 * sizeof(WorkItem));
    if (n0) std::memcpy(h + n1, plan.items[0].data(), n0 * sizeof(WorkItem));
    BatchBufs bb{(const WorkItem*)b.d_items, b.d_acc, b.d_left, b.d_cursor, h, plan.split_items.data()};
    return enqueue_batch_core(c, plan, bb, dAs, d_results, d_hist, stream);
}

static void free_graph(BatchGraphCache& g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    cudaFreeHost(g.h_items);
    cudaFreeHost(g.h_left);
    cudaFree(g.d_items);
    cudaFree(g.d_acc);
    cudaFree(g.d_left);
    cudaFree(g.d_cursor);
    g = BatchGraphCache();
}

static bool same_tuning(const BatchTuning& a, const BatchTuning& b)
{
    return a.tiny_cutoff == b.tiny_cutoff && a.cutoff == b.cutoff && a.chunk_log2 == b.chunk_log2 &&
           a.items_per_warp == b.items_per_warp && a.variant[0] == b.variant[0] && a.variant[1] == b.variant[1];
}

// Launch the instantiated graph on `stream`, after the previous replay (on
// any stream) has finished with the graph's buffers.
static int launch_batch_graph(DeviceCtx* c, cudaStream_t stream)
{
    bool capturing = false;
    int rc = scratch_acquire(c->bgraph_free, stream, &capturing);
    if (rc) return rc;
    if ((rc = cuda_rc(cudaGraphLaunch(c->bgraph.exec, stream)))) return rc;
    return scratch_release(c->bgraph_free, stream, capturing);
}

// Replay the captured launch sequence when nothing changed, else plan,
// capture on a private stream, instantiate and launch.
int enqueue_batch_graph(DeviceCtx* c, const int32_t* ns, int64_t count, const uint8_t* dAs, uint8_t* d_results,
                        unsigned long long* d_hist, cudaStream_t stream)
{
    BatchGraphCache& g = c->bgraph;
    if (g.valid && (int64_t)g.ns.size() == count && g.dAs == dAs && g.d_results == d_results && g.d_hist == d_hist &&
        same_tuning(g.tune, c->tune) && std::memcmp(g.ns.data(), ns, (size_t)count * sizeof(int32_t)) == 0)
        return launch_batch_graph(c, stream);
    // a previous replay, on this or another stream, may still read the
    // buffers about to be freed
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(c->bgraph_free);
    if (e != cudaSuccess) return cuda_rc(e);
    if (g.valid || g.exec) free_graph(g);
    BatchPlan plan;
    int warps[2];
    batch_warps(c, c->tune, warps);
    plan_batch(ns, count, c->tune, warps, plan);
    const size_t n0 = plan.items[0].size(), n1 = plan.items[1].size();
    const size_t ns_split = (size_t)plan.num_split + 1;
    bool ok = cudaMallocHost(&g.h_items, std::max<size_t>(1, n0 + n1) * sizeof(WorkItem)) == cudaSuccess;
    ok = ok && cudaMallocHost(&g.h_left, ns_split * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMalloc(&g.d_items, std::max<size_t>(1, n0 + n1) * sizeof(WorkItem)) == cudaSuccess;
    ok = ok && cudaMalloc(&g.d_acc, ns_split * 2 * sizeof(unsigned long long)) == cudaSuccess;
    ok = ok && cudaMalloc(&g.d_left, ns_split * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMalloc(&g.d_cursor, 4 * sizeof(unsigned)) == cudaSuccess;
    if (ok && !c->capture_stream)
        ok = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_graph(g);
        return PF3_ENOMEM;
    }
    WorkItem* h = (WorkItem*)g.h_items;
    if (n1) std::memcpy(h, plan.items[1].data(), n1 * sizeof(WorkItem));
    if (n0) std::memcpy(h + n1, plan.items[0].data(), n0 * sizeof(WorkItem));
    if (plan.num_split) std::memcpy(g.h_left, plan.split_items.data(), (size_t)plan.num_split * sizeof(unsigned));
    BatchBufs bb{(const WorkItem*)g.d_items, g.d_acc, g.d_left, g.d_cursor, g.h_items, g.h_left};
    e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_rc(e);
    }
    int rc = enqueue_batch_core(c, plan, bb, dAs, d_results, d_hist, c->capture_stream);
    e = cudaStreamEndCapture(c->capture_stream, &g.graph);
    if (rc || e != cudaSuccess) {
        cudaGetLastError();
        free_graph(g);
        return rc ? rc : cuda_rc(e);
    }
    e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_rc(e);
    }
    g.ns.assign(ns, ns + count);
    g.dAs = dAs;
    g.d_results = d_results;
    g.d_hist = d_hist;
    g.tune = c->tune;
    g.n_items[0] = (int)n0;
    g.n_items[1] = (int)n1;
    g.num_split = plan.num_split;
    g.valid = true;
    return launch_batch_graph(c, stream);
}

}  // namespace pf3

using namespace pf3;

extern "C" {

int pf3_batch_plan(const int32_t* ns, int64_t count, int tiny_cutoff, int split_cutoff, int chunk_log2,
                   int items_per_warp, const int* variant, const int* warps, pf3_plan_item* items, int64_t capacity,
                   int64_t* num_items, int* auto_chunk_log2)
{
    if (count < 0 || count > PF3_MAX_BATCH || (count > 0 && !ns) || !variant || !warps || !num_items ||
        capacity < 0)
        return PF3_EINVAL;
    if (tiny_cutoff < 0 || tiny_cutoff > kTinyMaxN || split_cutoff < 0 || split_cutoff > PF3_MAX_N ||
        (chunk_log2 != 0 && (chunk_log2 < 12 || chunk_log2 > 62)) || items_per_warp < 1 || items_per_warp > 1024)
        return PF3_EINVAL;
    for (int cls = 0; cls < 2; ++cls)
        if (variant[cls] < 0 || variant[cls] >= kNumBatchVariants || warps[cls] < 1) return PF3_EINVAL;
    for (int64_t k = 0; k < count; ++k)
        if (ns[k] < 0 || ns[k] > PF3_MAX_N) return PF3_EINVAL;
    BatchTuning t;
    t.tiny_cutoff = tiny_cutoff;
    t.cutoff = split_cutoff;
    t.chunk_log2 = chunk_log2;
    t.items_per_warp = items_per_warp;
    t.variant[0] = variant[0];
    t.variant[1] = variant[1];
    BatchPlan plan;
    const int w[2] = {warps[0], warps[1]};
    plan_batch(ns, count, t, w, plan);
    const int64_t total = (int64_t)(plan.items[0].size() + plan.items[1].size());
    *num_items = total;
    if (auto_chunk_log2) {
        auto_chunk_log2[0] = plan.chunk_log2[0];
        auto_chunk_log2[1] = plan.chunk_log2[1];
    }
    if (!items) return PF3_OK;
    if (capacity < total) return PF3_ETOOBIG;
    int64_t o = 0;
    for (int cls = 1; cls >= 0; --cls) {
        const int U = kBatchVariants[variant[cls]].U;
        for (const WorkItem& it : plan.items[cls]) {
            pf3_plan_item& x = items[o++];
            x.mat = it.mat;
            x.n = it.n;
            x.kind = it.split == kTinyItem ? 2 : (it.NB == 0 ? 3 : (it.split >= 0 ? 1 : 0));
            x.first_block = it.B0;
            x.num_blocks = it.NB;
            x.block_log2 = U;
            x.cls = cls;
        }
    }
    return PF3_OK;
}

int perm_f3_batch(const uint8_t* As, const int32_t* ns, int64_t count, uint8_t* results, uint64_t* hist)
{
    if (count < 0 || count > PF3_MAX_BATCH || (count > 0 && (!ns || !results))) return PF3_EINVAL;
    if (count == 0) {
        if (hist) hist[0] = hist[1] = hist[2] = 0;
        return PF3_OK;
    }
    size_t bytes = 0;
    for (int64_t k = 0; k < count; ++k) {
        if (ns[k] < 0 || ns[k] > PF3_MAX_N) return PF3_EINVAL;
        bytes += (size_t)ns[k] * ns[k];
    }
    if (bytes && !As) return PF3_EINVAL;
    for (size_t k = 0; k < bytes; ++k)
        if (As[k] > 2) return PF3_EDOMAIN;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    BatchPlan plan;
    int warps[2];
    batch_warps(c, c->tune, warps);
    plan_batch(ns, count, c->tune, warps, plan);
    if ((rc = ensure_batch_scratch(c, plan.items[0].size() + plan.items[1].size(), (size_t)plan.num_split, bytes,
                                   (size_t)count)))
        return rc;
    BatchScratch& b = c->batch;
    cudaError_t e = cudaSuccess;
    if (bytes) e = cudaMemcpyAsync(b.d_As, As, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    if ((rc = enqueue_batch(c, plan, b.d_As, b.d_results, b.d_hist, c->stream))) return rc;
    e = cudaMemcpyAsync(results, b.d_results, (size_t)count, cudaMemcpyDeviceToHost, c->stream);
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, b.d_hist, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    if (hist) {
        hist[0] = h[0];
        hist[1] = h[1];
        hist[2] = h[2];
    }
    return PF3_OK;
}

int perm_f3_batch_async(const uint8_t* dAs, const int32_t* ns, int64_t count, uint8_t* d_results, uint64_t* d_hist,
                        void* stream)
{
    if (count < 0 || count > PF3_MAX_BATCH || (count > 0 && (!ns || !d_results))) return PF3_EINVAL;
    size_t bytes = 0;
    for (int64_t k = 0; k < count; ++k) {
        if (ns[k] < 0 || ns[k] > PF3_MAX_N) return PF3_EINVAL;
        bytes += (size_t)ns[k] * ns[k];
    }
    if (bytes && !dAs) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    if (count == 0) {
        if (d_hist)
            return cuda_rc(cudaMemsetAsync(d_hist, 0, 3 * sizeof(unsigned long long), (cudaStream_t)stream));
        return PF3_OK;
    }
    return enqueue_batch_graph(c, ns, count, dAs, d_results, (unsigned long long*)d_hist, (cudaStream_t)stream);
}

}  // extern "C"
