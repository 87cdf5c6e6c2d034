// pf3_serve.cu -- continuous batching of permanent requests.
//
// The Monte Carlo studies of Sec. 4 consume perm(A) for a stream of random
// matrices; this runtime serves such a stream as requests arrive.  A
// scheduler thread owns a pool of device slots: every admitted job keeps its
// matrix, its two partial counts and its count of outstanding work items on
// the device until its last item finishes.  Each job's Gray range is cut into
// work items of 2^chunk_log2 indices (Sec. 3.1's blocks of consecutive Gray
// states).  Every launch of the persistent batch kernel takes items from many
// jobs at once under a work budget: first every job whose remaining work is
// small (at most 2^small_work_log2 indices), least remaining first, then the
// other jobs in arrival order.  Small jobs finish in the next launch, and
// since they carry a small share of the work the large ones are served much
// as first-come first-served would serve them, never behind a later large
// job.  A job whose equal columns merge into at most cfg.class_max_cols
// columns gets no work items: it is counted by column-sum vector
// (pf3_classes.cu) in the launch that admits it.  Up to two launches are in
// flight; new requests are admitted into free slots between launches, so
// work that arrives while other jobs run overlaps with them on the GPU.  Each launch's sequence of
// copies, kernels and event operations is one CUDA graph per buffer, replayed
// with that launch's sizes.  Nothing on the device waits on the host:
// completion is observed with CUDA events, and the host polls them with short
// sleeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "perm_f3.h"
#include "pf3_batch.h"
#include "pf3_context.h"
#include "pf3_internal.h"

using namespace pf3;

namespace {

constexpr int kSlotBytes = kMaxNN;
constexpr unsigned char kPending = 0xFEu;

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum JobState : int { kQueued = 0, kAdmitted = 1, kDone = 2, kFailed = 3 };

struct Job {
    int n = 0;
    int m = 0;                // columns walked: n, or fewer when equal columns were merged
    bool negate = false;      // the merge's sign factor: the result is negated
    bool by_class = false;    // counted by column-sum vector when admitted, not walked
    int state = kQueued;
    int slot = -1;
    int result = -1;
    int error = 0;
    std::vector<uint8_t> A;
    uint64_t nb = 0;          // Gray blocks of 2^U (0: one generic item)
    uint64_t per_item = 0;    // blocks per work item
    uint64_t cursor = 0;      // next block to issue
    uint64_t items_total = 0;
    uint64_t items_issued = 0;
    uint64_t t_submit = 0;
    uint64_t t_done = 0;
};

struct Launch {
    int buf = 0;
    std::vector<int64_t> finishing;
};

}  // namespace

struct pf3_ctx {
    pf3_config cfg;
    int device = 0;
    DeviceCtx* dc = nullptr;
    int U[2] = {8, 8};
    int variant[2] = {0, 0};
    int grid[2] = {1, 1};
    cudaStream_t streams[2] = {nullptr, nullptr};  // launches alternate between them
    cudaEvent_t kdone[2] = {nullptr, nullptr};     // after each launch's kernels
    // device state
    uint8_t* d_mats = nullptr;
    unsigned long long* d_acc = nullptr;
    unsigned* d_left = nullptr;
    uint8_t* d_results = nullptr;
    uint8_t* d_stage[2] = {nullptr, nullptr};
    void* d_table[2] = {nullptr, nullptr};    // SlotInit[max_admit] then WorkItem[max_items]
    unsigned* d_cursor = nullptr;             // 2 buffers x 2 classes
    // pinned host mirrors
    uint8_t* h_stage[2] = {nullptr, nullptr};
    void* h_table[2] = {nullptr, nullptr};
    uint8_t* h_results[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // One graph per buffer holds a launch's whole sequence; each launch sets
    // its sizes in the instantiated graph and replays it (see build_graph).
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraphNode_t g_stage[2] = {}, g_inits[2] = {}, g_items[2] = {}, g_slot[2] = {}, g_class[2] = {};
    cudaGraphNode_t g_batch[2][2] = {};  // [buffer][class]
    // host bookkeeping
    std::mutex mu;
    std::condition_variable cv_done;
    std::condition_variable cv_work;
    std::vector<Job> jobs;
    std::deque<int64_t> pending;
    std::vector<int64_t> active;  // admitted, items left to issue
    std::vector<int> free_slots;
    std::deque<Launch> inflight;
    std::thread th;
    bool stop = false;
    int fatal = 0;
    uint64_t launches = 0, items = 0, done = 0;
};

namespace {

size_t table_bytes(const pf3_config& c)
{
    return (size_t)c.max_admit * sizeof(SlotInit) + (size_t)c.launch_items * sizeof(WorkItem);
}

void fail_all(pf3_ctx* x, int code)
{
    // caller holds x->mu
    x->fatal = code;
    for (auto& j : x->jobs)
        if (j.state == kQueued || j.state == kAdmitted) {
            j.state = kFailed;
            j.error = code;
            j.t_done = now_ns();
        }
    x->pending.clear();
    x->active.clear();
    x->cv_done.notify_all();
}

// harvest the oldest in-flight launch once its event has completed
bool harvest(pf3_ctx* x, bool block)
{
    if (x->inflight.empty()) return false;
    Launch& L = x->inflight.front();
    cudaError_t e = block ? cudaEventSynchronize(x->ev[L.buf]) : cudaEventQuery(x->ev[L.buf]);
    if (e == cudaErrorNotReady) return false;
    std::lock_guard<std::mutex> g(x->mu);
    if (e != cudaSuccess) {
        fail_all(x, PF3_ECUDA);
        x->inflight.pop_front();
        return true;
    }
    const uint64_t t = now_ns();
    for (int64_t tk : L.finishing) {
        Job& j = x->jobs[tk];
        const unsigned char r = x->h_results[L.buf][j.slot];
        if (r < 3) {
            j.result = j.negate ? (3 - r) % 3 : r;
            j.state = kDone;
        } else {
            j.state = kFailed;
            j.error = (r == 255) ? PF3_EDOMAIN : PF3_ECUDA;
        }
        j.t_done = t;
        x->free_slots.push_back(j.slot);
        ++x->done;
    }
    x->inflight.pop_front();
    x->cv_done.notify_all();
    return true;
}

// The launch sequence of buffer b as a graph, one chain of nodes: copies of
// the staged matrices, the slot set-ups and the work items to the device; the
// slot set-up kernel; the count by column-sum vector of the admitted jobs
// whose merged matrix is narrow; the reset of the item cursors; the batch
// kernel for n > 32 and the one for n <= 32; then, after the other buffer's
// previous kernels (event wait), the copy of every slot's result byte to the
// host.
// Sizes, grids and item counts change from launch to launch: launch_once
// sets them in the instantiated graph and disables the nodes a launch does
// not need (no admissions, no items of a class).
int build_graph(pf3_ctx* x, int b)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return cuda_rc(e);
    x->graph[b] = g;
    const size_t inits_bytes = (size_t)x->cfg.max_admit * sizeof(SlotInit);
    cudaGraphNode_t prev = nullptr;
    auto dep = [&](cudaGraphNode_t node) { prev = node; };
    auto copy = [&](cudaGraphNode_t* node, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
        if (e == cudaSuccess) e = cudaGraphAddMemcpyNode1D(node, g, prev ? &prev : nullptr, prev ? 1 : 0, dst, src,
                                                          bytes, kind);
        if (e == cudaSuccess) dep(*node);
    };
    copy(&x->g_stage[b], x->d_stage[b], x->h_stage[b], kSlotBytes, cudaMemcpyHostToDevice);
    copy(&x->g_inits[b], x->d_table[b], x->h_table[b], sizeof(SlotInit), cudaMemcpyHostToDevice);
    copy(&x->g_items[b], (char*)x->d_table[b] + inits_bytes, (char*)x->h_table[b] + inits_bytes, sizeof(WorkItem),
         cudaMemcpyHostToDevice);
    // slot set-up kernel (sizes set per launch)
    const SlotInit* d_inits = (const SlotInit*)x->d_table[b];
    int count = 0, slot_bytes = kSlotBytes;
    const uint8_t* staging = x->d_stage[b];
    void* sargs[] = {(void*)&d_inits, (void*)&count, (void*)&staging, (void*)&x->d_mats, (void*)&slot_bytes,
                     (void*)&x->d_acc, (void*)&x->d_left, (void*)&x->d_results};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)slot_init_fn();
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(128);
    kp.kernelParams = sargs;
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&x->g_slot[b], g, &prev, 1, &kp);
    if (e == cudaSuccess) dep(x->g_slot[b]);
    // the jobs counted by column-sum vector (pf3_classes.cu), one CTA each
    int class_threads = 0;
    size_t class_smem = 0;
    const void* class_fn = class_slots_fn(&class_threads, &class_smem);
    if (e == cudaSuccess && !class_fn) e = cudaErrorInvalidValue;
    const uint8_t* mats = x->d_mats;
    void* cargs[] = {(void*)&d_inits, (void*)&count, (void*)&mats, (void*)&slot_bytes,
                     (void*)&x->d_acc, (void*)&x->d_left, (void*)&x->d_results};
    cudaKernelNodeParams cp = {};
    cp.func = (void*)class_fn;
    cp.gridDim = dim3(1);
    cp.blockDim = dim3((unsigned)class_threads);
    cp.sharedMemBytes = (unsigned)class_smem;
    cp.kernelParams = cargs;
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&x->g_class[b], g, &prev, 1, &cp);
    if (e == cudaSuccess) dep(x->g_class[b]);
    cudaMemsetParams mp = {};
    mp.dst = x->d_cursor + 2 * b;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = 2;
    mp.height = 1;
    cudaGraphNode_t n_cur = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&n_cur, g, &prev, 1, &mp);
    if (e == cudaSuccess) dep(n_cur);
    for (int cls = 1; cls >= 0 && e == cudaSuccess; --cls) {
        BatchArgs a = {};
        a.As = x->d_mats;
        a.items = (const WorkItem*)((char*)x->d_table[b] + inits_bytes);
        a.num_items = 0;
        a.cursor = x->d_cursor + 2 * b + cls;
        a.acc = x->d_acc;
        a.left = x->d_left;
        a.results = x->d_results;
        a.hist = nullptr;
        void* bargs[] = {(void*)&a};
        cudaKernelNodeParams bp = {};
        bp.func = (void*)batch_kernel_fn(cls + 1, x->variant[cls]);
        bp.gridDim = dim3(1);
        bp.blockDim = dim3(kBatchThreads);
        bp.kernelParams = bargs;
        e = cudaGraphAddKernelNode(&x->g_batch[b][cls], g, &prev, 1, &bp);
        if (e == cudaSuccess) dep(x->g_batch[b][cls]);
    }
    // the previous launch (other stream) may still run items of jobs that
    // finish here: results are copied once its kernels are done too
    cudaGraphNode_t n_rec = nullptr, n_wait = nullptr, n_res = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&n_rec, g, &prev, 1, x->kdone[b]);
    if (e == cudaSuccess) dep(n_rec);
    if (e == cudaSuccess) e = cudaGraphAddEventWaitNode(&n_wait, g, &prev, 1, x->kdone[b ^ 1]);
    if (e == cudaSuccess) dep(n_wait);
    copy(&n_res, x->h_results[b], x->d_results, (size_t)x->cfg.max_jobs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x->gexec[b], g, 0);
    return cuda_rc(e);
}

// The work split of an admitted job: Gray blocks of 2^U indices (U of the
// batch kernel variant of its plane width: one word for at most 32 columns)
// cut into work items of 2^chunk_log2 indices (Sec. 3.1's blocks of
// consecutive Gray states); a job of n <= U rows is one item walked by one
// lane.
void plan_job_items(Job& j, const pf3_config& cfg, const int U_cls[2])
{
    const int U = U_cls[j.m <= 32 ? 0 : 1];
    if (j.by_class) {  // no work items
        j.nb = 0;
        j.items_total = 0;
        return;
    }
    if (j.n <= U) {
        j.nb = 0;
        j.items_total = 1;
        return;
    }
    j.nb = (j.n == 64) ? (1ull << (64 - U)) : (1ull << (j.n - U));
    // items per job stay below 2^30 (the device counter's range)
    const int cl = std::max(std::max(cfg.chunk_log2, U + 5), j.n - 30);
    j.per_item = (cl - U >= 63) ? j.nb : (1ull << (cl - U));
    if (j.per_item > j.nb) j.per_item = j.nb;
    j.items_total = (j.nb + j.per_item - 1) / j.per_item;
}

// One launch's work items under the serving policy, at most
// cfg.launch_items and about cfg.launch_budget Gray indices (a job's first
// item always goes): first every active job whose remaining work is at most
// 2^small_work_log2 indices, least remaining first, then the others in
// arrival order (the order of `active`).  Items go to cls_items[0] (one
// plane word) or [1] (two), and to *issued in issue order when it is given;
// jobs whose last item was issued are appended to `finishing` and leave
// `active`.
void select_items(std::vector<Job>& jobs, std::vector<int64_t>& active, const pf3_config& cfg, const int U_cls[2],
                  std::vector<WorkItem> (&cls_items)[2], std::vector<int64_t>& finishing,
                  std::vector<WorkItem>* issued = nullptr)
{
    uint64_t budget = cfg.launch_budget;
    int n_items = 0;
    auto issue = [&](int64_t tk, uint64_t share) {
        Job& j = jobs[tk];
        while (j.items_issued < j.items_total && n_items < cfg.launch_items) {
            WorkItem it;
            std::memset(&it, 0, sizeof(it));
            it.offset = (long long)j.slot * kSlotBytes;
            it.mat = j.slot;
            it.n = j.n;
            it.cols = j.m;
            it.split = j.slot;
            uint64_t cost;
            if (j.nb == 0) {
                it.B0 = 0;
                it.NB = 0;
                cost = 1ull << j.n;
            } else {
                it.B0 = j.cursor;
                it.NB = std::min<unsigned long long>(j.per_item, j.nb - j.cursor);
                cost = (uint64_t)it.NB << U_cls[j.m <= 32 ? 0 : 1];
            }
            if (cost > share && n_items > 0) break;  // the first item always goes
            share = cost > share ? 0 : share - cost;
            budget = cost > budget ? 0 : budget - cost;
            j.cursor += it.NB;
            ++j.items_issued;
            cls_items[j.m <= 32 ? 0 : 1].push_back(it);
            if (issued) issued->push_back(it);
            ++n_items;
            if (j.items_issued == j.items_total) finishing.push_back(tk);
            if (share == 0) break;
        }
    };
    if (active.empty()) return;
    const int sl = cfg.small_work_log2;
    const uint64_t small = sl >= 64 ? ~0ull : (1ull << sl);
    auto remaining = [&](int64_t tk) -> uint64_t {
        const Job& j = jobs[tk];
        if (!j.nb) return 1ull << j.n;
        const int U = U_cls[j.m <= 32 ? 0 : 1];
        const uint64_t left = j.nb - j.cursor;
        return (left >> (64 - U)) ? ~0ull : left << U;  // 2^64 (n = 64) saturates
    };
    std::vector<int64_t> small_jobs, large_jobs;
    for (int64_t tk : active)
        if (jobs[tk].items_issued < jobs[tk].items_total)
            (remaining(tk) <= small ? small_jobs : large_jobs).push_back(tk);
    std::stable_sort(small_jobs.begin(), small_jobs.end(),
                     [&](int64_t a, int64_t b) { return remaining(a) < remaining(b); });
    for (const auto* list : {&small_jobs, &large_jobs})
        for (int64_t tk : *list) {
            if (budget == 0 || n_items >= cfg.launch_items) break;
            issue(tk, budget);
        }
    // drop fully issued jobs from the active list
    std::vector<int64_t> keep;
    for (int64_t tk : active)
        if (jobs[tk].items_issued < jobs[tk].items_total) keep.push_back(tk);
    active.swap(keep);
}

// build and enqueue one launch; returns false when there was nothing to do
bool launch_once(pf3_ctx* x)
{
    int buf;
    {
        std::lock_guard<std::mutex> g(x->mu);
        buf = (int)(x->launches & 1);
    }
    SlotInit* inits = (SlotInit*)x->h_table[buf];
    WorkItem* items = (WorkItem*)((char*)x->h_table[buf] + (size_t)x->cfg.max_admit * sizeof(SlotInit));
    std::vector<WorkItem> cls_items[2];
    Launch L;
    L.buf = buf;
    int n_inits = 0, n_class = 0;
    size_t stage_off = 0;
    {
        std::lock_guard<std::mutex> g(x->mu);
        if (x->fatal) return false;
        // admit queued jobs into free slots
        while (!x->pending.empty() && !x->free_slots.empty() && n_inits < x->cfg.max_admit) {
            const int64_t tk = x->pending.front();
            Job& j = x->jobs[tk];
            const size_t nn = (size_t)j.n * j.m;
            if (stage_off + nn > (size_t)x->cfg.max_admit * kSlotBytes) break;
            x->pending.pop_front();
            j.slot = x->free_slots.back();
            x->free_slots.pop_back();
            std::memcpy(x->h_stage[buf] + stage_off, j.A.data(), nn);
            std::vector<uint8_t>().swap(j.A);
            plan_job_items(j, x->cfg, x->U);
            j.state = kAdmitted;
            inits[n_inits].src = (long long)stage_off;
            inits[n_inits].slot = j.slot;
            inits[n_inits].n = j.n;
            inits[n_inits].cols = (unsigned)j.m;
            inits[n_inits].items = (unsigned)j.items_total;  // 0: counted by class in this launch
            ++n_inits;
            stage_off += nn;
            if (j.by_class) {
                ++n_class;
                L.finishing.push_back(tk);
            } else {
                x->active.push_back(tk);
            }
        }
        // choose items: small jobs first, then the others in arrival order
        select_items(x->jobs, x->active, x->cfg, x->U, cls_items, L.finishing);
        x->items += (uint64_t)(cls_items[0].size() + cls_items[1].size());
    }
    const size_t n1 = cls_items[1].size(), n0 = cls_items[0].size();
    if (n_inits == 0 && n0 + n1 == 0) return false;
    // items: class W = 2 first, then W = 1
    if (n1) std::memcpy(items, cls_items[1].data(), n1 * sizeof(WorkItem));
    if (n0) std::memcpy(items + n1, cls_items[0].data(), n0 * sizeof(WorkItem));
    // this launch's sizes into buffer buf's graph, then one replay of it
    cudaStream_t s = x->streams[buf];
    cudaGraphExec_t ge = x->gexec[buf];
    const size_t inits_bytes = (size_t)x->cfg.max_admit * sizeof(SlotInit);
    cudaError_t e = cudaSuccess;
    auto set_copy = [&](cudaGraphNode_t node, void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaGraphExecMemcpyNodeSetParams1D(ge, node, dst, src, bytes,
                                                                            cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaGraphNodeSetEnabled(ge, node, bytes ? 1u : 0u);
    };
    set_copy(x->g_stage[buf], x->d_stage[buf], x->h_stage[buf], stage_off);
    set_copy(x->g_inits[buf], x->d_table[buf], x->h_table[buf], (size_t)n_inits * sizeof(SlotInit));
    set_copy(x->g_items[buf], (char*)x->d_table[buf] + inits_bytes, items, (n0 + n1) * sizeof(WorkItem));
    if (e == cudaSuccess && n_inits) {
        const SlotInit* d_inits = (const SlotInit*)x->d_table[buf];
        int count = n_inits, slot_bytes = kSlotBytes;
        const uint8_t* staging = x->d_stage[buf];
        void* sargs[] = {(void*)&d_inits, (void*)&count, (void*)&staging, (void*)&x->d_mats, (void*)&slot_bytes,
                         (void*)&x->d_acc, (void*)&x->d_left, (void*)&x->d_results};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)slot_init_fn();
        kp.gridDim = dim3((unsigned)n_inits);
        kp.blockDim = dim3(128);
        kp.kernelParams = sargs;
        e = cudaGraphExecKernelNodeSetParams(ge, x->g_slot[buf], &kp);
    }
    if (e == cudaSuccess) e = cudaGraphNodeSetEnabled(ge, x->g_slot[buf], n_inits ? 1u : 0u);
    if (e == cudaSuccess && n_class) {
        const SlotInit* d_inits = (const SlotInit*)x->d_table[buf];
        int count = n_inits, slot_bytes = kSlotBytes;
        const uint8_t* mats = x->d_mats;
        void* cargs[] = {(void*)&d_inits, (void*)&count, (void*)&mats, (void*)&slot_bytes,
                         (void*)&x->d_acc, (void*)&x->d_left, (void*)&x->d_results};
        int threads = 0;
        size_t smem = 0;
        cudaKernelNodeParams cp = {};
        cp.func = (void*)class_slots_fn(&threads, &smem);
        cp.gridDim = dim3((unsigned)n_inits);
        cp.blockDim = dim3((unsigned)threads);
        cp.sharedMemBytes = (unsigned)smem;
        cp.kernelParams = cargs;
        e = cp.func ? cudaGraphExecKernelNodeSetParams(ge, x->g_class[buf], &cp) : cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) e = cudaGraphNodeSetEnabled(ge, x->g_class[buf], n_class ? 1u : 0u);
    const WorkItem* d_items = (const WorkItem*)((char*)x->d_table[buf] + inits_bytes);
    for (int cls = 1; cls >= 0 && e == cudaSuccess; --cls) {
        const size_t cnt = cls == 1 ? n1 : n0;
        if (cnt) {
            BatchArgs a = {};
            a.As = x->d_mats;
            a.items = d_items + (cls == 1 ? 0 : n1);
            a.num_items = (unsigned)cnt;
            a.cursor = x->d_cursor + 2 * buf + cls;
            a.acc = x->d_acc;
            a.left = x->d_left;
            a.results = x->d_results;
            a.hist = nullptr;
            const size_t ctas_needed = (cnt + kBatchThreads / 32 - 1) / (kBatchThreads / 32);
            int grid = x->grid[cls];
            if ((size_t)grid > ctas_needed) grid = (int)ctas_needed;
            void* bargs[] = {(void*)&a};
            cudaKernelNodeParams bp = {};
            bp.func = (void*)batch_kernel_fn(cls + 1, x->variant[cls]);
            bp.gridDim = dim3((unsigned)grid);
            bp.blockDim = dim3(kBatchThreads);
            bp.kernelParams = bargs;
            e = cudaGraphExecKernelNodeSetParams(ge, x->g_batch[buf][cls], &bp);
        }
        if (e == cudaSuccess) e = cudaGraphNodeSetEnabled(ge, x->g_batch[buf][cls], cnt ? 1u : 0u);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
    if (e == cudaSuccess) e = cudaEventRecord(x->ev[buf], s);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> g(x->mu);
        fail_all(x, cuda_rc(e));
        return false;
    }
    x->inflight.push_back(std::move(L));
    std::lock_guard<std::mutex> g(x->mu);
    ++x->launches;
    return true;
}

void scheduler(pf3_ctx* x)
{
    cudaSetDevice(x->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(x->mu);
            if (x->stop && x->pending.empty() && x->active.empty() && x->inflight.empty()) break;
            if (x->fatal && x->inflight.empty()) {
                if (x->stop) break;
                x->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
            const bool can_launch = !x->active.empty() || (!x->pending.empty() && !x->free_slots.empty());
            if (!can_launch && x->inflight.empty()) {
                x->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        // retire finished launches without blocking
        while (harvest(x, false)) {
        }
        if ((int)x->inflight.size() >= 2) {
            // both buffers busy: wait briefly for the oldest
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            continue;
        }
        if (!launch_once(x)) {
            if (!x->inflight.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" {

void pf3_config_default(pf3_config* cfg)
{
    if (!cfg) return;
    cfg->max_jobs = 4096;
    cfg->queue_depth = 1 << 20;
    cfg->chunk_log2 = 22;
    cfg->launch_items = 16384;
    cfg->max_admit = 1024;
    cfg->small_work_log2 = 33;
    cfg->launch_budget = 1ull << 33;
    cfg->class_max_cols = PF3_CLASS_MAX_COLS;
}

static bool valid_config(const pf3_config& cfg)
{
    return !(cfg.max_jobs < 1 || cfg.max_jobs > (1 << 20) || cfg.queue_depth < 1 || cfg.chunk_log2 < 13 ||
             cfg.chunk_log2 > 62 || cfg.launch_items < 1 || cfg.max_admit < 1 || cfg.launch_budget < 1 ||
             cfg.small_work_log2 < 0 || cfg.small_work_log2 > 64 || cfg.class_max_cols < 0 ||
             cfg.class_max_cols > PF3_CLASS_MAX_COLS);
}

int pf3_serve_plan(const int32_t* ns, const int32_t* ms, int64_t count, const pf3_config* cfg_in, const int* U,
                   int launches, pf3_serve_item* items, int64_t capacity, int64_t* num_items)
{
    if (count < 0 || (count > 0 && !ns) || !U || launches < 1 || !num_items || capacity < 0) return PF3_EINVAL;
    pf3_config cfg;
    pf3_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (!valid_config(cfg)) return PF3_EINVAL;
    if (U[0] < 1 || U[0] > 20 || U[1] < 1 || U[1] > 20) return PF3_EINVAL;
    std::vector<Job> jobs((size_t)count);
    std::vector<int64_t> active;
    for (int64_t k = 0; k < count; ++k) {
        const int n = ns[k], m = ms ? ms[k] : n;
        if (n < 1 || n > PF3_MAX_N || m < 1 || m > n) return PF3_EINVAL;
        Job& j = jobs[(size_t)k];
        j.n = n;
        j.m = m;
        j.slot = (int)k;
        j.by_class = m < n && n > 32 && m <= cfg.class_max_cols;
        plan_job_items(j, cfg, U);
        if (!j.by_class) active.push_back(k);
    }
    std::vector<pf3_serve_item> out;
    for (int l = 0; l < launches && !active.empty(); ++l) {
        std::vector<WorkItem> cls_items[2], all;
        std::vector<int64_t> finishing;
        select_items(jobs, active, cfg, U, cls_items, finishing, &all);
        for (const WorkItem& it : all) {
            const Job& j = jobs[(size_t)it.mat];
            pf3_serve_item o;
            o.request = it.mat;
            o.launch = l;
            o.cls = j.m <= 32 ? 0 : 1;
            o.first_block = it.B0;
            o.num_blocks = it.NB;
            o.block_log2 = U[o.cls];
            o.last = (j.nb == 0 || it.B0 + it.NB == j.nb) ? 1 : 0;
            out.push_back(o);
        }
    }
    *num_items = (int64_t)out.size();
    if (!items) return PF3_OK;
    if (capacity < (int64_t)out.size()) return PF3_ETOOBIG;  // nothing written
    std::copy(out.begin(), out.end(), items);
    return PF3_OK;
}

int pf3_create(pf3_ctx** out, const pf3_config* cfg_in)
{
    if (!out) return PF3_EINVAL;
    pf3_config cfg;
    pf3_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (!valid_config(cfg)) return PF3_EINVAL;
    int rc;
    DeviceCtx* dc = device_ctx(&rc);
    if (!dc) return rc;
    pf3_ctx* x = new pf3_ctx();
    x->cfg = cfg;
    x->dc = dc;
    x->device = dc->device;
    for (int cls = 0; cls < 2; ++cls) {
        x->variant[cls] = dc->tune.variant[cls];
        x->U[cls] = kBatchVariants[x->variant[cls]].U;
        x->grid[cls] = dc->sm_count * batch_ctas(dc, cls + 1, x->variant[cls]);
    }
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        ok = ok && cudaStreamCreateWithFlags(&x->streams[b], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&x->kdone[b], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&x->d_mats, (size_t)cfg.max_jobs * kSlotBytes) == cudaSuccess;
    ok = ok && cudaMalloc(&x->d_acc, (size_t)cfg.max_jobs * 2 * sizeof(unsigned long long)) == cudaSuccess;
    ok = ok && cudaMalloc(&x->d_left, (size_t)cfg.max_jobs * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMalloc(&x->d_results, (size_t)cfg.max_jobs) == cudaSuccess;
    ok = ok && cudaMalloc(&x->d_cursor, 4 * sizeof(unsigned)) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b) {
        ok = ok && cudaMalloc(&x->d_stage[b], (size_t)cfg.max_admit * kSlotBytes) == cudaSuccess;
        ok = ok && cudaMalloc(&x->d_table[b], table_bytes(cfg)) == cudaSuccess;
        ok = ok && cudaMallocHost(&x->h_stage[b], (size_t)cfg.max_admit * kSlotBytes) == cudaSuccess;
        ok = ok && cudaMallocHost(&x->h_table[b], table_bytes(cfg)) == cudaSuccess;
        ok = ok && cudaMallocHost(&x->h_results[b], (size_t)cfg.max_jobs) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&x->ev[b], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaMemset(x->d_results, kPending, (size_t)cfg.max_jobs) == cudaSuccess;
    // both "kernels done" events start recorded (complete), so the first
    // launch's wait on the other buffer's event is well defined
    for (int b = 0; b < 2 && ok; ++b) ok = cudaEventRecord(x->kdone[b], x->streams[b]) == cudaSuccess;
    ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pf3_destroy(x);
        return PF3_ENOMEM;
    }
    for (int b = 0; b < 2; ++b) {
        if ((rc = build_graph(x, b))) {
            cudaGetLastError();
            pf3_destroy(x);
            return rc;
        }
    }
    x->free_slots.reserve(cfg.max_jobs);
    for (int sl = cfg.max_jobs - 1; sl >= 0; --sl) x->free_slots.push_back(sl);
    x->th = std::thread(scheduler, x);
    *out = x;
    return PF3_OK;
}

void pf3_destroy(pf3_ctx* x)
{
    if (!x) return;
    if (x->th.joinable()) {
        {
            std::lock_guard<std::mutex> g(x->mu);
            x->stop = true;
            // requests not yet admitted are cancelled; admitted ones finish
            for (int64_t tk : x->pending) {
                x->jobs[tk].state = kFailed;
                x->jobs[tk].error = PF3_ECANCELED;
            }
            x->pending.clear();
            x->cv_work.notify_all();
            x->cv_done.notify_all();
        }
        x->th.join();
    }
    for (int b = 0; b < 2; ++b)
        if (x->streams[b]) cudaStreamSynchronize(x->streams[b]);
    cudaFree(x->d_mats);
    cudaFree(x->d_acc);
    cudaFree(x->d_left);
    cudaFree(x->d_results);
    cudaFree(x->d_cursor);
    for (int b = 0; b < 2; ++b) {
        cudaFree(x->d_stage[b]);
        cudaFree(x->d_table[b]);
        cudaFreeHost(x->h_stage[b]);
        cudaFreeHost(x->h_table[b]);
        cudaFreeHost(x->h_results[b]);
        if (x->ev[b]) cudaEventDestroy(x->ev[b]);
    }
    for (int b = 0; b < 2; ++b) {
        if (x->gexec[b]) cudaGraphExecDestroy(x->gexec[b]);
        if (x->graph[b]) cudaGraphDestroy(x->graph[b]);
    }
    for (int b = 0; b < 2; ++b) {
        if (x->kdone[b]) cudaEventDestroy(x->kdone[b]);
        if (x->streams[b]) cudaStreamDestroy(x->streams[b]);
    }
    delete x;
}

int pf3_cancel_queued(pf3_ctx* x)
{
    if (!x) return PF3_EINVAL;
    std::lock_guard<std::mutex> g(x->mu);
    int cnt = 0;
    for (int64_t tk : x->pending) {
        x->jobs[tk].state = kFailed;
        x->jobs[tk].error = PF3_ECANCELED;
        x->jobs[tk].t_done = now_ns();
        ++cnt;
    }
    x->pending.clear();
    x->cv_done.notify_all();
    return cnt;
}

int64_t perm_f3_submit(pf3_ctx* x, const uint8_t* A, int n)
{
    if (!x || n < 0 || n > PF3_MAX_N || (n > 0 && !A)) return PF3_EINVAL;
    for (int k = 0; k < n * n; ++k)
        if (A[k] > 2) return PF3_EDOMAIN;
    std::lock_guard<std::mutex> g(x->mu);
    if (x->stop) return PF3_ECANCELED;
    if (x->fatal) return x->fatal;
    if ((int64_t)x->pending.size() >= x->cfg.queue_depth) return PF3_EBUSY;
    const int64_t tk = (int64_t)x->jobs.size();
    x->jobs.emplace_back();
    Job& j = x->jobs.back();
    j.n = n;
    j.t_submit = now_ns();
    if (n == 0) {
        j.state = kDone;
        j.result = 1;
        j.t_done = j.t_submit;
        ++x->done;
        x->cv_done.notify_all();
        return tk;
    }
    // equal columns merged as for perm_f3 (pf3_capi.cu): one plane word
    // instead of two for requests whose terms are mostly nonzero
    std::vector<uint8_t> B;
    if (merge_columns(A, n, B, j.m, j.negate)) {
        j.A.swap(B);
        // few columns left: counted by column-sum vector (pf3_classes.cu)
        j.by_class = j.m <= x->cfg.class_max_cols;
    } else {
        j.m = n;
        j.A.assign(A, A + (size_t)n * n);
    }
    x->pending.push_back(tk);
    x->cv_work.notify_one();
    return tk;
}

int perm_f3_poll(pf3_ctx* x, int64_t ticket, uint8_t* result)
{
    if (!x) return PF3_EINVAL;
    std::lock_guard<std::mutex> g(x->mu);
    if (ticket < 0 || ticket >= (int64_t)x->jobs.size()) return PF3_EINVAL;
    const Job& j = x->jobs[ticket];
    if (j.state == kDone) {
        if (result) *result = (uint8_t)j.result;
        return PF3_OK;
    }
    if (j.state == kFailed) return j.error;
    return PF3_PENDING;
}

int perm_f3_wait(pf3_ctx* x, int64_t ticket, uint8_t* result, int64_t timeout_us)
{
    if (!x) return PF3_EINVAL;
    std::unique_lock<std::mutex> lk(x->mu);
    if (ticket < 0 || ticket >= (int64_t)x->jobs.size()) return PF3_EINVAL;
    auto ready = [&] { return x->jobs[ticket].state >= kDone; };
    if (timeout_us < 0) {
        x->cv_done.wait(lk, ready);
    } else if (!x->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return PF3_ETIMEDOUT;
    }
    const Job& j = x->jobs[ticket];
    if (j.state == kFailed) return j.error;
    if (result) *result = (uint8_t)j.result;
    return PF3_OK;
}

int pf3_job_times(pf3_ctx* x, int64_t ticket, uint64_t* submit_ns, uint64_t* done_ns)
{
    if (!x) return PF3_EINVAL;
    std::lock_guard<std::mutex> g(x->mu);
    if (ticket < 0 || ticket >= (int64_t)x->jobs.size()) return PF3_EINVAL;
    const Job& j = x->jobs[ticket];
    if (submit_ns) *submit_ns = j.t_submit;
    if (done_ns) *done_ns = j.t_done;
    return j.state >= kDone ? PF3_OK : PF3_PENDING;
}

int pf3_serve_stats(pf3_ctx* x, uint64_t* launches, uint64_t* items, uint64_t* jobs_done)
{
    if (!x) return PF3_EINVAL;
    std::lock_guard<std::mutex> g(x->mu);
    if (launches) *launches = x->launches;
    if (items) *items = x->items;
    if (jobs_done) *jobs_done = x->done;
    return PF3_OK;
}

uint64_t pf3_now_ns(void) { return now_ns(); }

}  // extern "C"
