// pf3_context.h -- per-device library state (host side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "perm_f3.h"
#include "pf3_batch.h"
#include "pf3_internal.h"

namespace pf3 {

constexpr int kMaxNN = 64 * 64;

// Batch scratch (grown on demand): the work-item table and per-matrix state.
struct BatchScratch {
    void* d_items = nullptr;              // WorkItem[items_cap]
    unsigned long long* d_acc = nullptr;  // 2 per matrix: plus, minus
    unsigned int* d_left = nullptr;       // work items left per matrix
    long long* d_offsets = nullptr;       // byte offset of each matrix
    int* d_ns = nullptr;                  // n of each matrix
    unsigned int* d_cursor = nullptr;     // 2 queue cursors (W = 1, W = 2)
    uint8_t* d_As = nullptr;              // staging for host-pointer batches
    uint8_t* d_results = nullptr;         // staging for host-pointer batches
    unsigned long long* d_hist = nullptr; // staging for host-pointer batches
    size_t items_cap = 0, mats_cap = 0, bytes_cap = 0, res_cap = 0;
    void* h_items = nullptr;              // pinned mirror of the item table
    size_t h_items_cap = 0;
};

// The launch sequence of the last device-pointer batch, captured as a CUDA
// graph and replayed while the plan (sizes, pointers, tuning) is unchanged.
struct BatchGraphCache {
    bool valid = false;
    std::vector<int32_t> ns;
    const uint8_t* dAs = nullptr;
    uint8_t* d_results = nullptr;
    unsigned long long* d_hist = nullptr;
    BatchTuning tune;
    int n_items[2] = {0, 0};
    int num_split = 0;
    void* h_items = nullptr;               // pinned, owned by the graph
    unsigned* h_left = nullptr;            // pinned, owned by the graph
    void* d_items = nullptr;
    unsigned long long* d_acc = nullptr;
    unsigned* d_left = nullptr;
    unsigned* d_cursor = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct DeviceCtx {
    int device = 0;
    int sm_count = 0;
    int single_variant[2] = {0, 0};        // tuned single-kernel variant for W = 1 / W = 2
    int single_variant_short[2] = {0, 0};  // the same for launches of fewer than kShortLaunch indices
    int single_variant_merged = 0;         // long launches of a matrix with merged columns (one word)
    int class_max_cols = PF3_CLASS_MAX_COLS;  // merged matrices this narrow are counted by class (0: never)
    int single_ctas[2][kMaxVariants] = {};  // resident CTAs per SM by W and variant (0 = not queried)
    int batch_ctas_cache[2][kMaxVariants] = {};
    int max_grid = 0;
    cudaStream_t stream = nullptr;
    // single-matrix scratch
    uint8_t* d_A = nullptr;                   // kMaxNN bytes
    unsigned long long* d_partials = nullptr; // 2 * max_grid
    unsigned int* d_flags = nullptr;          // ticket, error flag, chunk cursor (0 between launches)
    unsigned long long* d_out = nullptr;      // plus, minus, result
    uint8_t* h_A = nullptr;                   // pinned
    unsigned long long* h_out = nullptr;      // pinned
    // Recorded on the launching stream after every launch that uses
    // d_partials/d_flags; the next such launch, on whatever stream, waits for
    // it first, so calls on different streams never share the scratch at the
    // same time.  bgraph_free does the same for the captured batch graph's
    // buffers.
    cudaEvent_t scratch_free = nullptr;
    cudaEvent_t bgraph_free = nullptr;
    BatchScratch batch;
    BatchGraphCache bgraph;
    cudaStream_t capture_stream = nullptr;
    BatchTuning tune;
    std::mutex mu;
};

int cuda_rc(cudaError_t e);
DeviceCtx* device_ctx(int* rc);
// enqueue the single-matrix walk of Gray indices [first, last] of the device
// matrix dA (n rows of m columns; m = n unless equal columns were merged) on
// `stream`, results to d_out (plus, minus, perm mod 3)
int enqueue_range(DeviceCtx* c, const uint8_t* dA, int n, int m, uint64_t first, uint64_t last,
                  unsigned long long* d_out, cudaStream_t stream);
// the equal-column merge of the host-pointer calls (pf3_capi.cu): on true, B
// (n x m, row-major), m and negate describe the matrix to walk instead of A
bool merge_columns(const uint8_t* A, int n, std::vector<uint8_t>& B, int& m, bool& negate);
// the same merge for any n, on true when the merged matrix has at most
// max_cols columns
bool column_classes(const uint8_t* A, int n, int max_cols, std::vector<uint8_t>& B, int& m, bool& negate);
// Ryser counts of the whole range of the device matrix dB (n rows of m <=
// PF3_CLASS_MAX_COLS columns) by column-sum vector (pf3_classes.cu), to d_out
// as enqueue_range writes them; uses no scratch of the context
int enqueue_class_counts(const uint8_t* dB, int n, int m, unsigned long long* d_out, cudaStream_t stream);
size_t class_table_bytes(int m);
// the serving kernel that counts, one CTA each, the jobs of a launch's slot
// set-ups marked by items == 0 (args: const SlotInit* inits, int count, const
// uint8_t* mats, int slot_bytes, unsigned long long* acc, unsigned* left,
// uint8_t* results), with its block size and dynamic shared memory; nullptr
// on a CUDA error
const void* class_slots_fn(int* threads, size_t* smem);
// Order work on `stream` that uses the buffers guarded by `ev` after the
// previous user of those buffers (cudaStreamWaitEvent), and mark its end
// (cudaEventRecord).  Inside a stream capture both do nothing: ordering the
// captured work is then the capturing caller's job.
int scratch_acquire(cudaEvent_t ev, cudaStream_t stream, bool* capturing);
int scratch_release(cudaEvent_t ev, cudaStream_t stream, bool capturing);
int check_entries_host(const uint8_t* A, int n);
uint64_t full_range_last(int n);  // the last Gray index of an n-row walk
int single_ctas(DeviceCtx* c, int W, int v);
void load_tune_cache(DeviceCtx* c);
int batch_ctas(DeviceCtx* c, int W, int v);
struct BatchPlan;
int enqueue_batch(DeviceCtx* c, const BatchPlan& plan, const uint8_t* dAs, uint8_t* d_results,
                  unsigned long long* d_hist, cudaStream_t stream);

}  // namespace pf3
