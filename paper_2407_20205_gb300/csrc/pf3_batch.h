// pf3_batch.h -- work items and plans of the persistent batch kernel (host and
// device side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace pf3 {

constexpr int kBatchThreads = 128;  // 4 warps, one instance per warp
constexpr int kTinyMaxN = 16;       // largest n the one-matrix-per-lane path can hold
constexpr int kTinyItem = -2;       // WorkItem.split of a group of tiny matrices
constexpr int kMinChunkLog2 = 20;   // smallest automatic split item (2^20 Gray indices)

// One unit of batch work: Gray blocks [B0, B0 + NB) of matrix `mat` (block =
// 2^U indices); NB == 0 means "all 2^n indices, walked by one lane" (n <= U).
// A tiny item (split == kTinyItem) is NB <= 32 consecutive matrices of the
// same n <= tiny_cutoff starting at `mat` / `offset`: lane k walks matrix mat + k.
struct WorkItem {
    long long offset;         // byte offset of the matrix in the batch buffer
    unsigned long long B0;
    unsigned long long NB;
    int mat;                  // matrix index (result slot)
    int n;                    // rows
    int split;                // -1: the item is the whole matrix; else split slot
    int cols;                 // columns walked (0: n, a square matrix; fewer when equal columns were merged)
};

struct BatchArgs {
    const uint8_t* As;
    const WorkItem* items;
    unsigned num_items;
    unsigned* cursor;             // next item (0 at launch)
    unsigned long long* acc;      // 2 per split matrix, zero at launch
    unsigned* left;               // items left per split matrix (+ bad bit)
    uint8_t* results;
    unsigned long long* hist;     // 3 counters or null
};

// Tunables picked by the autotuner.
//  tiny_cutoff     packing cutoff: n <= tiny_cutoff is walked one matrix per
//                  lane, 32 matrices per warp (at most kTinyMaxN)
//  chunk_log2      > 0: matrices with n > cutoff are cut into items of
//                  2^chunk_log2 Gray indices;
//                  0: guided split (cutoff unused): the matrices of a class
//                  are taken largest first, and each is cut into pieces no
//                  longer than the work from it to the end of that order over
//                  (warps in the grid x items_per_warp), rounded down to a
//                  power of two and at least 2^kMinChunkLog2, so that the
//                  pieces handed out last are short and the warps finish
//                  together
//  items_per_warp  divisor of the guided split (more = shorter pieces, more
//                  warps, i.e. threads, sharing one matrix)
struct BatchTuning {
    int tiny_cutoff = 10;
    int cutoff = 28;
    int chunk_log2 = 0;
    int items_per_warp = 8;
    int variant[2] = {0, 0};  // batch kernel variant for W = 1 and W = 2
};

struct BatchPlan {
    std::vector<WorkItem> items[2];      // by class: n <= 32, n > 32
    std::vector<unsigned> split_items;   // items per split matrix
    int num_split = 0;
    long long total_bytes = 0;
    int chunk_log2[2] = {0, 0};          // split item length per class (log2)
};

// A job admitted into a serving slot: copy its matrix from the staging buffer
// into the slot and reset the slot's counters.
struct SlotInit {
    long long src;        // byte offset in the device staging buffer
    int slot;
    int n;                // rows
    unsigned items;       // work items the job will run in total
    unsigned cols;        // columns (0: n)
};

// warps[cls]: warps of the persistent grid of class cls (W = cls + 1); used
// by the automatic split only.
void plan_batch(const int32_t* ns, int64_t count, const BatchTuning& tune, const int warps[2], BatchPlan& plan);
// warps of the persistent grid of each class under the context's tuning
struct DeviceCtx;
void batch_warps(DeviceCtx* c, const BatchTuning& tune, int warps[2]);
cudaError_t launch_slot_init(const SlotInit* inits, int count, const uint8_t* staging, uint8_t* mats,
                             int slot_bytes, unsigned long long* acc, unsigned* left, uint8_t* results,
                             cudaStream_t stream);
int batch_max_ctas_per_sm(int W, int v);
// the kernels themselves, for graph nodes: variant v of the batch kernel for
// plane width W that reads each work item's column count (args: one
// BatchArgs; launch_batch runs the instance for square items), and the
// serving slot set-up kernel
// (args as launch_slot_init's, without the stream; 128 threads per CTA)
const void* batch_kernel_fn(int W, int v);
const void* slot_init_fn();
cudaError_t launch_batch(int W, int v, const BatchArgs& a, int grid, cudaStream_t stream);

}  // namespace pf3
