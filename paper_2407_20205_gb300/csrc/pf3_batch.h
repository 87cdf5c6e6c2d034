// pf3_batch.h -- work items and plans of the persistent batch kernel (host and
// device side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace pf3 {

constexpr int kBatchThreads = 128;  // 4 warps, one instance per warp
constexpr int kTinyN = 10;          // n <= kTinyN: one matrix per lane (32 per item)
constexpr int kTinyItem = -2;       // WorkItem.split of a group of tiny matrices

// One unit of batch work: Gray blocks [B0, B0 + NB) of matrix `mat` (block =
// 2^U indices); NB == 0 means "all 2^n indices, walked by one lane" (n <= U).
// A tiny item (split == kTinyItem) is NB <= 32 consecutive matrices of the
// same n <= kTinyN starting at `mat` / `offset`: lane k walks matrix mat + k.
struct WorkItem {
    long long offset;         // byte offset of the matrix in the batch buffer
    unsigned long long B0;
    unsigned long long NB;
    int mat;                  // matrix index (result slot)
    int n;
    int split;                // -1: the item is the whole matrix; else split slot
    int pad;
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
struct BatchTuning {
    int cutoff = 28;       // n above which a matrix is split over several items
    int chunk_log2 = 26;   // Gray indices per split item (log2)
    int variant[2] = {0, 0};  // batch kernel variant for W = 1 and W = 2
};

struct BatchPlan {
    std::vector<WorkItem> items[2];      // by class: n <= 32, n > 32
    std::vector<unsigned> split_items;   // items per split matrix
    int num_split = 0;
    long long total_bytes = 0;
};

// A job admitted into a serving slot: copy its matrix from the staging buffer
// into the slot and reset the slot's counters.
struct SlotInit {
    long long src;        // byte offset in the device staging buffer
    int slot;
    int n;
    unsigned items;       // work items the job will run in total
    unsigned pad;
};

void plan_batch(const int32_t* ns, int64_t count, const BatchTuning& tune, BatchPlan& plan);
cudaError_t launch_slot_init(const SlotInit* inits, int count, const uint8_t* staging, uint8_t* mats,
                             int slot_bytes, unsigned long long* acc, unsigned* left, uint8_t* results,
                             cudaStream_t stream);
int batch_max_ctas_per_sm(int W, int v);
cudaError_t launch_batch(int W, int v, const BatchArgs& a, int grid, cudaStream_t stream);

}  // namespace pf3
