// pf3_classes.cu -- Ryser counts of a matrix with few columns, by column-sum
// vector.
//
// Eq. (2)'s term for a row subset S depends on S only through two things: the
// vector of column sums sum_{i in S} B_i, a point w of F3^m, and the parity p
// of |S| (the sign (-1)^{|S|}).  For a matrix of m columns the 2^n subsets
// therefore fall on at most 2 * 3^m pairs (w, p), and the number of subsets
// on each pair follows one row at a time: the subsets of rows 0..i are those
// of rows 0..i-1 without row i (pair unchanged) and with it (pair moved to
// (w + B_i, 1 - p)).  After the n rows the +1 and -1 counts are read off the
// pairs whose m sums are all nonzero: the term there is (-1)^p times
// (-1)^{number of sums equal to -1}.  Every subset is counted once, by its own
// term, so the counts are exactly those of the Gray walk over the same matrix
// (Sec. 3); only the order of summation differs.  The work is n * 3^m table
// updates instead of 2^n walk states, which wins by far for the matrices whose
// equal columns merge into a handful (J_n merges into one or two columns).
//
// One CTA owns the table (2 * 3^m counters of 64 bits in shared memory,
// m <= PF3_CLASS_MAX_COLS).  Row i splits F3^m into orbits {w, w + B_i,
// w + 2 B_i} of three points (one point when B_i = 0); a thread updates a
// whole orbit in place, so the table needs no second copy.
#include <cuda_runtime.h>

#include <cstdint>

#include "perm_f3.h"
#include "pf3_batch.h"
#include "pf3_context.h"
#include "pf3_internal.h"

namespace pf3 {

namespace {

constexpr int kClassThreads = 1024;
constexpr int kClassMaxN = 64;

__host__ __device__ constexpr int pow3(int m) { return m <= 0 ? 1 : 3 * pow3(m - 1); }

// w + a in F3^m, w as a base-3 index (digit j of weight 3^j, digit 2 = -1)
__device__ __forceinline__ int add_point(int w, const int (&a)[PF3_CLASS_MAX_COLS], int m)
{
    int r = 0, weight = 1;
#pragma unroll
    for (int j = 0; j < PF3_CLASS_MAX_COLS; ++j) {
        if (j < m) {
            const int d = w % 3 + a[j];
            w /= 3;
            r += (d >= 3 ? d - 3 : d) * weight;
            weight *= 3;
        }
    }
    return r;
}

__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = 0;
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    }
    __syncthreads();
    return v;  // the total in thread 0
}

// Counts of +1 and -1 terms of the n x m matrix B (row-major, entries {0,1,2},
// 1 <= m <= PF3_CLASS_MAX_COLS, 1 <= n <= 64) by the whole CTA; tbl holds
// 2 * 3^m counters (even / odd |S| for each point).  P and M are valid in
// thread 0; bad (an entry above 2) in every thread.
__device__ void class_counts_block(const uint8_t* B, int n, int m, unsigned long long* tbl,
                                   unsigned long long& P, unsigned long long& M, bool& bad)
{
    __shared__ uint8_t rows[kClassMaxN * PF3_CLASS_MAX_COLS];
    __shared__ unsigned long long red[32];
    const int K = pow3(m);
    const int tid = threadIdx.x, nt = blockDim.x;
    int b = 0;
    for (int k = tid; k < n * m; k += nt) {
        const uint8_t e = B[k];
        b |= e > 2;
        rows[k] = e;
    }
    // the empty subset: the zero point, even size
    for (int k = tid; k < 2 * K; k += nt) tbl[k] = k == 0 ? 1ull : 0ull;
    bad = __syncthreads_or(b) != 0;
    P = M = 0;
    if (bad) return;
    for (int i = 0; i < n; ++i) {
        int a[PF3_CLASS_MAX_COLS];
        int lead = -1;  // first nonzero entry of row i
#pragma unroll
        for (int j = 0; j < PF3_CLASS_MAX_COLS; ++j) {
            a[j] = j < m ? rows[i * m + j] : 0;
            if (lead < 0 && a[j]) lead = j;
        }
        if (lead < 0) {
            // row i adds nothing: (w, p) and (w, 1 - p) exchange their subsets
            for (int w = tid; w < K; w += nt) {
                const unsigned long long s = tbl[2 * w] + tbl[2 * w + 1];
                tbl[2 * w] = s;
                tbl[2 * w + 1] = s;
            }
        } else {
            // orbit representatives: the points whose digit `lead` is 0
            int low = 1;
            for (int j = 0; j < lead; ++j) low *= 3;
            for (int r = tid; r < K / 3; r += nt) {
                const int w0 = (r / low) * (3 * low) + r % low;
                const int w1 = add_point(w0, a, m), w2 = add_point(w1, a, m);
                const unsigned long long e0 = tbl[2 * w0], o0 = tbl[2 * w0 + 1];
                const unsigned long long e1 = tbl[2 * w1], o1 = tbl[2 * w1 + 1];
                const unsigned long long e2 = tbl[2 * w2], o2 = tbl[2 * w2 + 1];
                // new (w, p) = old (w, p) + old (w - a, 1 - p); w0 - a = w2
                tbl[2 * w0] = e0 + o2;
                tbl[2 * w0 + 1] = o0 + e2;
                tbl[2 * w1] = e1 + o0;
                tbl[2 * w1 + 1] = o1 + e0;
                tbl[2 * w2] = e2 + o1;
                tbl[2 * w2 + 1] = o2 + e1;
            }
        }
        __syncthreads();
    }
    unsigned long long p = 0, q = 0;
    for (int w = tid; w < K; w += nt) {
        int t = w, neg = 0;
        bool nonzero = true;
        for (int j = 0; j < m; ++j) {
            const int d = t % 3;
            t /= 3;
            nonzero &= d != 0;
            neg ^= d == 2;
        }
        if (!nonzero) continue;
        // term of (w, p): (-1)^p * (-1)^neg
        p += neg ? tbl[2 * w + 1] : tbl[2 * w];
        q += neg ? tbl[2 * w] : tbl[2 * w + 1];
    }
    P = block_sum(p, red);
    M = block_sum(q, red);
}

// out: plus, minus, then perm mod 3 from those counts (~0 on an entry above 2)
__global__ void __launch_bounds__(kClassThreads, 1)
    class_count_kernel(const uint8_t* B, int n, int m, unsigned long long* out)
{
    extern __shared__ unsigned long long tbl[];
    unsigned long long P, M;
    bool bad;
    class_counts_block(B, n, m, tbl, P, M, bad);
    if (threadIdx.x == 0) {
        out[0] = bad ? 0ull : P;
        out[1] = bad ? 0ull : M;
        out[2] = bad ? ~0ull : (unsigned long long)perm_from_counts(n, P, M);
    }
}

// Serving: CTA k counts the job of inits[k] when it has no work items (the
// scheduler's mark for a job counted here) and finishes it as the batch
// kernel's last item would: counts into its accumulators, no items left, the
// result byte written.
__global__ void __launch_bounds__(kClassThreads, 1)
    class_slots_kernel(const SlotInit* inits, int count, const uint8_t* mats, int slot_bytes,
                       unsigned long long* acc, unsigned* left, uint8_t* results)
{
    extern __shared__ unsigned long long tbl[];
    const int k = blockIdx.x;
    if (k >= count) return;
    const SlotInit in = inits[k];
    if (in.items != 0 || in.cols == 0 || in.cols > PF3_CLASS_MAX_COLS) return;
    unsigned long long P, M;
    bool bad;
    class_counts_block(mats + (size_t)in.slot * slot_bytes, in.n, (int)in.cols, tbl, P, M, bad);
    if (threadIdx.x == 0) {
        acc[2 * in.slot] = P;
        acc[2 * in.slot + 1] = M;
        left[in.slot] = 0;
        results[in.slot] = bad ? 255u : (uint8_t)perm_from_counts(in.n, P, M);
    }
}

cudaError_t allow_table_smem(const void* fn)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)class_table_bytes(PF3_CLASS_MAX_COLS));
}

}  // namespace

size_t class_table_bytes(int m) { return 2 * sizeof(unsigned long long) * (size_t)pow3(m); }

int enqueue_class_counts(const uint8_t* dB, int n, int m, unsigned long long* d_out, cudaStream_t stream)
{
    if (n < 1 || n > kClassMaxN || m < 1 || m > PF3_CLASS_MAX_COLS) return PF3_EINVAL;
    cudaError_t e = allow_table_smem((const void*)class_count_kernel);
    if (e == cudaSuccess) {
        class_count_kernel<<<1, kClassThreads, class_table_bytes(m), stream>>>(dB, n, m, d_out);
        e = cudaGetLastError();
    }
    return cuda_rc(e);
}

const void* class_slots_fn(int* threads, size_t* smem)
{
    if (allow_table_smem((const void*)class_slots_kernel) != cudaSuccess) return nullptr;
    *threads = kClassThreads;
    *smem = class_table_bytes(PF3_CLASS_MAX_COLS);
    return (const void*)class_slots_kernel;
}

}  // namespace pf3
