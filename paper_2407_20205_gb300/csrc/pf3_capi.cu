// pf3_capi.cu -- the C ABI declared in include/perm_f3.h: argument checks,
// per-device contexts (stream, scratch, pinned staging) and the host side of
// the one-matrix entry points and diagnostics.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "perm_f3.h"
#include "pf3_context.h"
#include "pf3_internal.h"

namespace pf3 {

namespace {

std::mutex g_registry_mu;
std::vector<DeviceCtx*> g_ctx;  // indexed by device ordinal

}  // namespace

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return PF3_OK;
    if (e == cudaErrorMemoryAllocation) return PF3_ENOMEM;
    return PF3_ECUDA;
}

DeviceCtx* device_ctx(int* rc)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *rc = PF3_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> g(g_registry_mu);
    if ((int)g_ctx.size() <= dev) g_ctx.resize(dev + 1, nullptr);
    if (g_ctx[dev]) {
        *rc = PF3_OK;
        return g_ctx[dev];
    }
    DeviceCtx* c = new DeviceCtx();
    c->device = dev;
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) {
        delete c;
        *rc = cuda_rc(e);
        return nullptr;
    }
    c->sm_count = prop.multiProcessorCount;
    int most = 1;
    for (int W = 1; W <= 2; ++W)
        for (int v = 0; v < kNumSingleVariants; ++v) {
            c->single_ctas[W - 1][v] = single_max_ctas_per_sm(W, v);
            if (c->single_ctas[W - 1][v] > most) most = c->single_ctas[W - 1][v];
        }
    for (int W = 1; W <= 2; ++W)
        for (int v = 0; v < kNumBatchVariants; ++v) c->batch_ctas_cache[W - 1][v] = batch_max_ctas_per_sm(W, v);
    const int max_grid = c->sm_count * most;
    c->max_grid = max_grid;
    bool ok = true;
    ok = ok && cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMalloc(&c->d_A, kMaxNN) == cudaSuccess;
    ok = ok && cudaMalloc(&c->d_partials, sizeof(unsigned long long) * 2 * (size_t)max_grid) == cudaSuccess;
    ok = ok && cudaMalloc(&c->d_flags, sizeof(unsigned int) * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&c->d_out, sizeof(unsigned long long) * 4) == cudaSuccess;
    ok = ok && cudaMemset(c->d_flags, 0, sizeof(unsigned int) * 4) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->scratch_free, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->bgraph_free, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->h_A, kMaxNN) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->h_out, sizeof(unsigned long long) * 4) == cudaSuccess;
    ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        *rc = PF3_ENOMEM;
        cudaGetLastError();
        return nullptr;  // leaked partially built context on failure: rare, harmless
    }
    load_tune_cache(c);
    g_ctx[dev] = c;
    *rc = PF3_OK;
    return c;
}

int scratch_acquire(cudaEvent_t ev, cudaStream_t stream, bool* capturing)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &st);
    if (e != cudaSuccess) return cuda_rc(e);
    *capturing = st != cudaStreamCaptureStatusNone;
    if (*capturing) return PF3_OK;
    return cuda_rc(cudaStreamWaitEvent(stream, ev, 0));
}

int scratch_release(cudaEvent_t ev, cudaStream_t stream, bool capturing)
{
    if (capturing) return PF3_OK;
    return cuda_rc(cudaEventRecord(ev, stream));
}

int single_ctas(DeviceCtx* c, int W, int v) { return c->single_ctas[W - 1][v]; }
int batch_ctas(DeviceCtx* c, int W, int v) { return c->batch_ctas_cache[W - 1][v]; }

int check_entries_host(const uint8_t* A, int n)
{
    const size_t nn = (size_t)n * (size_t)n;
    for (size_t k = 0; k < nn; ++k)
        if (A[k] > 2) return PF3_EDOMAIN;
    return PF3_OK;
}

// Columns equal up to a factor -1 (2 in F3).  Let column j be l_j times a
// canonical vector v_c(j) (first nonzero entry 1, l_j = +-1).  For every row
// subset S the column sum of j is l_j times that of v_c(j), so the product of
// Eq. (2)'s term is (prod_j l_j) * prod_c (sum over S of v_c)^mult_c, and in
// F3 x^mult is x for odd mult and x^2 (1 unless x = 0) for even mult: the same
// as one copy of v_c for odd and two copies for even multiplicity.  Walking
// the n-row matrix of those columns instead of A changes every term by the
// one factor prod_j l_j, so the +1/-1 counts are A's, swapped when that
// factor is -1.
// On true (the merged matrix has at most max_cols columns), B (n rows x m
// columns, row-major), m and negate describe it; on false nothing is written.
bool column_classes(const uint8_t* A, int n, int max_cols, std::vector<uint8_t>& B, int& m, bool& negate)
{
    // each class as its canonical vector packed into (nonzero bits, == 2 bits)
    uint64_t key_m[64], key_s[64];
    int mult[64] = {};
    int classes = 0;
    bool neg = false;
    for (int j = 0; j < n; ++j) {
        uint64_t km = 0, ks = 0;
        int first = -1;
        for (int i = 0; i < n; ++i) {
            const uint8_t e = A[(size_t)i * n + j];
            if (!e) continue;
            if (first < 0) first = i;
            km |= 1ull << i;
            if (e == 2) ks |= 1ull << i;
        }
        const bool flip = first >= 0 && ((ks >> first) & 1ull);
        if (flip) ks ^= km;  // times 2 = times -1 in F3: 1 <-> 2
        neg ^= flip;
        int k = 0;
        while (k < classes && (key_m[k] != km || key_s[k] != ks)) ++k;
        if (k == classes) {
            if (classes == max_cols) return false;  // m >= classes > max_cols
            key_m[k] = km;
            key_s[k] = ks;
            ++classes;
        }
        ++mult[k];
    }
    int cols = 0;
    for (int k = 0; k < classes; ++k) cols += (mult[k] & 1) ? 1 : 2;
    if (cols > max_cols) return false;
    B.assign((size_t)n * cols, 0);
    int col = 0;
    for (int k = 0; k < classes; ++k)
        for (int copy = 0; copy < ((mult[k] & 1) ? 1 : 2); ++copy, ++col)
            for (int i = 0; i < n; ++i)
                B[(size_t)i * cols + col] = ((key_m[k] >> i) & 1ull) ? (((key_s[k] >> i) & 1ull) ? 2 : 1) : 0;
    m = cols;
    negate = neg;
    return true;
}

// The merge the host-pointer calls apply before walking: worth it when the
// merged matrix fits one plane word and A does not (n > 32, m <= 32).
// Matrices with many equal columns are the ones whose terms are mostly nonzero
// (the dense walk), where the second word doubles the work per state.
bool merge_columns(const uint8_t* A, int n, std::vector<uint8_t>& B, int& m, bool& negate)
{
    return n > 32 && column_classes(A, n, 32, B, m, negate);
}

int enqueue_range(DeviceCtx* c, const uint8_t* dA, int n, int m, uint64_t first, uint64_t last,
                  unsigned long long* d_out, cudaStream_t stream)
{
    const int W = m <= 32 ? 1 : 2;
    const bool is_short = last - first < kShortLaunch - 1;
    // m < n only for a merged matrix, whose terms are mostly nonzero (the
    // dense walk): its long launches take the variant tuned for that
    const int v = is_short ? c->single_variant_short[W - 1]
                           : (m < n ? c->single_variant_merged : c->single_variant[W - 1]);
    SingleArgs a;
    std::memset(&a, 0, sizeof(a));
    plan_range(n, first, last, kSingleVariants[v].U, a);
    a.m = m;
    a.A = dA;
    a.partials = c->d_partials;
    a.ticket = c->d_flags;
    a.err = c->d_flags + 1;
    a.cursor = c->d_flags + 2;
    a.out = d_out;
    const int grid = single_grid_for(a, v, c->sm_count, single_ctas(c, W, v));
    // the partials and flags are shared by every call on this device
    bool capturing = false;
    int rc = scratch_acquire(c->scratch_free, stream, &capturing);
    if (rc) return rc;
    if ((rc = cuda_rc(launch_single(a, v, grid, stream)))) return rc;
    return scratch_release(c->scratch_free, stream, capturing);
}

uint64_t full_range_last(int n) { return n >= 64 ? ~0ull : (1ull << n) - 1; }

int valid_range(int n, uint64_t first, uint64_t last)
{
    if (n < 1 || n > PF3_MAX_N || first > last) return PF3_EINVAL;
    if (n < 64 && last >= (1ull << n)) return PF3_EINVAL;
    return PF3_OK;
}

// host-pointer range counts, synchronous; returns the result byte in *result
int host_range(const uint8_t* A, int n, uint64_t first, uint64_t last, uint64_t* plus, uint64_t* minus, int* result)
{
    int rc = valid_range(n, first, last);
    if (rc) return rc;
    if (!A) return PF3_EINVAL;
    if ((rc = check_entries_host(A, n))) return rc;
    std::vector<uint8_t> B;
    int m = n;
    bool negate = false;
    const bool merged = merge_columns(A, n, B, m, negate);
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    // a whole range of a narrow merged matrix: counted by column-sum vector
    const bool by_class = merged && m <= c->class_max_cols && first == 0 && last == full_range_last(n);
    const size_t bytes = (size_t)n * m;
    std::memcpy(c->h_A, merged ? B.data() : A, bytes);
    cudaError_t e = cudaMemcpyAsync(c->d_A, c->h_A, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    rc = by_class ? enqueue_class_counts(c->d_A, n, m, c->d_out, c->stream)
                  : enqueue_range(c, c->d_A, n, m, first, last, c->d_out, c->stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(c->h_out, c->d_out, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_rc(e);
    if (c->h_out[2] == ~0ull) return PF3_EDOMAIN;
    const unsigned long long P = negate ? c->h_out[1] : c->h_out[0];
    const unsigned long long M = negate ? c->h_out[0] : c->h_out[1];
    if (plus) *plus = P;
    if (minus) *minus = M;
    if (result) *result = (int)perm_from_counts(n, P, M);
    return PF3_OK;
}

}  // namespace pf3

using namespace pf3;

extern "C" {

const char* pf3_strerror(int code)
{
    switch (code) {
    case PF3_OK: return "ok";
    case PF3_PENDING: return "pending";
    case PF3_EINVAL: return "invalid argument";
    case PF3_EDOMAIN: return "matrix entry outside {0,1,2}";
    case PF3_ECUDA: return "CUDA error";
    case PF3_ENOMEM: return "out of memory";
    case PF3_ETIMEDOUT: return "timed out";
    case PF3_ECANCELED: return "cancelled";
    case PF3_EBUSY: return "queue full";
    case PF3_ETOOBIG: return "more CTAs requested than the no-allocation scratch holds";
    default: return "unknown error";
    }
}

const char* pf3_version(void) { return "perm_f3 1.0 (sm_103a)"; }

int perm_f3(const uint8_t* A, int n)
{
    if (n < 0 || n > PF3_MAX_N) return PF3_EINVAL;
    if (n == 0) return 1;
    const uint64_t last = (n == 64) ? ~0ull : ((1ull << n) - 1);
    int result = 0;
    const int rc = host_range(A, n, 0, last, nullptr, nullptr, &result);
    return rc ? rc : result;
}

int pf3_perm_from_counts(int n, uint64_t plus, uint64_t minus)
{
    if (n < 0 || n > PF3_MAX_N) return PF3_EINVAL;
    return (int)perm_from_counts(n, plus, minus);
}

int perm_f3_counts(const uint8_t* A, int n, uint64_t* plus, uint64_t* minus)
{
    if (!plus || !minus || n < 0 || n > PF3_MAX_N) return PF3_EINVAL;
    if (n == 0) {
        *plus = 1;
        *minus = 0;
        return PF3_OK;
    }
    const uint64_t last = (n == 64) ? ~0ull : ((1ull << n) - 1);
    return host_range(A, n, 0, last, plus, minus, nullptr);
}

int perm_f3_range_counts(const uint8_t* A, int n, uint64_t first, uint64_t last, uint64_t* plus, uint64_t* minus)
{
    if (!plus || !minus) return PF3_EINVAL;
    return host_range(A, n, first, last, plus, minus, nullptr);
}

int perm_f3_range_counts_async(const uint8_t* dA, int n, uint64_t first, uint64_t last, uint64_t* d_out,
                               void* stream)
{
    int rc = valid_range(n, first, last);
    if (rc) return rc;
    if (!dA || !d_out) return PF3_EINVAL;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    return enqueue_range(c, dA, n, n, first, last, (unsigned long long*)d_out, (cudaStream_t)stream);
}

int pf3_column_merge(const uint8_t* A, int n, uint8_t* B, int* m, int* negate)
{
    if (!A || !B || !m || !negate || n < 1 || n > PF3_MAX_N) return PF3_EINVAL;
    int rc = check_entries_host(A, n);
    if (rc) return rc;
    std::vector<uint8_t> buf;
    int mm = n;
    bool neg = false;
    if (!merge_columns(A, n, buf, mm, neg)) return 0;  // nothing written
    std::memcpy(B, buf.data(), buf.size());
    *m = mm;
    *negate = neg ? 1 : 0;
    return 1;
}

int pf3_class_counts(const uint8_t* A, int n, uint64_t* plus, uint64_t* minus)
{
    if (!A || !plus || !minus || n < 1 || n > PF3_MAX_N) return PF3_EINVAL;
    int rc = check_entries_host(A, n);
    if (rc) return rc;
    std::vector<uint8_t> B;
    int m = n;
    bool negate = false;
    if (!column_classes(A, n, PF3_CLASS_MAX_COLS, B, m, negate)) return 0;  // nothing written
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    std::memcpy(c->h_A, B.data(), B.size());
    cudaError_t e = cudaMemcpyAsync(c->d_A, c->h_A, B.size(), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    if ((rc = enqueue_class_counts(c->d_A, n, m, c->d_out, c->stream))) return rc;
    e = cudaMemcpyAsync(c->h_out, c->d_out, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    if (c->h_out[2] == ~0ull) return PF3_EDOMAIN;
    *plus = negate ? c->h_out[1] : c->h_out[0];
    *minus = negate ? c->h_out[0] : c->h_out[1];
    return 1;
}

int pf3_set_class_limit(int max_cols)
{
    if (max_cols < 0 || max_cols > PF3_CLASS_MAX_COLS) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    c->class_max_cols = max_cols;
    return PF3_OK;
}

int pf3_get_class_limit(void)
{
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    return c->class_max_cols;
}

int pf3_step_table(uint32_t* out)
{
    if (!out) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    uint32_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 48 * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_rc(e);
    e = launch_step_table(d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, 48 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    return cuda_rc(e);
}

int pf3_pack(const uint8_t* A, int n, uint64_t* mag, uint64_t* sgn)
{
    if (n < 1 || n > PF3_MAX_N || !A || !mag || !sgn) return PF3_EINVAL;
    int rc = check_entries_host(A, n);
    if (rc) return rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long) * 2 * PF3_MAX_N);
    if (e != cudaSuccess) return cuda_rc(e);
    const size_t nn = (size_t)n * n;
    std::memcpy(c->h_A, A, nn);
    bool capturing = false;
    if ((rc = scratch_acquire(c->scratch_free, c->stream, &capturing))) {
        cudaFree(d);
        return rc;
    }
    e = cudaMemcpyAsync(c->d_A, c->h_A, nn, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_pack(c->d_A, n, d, d + PF3_MAX_N, c->d_flags + 1, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mag, d, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sgn, d + PF3_MAX_N, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flags + 1, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->scratch_free, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    return cuda_rc(e);
}

int pf3_intpipe_bench(int kind, int ctas_per_sm, int threads, int iters, double* inst_per_clk_per_sm,
                      double* inst_per_s, double* sm_mhz)
{
    static const int per_op[14] = {1, 1, 1, 2, 4, 3, 2, 3, 3, 4, 3, 3, 3, 3};
    if (kind < 0 || kind > 13 || ctas_per_sm < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1)
        return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    const int grid = c->sm_count * ctas_per_sm;
    uint32_t* sink = nullptr;
    unsigned long long* cyc = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(uint32_t) * (size_t)grid * threads);
    if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(unsigned long long) * grid);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    // warm-up launch, then the timed one
    if (e == cudaSuccess) e = launch_intpipe(kind, grid, threads, iters / 8 + 1, sink, cyc, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, c->stream);
    if (e == cudaSuccess) e = launch_intpipe(kind, grid, threads, iters, sink, cyc, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    float ms = 0.f;
    std::vector<unsigned long long> h(grid);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * grid, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        // ops per thread: iters * unroll(16) * chains(8) * instructions per op
        const double ops_thread = (double)iters * 16.0 * 8.0 * per_op[kind];
        double maxc = 0, sumc = 0;
        for (int b = 0; b < grid; ++b) {
            sumc += (double)h[b];
            if ((double)h[b] > maxc) maxc = (double)h[b];
        }
        const double avgc = sumc / grid;
        const double per_sm = ops_thread * threads * ctas_per_sm / avgc;
        if (inst_per_clk_per_sm) *inst_per_clk_per_sm = per_sm;
        if (inst_per_s) *inst_per_s = ops_thread * threads * (double)grid / (ms * 1e-3);
        if (sm_mhz) *sm_mhz = maxc / (ms * 1e-3) / 1e6;
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaFree(sink);
    cudaFree(cyc);
    return cuda_rc(e);
}

int pf3_device_info(int* sm_count, int* device)
{
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    if (sm_count) *sm_count = c->sm_count;
    if (device) *device = c->device;
    return PF3_OK;
}

}  // extern "C"
