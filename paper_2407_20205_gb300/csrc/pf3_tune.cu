// pf3_tune.cu -- variant selection and the autotuner.
//
// Each walk kernel is compiled in a few variants (unrolled block length 2^U,
// register budget).  The autotuner times every variant of the single-matrix
// kernel and of the batch kernel on the current device, separately for one
// and two words per plane, and keeps the fastest.  It then picks the batch
// packing cutoff (up to which n matrices are walked one per lane, 32 per
// warp) by timing both walks per n, and the batch split granularity (split
// items per warp, which sets the item length and so how many warps share one
// matrix) on mixed-size batches.  Sample matrices come from fixed xorshift
// streams (uniform entries in {0,1,2}).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "perm_f3.h"
#include "pf3_batch.h"
#include "pf3_context.h"
#include "pf3_internal.h"

namespace pf3 {

namespace {

void sample_matrix(uint8_t* A, int n, uint64_t seed)
{
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
    for (int k = 0; k < n * n;) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        const unsigned v = (unsigned)(x >> 60) & 3u;
        if (v < 3) A[k++] = (uint8_t)v;
    }
}

// `bytes` uniform entries in {0,1,2} from one stream (any n x n slice of it
// is a uniform matrix)
void fill_uniform(uint8_t* out, size_t bytes, uint64_t seed)
{
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
    for (size_t k = 0; k < bytes;) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        for (int f = 0; f < 32 && k < bytes; ++f) {
            const unsigned v = (unsigned)(x >> (2 * f)) & 3u;
            if (v < 3) out[k++] = (uint8_t)v;
        }
    }
}

constexpr int kSplitCandidates = PF3_SPLIT_CANDIDATES;  // items per warp 1, 2, 4, 8, 16
// Another variant replaces the default (variant 0) only when it is at least
// 1 % faster: below that the timings are noise, and a stable choice keeps
// profiles and benchmarks of the default kernel meaningful.
constexpr float kVariantMargin = 0.99f;
static_assert(kTinyMaxN == PF3_TINY_MAX_N, "packing capacity");

// average milliseconds of `reps` launches of fn after one warm-up
template <class F>
float time_ms(cudaStream_t s, int reps, F fn)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fn();
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) fn();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}

}  // namespace

// Autotune cache: a text file named by the environment variable
// PF3_TUNE_CACHE, one line per GPU model:
//   <device name>|<SM count>|<single W=1>|<single W=2>|<batch W=1>|<batch W=2>|
//   <packing cutoff>|<split items per warp>|<short single W=1>|<short single W=2>
// (shorter lines from earlier versions set only the fields they hold).
static std::string tune_key(int device)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return std::string();
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == '|' || ch == '\n') ch = '_';
    return name + "|" + std::to_string(prop.multiProcessorCount);
}

void load_tune_cache(DeviceCtx* c)
{
    const char* path = std::getenv("PF3_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    const std::string key = tune_key(c->device);
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        std::string l(line);
        if (l.compare(0, key.size(), key) != 0 || l.size() <= key.size() || l[key.size()] != '|') continue;
        int v[9];
        const int got = std::sscanf(l.c_str() + key.size() + 1, "%d|%d|%d|%d|%d|%d|%d|%d|%d", &v[0], &v[1], &v[2],
                                    &v[3], &v[4], &v[5], &v[6], &v[7], &v[8]);
        if (got != 4 && got != 6 && got != 8 && got != 9) continue;
        if (v[0] < 0 || v[0] >= kNumSingleVariants || v[1] < 0 || v[1] >= kNumSingleVariants || v[2] < 0 ||
            v[2] >= kNumBatchVariants || v[3] < 0 || v[3] >= kNumBatchVariants)
            continue;
        if (got >= 6 && (v[4] < 0 || v[4] > kTinyMaxN || v[5] < 1 || v[5] > 1024)) continue;
        if (got >= 8 && (v[6] < 0 || v[6] >= kNumSingleVariants || v[7] < 0 || v[7] >= kNumSingleVariants)) continue;
        if (got == 9 && (v[8] < 0 || v[8] >= kNumSingleVariants)) continue;
        c->single_variant[0] = v[0];
        c->single_variant[1] = v[1];
        c->tune.variant[0] = v[2];
        c->tune.variant[1] = v[3];
        if (got >= 6) {
            c->tune.tiny_cutoff = v[4];
            c->tune.items_per_warp = v[5];
            c->tune.chunk_log2 = 0;
        }
        if (got >= 8) {
            c->single_variant_short[0] = v[6];
            c->single_variant_short[1] = v[7];
        }
        if (got == 9) c->single_variant_merged = v[8];
    }
    std::fclose(f);
}

static void store_tune_cache(DeviceCtx* c)
{
    const char* path = std::getenv("PF3_TUNE_CACHE");
    if (!path || !*path) return;
    const std::string key = tune_key(c->device);
    std::vector<std::string> keep;
    if (FILE* f = std::fopen(path, "r")) {
        char line[512];
        while (std::fgets(line, sizeof(line), f)) {
            std::string l(line);
            if (l.compare(0, key.size() + 1, key + "|") != 0) keep.push_back(l);
        }
        std::fclose(f);
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto& l : keep) std::fputs(l.c_str(), f);
    std::fprintf(f, "%s|%d|%d|%d|%d|%d|%d|%d|%d|%d\n", key.c_str(), c->single_variant[0], c->single_variant[1],
                 c->tune.variant[0], c->tune.variant[1], c->tune.tiny_cutoff, c->tune.items_per_warp,
                 c->single_variant_short[0], c->single_variant_short[1], c->single_variant_merged);
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

}  // namespace pf3

using namespace pf3;

extern "C" {

int pf3_variant_count(int which)
{
    if (which == 0 || which == 2 || which == 3) return kNumSingleVariants;
    if (which == 1) return kNumBatchVariants;
    return PF3_EINVAL;
}

int pf3_set_variant(int which, int W, int v)
{
    if (W < 1 || W > 2 || v < 0 || which < 0 || which > 3 || (which == 3 && W != 1)) return PF3_EINVAL;
    if (v >= (which == 1 ? kNumBatchVariants : kNumSingleVariants)) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    if (which == 0) c->single_variant[W - 1] = c->single_variant_short[W - 1] = v;
    else if (which == 2) c->single_variant_short[W - 1] = v;
    else if (which == 3) c->single_variant_merged = v;
    else c->tune.variant[W - 1] = v;
    return PF3_OK;
}

int pf3_variant_info(int which, int v, int* U, int* G, int* min_ctas)
{
    const KernelVariant* t = nullptr;
    if ((which == 0 || which == 2 || which == 3) && v >= 0 && v < kNumSingleVariants) t = &kSingleVariants[v];
    if (which == 1 && v >= 0 && v < kNumBatchVariants) t = &kBatchVariants[v];
    if (!t) return PF3_EINVAL;
    if (U) *U = t->U;
    if (G) *G = t->G;
    if (min_ctas) *min_ctas = t->min_ctas;
    return PF3_OK;
}

int pf3_variant_threads(int which, int v)
{
    if ((which == 0 || which == 2) && v >= 0 && v < kNumSingleVariants) return kSingleVariants[v].threads;
    if (which == 1 && v >= 0 && v < kNumBatchVariants) return kBatchVariants[v].threads;
    return PF3_EINVAL;
}

int pf3_get_variant(int which, int W)
{
    if (W < 1 || W > 2 || which < 0 || which > 3 || (which == 3 && W != 1)) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    if (which == 2) return c->single_variant_short[W - 1];
    if (which == 3) return c->single_variant_merged;
    return which == 0 ? c->single_variant[W - 1] : c->tune.variant[W - 1];
}

int pf3_set_batch_split(int cutoff, int chunk_log2)
{
    if (cutoff < 0 || cutoff > PF3_MAX_N || (chunk_log2 != 0 && (chunk_log2 < 12 || chunk_log2 > 62)))
        return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    c->tune.cutoff = cutoff;
    c->tune.chunk_log2 = chunk_log2;
    return PF3_OK;
}

int pf3_set_batch_tuning(int tiny_cutoff, int split_cutoff, int chunk_log2, int items_per_warp)
{
    if (tiny_cutoff < 0 || tiny_cutoff > kTinyMaxN || split_cutoff < 0 || split_cutoff > PF3_MAX_N ||
        (chunk_log2 != 0 && (chunk_log2 < 12 || chunk_log2 > 62)) || items_per_warp < 1 || items_per_warp > 1024)
        return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    c->tune.tiny_cutoff = tiny_cutoff;
    c->tune.cutoff = split_cutoff;
    c->tune.chunk_log2 = chunk_log2;
    c->tune.items_per_warp = items_per_warp;
    return PF3_OK;
}

int pf3_get_batch_tuning(int* tiny_cutoff, int* split_cutoff, int* chunk_log2, int* items_per_warp)
{
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    if (tiny_cutoff) *tiny_cutoff = c->tune.tiny_cutoff;
    if (split_cutoff) *split_cutoff = c->tune.cutoff;
    if (chunk_log2) *chunk_log2 = c->tune.chunk_log2;
    if (items_per_warp) *items_per_warp = c->tune.items_per_warp;
    return PF3_OK;
}

int pf3_autotune_ex(double* single_ms, double* single_short_ms, double* batch_ms, double* pack_ms,
                    double* split_ms)
{
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaStream_t s = c->stream;
    // ---- single-matrix kernel: n = 32 over 2^31 indices (fixed shares), n =
    // 40 over 2^36 (long enough for the guided chunks the benchmark sizes use)
    const int nW[2] = {32, 40};
    const int lgW[2] = {31, 36};
    uint8_t* dA = nullptr;
    unsigned long long* dout = nullptr;
    cudaError_t e = cudaMalloc(&dA, kMaxNN);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(dA);
        return cuda_rc(e);
    }
    std::vector<uint8_t> hA(kMaxNN);
    for (int W = 1; W <= 2; ++W) {
        const int n = nW[W - 1];
        sample_matrix(hA.data(), n, 1000 + n);
        cudaMemcpy(dA, hA.data(), (size_t)n * n, cudaMemcpyHostToDevice);
        float best = 1e30f;
        int bestv = 0;
        for (int v = 0; v < kNumSingleVariants; ++v) {
            c->single_variant[W - 1] = v;
            const float ms = time_ms(s, 2, [&] {
                enqueue_range(c, dA, n, n, 0, (1ull << lgW[W - 1]) - 1, dout, s);
            });
            if (single_ms) single_ms[(W - 1) * kNumSingleVariants + v] = ms;
            if (v == 0 || ms < kVariantMargin * best) {
                best = ms;
                bestv = v;
            }
        }
        c->single_variant[W - 1] = bestv;
    }
    // ---- short single-matrix launches (under kShortLaunch indices), where
    // the fixed costs of a launch decide: n = 24 over all 2^24 indices (W = 1)
    // and n = 36 over 2^27 (W = 2), 20 launches per variant
    const int nS[2] = {24, 36};
    const int lgS[2] = {24, 27};
    for (int W = 1; W <= 2; ++W) {
        const int n = nS[W - 1];
        sample_matrix(hA.data(), n, 2000 + n);
        cudaMemcpy(dA, hA.data(), (size_t)n * n, cudaMemcpyHostToDevice);
        float best = 1e30f;
        int bestv = 0;
        for (int v = 0; v < kNumSingleVariants; ++v) {
            c->single_variant_short[W - 1] = v;
            const float ms = time_ms(s, 20, [&] {
                enqueue_range(c, dA, n, n, 0, (1ull << lgS[W - 1]) - 1, dout, s);
            });
            if (single_short_ms) single_short_ms[(W - 1) * kNumSingleVariants + v] = ms;
            if (v == 0 || ms < kVariantMargin * best) {
                best = ms;
                bestv = v;
            }
        }
        c->single_variant_short[W - 1] = bestv;
    }
    // ---- long launches of a merged matrix (equal columns merged into one
    // word; its terms are mostly nonzero, so the dense walk runs): J_36 as
    // the host-pointer calls walk it, 36 rows of two columns of ones, over
    // 2^33 indices
    {
        const int n = 36, m = 2;
        for (int k = 0; k < n * m; ++k) hA[k] = 1;
        cudaMemcpy(dA, hA.data(), (size_t)n * m, cudaMemcpyHostToDevice);
        float best = 1e30f;
        int bestv = 0;
        for (int v = 0; v < kNumSingleVariants; ++v) {
            c->single_variant_merged = v;
            const float ms = time_ms(s, 2, [&] { enqueue_range(c, dA, n, m, 0, (1ull << 33) - 1, dout, s); });
            if (v == 0 || ms < kVariantMargin * best) {
                best = ms;
                bestv = v;
            }
        }
        c->single_variant_merged = bestv;
    }
    // ---- batch kernel variants, each under the guided split: 8192 matrices
    // of n = 24 (W = 1) and 32 of n = 33 (W = 2), a few grids' worth of work,
    // so that the variants are compared on throughput, not on how their
    // warp counts happen to fit the last round
    int warps[2];
    const int bn[2] = {24, 33};
    const int bcount[2] = {8192, 32};
    for (int W = 1; W <= 2 && e == cudaSuccess; ++W) {
        const int n = bn[W - 1], cnt = bcount[W - 1];
        std::vector<int32_t> ns(cnt, n);
        std::vector<uint8_t> hAs((size_t)cnt * n * n);
        for (int k = 0; k < cnt; ++k) sample_matrix(hAs.data() + (size_t)k * n * n, n, 77 + k);
        uint8_t* dAs = nullptr;
        uint8_t* dres = nullptr;
        e = cudaMalloc(&dAs, hAs.size());
        if (e == cudaSuccess) e = cudaMalloc(&dres, cnt);
        if (e != cudaSuccess) {
            cudaFree(dAs);
            break;
        }
        cudaMemcpy(dAs, hAs.data(), hAs.size(), cudaMemcpyHostToDevice);
        const BatchTuning keep = c->tune;
        c->tune.chunk_log2 = 0;
        float best = 1e30f;
        int bestv = 0;
        for (int v = 0; v < kNumBatchVariants; ++v) {
            c->tune.variant[W - 1] = v;
            batch_warps(c, c->tune, warps);
            BatchPlan plan;
            plan_batch(ns.data(), cnt, c->tune, warps, plan);
            const float ms = time_ms(s, 1, [&] { enqueue_batch(c, plan, dAs, dres, nullptr, s); });
            if (batch_ms) batch_ms[(W - 1) * kNumBatchVariants + v] = ms;
            if (v == 0 || ms < kVariantMargin * best) {
                best = ms;
                bestv = v;
            }
        }
        c->tune = keep;
        c->tune.variant[W - 1] = bestv;
        cudaFree(dAs);
        cudaFree(dres);
    }
    batch_warps(c, c->tune, warps);

    // ---- packing cutoff: for each n above the W = 1 variant's block length,
    // a full grid of n x n matrices (two packed items per warp) walked one
    // matrix per lane against one matrix per warp; the cutoff is the last n
    // (counting up) at which the packed walk is faster.  Below U + 1 a warp
    // would leave all but one lane idle, so packing always wins there.
    if (pack_ms)
        for (int k = 0; k < 2 * (kTinyMaxN + 1); ++k) pack_ms[k] = 0.0;
    if (e == cudaSuccess) {
        const int U = kBatchVariants[c->tune.variant[0]].U;
        const int64_t K = (int64_t)warps[0] * 32 * 2;
        uint8_t* dAs = nullptr;
        uint8_t* dres = nullptr;
        const size_t bytes = (size_t)K * kTinyMaxN * kTinyMaxN;
        e = cudaMalloc(&dAs, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&dres, (size_t)K);
        if (e == cudaSuccess) {
            std::vector<uint8_t> hAs(bytes);
            fill_uniform(hAs.data(), bytes, 4242);
            e = cudaMemcpy(dAs, hAs.data(), bytes, cudaMemcpyHostToDevice);
        }
        int tiny = std::min(U, kTinyMaxN);
        const BatchTuning keep = c->tune;
        for (int n = U + 1; n <= kTinyMaxN && e == cudaSuccess; ++n) {
            std::vector<int32_t> ns((size_t)K, n);
            float t[2];
            for (int path = 0; path < 2; ++path) {
                c->tune.tiny_cutoff = path == 0 ? n : n - 1;
                BatchPlan plan;
                plan_batch(ns.data(), K, c->tune, warps, plan);
                t[path] = time_ms(s, 1, [&] { enqueue_batch(c, plan, dAs, dres, nullptr, s); });
                if (pack_ms) pack_ms[path * (kTinyMaxN + 1) + n] = t[path];
            }
            if (t[0] >= t[1]) break;
            tiny = n;
        }
        c->tune = keep;
        c->tune.tiny_cutoff = tiny;
        cudaFree(dAs);
        cudaFree(dres);
    }

    // ---- split granularity: the guided split with 1..16 items per warp,
    // timed on three batches (3000 x n = 26, where the last partial round
    // matters; 300 x 28 + 600 x 26 + 1200 x 24; 20 x 33 + 6 x 34, fewer
    // matrices than warps); the fastest total wins, ties within 1 % going to
    // fewer, longer items.
    if (e == cudaSuccess) {
        const int mixes[3][3][2] = {{{26, 3000}, {0, 0}, {0, 0}},
                                    {{28, 300}, {26, 600}, {24, 1200}},
                                    {{33, 20}, {34, 6}, {0, 0}}};
        std::vector<int32_t> ns[3];
        size_t bytes[3] = {0, 0, 0}, max_bytes = 0, max_count = 0;
        for (int w = 0; w < 3; ++w) {
            for (const auto& m : mixes[w])
                for (int k = 0; k < m[1]; ++k) {
                    ns[w].push_back(m[0]);
                    bytes[w] += (size_t)m[0] * m[0];
                }
            max_bytes = std::max(max_bytes, bytes[w]);
            max_count = std::max(max_count, ns[w].size());
        }
        uint8_t* dAs = nullptr;
        uint8_t* dres = nullptr;
        e = cudaMalloc(&dAs, max_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&dres, max_count);
        if (e == cudaSuccess) {
            std::vector<uint8_t> hAs(max_bytes);
            fill_uniform(hAs.data(), max_bytes, 4343);
            e = cudaMemcpy(dAs, hAs.data(), max_bytes, cudaMemcpyHostToDevice);
        }
        const BatchTuning keep = c->tune;
        c->tune.chunk_log2 = 0;
        float best = 1e30f;
        int bestg = keep.items_per_warp;
        for (int k = 0; k < kSplitCandidates && e == cudaSuccess; ++k) {
            c->tune.items_per_warp = 1 << k;
            float ms = 0.f;
            for (int w = 0; w < 3; ++w) {
                BatchPlan plan;
                plan_batch(ns[w].data(), (int64_t)ns[w].size(), c->tune, warps, plan);
                ms += time_ms(s, 1, [&] { enqueue_batch(c, plan, dAs, dres, nullptr, s); });
            }
            if (split_ms) split_ms[k] = ms;
            if (ms < 0.99f * best) {
                best = ms;
                bestg = 1 << k;
            }
        }
        c->tune = keep;
        c->tune.chunk_log2 = 0;
        c->tune.items_per_warp = bestg;
        cudaFree(dAs);
        cudaFree(dres);
    }
    cudaFree(dA);
    cudaFree(dout);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) store_tune_cache(c);
    return cuda_rc(e);
}

int pf3_autotune(double* single_ms, double* batch_ms)
{
    return pf3_autotune_ex(single_ms, nullptr, batch_ms, nullptr, nullptr);
}

}  // extern "C"
