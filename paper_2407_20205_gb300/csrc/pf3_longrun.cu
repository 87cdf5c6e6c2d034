// pf3_longrun.cu -- long single-matrix walks in bounded launches with a
// checkpoint of the range cursor.
//
// Sec. 3.1 computes perm(Pi_50) as many jobs over blocks of consecutive Gray
// states whose partial sums are added.  On one GPU the same split keeps every
// launch short: the range [0, 2^n) is walked in launches of at most
// 2^chunk_log2 indices; after each launch the exact 64-bit counts and the
// next index are written to a checkpoint file (written to a temporary name,
// then renamed), so an interrupted run resumes where it stopped and produces
// the same counts as an uninterrupted one.  Between launches the loop
// honours a wall-clock limit and a cancellation flag; no launch waits on the
// host.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "perm_f3.h"
#include "pf3_context.h"
#include "pf3_internal.h"

using namespace pf3;

namespace {

std::atomic<int> g_cancel{0};

uint64_t fnv1a64(const uint8_t* p, size_t len, int n)
{
    uint64_t h = 1469598103934665603ull;
    h = (h ^ (uint64_t)n) * 1099511628211ull;
    for (size_t i = 0; i < len; ++i) h = (h ^ p[i]) * 1099511628211ull;
    return h;
}

struct Checkpoint {
    int n = 0;
    uint64_t hash = 0, cursor = 0, plus = 0, minus = 0;
    int done = 0;
};

bool read_checkpoint(const char* path, Checkpoint& c)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char magic[64] = {0};
    unsigned long long h = 0, cur = 0, p = 0, m = 0;
    int n = 0, done = 0;
    const int got = std::fscanf(f, "%63s n=%d hash=%llx cursor=%llu plus=%llu minus=%llu done=%d", magic, &n, &h,
                                &cur, &p, &m, &done);
    std::fclose(f);
    if (got != 7 || std::strcmp(magic, "pf3-checkpoint-v1") != 0) return false;
    c.n = n;
    c.hash = h;
    c.cursor = cur;
    c.plus = p;
    c.minus = m;
    c.done = done;
    return true;
}

bool write_checkpoint(const char* path, const Checkpoint& c)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "pf3-checkpoint-v1\nn=%d\nhash=%llx\ncursor=%llu\nplus=%llu\nminus=%llu\ndone=%d\n", c.n,
                 (unsigned long long)c.hash, (unsigned long long)c.cursor, (unsigned long long)c.plus,
                 (unsigned long long)c.minus, c.done);
    const bool ok = std::fflush(f) == 0;
    std::fclose(f);
    return ok && std::rename(tmp.c_str(), path) == 0;
}

}  // namespace

extern "C" {

void pf3_longrun_cancel(int on) { g_cancel.store(on ? 1 : 0); }

int pf3_longrun(const uint8_t* A, int n, int chunk_log2, const char* checkpoint_path, double max_seconds,
                uint64_t* plus, uint64_t* minus, uint64_t* next_index, int* finished, int* result)
{
    if (!A || n < 1 || n > PF3_MAX_N || chunk_log2 < 10 || chunk_log2 > PF3_LONGRUN_MAX_CHUNK_LOG2 || !plus ||
        !minus)
        return PF3_EINVAL;
    int rc = check_entries_host(A, n);
    if (rc) return rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    const uint64_t hash = fnv1a64(A, (size_t)n * n, n);
    Checkpoint ck;
    ck.n = n;
    ck.hash = hash;
    if (checkpoint_path && read_checkpoint(checkpoint_path, ck)) {
        if (ck.n != n || ck.hash != hash) return PF3_EINVAL;  // checkpoint of another matrix
    } else {
        ck = Checkpoint();
        ck.n = n;
        ck.hash = hash;
    }
    const uint64_t last = (n == 64) ? ~0ull : ((1ull << n) - 1);
    const uint64_t step_m1 = (1ull << chunk_log2) - 1;
    const auto t0 = std::chrono::steady_clock::now();
    // equal columns merged as for perm_f3 (pf3_capi.cu); the counts are A's
    std::vector<uint8_t> B;
    int m = n;
    bool negate = false;
    const bool merged = merge_columns(A, n, B, m, negate);
    const uint8_t* src = merged ? B.data() : A;
    const size_t bytes = (size_t)n * m;
    if (merged && ck.cursor == 0 && !ck.done && !g_cancel.load()) {
        // a fresh run of a narrow merged matrix: the whole range at once by
        // column-sum vector (pf3_classes.cu), one short launch
        std::lock_guard<std::mutex> g(c->mu);
        if (m <= c->class_max_cols) {
            std::memcpy(c->h_A, src, bytes);
            cudaError_t e = cudaMemcpyAsync(c->d_A, c->h_A, bytes, cudaMemcpyHostToDevice, c->stream);
            if (!(rc = cuda_rc(e))) rc = enqueue_class_counts(c->d_A, n, m, c->d_out, c->stream);
            if (!rc) {
                e = cudaMemcpyAsync(c->h_out, c->d_out, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                    c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                rc = cuda_rc(e);
            }
            if (!rc) {
                ck.plus = negate ? c->h_out[1] : c->h_out[0];
                ck.minus = negate ? c->h_out[0] : c->h_out[1];
                ck.done = 1;
                if (checkpoint_path && !write_checkpoint(checkpoint_path, ck)) rc = PF3_EINVAL;
            }
        }
    }
    while (!rc && !ck.done) {
        if (g_cancel.load()) {
            rc = PF3_ECANCELED;
            break;
        }
        const uint64_t first = ck.cursor;
        const uint64_t stop = (last - first <= step_m1) ? last : first + step_m1;
        {
            // the device context is held for one launch at a time, so other
            // calls on this device interleave with a long walk; the matrix is
            // copied again each time because they share the staging buffers
            std::lock_guard<std::mutex> g(c->mu);
            std::memcpy(c->h_A, src, bytes);
            cudaError_t e = cudaMemcpyAsync(c->d_A, c->h_A, bytes, cudaMemcpyHostToDevice, c->stream);
            if ((rc = cuda_rc(e))) break;
            if ((rc = enqueue_range(c, c->d_A, n, m, first, stop, c->d_out, c->stream))) break;
            e = cudaMemcpyAsync(c->h_out, c->d_out, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if ((rc = cuda_rc(e))) break;
            ck.plus += negate ? c->h_out[1] : c->h_out[0];
            ck.minus += negate ? c->h_out[0] : c->h_out[1];
        }
        if (stop == last) ck.done = 1;
        else ck.cursor = stop + 1;
        if (checkpoint_path && !write_checkpoint(checkpoint_path, ck)) {
            rc = PF3_EINVAL;
            break;
        }
        // the wall-clock limit is checked after each launch: every call makes progress
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (!ck.done && max_seconds > 0 && el >= max_seconds) rc = PF3_ETIMEDOUT;
    }
    *plus = ck.plus;
    *minus = ck.minus;
    if (next_index) *next_index = ck.done ? 0 : ck.cursor;
    if (finished) *finished = ck.done;
    if (result && ck.done) *result = (int)perm_from_counts(n, ck.plus, ck.minus);
    return rc;
}

}  // extern "C"
