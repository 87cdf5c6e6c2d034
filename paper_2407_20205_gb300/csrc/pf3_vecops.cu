// pf3_vecops.cu -- the bipedal vector operations of Sec. 2 (Theorem 2.1) on
// arrays of vectors of any length n, ceil(n / 64) 64-bit words per plane.
//
// Theorem 2.1 gives, for bipedal representations (m1, s1) of alpha and
// (m2, s2) of beta:
//   sum:        x = m2 & (m1 ^ s1 ^ s2);  m = x | (m1 ^ m2);  s = x ^ s1
//   difference: x = m1 & (s1 ^ s2);       m = x | (m1 ^ m2);  s = x ^ (m2 ^ s2)
//   product:    m = m1 & m2;              s = s1 ^ s2
//   quotient:   m = m1;                   s = s1 ^ s2   (beta nonzero)
// (the paper's forms, six two-input operations for the sum and difference).
// These are the library forms for vectors; the permanent walk uses its own
// three-gate row step.  Off the permanent's hot path.
#include <cuda_runtime.h>

#include "perm_f3.h"
#include "pf3_context.h"

namespace pf3 {

namespace {

// Vector k of length n is w = ceil(n / 64) words per plane, words k*w ..
// k*w + w - 1, column j in bit j % 64 of word j / 64 (the footnote of Sec. 3
// on rows longer than one machine word); bits at and above n are cleared in
// every result.  One thread per word, grid-stride.
__global__ void vecop_kernel(int op, const unsigned long long* m1, const unsigned long long* s1,
                             const unsigned long long* m2, const unsigned long long* s2, unsigned long long* m3,
                             unsigned long long* s3, long long words, int w, unsigned long long last_mask)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < words;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long a = m1[k], b = s1[k], c = m2[k], d = s2[k];
        unsigned long long m, s;
        switch (op) {
        case PF3_OP_ADD: {
            const unsigned long long x = c & (a ^ b ^ d);
            m = x | (a ^ c);
            s = x ^ b;
            break;
        }
        case PF3_OP_SUB: {
            const unsigned long long x = a & (b ^ d);
            m = x | (a ^ c);
            s = x ^ (c ^ d);
            break;
        }
        case PF3_OP_MUL:
            m = a & c;
            s = b ^ d;
            break;
        default:  // PF3_OP_DIV
            m = a;
            s = b ^ d;
            break;
        }
        const unsigned long long mask = (k % w == w - 1) ? last_mask : ~0ull;
        m3[k] = m & mask;
        s3[k] = s & mask;
    }
}

// psi of Sec. 2, one thread per (vector, column): 0 where mag = 0, else 1 or
// 2 (== -1) by sgn
__global__ void unpack_kernel(const unsigned long long* mag, const unsigned long long* sgn, uint8_t* out, int n,
                              int w, long long total)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long v = k / n;
        const int j = (int)(k % n);
        const long long word = v * w + (j >> 6);
        const unsigned m = (unsigned)((mag[word] >> (j & 63)) & 1ull);
        const unsigned s = (unsigned)((sgn[word] >> (j & 63)) & 1ull);
        out[k] = (uint8_t)(m ? (s ? 2u : 1u) : 0u);
    }
}

// phi of Sec. 2, one warp per 32 columns of a vector: ballots of "nonzero"
// and "== 2" give the two planes' bits; bad is set on an entry above 2
__global__ void pack_kernel_vec(const uint8_t* in, unsigned long long* mag, unsigned long long* sgn, int n, int w,
                                long long count, unsigned int* bad)
{
    const int lane = threadIdx.x & 31;
    const long long halves = count * (long long)w * 2;  // 32-column pieces
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long h = (((long long)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; h < halves; h += warps) {
        const long long v = h / (2 * w);
        const int piece = (int)(h % (2 * w));
        const int col = piece * 32 + lane;
        unsigned a = 0;
        if (col < n) a = in[v * n + col];
        const unsigned mb = __ballot_sync(0xFFFFFFFFu, a == 1u || a == 2u);
        const unsigned sb = __ballot_sync(0xFFFFFFFFu, a == 2u);
        if (__any_sync(0xFFFFFFFFu, a > 2u) && lane == 0) atomicOr(bad, 1u);
        if (lane == 0) {
            unsigned* mw = (unsigned*)(mag + v * w + (piece >> 1));
            unsigned* sw = (unsigned*)(sgn + v * w + (piece >> 1));
            mw[piece & 1] = mb;  // little-endian halves of the 64-bit word
            sw[piece & 1] = sb;
        }
    }
}

unsigned grid_for(long long items, int threads)
{
    long long b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    return (unsigned)(b > (1 << 20) ? (1 << 20) : b);
}

}  // namespace

}  // namespace pf3

using namespace pf3;

namespace {

// words per plane of one vector, or 0 when n or the total is out of range
long long vec_words(int n, int64_t count)
{
    if (n < 1 || n > PF3_VEC_MAX_N || count < 0) return 0;
    const long long w = (n + 63) / 64;
    if (count > 0 && w > PF3_VEC_MAX_WORDS / count) return 0;
    return w;
}

}  // namespace

extern "C" int pf3_vec_unpack(int n, int64_t count, const uint64_t* mag, const uint64_t* sgn, uint8_t* out)
{
    const long long w = vec_words(n, count);
    if (!w) return PF3_EINVAL;
    if (count == 0) return PF3_OK;
    if (!mag || !sgn || !out) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    const size_t bytes = (size_t)count * w * sizeof(uint64_t);
    const long long total = (long long)count * n;
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * bytes + (size_t)total);
    if (e != cudaSuccess) return cuda_rc(e);
    uint8_t* dout = (uint8_t*)(d + 2 * (size_t)count * w);
    e = cudaMemcpyAsync(d, mag, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + (size_t)count * w, sgn, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        unpack_kernel<<<grid_for(total, 256), 256, 0, c->stream>>>(d, d + (size_t)count * w, dout, n, (int)w, total);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)total, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    return cuda_rc(e);
}

extern "C" int pf3_vec_pack(int n, int64_t count, const uint8_t* in, uint64_t* mag, uint64_t* sgn)
{
    const long long w = vec_words(n, count);
    if (!w) return PF3_EINVAL;
    if (count == 0) return PF3_OK;
    if (!in || !mag || !sgn) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    const size_t bytes = (size_t)count * w * sizeof(uint64_t);
    const size_t in_bytes = (size_t)count * n;
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * bytes + in_bytes + 16);
    if (e != cudaSuccess) return cuda_rc(e);
    unsigned int* dbad = (unsigned int*)(d + 2 * (size_t)count * w);
    uint8_t* din = (uint8_t*)(dbad + 4);
    unsigned int hbad = 0;
    e = cudaMemsetAsync(dbad, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(din, in, in_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        const long long threads = (long long)count * w * 2 * 32;
        pack_kernel_vec<<<grid_for(threads, 256), 256, 0, c->stream>>>(din, d, d + (size_t)count * w, n, (int)w,
                                                                          count, dbad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, dbad, sizeof(hbad), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && !hbad) {
        e = cudaMemcpy(mag, d, bytes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sgn, d + (size_t)count * w, bytes, cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    if (e != cudaSuccess) return cuda_rc(e);
    return hbad ? PF3_EDOMAIN : PF3_OK;
}

extern "C" int pf3_vec_op(int op, int n, int64_t count, const uint64_t* m1, const uint64_t* s1, const uint64_t* m2,
                          const uint64_t* s2, uint64_t* m3, uint64_t* s3)
{
    if (op < PF3_OP_ADD || op > PF3_OP_DIV) return PF3_EINVAL;
    const long long w = vec_words(n, count);
    if (!w) return PF3_EINVAL;
    if (count == 0) return PF3_OK;
    if (!m1 || !s1 || !m2 || !s2 || !m3 || !s3) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    const long long words = (long long)count * w;
    const size_t bytes = (size_t)words * sizeof(uint64_t);
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 6 * bytes);
    if (e != cudaSuccess) return cuda_rc(e);
    const uint64_t* in[4] = {m1, s1, m2, s2};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(d + (size_t)k * words, in[k], bytes, cudaMemcpyHostToDevice, c->stream);
    const int r = n % 64;
    const unsigned long long last_mask = r ? ((1ull << r) - 1) : ~0ull;
    if (e == cudaSuccess) {
        vecop_kernel<<<grid_for(words, 256), 256, 0, c->stream>>>(op, d, d + words, d + 2 * words, d + 3 * words,
                                                                   d + 4 * words, d + 5 * words, words, (int)w,
                                                                   last_mask);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(m3, d + 4 * words, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s3, d + 5 * words, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    return cuda_rc(e);
}
