// pf3_vecops.cu -- the bipedal vector operations of Sec. 2 (Theorem 2.1) on
// arrays of vectors of length n <= 64, one 64-bit (mag, sgn) pair per vector.
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

__global__ void vecop_kernel(int op, const unsigned long long* m1, const unsigned long long* s1,
                             const unsigned long long* m2, const unsigned long long* s2, unsigned long long* m3,
                             unsigned long long* s3, long long count, unsigned long long mask)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
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
    m3[k] = m & mask;
    s3[k] = s & mask;
}

// psi of Sec. 2, one thread per (vector, column): 0 where mag = 0, else 1 or
// 2 (== -1) by sgn; column j is bit j
__global__ void unpack_kernel(const unsigned long long* mag, const unsigned long long* sgn, uint8_t* out, int n,
                              long long count)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count * n) return;
    const long long v = k / n;
    const int j = (int)(k % n);
    const unsigned m = (unsigned)((mag[v] >> j) & 1ull), s = (unsigned)((sgn[v] >> j) & 1ull);
    out[k] = (uint8_t)(m ? (s ? 2u : 1u) : 0u);
}

}  // namespace

}  // namespace pf3

using namespace pf3;

extern "C" int pf3_vec_unpack(int n, int64_t count, const uint64_t* mag, const uint64_t* sgn, uint8_t* out)
{
    if (n < 1 || n > PF3_MAX_N || count < 0) return PF3_EINVAL;
    if (count == 0) return PF3_OK;
    if (!mag || !sgn || !out) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    const size_t bytes = (size_t)count * sizeof(uint64_t);
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * bytes + (size_t)count * n);
    if (e != cudaSuccess) return cuda_rc(e);
    uint8_t* dout = (uint8_t*)(d + 2 * count);
    e = cudaMemcpyAsync(d, mag, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + count, sgn, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        const long long total = count * n;
        unpack_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(d, d + count, dout, n, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)count * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    return cuda_rc(e);
}

extern "C" int pf3_vec_op(int op, int n, int64_t count, const uint64_t* m1, const uint64_t* s1, const uint64_t* m2,
                          const uint64_t* s2, uint64_t* m3, uint64_t* s3)
{
    if (op < PF3_OP_ADD || op > PF3_OP_DIV || n < 1 || n > PF3_MAX_N || count < 0) return PF3_EINVAL;
    if (count == 0) return PF3_OK;
    if (!m1 || !s1 || !m2 || !s2 || !m3 || !s3) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    const size_t bytes = (size_t)count * sizeof(uint64_t);
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 6 * bytes);
    if (e != cudaSuccess) return cuda_rc(e);
    const uint64_t* in[4] = {m1, s1, m2, s2};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(d + (size_t)k * count, in[k], bytes, cudaMemcpyHostToDevice, c->stream);
    const unsigned long long mask = (n == 64) ? ~0ull : ((1ull << n) - 1);
    if (e == cudaSuccess) {
        const int threads = 256;
        const long long blocks = (count + threads - 1) / threads;
        vecop_kernel<<<(unsigned)blocks, threads, 0, c->stream>>>(op, d, d + count, d + 2 * count, d + 3 * count,
                                                                   d + 4 * count, d + 5 * count, count, mask);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(m3, d + 4 * count, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s3, d + 5 * count, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    return cuda_rc(e);
}
