// pf3_zcount.cu -- perm(A) mod 3 of EVERY n x n matrix over F3 (n <= 5),
// counted by value: Table 2 of the paper (z(n) = #{A : perm(A) = 0}).
//
// Matrix index idx in [0, 3^(n^2)): row r is the base-3^n digit r of idx, and
// inside a row, column j is base-3 digit j (value 2 == -1).  The outer index
// runs over rows 1..n-1; for each outer configuration the 2^(n-1) subset sums
// of rows 1..n-1 (bipedal pairs, Sec. 2) are formed once, together with the
// part of Eq. (2)'s sum over the subsets that do not contain row 0.  Then all
// 3^n choices of row 0 are evaluated: the subsets containing row 0 are the
// probes v_S + row0, each one row step (Theorem 2.1 semantics, our 3-LOP3
// form), a zero test on mag and a popcount sign.
#include <cuda_runtime.h>

#include "perm_f3.h"
#include "pf3_context.h"
#include "pf3_device.cuh"

namespace pf3 {

namespace {

constexpr int kZThreads = 256;

__device__ __forceinline__ void row_bits(uint32_t code, int n, uint32_t& mag, uint32_t& sgn)
{
    mag = 0;
    sgn = 0;
    for (int j = 0; j < n; ++j) {
        const uint32_t d = code % 3u;
        code /= 3u;
        mag |= (uint32_t)(d != 0u) << j;
        sgn |= (uint32_t)(d == 2u) << j;
    }
}

__host__ __device__ constexpr uint32_t pow3(int k)
{
    return k == 0 ? 1u : 3u * pow3(k - 1);
}

// counts[v] += number of matrices with outer index in [o0, o1) whose perm is v
template <int N>
__global__ void __launch_bounds__(kZThreads) zcount_kernel(unsigned long long o0, unsigned long long o1,
                                                            unsigned long long* counts)
{
    constexpr int n = N;
    constexpr uint32_t R = pow3(N);  // 3^n values of a row
    __shared__ uint32_t s_k1[R], s_k2p[R], s_k2m[R];
    __shared__ unsigned long long red[3][kZThreads / 32];
    for (uint32_t c = threadIdx.x; c < R; c += blockDim.x) {
        uint32_t mag, sgn;
        row_bits(c, n, mag, sgn);
        row_masks(mag, sgn, s_k1[c], s_k2p[c], s_k2m[c]);
    }
    __syncthreads();

    const unsigned long long total = o1 - o0;
    const unsigned long long T = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t s, len;
    split_range(total, T, tid, s, len);
    unsigned long long c0 = 0, c1 = 0, c2 = 0;
    const uint32_t pad = ~((1u << n) - 1u);  // padding columns hold the constant 1
    constexpr int h = n - 1;                 // rows 1..n-1
    // decode the first outer index into row codes (rows 1..n-1)
    uint32_t code[h > 0 ? h : 1] = {};
    {
        unsigned long long o = o0 + s;
        for (int r = 0; r < h; ++r) {
            code[r] = (uint32_t)(o % R);
            o /= R;
        }
    }
    for (uint64_t q = 0; q < len; ++q) {
        // subset sums over rows 1..n-1 (bit r of S = row r+1) in Gray order
        uint32_t bm[1 << h], bs[1 << h];
        int dsum = 0;  // sum over S without row 0 of (-1)^{|S|} * prod
        bm[0] = pad;
        bs[0] = 0u;
#pragma unroll
        for (int S = 1; S < (1 << h); ++S) {
            // build from S without its lowest set bit
            const int low = __ffs(S) - 1;
            const int prev = S & (S - 1);
            uint32_t m = bm[prev], sg = bs[prev];
            const uint32_t c = code[low];
            add_word(m, sg, s_k1[c], s_k2p[c]);
            bm[S] = m;
            bs[S] = sg;
            if (m == 0xFFFFFFFFu) dsum += ((__popc(sg) + __popc((unsigned)S)) & 1) ? -1 : 1;
        }
        // the empty subset: product of n zeros = 0 for n >= 1
        for (uint32_t c = 0; c < R; ++c) {
            int d = dsum;
            const uint32_t k1 = s_k1[c], k2 = s_k2p[c];
#pragma unroll
            for (int S = 0; S < (1 << h); ++S) {
                uint32_t m = bm[S], sg = bs[S];
                add_word(m, sg, k1, k2);
                if (m == 0xFFFFFFFFu) d += ((__popc(sg) + __popc((unsigned)S) + 1) & 1) ? -1 : 1;
            }
            if (n & 1) d = -d;
            const int v = ((d % 3) + 3) % 3;
            c0 += (v == 0);
            c1 += (v == 1);
            c2 += (v == 2);
        }
        // next outer configuration (odometer over rows 1..n-1)
#pragma unroll
        for (int r = 0; r < h; ++r) {
            if (++code[r] < R) break;
            code[r] = 0;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    c0 = warp_sum(c0);
    c1 = warp_sum(c1);
    c2 = warp_sum(c2);
    if (lane == 0) {
        red[0][warp] = c0;
        red[1][warp] = c1;
        red[2][warp] = c2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        unsigned long long t = 0;
        for (int w = 0; w < kZThreads / 32; ++w) t += red[threadIdx.x][w];
        atomicAdd(counts + threadIdx.x, t);
    }
}

}  // namespace

}  // namespace pf3

using namespace pf3;

extern "C" int pf3_count_exhaustive(int n, uint64_t* counts)
{
    if (n < 1 || n > 5 || !counts) return PF3_EINVAL;
    int rc;
    DeviceCtx* c = device_ctx(&rc);
    if (!c) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    unsigned long long R = 1, outer = 1;
    for (int j = 0; j < n; ++j) R *= 3ull;
    for (int r = 1; r < n; ++r) outer *= R;
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, 3 * sizeof(unsigned long long), c->stream);
    // bounded launches: at most 2^26 outer configurations (about 0.3 s at n = 5) each
    const unsigned long long step = 1ull << 26;
    const int grid = c->sm_count * 8;
    for (unsigned long long o = 0; o < outer && e == cudaSuccess; o += step) {
        const unsigned long long o1 = (outer - o > step) ? o + step : outer;
        switch (n) {
        case 1: zcount_kernel<1><<<grid, kZThreads, 0, c->stream>>>(o, o1, d); break;
        case 2: zcount_kernel<2><<<grid, kZThreads, 0, c->stream>>>(o, o1, d); break;
        case 3: zcount_kernel<3><<<grid, kZThreads, 0, c->stream>>>(o, o1, d); break;
        case 4: zcount_kernel<4><<<grid, kZThreads, 0, c->stream>>>(o, o1, d); break;
        default: zcount_kernel<5><<<grid, kZThreads, 0, c->stream>>>(o, o1, d); break;
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_rc(e);
    counts[0] = h[0];
    counts[1] = h[1];
    counts[2] = h[2];
    return PF3_OK;
}
