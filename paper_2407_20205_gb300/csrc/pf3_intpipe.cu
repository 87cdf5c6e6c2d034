// pf3_intpipe.cu -- issue-rate microbenchmark of the integer/logic pipe.
//
// The Gray walk is bound by the rate at which an SM issues 32-bit logic and
// compare instructions (three LOP3 and one compare per subset and word), so
// its roofline denominator is that rate measured on the chip itself.  Each
// thread runs 8 independent dependency chains so that latency is hidden; each
// CTA times itself with the SM cycle counter.
//
// kinds: 0 = LOP3, 1 = IMAD (multiplier opaque to the compiler), 2 = integer
// add, 3 = LOP3 and IMAD interleaved 1:1, 4 = the full row step (three LOP3
// and an accumulating compare), 5 = POPC, 6 = unsigned max, 7 = two LOP3 and
// one max, 8 = two LOP3 and an accumulating compare (the probe of the walk),
// 9 = three LOP3 and one IMAD, 10 = two LOP3 and one integer add, 11 = the
// probe with an inverted last gate tested against zero, 12 = the probe tested
// against all ones, 13 = the inverted probe accumulated with AND of "nonzero"
// (each: two LOP3 and one compare per op).
#include <cuda_runtime.h>

#include "pf3_device.cuh"
#include "pf3_internal.h"

namespace pf3 {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <int KIND>
__global__ void intpipe_kernel(uint32_t* sink, unsigned long long* cycles, int iters, uint32_t one)
{
    uint32_t x[kChains], y[kChains], z[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = threadIdx.x * 0x9E3779B9u + c * 0x85EBCA6Bu + blockIdx.x;
        y[c] = x[c] ^ 0x5bd1e995u;
        z[c] = y[c] + 7u;
    }
    const uint32_t ka = one * 0x0F0F0F0Fu, kb = one * 0x33333333u, kc = one * 0x55555555u,
                   kd = one * 0x00FF00FFu;
    bool hit = false;
    bool allnz = true;
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == 0) {
                    // alternate operands so consecutive gates never fold into one
                    x[c] = (u & 1) ? lop3<0x96>(x[c], ka, kb) : lop3<0xE8>(x[c], kc, kd);
                } else if (KIND == 1) {
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(one), "r"((u & 1) ? ka : kb));
                } else if (KIND == 2) {
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(x[c]) : "r"((u & 1) ? ka : kc));
                } else if (KIND == 3) {
                    x[c] = lop3<0x96>(x[c], ka, kb);
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(y[c]) : "r"(one), "r"(kc));
                } else if (KIND == 4) {
                    add_word(x[c], y[c], (u & 1) ? ka : kc, (u & 1) ? kb : kd);
                    hit |= (x[c] == 0xFFFFFFFFu);
                } else if (KIND == 5) {
                    x[c] = __popc(x[c]) + y[c];
                    y[c] ^= 1u;
                } else if (KIND == 6) {
                    asm volatile("max.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(y[c]));
                    y[c] = y[c] * 0x9E3779B9u + 1u;  // keeps operands distinct (IMAD)
                } else if (KIND == 7) {
                    x[c] = lop3<0x96>(x[c], ka, kb);
                    x[c] = lop3<0xE8>(x[c], kc, kd);
                    asm volatile("max.u32 %0, %0, %1;" : "+r"(y[c]) : "r"(x[c]));
                } else if (KIND == 8) {
                    x[c] = lop3<0x96>(x[c], ka, kb);
                    x[c] = lop3<0xE8>(x[c], kc, kd);
                    hit |= (x[c] == 0xFFFFFFFFu);
                } else if (KIND == 9) {
                    add_word(x[c], y[c], (u & 1) ? ka : kc, (u & 1) ? kb : kd);
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(z[c]) : "r"(one), "r"(x[c]));
                } else if (KIND == 10) {
                    x[c] = lop3<0x96>(x[c], ka, kb);
                    x[c] = lop3<0xE8>(x[c], kc, kd);
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(y[c]) : "r"(x[c]));
                } else if (KIND == 11) {
                    // probe with an inverted last gate tested against zero; the
                    // two gate outputs feed the next probe (no folding possible)
                    const uint32_t gq = lop3<kLutG>(y[c], (u & 1) ? ka : kc, (u & 1) ? kb : kd);
                    const uint32_t nm = lop3<(~kLutMag) & 0xFF>(x[c], (u & 1) ? ka : kc, gq);
                    hit |= (nm == 0u);
                    x[c] = gq;
                    y[c] = nm;
                } else if (KIND == 13) {
                    // inverted gate, accumulated as "every probe has a zero column"
                    const uint32_t gq = lop3<kLutG>(y[c], (u & 1) ? ka : kc, (u & 1) ? kb : kd);
                    const uint32_t nm = lop3<(~kLutMag) & 0xFF>(x[c], (u & 1) ? ka : kc, gq);
                    allnz &= (nm != 0u);
                    x[c] = gq;
                    y[c] = nm;
                } else if (KIND == 12) {
                    // the walk's probe as written (test against all ones), same chain
                    const uint32_t gq = lop3<kLutG>(y[c], (u & 1) ? ka : kc, (u & 1) ? kb : kd);
                    const uint32_t mq = lop3<kLutMag>(x[c], (u & 1) ? ka : kc, gq);
                    hit |= (mq == 0xFFFFFFFFu);
                    x[c] = gq;
                    y[c] = mq;
                }
            }
        }
    }
    const unsigned long long t1 = clock64();
    uint32_t acc = (hit ? 1u : 0u) ^ (allnz ? 2u : 0u);
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= x[c] ^ y[c] ^ z[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

cudaError_t launch_intpipe(int kind, int grid, int threads, int iters, uint32_t* sink, unsigned long long* cycles,
                           cudaStream_t stream)
{
    switch (kind) {
    case 0: intpipe_kernel<0><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 1: intpipe_kernel<1><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 2: intpipe_kernel<2><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 3: intpipe_kernel<3><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 4: intpipe_kernel<4><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 5: intpipe_kernel<5><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 6: intpipe_kernel<6><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 7: intpipe_kernel<7><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 8: intpipe_kernel<8><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 9: intpipe_kernel<9><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 10: intpipe_kernel<10><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 11: intpipe_kernel<11><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 12: intpipe_kernel<12><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    case 13: intpipe_kernel<13><<<grid, threads, 0, stream>>>(sink, cycles, iters, 1u); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pf3
