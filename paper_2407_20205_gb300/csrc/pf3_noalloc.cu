// pf3_noalloc.cu -- the Gray-walk range entry point for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a process whose memory
// manager reserves the whole device up front and forbids allocations it did
// not make, or a latency-sensitive caller for whom cudaMalloc/cudaFree (which
// may synchronise the device and stall every stream) is not acceptable.  This
// file gives them perm_f3_range_counts_noalloc: the same walk as
// perm_f3_range_counts_async, with the kernel's scratch (one pair of partial
// counts per CTA, the last-CTA ticket, the error flag and the chunk cursor)
// in a fixed file-scope device array instead of memory the library
// allocates.  The caller still owns and passes the matrix and the output
// buffer.
//
// The array is part of the module: every GPU that loads the library holds its
// PF3_NOALLOC_MAX_CTAS * 16 + 256 bytes until the process exits.  All calls on
// a device share it and it keeps the last call's contents, so each call first
// clears the ticket, error flag and cursor (cudaMemsetAsync, no allocation),
// and two calls that overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "perm_f3.h"
#include "pf3_internal.h"

namespace pf3 {

namespace {

constexpr int kNoAllocFlagsBytes = 256;
constexpr size_t kNoAllocBytes = (size_t)PF3_NOALLOC_MAX_CTAS * 2 * sizeof(unsigned long long) + kNoAllocFlagsBytes;

// flags first (ticket, error, chunk cursor), then 2 x uint64 per CTA
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};  // device address per device ordinal
int g_noalloc_sms[kMaxDevices] = {};
int g_noalloc_ctas[kMaxDevices][2] = {};

// once per device, with that device current: the array's device address (the
// host-side name g_noalloc_scratch is only a stand-in, not a device pointer)
int noalloc_setup(int dev)
{
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (g_noalloc_ptr[dev]) return PF3_OK;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return PF3_ECUDA;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) return PF3_ECUDA;
    g_noalloc_sms[dev] = sms;
    g_noalloc_ctas[dev][0] = single_max_ctas_per_sm(1, 0);
    g_noalloc_ctas[dev][1] = single_max_ctas_per_sm(2, 0);
    g_noalloc_ptr[dev] = (unsigned char*)p;
    return PF3_OK;
}

}  // namespace

}  // namespace pf3

using namespace pf3;

extern "C" int perm_f3_range_counts_noalloc(const uint8_t* dA, int n, uint64_t first, uint64_t last,
                                            uint64_t* d_out, int ctas, void* stream)
{
    if (n < 1 || n > PF3_MAX_N || first > last || !dA || !d_out || ctas < 0) return PF3_EINVAL;
    if (n < 64 && last >= (1ull << n)) return PF3_EINVAL;
    if (ctas > PF3_NOALLOC_MAX_CTAS) return PF3_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PF3_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return PF3_ECUDA;
    int rc = noalloc_setup(dev);
    if (rc) return rc;
    unsigned char* base = g_noalloc_ptr[dev];
    const int W = n <= 32 ? 1 : 2;
    const int v = 0;  // the default variant: the same code as the allocating entry point's default
    SingleArgs a;
    std::memset(&a, 0, sizeof(a));
    plan_range(n, first, last, kSingleVariants[v].U, a);
    a.A = dA;
    a.ticket = (unsigned int*)base;
    a.err = (unsigned int*)base + 1;
    a.cursor = (unsigned int*)base + 2;
    a.partials = (unsigned long long*)(base + kNoAllocFlagsBytes);
    a.out = (unsigned long long*)d_out;
    int grid = single_grid_for(a, v, g_noalloc_sms[dev], g_noalloc_ctas[dev][W - 1]);
    if (ctas > 0 && grid > ctas) grid = ctas;
    if (grid > PF3_NOALLOC_MAX_CTAS) grid = PF3_NOALLOC_MAX_CTAS;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(base, 0, 3 * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = launch_single(a, v, grid, s);
    return e == cudaSuccess ? PF3_OK : PF3_ECUDA;
}
