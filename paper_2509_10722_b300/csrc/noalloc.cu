// Utility evaluation that allocates nothing (num_objective_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the number: code
// running inside another framework's memory pool with allocation locked, a real-time
// loop that forbids cudaMalloc (it synchronizes the device), or a fixed-budget embedded
// deployment.  For them this is a variant of the objective reduction that num_get runs
// (sum_j U_j(x_j) in FP64 over block partials): the block partials live in the file-scope
// static device array below instead of handle-owned scratch, so the call allocates
// nothing.  The paper has no counterpart; it is a service of this library.
//
// The array is at most kNoAllocMaxBlocks doubles (32 KB); every GPU that loads this
// library holds it until the process exits.  All calls share it: the last call's contents
// stay there, and calls that overlap on the GPU (different streams, or different host
// threads) race on it.  Every slot a call reads is written by the same call first, so
// nothing needs clearing between calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "num_pmp.h"
#include "pmp_device.cuh"
#include "pmp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 32;
constexpr long long kPerBlock = (long long)kThreads * kPerThread;  // streams per block
constexpr int kNoAllocMaxBlocks = 4096;                              // 32 KB of partials
constexpr long long kNoAllocMaxN = kPerBlock * kNoAllocMaxBlocks;    // 33,554,432 streams
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

// Device address of g_noalloc_partials per device, looked up once (host code may not use
// the symbol's name as an address: on the host it only stands for the device variable).
// Kept for the life of the process: one CUDA context per device is assumed throughout.
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Block b sums U_j(x_j) over streams [b * kPerBlock, (b + 1) * kPerBlock), fixed order.
__global__ void __launch_bounds__(kThreads)
k_noalloc_partials(long long n, const double* __restrict__ x, const uint8_t* __restrict__ utype,
                   const double* __restrict__ w, double* part) {
    __shared__ double red[kThreads / 32];
    const long long base = (long long)blockIdx.x * kPerBlock;
    double s = 0.0;
    for (int k = 0; k < kPerThread; ++k) {
        const long long j = base + (long long)k * kThreads + threadIdx.x;
        if (j < n) {
            const double xj = x[j];
            const uint8_t t = utype[j];
            s += t == 0 ? w[j] * log(xj) : (t == 2 ? -w[j] / xj : w[j] * xj);  // U_j, Sec. II
        }
    }
    s = pmp::block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads)
k_noalloc_total(const double* part, int nb, double* out) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) s += part[i];
    s = pmp::block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace

extern "C" int num_objective_noalloc(int64_t n, const double* x, const uint8_t* utype,
                                     const double* w, double* objective, void* cuda_stream) {
    if (!x || !utype || !w || !objective)
        return pmp::report_error(NUM_ERR_INVALID, "a required pointer is NULL");
    if (n < 1) return pmp::report_error(NUM_ERR_INVALID, "n must be >= 1");
    if (n > kNoAllocMaxN)
        return pmp::report_error(NUM_ERR_INVALID,
                                 "n exceeds the no-allocation maximum of " +
                                     std::to_string(kNoAllocMaxN) +
                                     " streams (use num_get on a handle instead)");
    // a non-sticky error left on this thread by an earlier runtime call would otherwise be
    // reported below as this call's launch failure
    (void)cudaGetLastError();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pmp::report_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return pmp::report_error(NUM_ERR_INVALID, "device index");
    void* part = nullptr;
    {
        // first call on this device (with it current): find the array's device address
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_partials);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                return pmp::report_cuda_error(e, "cudaGetSymbolAddress");
            }
        }
        part = g_addr[dev];
    }
    const int nb = (int)((n + kPerBlock - 1) / kPerBlock);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_noalloc_partials<<<nb, kThreads, 0, st>>>((long long)n, x, utype, w, (double*)part);
    k_noalloc_total<<<1, kThreads, 0, st>>>((const double*)part, nb, objective);
    pmp::note_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pmp::report_cuda_error(e, "launching the reduction");
    pmp::clear_error();
    return NUM_OK;
}
