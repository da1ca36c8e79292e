// Random-gather rate of the current GPU (num_measure_gather_rate).
//
// Both passes of a PMP iteration (Sec. III-D) gather one value per route entry: the link
// pass reads x of every stream of a link, the stream pass reads the (pbar, y) pair of every
// link of a route.  On a random link-route incidence these are uniformly random reads of a
// vector that lives in L2, one 32-byte sector each, and their rate, not HBM bandwidth,
// bounds the iteration.  This file measures that rate on the GPU at hand: `count` uniformly
// random 4- or 8-byte reads from a vector of `vec_len` elements, four reads in flight per
// thread at full occupancy, timed with CUDA events.  The same with plain stores to random
// positions (num_measure_scatter_rate) measures the alternative of pushing each value to
// a permuted copy and reading that contiguously.  The paper has no counterpart; it is a
// measurement service for reporting the kernels against the ceiling that bounds them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "num_pmp.h"
#include "pmp_internal.cuh"

namespace {

constexpr int kThreads = 256;

// uniformly distributed indices in [0, len): a 64-bit mix of the position, reduced by a
// multiply-shift (no modulo bias worth speaking of at these lengths)
__global__ void k_random_indices(int* idx, long long count, unsigned long long len,
                                 unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long h = (unsigned long long)i + seed;
        h = (h ^ (h >> 30)) * 0xbf58476d1ce4e5b9ULL;
        h = (h ^ (h >> 27)) * 0x94d049bb133111ebULL;
        h ^= h >> 31;
        idx[i] = (int)(((h >> 32) * len) >> 32);
    }
}

template <typename V>
__global__ void k_fill(V* v, long long len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        v[i] = V{};
    }
}

__device__ __forceinline__ float first(float v) { return v; }
__device__ __forceinline__ float first(float2 v) { return v.x + v.y; }

// each thread keeps four independent reads in flight; the sum goes to *sink only if it
// takes an impossible value, so the reads cannot be optimized away
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_gather(const int* __restrict__ idx, long long count, const V* __restrict__ v, float* sink) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float s = 0.f;
    for (; i + 3 * stride < count; i += 4 * stride) {
        const int j0 = __ldg(idx + i), j1 = __ldg(idx + i + stride);
        const int j2 = __ldg(idx + i + 2 * stride), j3 = __ldg(idx + i + 3 * stride);
        s += first(__ldg(v + j0)) + first(__ldg(v + j1)) + first(__ldg(v + j2)) +
             first(__ldg(v + j3));
    }
    for (; i < count; i += stride) s += first(__ldg(v + __ldg(idx + i)));
    if (s == -1.f) *sink = s;
}

// each thread writes four independent values per round to uniformly random positions
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_scatter(const int* __restrict__ idx, long long count, V* __restrict__ v) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < count; i += 4 * stride) {
        const int j0 = __ldg(idx + i), j1 = __ldg(idx + i + stride);
        const int j2 = __ldg(idx + i + 2 * stride), j3 = __ldg(idx + i + 3 * stride);
        v[j0] = V{};
        v[j1] = V{};
        v[j2] = V{};
        v[j3] = V{};
    }
    for (; i < count; i += stride) v[__ldg(idx + i)] = V{};
}

struct Buffers {
    int* idx = nullptr;
    void* vec = nullptr;
    float* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Buffers() {
        if (st) cudaStreamSynchronize(st);
        if (idx) cudaFree(idx);
        if (vec) cudaFree(vec);
        if (sink) cudaFree(sink);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    }
};

int fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return pmp::report_error(NUM_ERR_OOM, std::string("out of device memory: ") + what);
    }
    return pmp::report_cuda_error(e, what);
}

template <typename V>
int measure(long long count, long long len, int repeats, double* rate, bool stores) {
    Buffers b;
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return fail(e, "cudaDeviceGetAttribute");
    if ((e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(e, "cudaStreamCreate");
    if ((e = cudaMalloc(&b.idx, (size_t)count * sizeof(int))) != cudaSuccess)
        return fail(e, "index buffer");
    if ((e = cudaMalloc(&b.vec, (size_t)len * sizeof(V))) != cudaSuccess)
        return fail(e, "gathered vector");
    if ((e = cudaMalloc(&b.sink, sizeof(float))) != cudaSuccess) return fail(e, "sink");
    if ((e = cudaEventCreate(&b.e0)) != cudaSuccess || (e = cudaEventCreate(&b.e1)) != cudaSuccess)
        return fail(e, "cudaEventCreate");
    const int fill_grid = sms * 8;
    k_random_indices<<<fill_grid, kThreads, 0, b.st>>>(b.idx, count, (unsigned long long)len,
                                                       0x9e3779b97f4a7c15ULL);
    k_fill<V><<<fill_grid, kThreads, 0, b.st>>>((V*)b.vec, len);
    // full occupancy: 2048 resident threads per SM
    const int grid = sms * (2048 / kThreads);
    auto pass = [&]() {
        if (stores)
            k_scatter<V><<<grid, kThreads, 0, b.st>>>(b.idx, count, (V*)b.vec);
        else
            k_gather<V><<<grid, kThreads, 0, b.st>>>(b.idx, count, (const V*)b.vec, b.sink);
    };
    pass();  // warm-up
    cudaEventRecord(b.e0, b.st);
    for (int r = 0; r < repeats; ++r) pass();
    cudaEventRecord(b.e1, b.st);
    pmp::note_launches(3 + repeats);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "launching the gather kernels");
    if ((e = cudaEventSynchronize(b.e1)) != cudaSuccess) return fail(e, "gather kernels");
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, b.e0, b.e1)) != cudaSuccess)
        return fail(e, "cudaEventElapsedTime");
    if (!(ms > 0.f)) return pmp::report_error(NUM_ERR_CUDA, "zero elapsed time");
    *rate = (double)count * repeats / (ms * 1e-3);
    return NUM_OK;
}

}  // namespace

namespace {

int measure_rate(int64_t count, int64_t vec_len, int32_t vec_bytes, int32_t repeats,
                 double* rate, bool stores) {
    if (!rate) return pmp::report_error(NUM_ERR_INVALID, "the result pointer is NULL");
    if (count < 1 || count > 2000000000LL)
        return pmp::report_error(NUM_ERR_INVALID, "count must be in [1, 2e9]");
    if (vec_len < 1 || vec_len > 2147483647LL)
        return pmp::report_error(NUM_ERR_INVALID, "vec_len must be in [1, 2^31 - 1]");
    if (vec_bytes != 4 && vec_bytes != 8)
        return pmp::report_error(NUM_ERR_INVALID, "vec_bytes must be 4 or 8");
    if (repeats < 1 || repeats > 1000)
        return pmp::report_error(NUM_ERR_INVALID, "repeats must be in [1, 1000]");
    const int rc = vec_bytes == 4 ? measure<float>(count, vec_len, repeats, rate, stores)
                                  : measure<float2>(count, vec_len, repeats, rate, stores);
    if (rc == NUM_OK) pmp::clear_error();
    return rc;
}

}  // namespace

extern "C" int num_measure_gather_rate(int64_t count, int64_t vec_len, int32_t vec_bytes,
                                       int32_t repeats, double* gathers_per_s) {
    return measure_rate(count, vec_len, vec_bytes, repeats, gathers_per_s, false);
}

extern "C" int num_measure_scatter_rate(int64_t count, int64_t vec_len, int32_t vec_bytes,
                                        int32_t repeats, double* stores_per_s) {
    return measure_rate(count, vec_len, vec_bytes, repeats, stores_per_s, true);
}
