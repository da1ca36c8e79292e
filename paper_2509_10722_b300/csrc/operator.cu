// Setup of one NUM instance on the device: input validation, the link-major (CSR) copy of
// the 0/1 link-route matrix R of Sec. II built from its routes (CSC) by a stable radix sort,
// the tile tables of the fused kernels, parameter conversion, and the small control and
// export kernels.  None of this runs per iteration.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "pmp_device.cuh"
#include "pmp_internal.cuh"

namespace pmp {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long count, int per_block = kThreads, int cap = 1 << 20) {
    long long b = (count + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// order-preserving map of a double onto unsigned 64-bit keys (for atomic min / max)
__device__ __forceinline__ unsigned long long ordered_key(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// Every route nonempty, the pointers increasing from 0.
__global__ void k_validate_routes(int n, const int64_t* __restrict__ route_ptr, int* err) {
    int bits = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int64_t p0 = route_ptr[j], p1 = route_ptr[j + 1];
        if (p1 <= p0 || (j == 0 && p0 != 0)) bits |= VB_ROUTE;
    }
    if (bits) atomicOr(err, bits);
}

__global__ void k_validate_streams(int n, const uint8_t* __restrict__ utype,
                                   const double* __restrict__ w, const double* __restrict__ lo,
                                   const double* __restrict__ hi, int* err,
                                   unsigned long long* box) {
    int bits = 0, alpha2 = 0;
    unsigned long long lo_min = ~0ull, lo_max = 0ull, hi_min = ~0ull, hi_max = 0ull;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double wj = w[j];
        if (!(wj > 0.0) || !isfinite(wj)) bits |= VB_WEIGHT;
        const uint8_t t = utype[j];
        if (t > 2) bits |= VB_UTYPE;
        if (t == 2) alpha2 = 1;
        const double l = lo ? lo[j] : 0.0, h = hi[j];
        if (!isfinite(l) || !isfinite(h) || l > h || (t != 1 && !(h > 0.0))) bits |= VB_BOX;
        const unsigned long long kl = ordered_key(l), kh = ordered_key(h);
        lo_min = kl < lo_min ? kl : lo_min;
        lo_max = kl > lo_max ? kl : lo_max;
        hi_min = kh < hi_min ? kh : hi_min;
        hi_max = kh > hi_max ? kh : hi_max;
    }
    if (bits) atomicOr(err, bits);
    if (alpha2) atomicOr(err + 1, 1);  // some stream has U = -w / x
    // box extremes: warp shuffles, then the block, then one atomic per block and value
    // (a global atomic per thread on four shared addresses serialises in L2)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo_min, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, lo_max, o);
        const unsigned long long c = __shfl_xor_sync(0xffffffffu, hi_min, o);
        const unsigned long long d = __shfl_xor_sync(0xffffffffu, hi_max, o);
        lo_min = a < lo_min ? a : lo_min;
        lo_max = b > lo_max ? b : lo_max;
        hi_min = c < hi_min ? c : hi_min;
        hi_max = d > hi_max ? d : hi_max;
    }
    __shared__ unsigned long long ext[4][kThreads / 32];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        ext[0][warp] = lo_min;
        ext[1][warp] = lo_max;
        ext[2][warp] = hi_min;
        ext[3][warp] = hi_max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            lo_min = ext[0][q] < lo_min ? ext[0][q] : lo_min;
            lo_max = ext[1][q] > lo_max ? ext[1][q] : lo_max;
            hi_min = ext[2][q] < hi_min ? ext[2][q] : hi_min;
            hi_max = ext[3][q] > hi_max ? ext[3][q] : hi_max;
        }
        atomicMin(box + 0, lo_min);
        atomicMax(box + 1, lo_max);
        atomicMin(box + 2, hi_min);
        atomicMax(box + 3, hi_max);
    }
}

__global__ void k_validate_link_ids(int m, long long nnz, const int* __restrict__ route_links,
                                    int* err) {
    int bits = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int l = route_links[e];
        if (l < 0 || l >= m) bits |= VB_LINK_ID;
    }
    if (bits) atomicOr(err, bits);
}

__global__ void k_validate_capacities(int m, const double* __restrict__ c, int* err) {
    int bits = 0;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < m; l += gridDim.x * blockDim.x) {
        const double cl = c[l];
        if (!(cl > 0.0) || !isfinite(cl)) bits |= VB_CAPACITY;
    }
    if (bits) atomicOr(err, bits);
}

__global__ void k_validate_positive(int count, const double* __restrict__ a, int* err) {
    int bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const double v = a[i];
        if (!(v > 0.0) || !isfinite(v)) bad = 1;
    }
    if (bad) atomicOr(err, 1);
}

__global__ void k_init_box(unsigned long long* box) {
    box[0] = ~0ull;
    box[1] = 0ull;
    box[2] = ~0ull;
    box[3] = 0ull;
}

// CSC pointer to int32, and the stream id of every route entry (the sort's payload)
__global__ void k_expand_routes(int n, const int64_t* __restrict__ route_ptr, int* col_ptr,
                                int* stream_of) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += gridDim.x * blockDim.x) {
        const int p0 = (int)route_ptr[j];
        col_ptr[j] = p0;
        if (j < n) {
            const int p1 = (int)route_ptr[j + 1];
            for (int e = p0; e < p1; ++e) stream_of[e] = j;
        }
    }
}

// ---- stable LSD radix sort of (link id, stream id) pairs by link id ----------------------------
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const int* __restrict__ keys, int count, int shift, int* hist, int nblocks) {
    __shared__ int cnt[kRadix];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
        const int e = base + k * kSortThreads + threadIdx.x;
        if (e < count) atomicAdd(&cnt[(keys[e] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter with the offsets of an exclusive scan of the digit-major histogram.  Within a
// block, keys are ranked in their original order (rounds of 256 in order; inside a round,
// warps in order and lanes in order), which makes every pass stable.
__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const int* __restrict__ keys_in, const int* __restrict__ vals_in, int count,
                int shift, const int* __restrict__ offs, int nblocks, int* keys_out,
                int* vals_out) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ int run[kRadix];
    __shared__ int wcnt[kWarps][kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offs[(size_t)tid * nblocks + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int base = blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        for (int i = tid; i < kWarps * kRadix; i += kSortThreads) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int e = base + k * kSortThreads + tid;
        const bool valid = e < count;
        const int key = valid ? keys_in[e] : 0;
        const int d = valid ? ((key >> shift) & (kRadix - 1)) : kRadix;  // kRadix: no digit
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        int total = 0;
        for (int w = 0; w < kWarps; ++w) {  // exclusive prefix over warps of digit `tid`
            const int cw = wcnt[w][tid];
            wcnt[w][tid] = total;
            total += cw;
        }
        __syncthreads();
        if (valid) {
            const int pos = run[d] + wcnt[warp][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = vals_in[e];
        }
        __syncthreads();
        run[tid] += total;
    }
}

// ---- exclusive scan of int32 (values and total < 2^31) ----------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const int* in, int* out, size_t len, int* tile_sums) {  // in may equal out
    __shared__ int wsum[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)tid * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < len) ? in[base + i] : 0;
        s += v[i];
    }
    int incl = s;  // inclusive scan of the thread sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += wsum[w];
    int run = wbase + incl - s;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < len) out[base + i] = run;
        run += v[i];
    }
    if (tid == kScanThreads - 1 && tile_sums) tile_sums[blockIdx.x] = wbase + incl;
}

__global__ void k_scan_add(int* out, size_t len, const int* __restrict__ tile_offs) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += stride)
        out[i] += tile_offs[i / kScanTile];
}

cudaError_t scan_exclusive(const int* in, int* out, size_t len, int* tmp, cudaStream_t st) {
    const size_t tiles = (len + kScanTile - 1) / kScanTile;
    if (tiles <= 1) {
        k_scan_tiles<<<1, kScanThreads, 0, st>>>(in, out, len, nullptr);
        note_launches(1);
        return cudaGetLastError();
    }
    int* sums = tmp;
    int* sums_scanned = tmp + tiles;
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, len, sums);
    note_launches(1);
    cudaError_t e = scan_exclusive(sums, sums_scanned, tiles, tmp + 2 * tiles, st);
    if (e != cudaSuccess) return e;
    k_scan_add<<<blocks_for((long long)len, kThreads, 65535), kThreads, 0, st>>>(out, len,
                                                                                 sums_scanned);
    note_launches(1);
    return cudaGetLastError();
}

// row_ptr from link ids sorted ascending: row_ptr[l] = first position with key >= l
__global__ void k_row_ptr(const int* __restrict__ keys, int nnz, int m, int* row_ptr) {
    const int stride = gridDim.x * blockDim.x;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= nnz; e += stride) {
        const int prev = e == 0 ? -1 : keys[e - 1];
        const int cur = e == nnz ? m : keys[e];
        for (int l = prev + 1; l <= cur; ++l) row_ptr[l] = e;
    }
}

// a duplicate link in one route shows up as two equal (link, stream) pairs side by side
__global__ void k_find_duplicates(const int* __restrict__ keys, const int* __restrict__ vals,
                                  int nnz, int* err) {
    const int stride = gridDim.x * blockDim.x;
    bool dup = false;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x + 1; e < nnz; e += stride)
        dup |= (keys[e] == keys[e - 1]) && (vals[e] == vals[e - 1]);
    if (dup) atomicOr(err, VB_DUPLICATE);
}

// ---- stream relabeling: streams ordered by the first link of their route ---------------------
__global__ void k_first_link(int n, const int64_t* __restrict__ route_ptr,
                             const int* __restrict__ route_links, int* keys, int* vals) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        keys[j] = route_links[route_ptr[j]];
        vals[j] = j;
    }
}

// lens[j] = route length of the stream placed at position j (lens[n] = 0, for the scan)
__global__ void k_perm_lengths(int n, const int64_t* __restrict__ route_ptr,
                               const int* __restrict__ perm, int* lens) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += gridDim.x * blockDim.x)
        lens[j] = j < n ? (int)(route_ptr[perm[j] + 1] - route_ptr[perm[j]]) : 0;
}

__global__ void k_perm_routes(int n, const int64_t* __restrict__ route_ptr,
                              const int* __restrict__ route_links, const int* __restrict__ perm,
                              const int* __restrict__ ptr32, int64_t* route_ptr_new,
                              int* route_links_new) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += gridDim.x * blockDim.x) {
        route_ptr_new[j] = ptr32[j];
        if (j < n) {
            const int64_t src = route_ptr[perm[j]];
            const int len = ptr32[j + 1] - ptr32[j];
            for (int e = 0; e < len; ++e) route_links_new[ptr32[j] + e] = route_links[src + e];
        }
    }
}

__global__ void k_chunk_counts(const int* __restrict__ row_ptr, int m, int* counts) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l <= m; l += gridDim.x * blockDim.x) {
        int c = 0;
        if (l < m) {
            const int deg = row_ptr[l + 1] - row_ptr[l];
            c = deg > kLongRow ? (deg + kChunk - 1) / kChunk : 0;
        }
        counts[l] = c;
    }
}

// flags[j] = 1 for a stream with more than kLongRoute links (j < n), 0 otherwise (j <= n)
__global__ void k_long_route_flags(const int* __restrict__ col_ptr, int n, int* flags) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += gridDim.x * blockDim.x)
        flags[j] = j < n && col_ptr[j + 1] - col_ptr[j] > kLongRoute ? 1 : 0;
}

__global__ void k_long_route_fill(const int* __restrict__ col_ptr, int n,
                                  const int* __restrict__ offs, int* list) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (col_ptr[j + 1] - col_ptr[j] > kLongRoute) list[offs[j]] = j;
}

__global__ void k_chunk_fill(const int* __restrict__ row_ptr, int m, const int* __restrict__ offs,
                             int4* chunks) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < m; l += gridDim.x * blockDim.x) {
        const int p0 = row_ptr[l], p1 = row_ptr[l + 1];
        if (p1 - p0 <= kLongRow) continue;
        const int first = offs[l];
        for (int c = 0; first + c < offs[l + 1]; ++c) {
            const int e0 = p0 + c * kChunk;
            const int e1 = e0 + kChunk < p1 ? e0 + kChunk : p1;
            chunks[first + c] = make_int4(l, e0, e1, first);
        }
    }
}

// Sort keys of the chunk queue: kChunk - length (0 for a full chunk), value the chunk index.
__global__ void k_chunk_keys(const int4* __restrict__ chunks, int nchunks, int* keys, int* vals) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nchunks; q += gridDim.x * blockDim.x) {
        const int4 ch = chunks[q];
        keys[q] = kChunk - (ch.z - ch.y);
        vals[q] = q;
    }
}

template <typename T>
__global__ void k_convert(int n, int m, const double* __restrict__ c,
                          const uint8_t* __restrict__ utype, const double* __restrict__ w,
                          const double* __restrict__ lo, const double* __restrict__ hi,
                          const int* __restrict__ perm, T* c_t, T* wt_t, T* lo_t, T* hi_t,
                          uint8_t* ut_out) {
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const int o = perm ? perm[j] : j;  // original index of the stream at position j
        const T wj = (T)w[o];
        wt_t[j] = utype[o] == 1 ? -wj : wj;  // log and alpha = 2: +w; linear: -w
        if (ut_out) ut_out[j] = utype[o];
        if (lo_t) lo_t[j] = lo ? (T)lo[o] : T(0);
        if (hi_t) hi_t[j] = (T)hi[o];
    }
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < m; l += stride) c_t[l] = (T)c[l];
}

__global__ void k_ctl_arm(Ctl* ctl, long long k_limit, double eps_tol) {
    ctl->k_limit = k_limit;
    ctl->eps_tol = eps_tol;
    ctl->stop = RUNNING;
}

__global__ void k_ctl_reset(Ctl* ctl, double rho0, double alpha, double mu, double gamma,
                            int period, int hist_len) {
    Ctl c;
    memset(&c, 0, sizeof(c));
    c.rho = rho0;
    c.alpha = alpha;
    c.mu = mu;
    c.gamma = gamma;
    c.period = period;
    c.hist_len = hist_len;
    *ctl = c;
}

__global__ void k_ctl_sched(Ctl* ctl, int len) { ctl->sched_len = len; }

// ---- solution export ------------------------------------------------------------------------
constexpr int kExportThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kExportThreads)
k_export(View<T> v, double* x_out, double* y_out, double* part) {
    __shared__ double red[kExportThreads / 32];
    double obj = 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += stride) {
        const double xj = (double)v.x[j];
        const double wt = (double)v.wt[j];
        if (x_out) x_out[v.perm ? v.perm[j] : j] = xj;  // back to the caller's stream order
        if (v.ut && v.ut[j] == 2)
            obj += -wt / xj;  // U_j(x_j), Sec. II
        else
            obj += wt > 0.0 ? wt * log(xj) : -wt * xj;
    }
    if (y_out) {
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < v.m; l += stride)
            y_out[l] = v.y ? (double)v.y[l] : (double)v.pby[l].y;
    }
    const double s = block_sum(obj, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s;
        __threadfence();
        const unsigned t = atomicAdd(&v.ctl->ticket2, 1u);
        red[0] = (t == gridDim.x - 1) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (red[0] != 0.0) {  // last block: FP64 sum of the block partials in block order
        __syncthreads();
        __threadfence();
        const double tot = block_sum_global(part, gridDim.x, 1, red);
        if (threadIdx.x == 0) {
            v.ctl->objective = tot;
            v.ctl->ticket2 = 0;
        }
    }
}

// ---- iterate export / import (warm starts) -----------------------------------------------------
// which: 0 x, 1 Z (per stream, caller order); 2 pbar, 3 y, 4 zs, 5 Rx, 6 ps (per link)
template <typename T>
__device__ __forceinline__ T* state_array(const View<T>& v, int which) {
    switch (which) {
        case 0: return v.x;
        case 1: return v.Z;
        case 4: return v.zs;
        case 5: return v.Rx;
        case 6: return v.ps;
        default: return nullptr;
    }
}

template <typename T>
__global__ void k_state_out(View<T> v, int which, double* out) {
    const int count = which < 2 ? v.n : v.m;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x) {
        double val;
        if (which == 2)
            val = v.pbar ? (double)v.pbar[j] : (double)v.pby[j].x;
        else if (which == 3)
            val = v.y ? (double)v.y[j] : (double)v.pby[j].y;
        else
            val = (double)state_array(v, which)[j];
        const int dst = (which < 2 && v.perm) ? v.perm[j] : j;  // caller's stream order
        out[dst] = val;
    }
}

template <typename T>
__global__ void k_state_in(View<T> v, int which, const double* in) {
    const int count = which < 2 ? v.n : v.m;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x) {
        const double val = in[(which < 2 && v.perm) ? v.perm[j] : j];
        if (which == 2) {
            if (v.pbar) v.pbar[j] = (T)val; else v.pby[j].x = (T)val;
        } else if (which == 3) {
            if (v.y) v.y[j] = (T)val; else v.pby[j].y = (T)val;
        } else {
            state_array(v, which)[j] = (T)val;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------

size_t radix_hist_len(int nnz) {
    const size_t nblocks = ((size_t)nnz + kSortTile - 1) / kSortTile;
    return (nblocks < 1 ? 1 : nblocks) * kRadix;
}

size_t scan_tmp_len(size_t len) {
    size_t total = 0;
    size_t tiles = (len + kScanTile - 1) / kScanTile;
    while (tiles > 1) {
        total += 2 * tiles;
        tiles = (tiles + kScanTile - 1) / kScanTile;
    }
    return total + 2;
}

double ordered_key_to_double(unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ull) ? (k & ~0x8000000000000000ull) : ~k;
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
}

cudaError_t validate_routes(int n, int m, long long nnz, const int64_t* route_ptr,
                            const int* route_links, int* err_bits, cudaStream_t st) {
    k_validate_routes<<<blocks_for(n, kThreads, 4096), kThreads, 0, st>>>(n, route_ptr, err_bits);
    note_launches(1);
    k_validate_link_ids<<<blocks_for(nnz, kThreads, 8192), kThreads, 0, st>>>(m, nnz, route_links,
                                                                              err_bits);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t validate_positive(int count, const double* a, int* err, cudaStream_t st) {
    k_validate_positive<<<blocks_for(count, kThreads, 4096), kThreads, 0, st>>>(count, a, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t validate_values(int n, int m, const double* c, const uint8_t* utype,
                            const double* w, const double* lo, const double* hi, int* err_bits,
                            unsigned long long* box_minmax, cudaStream_t st) {
    k_init_box<<<1, 1, 0, st>>>(box_minmax);
    note_launches(1);
    k_validate_streams<<<blocks_for(n, kThreads, 4096), kThreads, 0, st>>>(
        n, utype, w, lo, hi, err_bits, box_minmax);
    note_launches(1);
    k_validate_capacities<<<blocks_for(m, kThreads, 4096), kThreads, 0, st>>>(m, c, err_bits);
    note_launches(1);
    return cudaGetLastError();
}

// Stable LSD radix sort of `count` (key, value) pairs held in s.keys_a / s.vals_a by key
// (keys in [0, key_bound)); *keys / *vals receive the buffers holding the sorted pairs.
cudaError_t radix_sort_pairs(int count, int key_bound, const Scratch& s, int** keys, int** vals,
                             cudaStream_t st) {
    cudaError_t e;
    int bits = 0;
    while (bits < 31 && (1ll << bits) < (long long)key_bound) ++bits;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    int *ki = s.keys_a, *vi = s.vals_a, *ko = s.keys_b, *vo = s.vals_b;
    const int nblocks = count > 0 ? (count + kSortTile - 1) / kSortTile : 0;
    for (int p = 0; p < passes && nblocks > 0; ++p) {
        const int shift = p * kRadixBits;
        k_radix_hist<<<nblocks, kSortThreads, 0, st>>>(ki, count, shift, s.hist, nblocks);
        note_launches(1);
        if ((e = scan_exclusive(s.hist, s.hist, (size_t)nblocks * kRadix, s.scan_tmp, st)) !=
            cudaSuccess)
            return e;
        k_radix_scatter<<<nblocks, kSortThreads, 0, st>>>(ki, vi, count, shift, s.hist, nblocks,
                                                          ko, vo);
        note_launches(1);
        int* t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    *keys = ki;
    *vals = vi;
    return cudaGetLastError();
}

cudaError_t build_operator(int n, int m, int nnz, const int64_t* route_ptr,
                           const int* route_links, int* col_ptr, int* row_idx, int* row_ptr,
                           int* col_idx, const Scratch& s, int* err_bits, cudaStream_t st) {
    cudaError_t e;
    k_expand_routes<<<blocks_for(n + 1, kThreads, 65535), kThreads, 0, st>>>(n, route_ptr, col_ptr,
                                                                              s.vals_a);
    note_launches(1);
    if ((e = cudaMemcpyAsync(row_idx, route_links, sizeof(int) * (size_t)nnz,
                             cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(s.keys_a, route_links, sizeof(int) * (size_t)nnz,
                             cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    int *ki = nullptr, *vi = nullptr;
    if ((e = radix_sort_pairs(nnz, m, s, &ki, &vi, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(col_idx, vi, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice,
                             st)) != cudaSuccess)
        return e;
    k_row_ptr<<<blocks_for((long long)nnz + 1, kThreads, 65535), kThreads, 0, st>>>(ki, nnz, m,
                                                                                    row_ptr);
    note_launches(1);
    if (nnz > 1) {
        k_find_duplicates<<<blocks_for(nnz, kThreads, 8192), kThreads, 0, st>>>(ki, vi, nnz,
                                                                                err_bits);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t relabel_streams(int n, int m, const int64_t* route_ptr, const int* route_links,
                            const Scratch& s, int* perm, int* lens, int* ptr32, int* scan_tmp,
                            int64_t* route_ptr_new, int* route_links_new, cudaStream_t st) {
    cudaError_t e;
    k_first_link<<<blocks_for(n, kThreads, 65535), kThreads, 0, st>>>(n, route_ptr, route_links,
                                                                       s.keys_a, s.vals_a);
    note_launches(1);
    int *ki = nullptr, *vi = nullptr;
    if ((e = radix_sort_pairs(n, m, s, &ki, &vi, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(perm, vi, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
        return e;
    k_perm_lengths<<<blocks_for((long long)n + 1, kThreads, 65535), kThreads, 0, st>>>(
        n, route_ptr, perm, lens);
    note_launches(1);
    if ((e = scan_exclusive(lens, ptr32, (size_t)n + 1, scan_tmp, st)) != cudaSuccess) return e;
    k_perm_routes<<<blocks_for((long long)n + 1, kThreads, 65535), kThreads, 0, st>>>(
        n, route_ptr, route_links, perm, ptr32, route_ptr_new, route_links_new);
    note_launches(1);
    return cudaGetLastError();
}


cudaError_t count_chunks(const int* row_ptr, int m, int* counts, int* offs, int* tmp,
                         int* nchunks, cudaStream_t st) {
    k_chunk_counts<<<blocks_for((long long)m + 1, kThreads, 65535), kThreads, 0, st>>>(row_ptr, m,
                                                                                       counts);
    note_launches(1);
    cudaError_t e = scan_exclusive(counts, offs, (size_t)m + 1, tmp, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(nchunks, offs + m, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t count_long_routes(const int* col_ptr, int n, int* flags, int* offs, int* tmp,
                              int* nlong, cudaStream_t st) {
    k_long_route_flags<<<blocks_for((long long)n + 1, kThreads, 65535), kThreads, 0, st>>>(
        col_ptr, n, flags);
    note_launches(1);
    cudaError_t e = scan_exclusive(flags, offs, (size_t)n + 1, tmp, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(nlong, offs + n, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t fill_long_routes(const int* col_ptr, int n, const int* offs, int* list,
                             cudaStream_t st) {
    k_long_route_fill<<<blocks_for(n, kThreads, 65535), kThreads, 0, st>>>(col_ptr, n, offs,
                                                                           list);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t fill_chunks(const int* row_ptr, int m, const int* offs, int4* chunks,
                        cudaStream_t st) {
    k_chunk_fill<<<blocks_for(m, kThreads, 65535), kThreads, 0, st>>>(row_ptr, m, offs, chunks);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t order_chunks(const int4* chunks, int nchunks, const Scratch& s, int* queue,
                         cudaStream_t st) {
    k_chunk_keys<<<blocks_for(nchunks, kThreads, 65535), kThreads, 0, st>>>(chunks, nchunks,
                                                                           s.keys_a, s.vals_a);
    note_launches(1);
    int *ki = nullptr, *vi = nullptr;
    cudaError_t e = radix_sort_pairs(nchunks, kChunk, s, &ki, &vi, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(queue, vi, sizeof(int) * (size_t)nchunks, cudaMemcpyDeviceToDevice, st);
}

template <typename T>
cudaError_t convert_params(int n, int m, const double* c, const uint8_t* utype,
                           const double* w, const double* lo, const double* hi, const int* perm,
                           T* c_t, T* wt_t, T* lo_t, T* hi_t, cudaStream_t st,
                           uint8_t* ut_out) {
    k_convert<T><<<blocks_for(n > m ? n : m, kThreads, 65535), kThreads, 0, st>>>(
        n, m, c, utype, w, lo, hi, perm, c_t, wt_t, lo_t, hi_t, ut_out);
    note_launches(1);
    return cudaGetLastError();
}
template cudaError_t convert_params<float>(int, int, const double*, const uint8_t*,
                                           const double*, const double*, const double*,
                                           const int*, float*, float*, float*, float*,
                                           cudaStream_t, uint8_t*);
template cudaError_t convert_params<double>(int, int, const double*, const uint8_t*,
                                            const double*, const double*, const double*,
                                            const int*, double*, double*, double*, double*,
                                            cudaStream_t, uint8_t*);

int export_partial_blocks(int n) { return blocks_for(n, kExportThreads, 1024); }

template <typename T>
cudaError_t state_transfer(const View<T>& v, int which, double* buf, bool out, cudaStream_t st) {
    const int count = which < 2 ? v.n : v.m;
    if (out)
        k_state_out<T><<<blocks_for(count, kThreads, 65535), kThreads, 0, st>>>(v, which, buf);
    else
        k_state_in<T><<<blocks_for(count, kThreads, 65535), kThreads, 0, st>>>(v, which, buf);
    note_launches(1);
    return cudaGetLastError();
}
template cudaError_t state_transfer<float>(const View<float>&, int, double*, bool, cudaStream_t);
template cudaError_t state_transfer<double>(const View<double>&, int, double*, bool, cudaStream_t);

template <typename T>
cudaError_t export_solution(const View<T>& v, double* x_out, double* y_out, double* part,
                            int part_blocks, cudaStream_t st) {
    k_export<T><<<part_blocks, kExportThreads, 0, st>>>(v, x_out, y_out, part);
    note_launches(1);
    return cudaGetLastError();
}
template cudaError_t export_solution<float>(const View<float>&, double*, double*, double*, int,
                                            cudaStream_t);
template cudaError_t export_solution<double>(const View<double>&, double*, double*, double*,
                                             int, cudaStream_t);

cudaError_t ctl_arm(Ctl* ctl, long long k_limit, double eps_tol, cudaStream_t st) {
    k_ctl_arm<<<1, 1, 0, st>>>(ctl, k_limit, eps_tol);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t ctl_reset(Ctl* ctl, double rho0, double alpha, double mu, double gamma, int period,
                      int hist_len, cudaStream_t st) {
    k_ctl_reset<<<1, 1, 0, st>>>(ctl, rho0, alpha, mu, gamma, period, hist_len);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t ctl_set_schedule_len(Ctl* ctl, int len, cudaStream_t st) {
    k_ctl_sched<<<1, 1, 0, st>>>(ctl, len);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pmp
