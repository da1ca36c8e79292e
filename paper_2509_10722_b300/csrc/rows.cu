// Row-parallel variant of the two fused kernels of one PMP iteration (same arithmetic as
// the tile engine in fused.cu; see the derivation there).  On this GPU the iteration is
// bound by random gathers from L2 (one 32-byte sector per gathered value), so the design
// goal is to keep as many gathers in flight as possible with no block-wide barriers:
//
//   stream kernel: one warp takes 32 consecutive streams, loads their route entries as
//     one contiguous coalesced segment, gathers (pbar, y) for every entry into a
//     warp-private shared buffer, then each lane sums its own route and runs the prox
//     epilogue for its stream (routes longer than the buffer: the lane gathers directly);
//   link kernel: one warp per link (two entries per lane in flight), the link epilogue by
//     lane 0; links with more than kLongRow streams are cut into fixed chunks of kChunk
//     entries, each chunk summed by one warp into its own slot, and the warp that brings
//     the row's arrival count to the number of chunks sums the slots in chunk order and
//     runs the epilogue (no waiting, deterministic);
//   the last block of the link kernel finishes the iteration (FP64 residual sums, stopping
//   test, rho), as in the tile engine.
#include <cuda_runtime.h>

#include "pmp_device.cuh"
#include "pmp_internal.cuh"

namespace pmp {

namespace {

constexpr int kTh = 256;
constexpr int kWarps = kTh / 32;
constexpr int kCap = 512;  // route entries of one warp tile held in shared memory

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ---- stream kernel -------------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kTh) k_stream_rows(View<T> v) {
    using V = typename Pair<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw) + (threadIdx.x >> 5) * kCap;
    __shared__ double red[kWarps];
    const Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    const T alpha = (T)ctl->alpha;
    const T inv_rho = (T)(1.0 / ctl->rho);
    const int lane = threadIdx.x & 31;
    const int n = v.n;
    const int* __restrict__ col_ptr = v.col_ptr;
    const int* __restrict__ row_idx = v.row_idx;
    const V* __restrict__ pby = v.pby;
    double dacc = 0.0;
    const int wstride = gridDim.x * kWarps * 32;
    for (int j0 = (blockIdx.x * kWarps + (threadIdx.x >> 5)) * 32; j0 < n; j0 += wstride) {
        const int j = j0 + lane;
        const bool valid = j < n;
        const int jc = valid ? j : n;
        const int p = __ldg(col_ptr + jc);
        int pn = __shfl_down_sync(0xffffffffu, p, 1);
        if (lane == 31 || jc == n) pn = __ldg(col_ptr + (jc < n ? jc + 1 : n));
        // epilogue state early, so its loads overlap the gathers
        T xo = T(0), Zo = T(0), wt = T(0), lo = v.lo_u, hi = v.hi_u;
        if (valid) {
            xo = v.x[j];
            Zo = v.Z[j];
            wt = __ldg(v.wt + j);
            if (!v.box_uniform) {
                lo = __ldg(v.lo + j);
                hi = __ldg(v.hi + j);
            }
        }
        const int seg0 = __shfl_sync(0xffffffffu, p, 0);
        const int seg1 = __shfl_sync(0xffffffffu, pn, 31);
        const int cnt = seg1 - seg0;
        V sum = vzero(V());
        if (cnt <= kCap) {
            for (int e0 = 0; e0 < cnt; e0 += 128) {
                int l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * 32 + lane;
                    l[u] = e < cnt ? __ldg(row_idx + seg0 + e) : -1;
                }
                V g[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) g[u] = l[u] >= 0 ? __ldg(pby + l[u]) : vzero(V());
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * 32 + lane;
                    if (e < cnt) buf[e] = g[u];
                }
            }
            __syncwarp();
            if (valid)
                for (int e = p - seg0; e < pn - seg0; ++e) sum = vadd(sum, buf[e]);
            __syncwarp();
        } else if (valid) {
            for (int e = p; e < pn; ++e) sum = vadd(sum, __ldg(pby + __ldg(row_idx + e)));
        }
        if (valid) {
            const T L = (T)(pn - p);
            const T Zn = alpha * L * xo + (T(1) - alpha) * Zo - alpha * sum.x;
            const T S = Zn - sum.y * inv_rho;
            const T xn = stream_prox<T>(S, L, wt, inv_rho, lo, hi);
            v.Z[j] = Zn;
            v.x[j] = xn;
            const T dx = xn - xo;
            dacc += (double)(L * dx * dx);
        }
    }
    const double s = block_sum(dacc, red);
    if (threadIdx.x == 0) v.part_s[blockIdx.x] = s;
}

// ---- link kernel ---------------------------------------------------------------------------------

// Link epilogue (slack prox, average, z and price updates) and its residual terms.
template <typename T>
__device__ __forceinline__ void link_epilogue(const View<T>& v, int l, T Rxn, int deg, T alpha,
                                              T rho, T inv_rho, double& r2, double& s2) {
    using T2 = typename Pair<T>::type;
    const T2 py = v.pby[l];
    const T pbo = py.x, y = py.y;
    const T Rxo = v.Rx[l], pso = v.ps[l], zso = v.zs[l], cl = __ldg(v.c + l);
    T psn = zso - y * inv_rho;
    psn = psn < -cl ? -cl : psn;
    const T degf = (T)deg;
    const T pbn = (Rxn + psn) / (degf + T(1));
    T2 out;
    out.x = pbn;
    out.y = y + alpha * rho * pbn;
    v.pby[l] = out;
    v.zs[l] = alpha * (psn - pbn) + (T(1) - alpha) * zso;
    v.Rx[l] = Rxn;
    v.ps[l] = psn;
    const T dpb = pbn - pbo, dRx = Rxn - Rxo, dd = (psn - pbn) - (pso - pbo);
    r2 += (double)((degf + T(1)) * pbn * pbn);
    s2 += (double)(degf * dpb * dpb - T(2) * dpb * dRx + dd * dd);
}

// Sum of x over entries [e0, e1) of the link-major index array, by the whole warp, in a
// fixed order (lane-strided, two loads in flight per lane, then a shuffle tree).
template <typename T>
__device__ __forceinline__ T warp_gather_sum(const int* __restrict__ col_idx,
                                             const T* __restrict__ x, int e0, int e1, int lane) {
    T s = T(0);
    for (int e = e0 + lane; e < e1; e += 64) {
        const int i0 = __ldg(col_idx + e);
        const int i1 = e + 32 < e1 ? __ldg(col_idx + e + 32) : -1;
        const T a = __ldg(x + i0);
        const T b = i1 >= 0 ? __ldg(x + i1) : T(0);
        s += a + b;
    }
    return warp_sum_t(s);
}

template <typename T>
__global__ void __launch_bounds__(kTh) k_link_rows(View<T> v) {
    __shared__ double red[kWarps];
    __shared__ int last;
    Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    const T alpha = (T)ctl->alpha, rho = (T)ctl->rho, inv_rho = (T)(1.0 / ctl->rho);
    const int lane = threadIdx.x & 31;
    const int m = v.m;
    const int* __restrict__ row_ptr = v.row_ptr;
    const int* __restrict__ col_idx = v.col_idx;
    const T* __restrict__ x = v.x;
    double r2 = 0.0, s2 = 0.0;
    const int items = m + v.nchunks;
    const int wstride = gridDim.x * kWarps;
    for (int it = blockIdx.x * kWarps + (threadIdx.x >> 5); it < items; it += wstride) {
        if (it < m) {
            const int p0 = __ldg(row_ptr + it), p1 = __ldg(row_ptr + it + 1);
            if (p1 - p0 > kLongRow) continue;  // done by its chunks
            const T s = warp_gather_sum(col_idx, x, p0, p1, lane);
            if (lane == 0) link_epilogue(v, it, s, p1 - p0, alpha, rho, inv_rho, r2, s2);
        } else {
            const int4 ch = __ldg(v.chunks + (it - m));  // (row, first entry, end entry, first chunk)
            const T s = warp_gather_sum(col_idx, x, ch.y, ch.z, lane);
            int fin = 0;
            if (lane == 0) {
                v.carry_l[it - m] = s;
                __threadfence();
                const int p0 = __ldg(row_ptr + ch.x), p1 = __ldg(row_ptr + ch.x + 1);
                const int nch = (p1 - p0 + kChunk - 1) / kChunk;
                fin = atomicAdd(v.arrive_l + ch.w, 1) == nch - 1;
            }
            fin = __shfl_sync(0xffffffffu, fin, 0);
            if (fin) {  // every chunk of the row is in: sum the slots in chunk order
                __threadfence();
                const int p0 = __ldg(row_ptr + ch.x), p1 = __ldg(row_ptr + ch.x + 1);
                const int nch = (p1 - p0 + kChunk - 1) / kChunk;
                T t = T(0);
                for (int q = lane; q < nch; q += 32) t += __ldcg(v.carry_l + ch.w + q);
                t = warp_sum_t(t);
                if (lane == 0) {
                    v.arrive_l[ch.w] = 0;
                    link_epilogue(v, ch.x, t, p1 - p0, alpha, rho, inv_rho, r2, s2);
                }
            }
        }
    }
    const double R2 = block_sum(r2, red);
    const double S2 = block_sum(s2, red);
    if (threadIdx.x == 0) {
        v.part_l[2 * blockIdx.x] = R2;
        v.part_l[2 * blockIdx.x + 1] = S2;
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        const double a = block_sum_global(v.part_l, gridDim.x, 2, red);
        const double b = block_sum_global(v.part_l + 1, gridDim.x, 2, red);
        const double c = block_sum_global(v.part_s, v.grid_s, 1, red);
        if (threadIdx.x == 0) {
            ctl->ticket = 0;
            finalize_iteration(ctl, a, c + b, v.hist, v.sched);
        }
    }
}

template <typename T>
size_t stream_smem() {
    return sizeof(typename Pair<T>::type) * kCap * kWarps;
}

template <typename T>
cudaError_t rows_occupancy(int* occ_s, int* occ_l) {
    cudaError_t e = cudaFuncSetAttribute(k_stream_rows<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)stream_smem<T>());
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_s, k_stream_rows<T>, kTh,
                                                      stream_smem<T>());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_l, k_link_rows<T>, kTh, 0);
}

}  // namespace

cudaError_t rows_grids(int precision, int n, int m, int nchunks, int* grid_s, int* grid_l) {
    int dev = 0, sms = 0, occ_s = 0, occ_l = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = precision == 0 ? rows_occupancy<float>(&occ_s, &occ_l) : rows_occupancy<double>(&occ_s, &occ_l);
    if (e != cudaSuccess) return e;
    if (occ_s < 1 || occ_l < 1) return cudaErrorInvalidConfiguration;
    const long long need_s = ((long long)n + kTh - 1) / kTh;
    const long long need_l = ((long long)m + nchunks + kWarps - 1) / kWarps;
    long long gs = (long long)occ_s * sms, gl = (long long)occ_l * sms;
    gs = gs < need_s ? gs : need_s;
    gl = gl < need_l ? gl : need_l;
    *grid_s = (int)(gs < kMaxRowsGrid ? gs : kMaxRowsGrid);
    *grid_l = (int)(gl < kMaxRowsGrid ? gl : kMaxRowsGrid);
    return cudaSuccess;
}

template <typename T>
cudaError_t rows_iteration(const View<T>& v, cudaStream_t st, cudaEvent_t* evs) {
    k_stream_rows<T><<<v.grid_s, kTh, stream_smem<T>(), st>>>(v);
    if (evs) cudaEventRecordWithFlags(evs[0], st, cudaEventRecordExternal);
    k_link_rows<T><<<v.grid_l, kTh, 0, st>>>(v);
    if (evs) cudaEventRecordWithFlags(evs[1], st, cudaEventRecordExternal);
    return cudaGetLastError();
}
template cudaError_t rows_iteration<float>(const View<float>&, cudaStream_t, cudaEvent_t*);
template cudaError_t rows_iteration<double>(const View<double>&, cudaStream_t, cudaEvent_t*);

}  // namespace pmp
