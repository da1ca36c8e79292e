// The two fused kernels of one PMP iteration (Sec. III-D..G) on one GPU.
//
// Per-terminal ADMM collapses to per-stream / per-link state (u is the same on every
// terminal of a link, z sums to zero over a link, and the log / linear prox of Sec. III-E
// depend on their argument only through its sum).  With Z_j = sum of z over stream j's
// terminals, y_l = rho u_l (the unscaled price, so the rescale of Eq. dual-rescale is a
// no-op), and iteration k using rho_k:
//
//   stream kernel (routes, CSC):  A_j = sum_{l in j} pbar_l,  B_j = sum_{l in j} y_l
//       Z_j  <- alpha |j| x_j + (1 - alpha) Z_j - alpha A_j          (z update, Sec. III-G)
//       x_j  <- clip( prox_j( Z_j - B_j / rho ) )                     (prox, Sec. III-E)
//       partial  sum_j |j| (x_j - x_j_prev)^2                         (dual residual)
//   link kernel (CSR):            Rx_l = sum_{j in l} x_j
//       ps_l   <- max(zs_l - y_l / rho, -c_l)                         (slack prox)
//       pbar_l <- (Rx_l + ps_l) / (deg_l + 1)                         (link average)
//       zs_l   <- alpha (ps_l - pbar_l) + (1 - alpha) zs_l
//       y_l    <- y_l + alpha rho pbar_l                              (price update)
//       partials  sum_l (deg_l + 1) pbar_l^2                          (||r||^2)
//                 sum_l [deg_l dpbar^2 - 2 dpbar dRx + (dps - dpbar)^2]  (rest of ||s||^2/rho^2)
//   last block of the link kernel: FP64 sums, norms, stopping test, rho update.
//
// Both kernels are one tile engine: a segmented gather-sum over an "item space" in which
// row r (a stream's route, or a link's stream list) owns its entries followed by one
// row-end item.  Tiles hold a fixed number of items, so a tile's work does not depend on
// how long the rows are (merge-path balancing, needed for Zipf-skewed link degrees).  A
// row cut by tile boundaries is summed from per-tile partials by whichever tile arrives
// last (an arrival counter, no waiting), in tile order, so results are deterministic.
#include <cuda_runtime.h>

#include "pmp_device.cuh"
#include "pmp_internal.cuh"

namespace pmp {

namespace {

constexpr int kTh = 256;           // threads per block of both fused kernels
constexpr int kMaxGrid = 8192;     // upper bound of the persistent grids (partials buffers)
constexpr int kSerialSplitSum = 8; // split rows over at most this many tiles: one-thread sum

__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

template <typename V> __device__ __forceinline__ V ld_cg(const V* p);
template <> __device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ld_cg(const double2* p) { return __ldcg(p); }

__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 shfl_down(float2 v, int o) {
    return make_float2(shfl_down(v.x, o), shfl_down(v.y, o));
}
__device__ __forceinline__ double2 shfl_down(double2 v, int o) {
    return make_double2(shfl_down(v.x, o), shfl_down(v.y, o));
}

// Block sum of a V, valid in thread 0 (fixed order).  `buf` holds kTh / 32 V's.
template <typename V>
__device__ __forceinline__ V block_vsum(V v, V* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = vadd(v, shfl_down(v, o));
    __syncthreads();
    if (lane == 0) buf[warp] = v;
    __syncthreads();
    V s = vzero(V());
    if (threadIdx.x == 0)
        for (int i = 0; i < kTh / 32; ++i) s = vadd(s, buf[i]);
    return s;
}

// Shared-memory carve-up of one tile (sizes in bytes; every V array starts 16-aligned).
template <typename V>
struct TileLayout {
    int tile, maxrows;
    __host__ __device__ size_t red_off() const { return 0; }
    __host__ __device__ size_t vals_off() const { return 64; }
    __host__ __device__ size_t vals_len() const { return (size_t)tile + tile / 16 + 1; }
    __host__ __device__ size_t rsum_off() const { return vals_off() + sizeof(V) * vals_len(); }
    __host__ __device__ size_t cval_off() const { return rsum_off() + sizeof(V) * maxrows; }
    __host__ __device__ size_t split_off() const { return cval_off() + sizeof(V) * kTh; }
    __host__ __device__ size_t sptr_off() const { return split_off() + sizeof(V) * 4; }
    __host__ __device__ size_t crow_off() const { return sptr_off() + 4 * (size_t)(maxrows + 1); }
    __host__ __device__ size_t sinfo_off() const { return crow_off() + 4 * (size_t)kTh; }
    __host__ __device__ size_t bytes() const { return sinfo_off() + 4 * 8; }
};

// Rows intersecting one tile: every row has >= 1 item (link rows may have no entries);
// stream rows have >= 2 (routes are nonempty).
__host__ __device__ inline int max_rows_link(int tile) { return tile; }
__host__ __device__ inline int max_rows_stream(int tile) { return tile / 2 + 1; }

// ---- policies: what is gathered and what the row-end epilogue does -----------------------------

template <typename T>
struct StreamPolicy {
    using V = typename Pair<T>::type;
    View<T> v;
    T alpha, inv_rho;
    __device__ const int* ptr() const { return v.col_ptr; }
    __device__ const int* idx() const { return v.row_idx; }
    __device__ int J() const { return v.Js; }
    __device__ const int2* tiles() const { return v.tiles_s; }
    __device__ int ntiles() const { return v.ntiles_s; }
    __device__ V* carry() const { return v.carry_s; }
    __device__ int* arrive() const { return v.arrive_s; }
    __device__ V gather(int l) const { return __ldg(v.pby + checked_index(l, v.m, v.dbg)); }
    // stream j: sum = (A_j, B_j), L = |j|
    __device__ void epilogue(int j, V sum, int L, double& acc0, double&) const {
        const T Lf = (T)L;
        const T xo = v.x[j], Zo = v.Z[j], wt = __ldg(v.wt + j);
        const T Zn = alpha * Lf * xo + (T(1) - alpha) * Zo - alpha * sum.x;
        const T S = Zn - sum.y * inv_rho;
        const T lo = v.box_uniform ? v.lo_u : __ldg(v.lo + j);
        const T hi = v.box_uniform ? v.hi_u : __ldg(v.hi + j);
        const T xn = stream_prox<T>(S, Lf, wt, inv_rho, lo, hi, v.ut && v.ut[j] == 2);
        v.Z[j] = Zn;
        v.x[j] = xn;
        const T dx = xn - xo;
        acc0 += (double)(Lf * dx * dx);
    }
};

template <typename T>
struct LinkPolicy {
    using V = T;
    using T2 = typename Pair<T>::type;
    View<T> v;
    T alpha, rho, inv_rho;
    __device__ const int* ptr() const { return v.row_ptr; }
    __device__ const int* idx() const { return v.col_idx; }
    __device__ int J() const { return v.Jl; }
    __device__ const int2* tiles() const { return v.tiles_l; }
    __device__ int ntiles() const { return v.ntiles_l; }
    __device__ V* carry() const { return v.carry_l; }
    __device__ int* arrive() const { return v.arrive_l; }
    __device__ V gather(int j) const { return __ldg(v.x + checked_index(j, v.n, v.dbg)); }
    // link l: sum = (R x)_l, deg = number of streams on l
    __device__ void epilogue(int l, V Rxn, int deg, double& acc0, double& acc1) const {
        const T2 py = v.pby[l];
        const T pbo = py.x, y = py.y;
        const T Rxo = v.Rx[l], pso = v.ps[l], zso = v.zs[l], cl = __ldg(v.c + l);
        T psn = zso - y * inv_rho;
        psn = psn < -cl ? -cl : psn;  // comparison form keeps a NaN visible
        const T degf = (T)deg;
        const T pbn = (Rxn + psn) / (degf + T(1));
        const T zsn = alpha * (psn - pbn) + (T(1) - alpha) * zso;
        const T yn = y + alpha * rho * pbn;
        T2 out;
        out.x = pbn;
        out.y = yn;
        v.pby[l] = out;
        v.zs[l] = zsn;
        v.Rx[l] = Rxn;
        v.ps[l] = psn;
        acc0 += (double)((degf + T(1)) * pbn * pbn);
        const T dpb = pbn - pbo, dRx = Rxn - Rxo, dd = (psn - pbn) - (pso - pbo);
        acc1 += (double)(degf * dpb * dpb - T(2) * dpb * dRx + dd * dd);
    }
};

// ---- the tile engine -------------------------------------------------------------------------------
// Processes tiles blockIdx.x, blockIdx.x + gridDim.x, ... and adds the epilogues' residual
// partials of this thread to dacc0 / dacc1 (FP64).
template <typename T, int ITEMS, class P>
__device__ __forceinline__ void seg_tiles(const P& p, unsigned char* smem, int maxrows,
                                          double& dacc0, double& dacc1) {
    using V = typename P::V;
    constexpr int TILE = kTh * ITEMS;
    TileLayout<V> lay{TILE, maxrows};
    V* vals = (V*)(smem + lay.vals_off());
    V* rsum = (V*)(smem + lay.rsum_off());
    V* cval = (V*)(smem + lay.cval_off());
    V* split = (V*)(smem + lay.split_off());
    int* sptr = (int*)(smem + lay.sptr_off());
    int* crow = (int*)(smem + lay.crow_off());
    int* sinfo = (int*)(smem + lay.sinfo_off());

    const int tid = threadIdx.x;
    const int* __restrict__ ptr = p.ptr();
    const int* __restrict__ idx = p.idx();
    const int J = p.J();
    const int ntiles = p.ntiles();

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int j0 = t * TILE;
        const int j1 = min(j0 + TILE, J);
        const int2 tr = __ldg(p.tiles() + t);
        const int r0 = tr.x, rl = tr.y, nr = rl - r0 + 1;
        const int end_last = __ldg(ptr + rl + 1) + rl;  // row-end item of the tile's last row
        const bool last_ends = end_last < j1;
        const int nnz_lo = j0 - r0;                      // entries before the tile
        const int cnt = (j1 - j0) - (rl - r0) - (last_ends ? 1 : 0);

        // 1. row starts (item space) and gathered values of the tile's entries
        for (int i = tid; i <= nr; i += kTh) sptr[i] = __ldg(ptr + r0 + i) + r0 + i;
        {
            int ix[ITEMS];
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) {
                const int e = k * kTh + tid;
                ix[k] = e < cnt ? __ldg(idx + nnz_lo + e) : -1;
            }
            V gv[ITEMS];
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) gv[k] = ix[k] >= 0 ? p.gather(ix[k]) : vzero(V());
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) {
                const int e = k * kTh + tid;
                if (e < cnt) vals[pad16(e)] = gv[k];
            }
        }
        if (tid < 4) sinfo[tid] = -1;
        __syncthreads();

        // 2. walk this thread's ITEMS consecutive items: complete row sums into rsum, the
        //    first row-end (if its row began earlier) kept pending, carry-out recorded
        const int jb = j0 + tid * ITEMS;
        const int je = min(jb + ITEMS, j1);
        int pend_row = -1;
        V pend_val = vzero(V());
        V acc = vzero(V());
        int my_row = -1;
        if (jb < j1) {
            int lo = 0, hi = nr - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sptr[mid] <= jb)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            int i = lo;
            int rend = sptr[i + 1] - 1;
            int ebase = r0 + i + nnz_lo;  // entry index of item j in row i: j - ebase
            bool first = true;
            for (int j = jb; j < je; ++j) {
                if (j < rend) {
                    acc = vadd(acc, vals[pad16(j - ebase)]);
                } else {
                    if (first && sptr[i] < jb) {
                        pend_row = i;
                        pend_val = acc;
                    } else {
                        rsum[i] = acc;
                    }
                    first = false;
                    acc = vzero(V());
                    ++i;
                    ++ebase;
                    if (i < nr) rend = sptr[i + 1] - 1;
                }
            }
            my_row = i;
        }
        crow[tid] = my_row;
        cval[tid] = acc;
        __syncthreads();

        // 3. carry-in of the pending row from the threads before; the in-tile part of a
        //    last row that continues into the next tile
        if (pend_row >= 0) {
            V c = vzero(V());
            for (int t2 = tid - 1; t2 >= 0 && crow[t2] == pend_row; --t2) c = vadd(c, cval[t2]);
            const V tot = vadd(c, pend_val);
            if (sptr[pend_row] < j0)
                split[0] = tot;  // row r0 began in an earlier tile and ends here
            else
                rsum[pend_row] = tot;
        }
        const int tl = (j1 - 1 - j0) / ITEMS;  // last thread holding items
        if (!last_ends && tid == tl) {
            V c = vzero(V());
            for (int t2 = tl; t2 >= 0 && crow[t2] == nr - 1; --t2) c = vadd(c, cval[t2]);
            split[1] = c;
        }
        __syncthreads();

        // 4. rows cut by tile boundaries: deposit this tile's part, count arrivals; the last
        //    tile to arrive sums the parts in tile order and runs the epilogue
        double a0 = 0.0, a1 = 0.0;
        if (tid == 0) {
            V* carry = p.carry();
            int* arrive = p.arrive();
            const bool first_split = sptr[0] < j0;
            int nfin = 0;
            auto deposit = [&](int slot, V val, int row, int ta, int tb) {
                carry[slot] = val;
                __threadfence();
                const int span = tb - ta + 1;
                const int old = atomicAdd(arrive + ta, 1);
                if (old == span - 1) {
                    __threadfence();
                    if (span <= kSerialSplitSum) {
                        V s = ld_cg(carry + 2 * ta + 1);
                        for (int q = ta + 1; q <= tb; ++q) s = vadd(s, ld_cg(carry + 2 * q));
                        arrive[ta] = 0;
                        const int len = (__ldg(ptr + row + 1) - __ldg(ptr + row));
                        p.epilogue(row, s, len, a0, a1);
                    } else {
                        sinfo[2 * nfin] = row;
                        sinfo[2 * nfin + 1] = ta;
                        sinfo[4 + nfin] = tb;
                        ++nfin;
                    }
                }
            };
            if (first_split && (nr > 1 || last_ends))
                deposit(2 * t, split[0], r0, (sptr[0]) / TILE, t);
            if (!last_ends) {
                const int tb = end_last / TILE;
                if (nr == 1 && first_split)
                    deposit(2 * t, split[1], r0, sptr[0] / TILE, tb);
                else
                    deposit(2 * t + 1, split[1], rl, t, tb);
            }
        }
        __syncthreads();
        for (int f = 0; f < 2; ++f) {  // block-uniform: rows split over many tiles
            const int row = sinfo[2 * f];
            if (row < 0) break;
            const int ta = sinfo[2 * f + 1], tb = sinfo[4 + f];
            __threadfence();
            const V* carry = p.carry();
            V s = vzero(V());
            for (int q = tid; q <= tb - ta; q += kTh)
                s = vadd(s, ld_cg(carry + (q == 0 ? 2 * ta + 1 : 2 * (ta + q))));
            s = block_vsum(s, cval);
            if (tid == 0) {
                p.arrive()[ta] = 0;
                const int len = (__ldg(ptr + row + 1) - __ldg(ptr + row));
                p.epilogue(row, s, len, a0, a1);
            }
        }

        // 5. epilogue of every row that lies inside the tile, one thread per row
        const int ib = (sptr[0] < j0) ? 1 : 0;
        const int ie = last_ends ? nr : nr - 1;
        for (int i = ib + tid; i < ie; i += kTh)
            p.epilogue(r0 + i, rsum[i], sptr[i + 1] - sptr[i] - 1, a0, a1);
        dacc0 += a0;
        dacc1 += a1;
        __syncthreads();
    }
}

template <typename T, int ITEMS>
__global__ void __launch_bounds__(kTh) k_stream(View<T> v) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    StreamPolicy<T> p;
    p.v = v;
    p.alpha = (T)ctl->alpha;
    p.inv_rho = (T)(1.0 / ctl->rho);
    double d0 = 0.0, d1 = 0.0;
    seg_tiles<T, ITEMS>(p, smem, max_rows_stream(kTh * ITEMS), d0, d1);
    double* red = (double*)smem;
    const double s = block_sum(d0, red);
    if (threadIdx.x == 0) v.part_s[blockIdx.x] = s;
}

template <typename T, int ITEMS>
__global__ void __launch_bounds__(kTh) k_link(View<T> v) {
    extern __shared__ __align__(16) unsigned char smem[];
    Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    LinkPolicy<T> p;
    p.v = v;
    p.alpha = (T)ctl->alpha;
    p.rho = (T)ctl->rho;
    p.inv_rho = (T)(1.0 / ctl->rho);
    double d0 = 0.0, d1 = 0.0;
    seg_tiles<T, ITEMS>(p, smem, max_rows_link(kTh * ITEMS), d0, d1);
    double* red = (double*)smem;  // the tile staging area, far larger than 3 * kTh / 32 doubles
    double rs[2] = {d0, d1};
    block_sum_n<2>(rs, red);
    __shared__ int last;
    if (threadIdx.x == 0) {
        v.part_l[2 * blockIdx.x] = rs[0];
        v.part_l[2 * blockIdx.x + 1] = rs[1];
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {  // every block's partials are visible: finish the iteration
        __threadfence();
        double R2, S2l, S2s;
        grid_residual_sums(v.part_l, gridDim.x, v.part_s, v.grid_s, red, R2, S2l, S2s);
        if (threadIdx.x == 0) {
            ctl->ticket = 0;
            finalize_iteration(ctl, R2, S2s + S2l, v.hist, v.sched);
        }
    }
}

template <typename T>
size_t smem_stream(int tile) {
    TileLayout<typename Pair<T>::type> lay{tile, max_rows_stream(tile)};
    return lay.bytes();
}
template <typename T>
size_t smem_link(int tile) {
    TileLayout<T> lay{tile, max_rows_link(tile)};
    return lay.bytes();
}

template <typename T, int IS, int IL>
cudaError_t launch_fixed(const View<T>& v, cudaStream_t st, cudaEvent_t* evs) {
    k_stream<T, IS><<<v.grid_s, kTh, smem_stream<T>(kTh * IS), st>>>(v);
    if (evs) record_kernel_event(evs[0], st);
    k_link<T, IL><<<v.grid_l, kTh, smem_link<T>(kTh * IL), st>>>(v);
    if (evs) record_kernel_event(evs[1], st);
    return cudaGetLastError();
}

template <typename T, int IS>
cudaError_t launch_by_link(const View<T>& v, cudaStream_t st, cudaEvent_t* evs) {
    switch (v.tile_l / kTh) {
        case 1: return launch_fixed<T, IS, 1>(v, st, evs);
        case 2: return launch_fixed<T, IS, 2>(v, st, evs);
        case 4: return launch_fixed<T, IS, 4>(v, st, evs);
        case 8: return launch_fixed<T, IS, 8>(v, st, evs);
        case 16: return launch_fixed<T, IS, 16>(v, st, evs);
        case 32: return launch_fixed<T, IS, 32>(v, st, evs);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int ITEMS>
cudaError_t set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_stream<T, ITEMS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_stream<T>(kTh * ITEMS));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_link<T, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_link<T>(kTh * ITEMS));
}

template <typename T>
cudaError_t occupancy(int tile_s, int tile_l, int* occ_s, int* occ_l) {
    cudaError_t e = cudaSuccess;
    const void* fs = nullptr;
    const void* fl = nullptr;
    switch (tile_s / kTh) {
        case 1: e = set_attrs<T, 1>(); fs = (const void*)k_stream<T, 1>; break;
        case 2: e = set_attrs<T, 2>(); fs = (const void*)k_stream<T, 2>; break;
        case 4: e = set_attrs<T, 4>(); fs = (const void*)k_stream<T, 4>; break;
        case 8: e = set_attrs<T, 8>(); fs = (const void*)k_stream<T, 8>; break;
        case 16: e = set_attrs<T, 16>(); fs = (const void*)k_stream<T, 16>; break;
        case 32: e = set_attrs<T, 32>(); fs = (const void*)k_stream<T, 32>; break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    switch (tile_l / kTh) {
        case 1: e = set_attrs<T, 1>(); fl = (const void*)k_link<T, 1>; break;
        case 2: e = set_attrs<T, 2>(); fl = (const void*)k_link<T, 2>; break;
        case 4: e = set_attrs<T, 4>(); fl = (const void*)k_link<T, 4>; break;
        case 8: e = set_attrs<T, 8>(); fl = (const void*)k_link<T, 8>; break;
        case 16: e = set_attrs<T, 16>(); fl = (const void*)k_link<T, 16>; break;
        case 32: e = set_attrs<T, 32>(); fl = (const void*)k_link<T, 32>; break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_s, fs, kTh, smem_stream<T>(tile_s));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_l, fl, kTh, smem_link<T>(tile_l));
}

}  // namespace

// Default tile sizes (items = nonzeros + rows per tile); the same for both precisions.
int fused_tile_items_stream(int /*precision*/) { return 2048; }
int fused_tile_items_link(int /*precision*/) { return 4096; }

size_t fused_smem_stream(int precision, int tile) {
    return precision == 0 ? smem_stream<float>(tile) : smem_stream<double>(tile);
}
size_t fused_smem_link(int precision, int tile) {
    return precision == 0 ? smem_link<float>(tile) : smem_link<double>(tile);
}

cudaError_t fused_grids(int precision, int tile_s, int tile_l, int ntiles_s, int ntiles_l,
                        int* grid_s, int* grid_l) {
    int dev = 0, sms = 0, occ_s = 0, occ_l = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = precision == 0 ? occupancy<float>(tile_s, tile_l, &occ_s, &occ_l)
                       : occupancy<double>(tile_s, tile_l, &occ_s, &occ_l);
    if (e != cudaSuccess) return e;
    if (occ_s < 1 || occ_l < 1) return cudaErrorInvalidConfiguration;
    long long gs = (long long)occ_s * sms, gl = (long long)occ_l * sms;
    gs = gs < ntiles_s ? gs : ntiles_s;
    gl = gl < ntiles_l ? gl : ntiles_l;
    *grid_s = (int)(gs < kMaxGrid ? gs : kMaxGrid);
    *grid_l = (int)(gl < kMaxGrid ? gl : kMaxGrid);
    return cudaSuccess;
}

template <typename T>
cudaError_t fused_iteration(const View<T>& v, cudaStream_t st, cudaEvent_t* evs) {
    switch (v.tile_s / kTh) {
        case 1: return launch_by_link<T, 1>(v, st, evs);
        case 2: return launch_by_link<T, 2>(v, st, evs);
        case 4: return launch_by_link<T, 4>(v, st, evs);
        case 8: return launch_by_link<T, 8>(v, st, evs);
        case 16: return launch_by_link<T, 16>(v, st, evs);
        case 32: return launch_by_link<T, 32>(v, st, evs);
        default: return cudaErrorInvalidValue;
    }
}
template cudaError_t fused_iteration<float>(const View<float>&, cudaStream_t, cudaEvent_t*);
template cudaError_t fused_iteration<double>(const View<double>&, cudaStream_t, cudaEvent_t*);

}  // namespace pmp
