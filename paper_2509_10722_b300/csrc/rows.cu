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
// On this GPU the iteration is bound by random gathers from L2 (one 32-byte sector per
// gathered value), so the design goal is to keep as many gathers in flight as possible
// with no block-wide barriers:
//
//   stream kernel: one thread per stream; the stream's state is loaded first, then its
//     route entries four at a time (four independent gathers of (pbar, y) in flight);
//     streams with more than kLongRoute (32) links are summed by one warp each instead;
//   link kernel: a group of 8 lanes sums R x of a link in a fixed order; with few links
//     per group (a small instance) each link has its own group, whose leader loads the
//     link's state before the gathers and runs the epilogue; with many, a group sums 8
//     consecutive links one after the other and its 8 lanes run their epilogues; links
//     with more than kLongRow (256)
//     streams are cut into fixed chunks of kChunk (2048) entries, each chunk summed by one
//     warp (four gathers in flight per lane) into its own slot, and the warp that brings
//     the row's arrival count to the number of chunks sums the slots in a fixed order and
//     runs the epilogue (no waiting, deterministic): the long links' work is cut into
//     equal pieces, which the warps take from a grid-wide queue, longest first, once
//     their own links are done; that is what balances the Zipf-skewed link degrees;
//   the last block of the link kernel finishes the iteration (FP64 residual sums, stopping
//   test, rho).
// Residual terms are summed in FP64 (per thread, per block, over the grid) in both
// precisions.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "pmp_device.cuh"
#include "pmp_internal.cuh"
#include "pmp_rows.cuh"

namespace cg = cooperative_groups;

namespace pmp {

namespace {

constexpr int kTh = 256;
constexpr int kWarps = kTh / 32;
constexpr int kGroup = 8;  // lanes per link (4 links per warp); 4 to 32 measured, 8 kept

// kSplit: the instance has streams with long routes (v.nlong > 0); without them the kernel
// is compiled without the warp phase, and the common loop without its length test.
// kTape: the adjoint tape is being written (the forward runs of num_adjoint_forward and
// the backward sweep's recomputation); it receives every stream's new rate.
template <typename T, bool kSplit, bool kTape>
__global__ void __launch_bounds__(kTh) k_stream_rows(View<T> v) {
    using V = typename Pair<T>::type;
    __shared__ double red[kWarps];
    const Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    const long long tk = kTape ? ctl->k - v.tape_k0 : -1;  // tape slot of this iteration
    T* const tape = kTape && tk >= 0 && tk < v.tape_len ? v.tape_x + (size_t)tk * v.n : nullptr;
    const T alpha = (T)ctl->alpha;
    const T inv_rho = (T)(1.0 / ctl->rho);
    const int n = v.n;
    const int* __restrict__ col_ptr = v.col_ptr;
    const int* __restrict__ row_idx = v.row_idx;
    const V* __restrict__ pby = v.pby;
    Acc<T> acc;
    for (int j = blockIdx.x * kTh + threadIdx.x; j < n; j += gridDim.x * kTh) {
        const int p = __ldg(col_ptr + j), pn = __ldg(col_ptr + j + 1);
        if (kSplit && pn - p > kLongRoute) continue;  // summed by a warp below
        const T xo = v.x[j], Zo = v.Z[j], wt = __ldg(v.wt + j);
        const T lo = v.box_uniform ? v.lo_u : __ldg(v.lo + j);
        const T hi = v.box_uniform ? v.hi_u : __ldg(v.hi + j);
        const V sum = route_sum<T>(row_idx, pby, p, pn, v.m, v.dbg);
        const T xn = stream_epilogue(v, j, sum, (T)(pn - p), xo, Zo, wt, lo, hi, alpha, inv_rho, acc);
        if (kTape && tape) tape[j] = xn;
    }
    // streams with more than kLongRoute links: one warp each
    const int lane = threadIdx.x & 31;
    for (int q = blockIdx.x * kWarps + (int)(threadIdx.x >> 5); kSplit && q < v.nlong;
         q += gridDim.x * kWarps) {
        const int j = __ldg(v.long_routes + q);
        const int p = __ldg(col_ptr + j), pn = __ldg(col_ptr + j + 1);
        const V sum = warp_route_sum<T>(row_idx, pby, p, pn, lane, v.m, v.dbg);
        if (lane == 0) {
            const T xo = v.x[j], Zo = v.Z[j], wt = __ldg(v.wt + j);
            const T lo = v.box_uniform ? v.lo_u : __ldg(v.lo + j);
            const T hi = v.box_uniform ? v.hi_u : __ldg(v.hi + j);
            const T xn = stream_epilogue(v, j, sum, (T)(pn - p), xo, Zo, wt, lo, hi, alpha,
                                         inv_rho, acc);
            if (kTape && tape) tape[j] = xn;
        }
    }
    const double s = block_sum(acc.value(), red);
    if (threadIdx.x == 0) v.part_s[blockIdx.x] = s;
}
// ---- link kernel ---------------------------------------------------------------------------------

// kSpread: the epilogues of a group's links run on all its lanes (many links per group)
// rather than on its leader (few).  Two pairs of gathers are in flight per lane.
// kTape: as in the stream kernel; the tape receives every link's slack flow and the rho
// of the iteration.
// kChunks: the instance has links of more than kLongRow streams (v.nchunks > 0); without
// them the kernel is compiled without the chunk phase (which costs the other phases
// registers: 48 against 40 per thread, 5 resident blocks per SM instead of 6).
// Resident blocks per SM each variant asks of the compiler (0: no request), as measured.
// The FP32 taping variants and the FP32 spread variant with chunks ask for 6 (40 registers,
// a few bytes of spills): left free, the taping one-group-per-link variant takes 56
// registers (4 blocks), which made the adjoint's recomputation 10% slower at c5, and the
// spread variant with chunks 48 (5 blocks).  The FP32 one-group-per-link variant asks for 1,
// which lets it take 48 registers: 8% faster on a network of 1e5 links than at 40.  The
// FP32 spread variant without chunks compiles to 40 registers without spills with no
// request, and FP64 to 62-64.
template <typename T, bool kSpread, bool kTape, bool kChunks>
constexpr int link_min_blocks() {
    if (sizeof(T) != 4) return 0;
    if (kTape || (kSpread && kChunks)) return 6;
    return kSpread ? 0 : 1;
}

template <typename T, bool kSpread, bool kTape, bool kChunks>
__global__ void __launch_bounds__(kTh, (link_min_blocks<T, kSpread, kTape, kChunks>()))
    k_link_rows(View<T> v) {
    __shared__ double red[3 * kWarps];
    __shared__ int last;
    Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    const long long tk = kTape ? ctl->k - v.tape_k0 : -1;  // tape slot of this iteration
    const bool taping = kTape && tk >= 0 && tk < v.tape_len;
    T* const tape = taping ? v.tape_ps + (size_t)tk * v.m : nullptr;
    const T alpha = (T)ctl->alpha, rho = (T)ctl->rho, inv_rho = (T)(1.0 / ctl->rho);
    auto g = cg::tiled_partition<kGroup>(cg::this_thread_block());
    const bool leader = g.thread_rank() == 0;
    const int m = v.m;
    const int* __restrict__ row_ptr = v.row_ptr;
    const int* __restrict__ col_idx = v.col_idx;
    const T* __restrict__ x = v.x;
    Acc<T> r2, s2;
    constexpr int kGroups = kTh / kGroup;
    if (kSpread) {
        // links of up to kLongRow streams, many per group: a group takes kGroup consecutive
        // links at a time and sums them one after the other with all its lanes; lane k then
        // runs the epilogue of the k-th of them, so that the epilogues use every lane.
        // Rounds of kGroup links per group are dealt out in turn (groups side by side take
        // links side by side, whose first-link streams share sectors).
        const int sl = g.thread_rank();
        if constexpr (kChunks) {
            // the links left after the full rounds are split evenly, fewer than kGroup per
            // group, so that no group has a round more than another
            const int ngroups = gridDim.x * kGroups;
            const int gid = blockIdx.x * kGroups + (int)(threadIdx.x / kGroup);
            const int per_round = ngroups * kGroup;
            const int rounds = m / per_round;
            const int rest0 = rounds * per_round;  // first link left over
            const int rest = m - rest0;
            const int last0 = rest0 + (int)((long long)gid * rest / ngroups);
            const int last1 = rest0 + (int)((long long)(gid + 1) * rest / ngroups);
            for (int k = 0; k <= rounds; ++k) {
                // this round's links of the group: [base, end)
                const int base = k < rounds ? (k * ngroups + gid) * kGroup : last0;
                const int end = k < rounds ? base + kGroup : last1;
                const int lk = base + sl;  // this lane's link
                int q0 = 0, q1 = 0;
                if (lk < end) {
                    q0 = __ldg(row_ptr + lk);
                    q1 = __ldg(row_ptr + lk + 1);
                }
                T mine = T(0);
#pragma unroll 1
                for (int j = 0; j < kGroup; ++j) {
                    if (base + j >= end) break;  // the same for the whole group
                    const int p0 = g.shfl(q0, j), p1 = g.shfl(q1, j);
                    if (p1 - p0 > kLongRow) continue;  // done by its chunks
                    const T s = group_gather_sum<kGroup, 2>(g, col_idx, x, p0, p1, v.n, v.dbg);
                    const T sj = g.shfl(s, 0);
                    if (sl == j) mine = sj;
                }
                if (lk < end && q1 - q0 <= kLongRow) {
                    const LinkState<T> st = load_link(v, lk);
                    const T psn = link_epilogue(v, lk, st, mine, q1 - q0, alpha, rho, inv_rho, r2, s2);
                    if (kTape && tape) tape[lk] = psn;
                }
            }
        } else {
            // the rounds go on to the end: split evenly, the last round took this variant
            // registers (or spills) that cost more than the split saved on short links
            const long long stride = (long long)gridDim.x * kGroups * kGroup;
            for (long long base = ((long long)blockIdx.x * kGroups + threadIdx.x / kGroup) * kGroup;
                 base < m; base += stride) {
                const long long lk = base + sl;  // this lane's link
                int q0 = 0, q1 = 0;
                if (lk < m) {
                    q0 = __ldg(row_ptr + lk);
                    q1 = __ldg(row_ptr + lk + 1);
                }
                T mine = T(0);
#pragma unroll 1
                for (int j = 0; j < kGroup; ++j) {
                    if (base + j >= m) break;  // the same for the whole group
                    const int p0 = g.shfl(q0, j), p1 = g.shfl(q1, j);
                    const T s = group_gather_sum<kGroup, 2>(g, col_idx, x, p0, p1, v.n, v.dbg);
                    const T sj = g.shfl(s, 0);
                    if (sl == j) mine = sj;
                }
                if (lk < m) {
                    const LinkState<T> st = load_link(v, (int)lk);
                    const T psn = link_epilogue(v, (int)lk, st, mine, q1 - q0, alpha, rho, inv_rho, r2, s2);
                    if (kTape && tape) tape[lk] = psn;
                }
            }
        }
    } else {
        // links of up to kLongRow streams, few per group: one group per link, its leader
        // runs the epilogue; the bounds of the group's next link are loaded before the
        // current link is summed, so they are at hand when it is done
        int l = blockIdx.x * kGroups + (int)(threadIdx.x / kGroup);
        int p0 = 0, p1 = 0;
        if (l < m) {
            p0 = __ldg(row_ptr + l);
            p1 = __ldg(row_ptr + l + 1);
        }
        while (l < m) {
            const int ln = l + gridDim.x * kGroups;
            int q0 = 0, q1 = 0;
            if (ln < m) {
                q0 = __ldg(row_ptr + ln);
                q1 = __ldg(row_ptr + ln + 1);
            }
            if (!kChunks || p1 - p0 <= kLongRow) {  // longer links are done by their chunks
                LinkState<T> st;
                if (leader) st = load_link(v, l);
                const T s = group_gather_sum<kGroup, 2>(g, col_idx, x, p0, p1, v.n, v.dbg);
                if (leader) {
                    const T psn = link_epilogue(v, l, st, s, p1 - p0, alpha, rho, inv_rho, r2, s2);
                    if (kTape && tape) tape[l] = psn;
                }
            }
            l = ln;
            p0 = q0;
            p1 = q1;
        }
    }
    // chunks of the longer links: one warp each (four gathers in flight per lane), so that
    // a chunk is a short chain of round trips.  The warps take them from a queue shared by
    // the grid, longest first, and each warp takes its next chunk before it sums the
    // current one: a warp that is done with its links takes more chunks, so that the
    // Zipf-skewed work evens out over the SMs, and the chunks taken last are the shortest.
    // Which warp sums a chunk does not change the result: every chunk has its own slot, and
    // the slots of a link are summed in a fixed order.
    const int lane = threadIdx.x & 31;
    if (kChunks) {
        int t = 0;  // queue position
        if (lane == 0) t = (int)atomicAdd(&ctl->chunk_next, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        while (t < v.nchunks) {
            int tn = 0;
            if (lane == 0) tn = (int)atomicAdd(&ctl->chunk_next, 1u);
            const int q = __ldg(v.chunk_queue + t);
            const int4 ch = __ldg(v.chunks + q);  // (row, first entry, end entry, first chunk)
            const T s = warp_gather_sum(col_idx, x, ch.y, ch.z, lane, v.n, v.dbg);
            int fin = 0;
            if (lane == 0) {
                v.carry_l[q] = s;
                __threadfence();
                const int p0 = __ldg(row_ptr + ch.x), p1 = __ldg(row_ptr + ch.x + 1);
                const int nch = (p1 - p0 + kChunk - 1) / kChunk;
                fin = atomicAdd(v.arrive_l + ch.w, 1) == nch - 1;
            }
            fin = __shfl_sync(0xffffffffu, fin, 0);
            if (fin) {  // every chunk of the row is in: sum the slots in a fixed order
                __threadfence();
                const int p0 = __ldg(row_ptr + ch.x), p1 = __ldg(row_ptr + ch.x + 1);
                const int nch = (p1 - p0 + kChunk - 1) / kChunk;
                const T tot = warp_sum_slots(v.carry_l + ch.w, nch, lane);
                if (lane == 0) {
                    v.arrive_l[ch.w] = 0;
                    const LinkState<T> st = load_link(v, ch.x);
                    const T psn = link_epilogue(v, ch.x, st, tot, p1 - p0, alpha, rho, inv_rho, r2, s2);
                    if (kTape && tape) tape[ch.x] = psn;
                }
            }
            t = __shfl_sync(0xffffffffu, tn, 0);
        }
    }
    double rs[2] = {r2.value(), s2.value()};
    block_sum_n<2>(rs, red);
    if (threadIdx.x == 0) {
        v.part_l[2 * blockIdx.x] = rs[0];
        v.part_l[2 * blockIdx.x + 1] = rs[1];
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double a, b, c;
        grid_residual_sums(v.part_l, gridDim.x, v.part_s, v.grid_s, red, a, b, c);
        if (threadIdx.x == 0) {
            ctl->ticket = 0;
            ctl->chunk_next = 0;  // every warp of the grid has left the chunk queue
            if (kTape && taping) v.tape_rho[tk] = ctl->rho;  // the rho this iteration used
            finalize_iteration(ctl, a, c + b, v.hist, v.sched);
        }
    }
}

template <typename T, bool kChunks>
cudaError_t rows_occupancy(int* occ_s, int* occ_spread, int* occ_leader) {
    // the variant with the warp phase uses at least as many registers
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        occ_s, k_stream_rows<T, true, false>, kTh, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        occ_spread, k_link_rows<T, true, false, kChunks>, kTh, 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        occ_leader, k_link_rows<T, false, false, kChunks>, kTh, 0);
}

// With about 4 links to sum per group slot of a resident grid (c5: 1e5 links), one group
// per link was fastest; with about 42 (c2: 1e6 links) or more (4.2e2 for 1e7 links),
// spreading the epilogues over the lanes.  The switch sits between the two.
constexpr int kFewLinksPerGroup = 16;

}  // namespace

cudaError_t rows_grids(int precision, int n, int m, int nchunks, int* grid_s, int* grid_l,
                       int* link_spread) {
    int dev = 0, sms = 0, occ_s = 0, occ_spread = 0, occ_leader = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (precision == 0)
        e = nchunks > 0 ? rows_occupancy<float, true>(&occ_s, &occ_spread, &occ_leader)
                        : rows_occupancy<float, false>(&occ_s, &occ_spread, &occ_leader);
    else
        e = nchunks > 0 ? rows_occupancy<double, true>(&occ_s, &occ_spread, &occ_leader)
                        : rows_occupancy<double, false>(&occ_s, &occ_spread, &occ_leader);
    if (e != cudaSuccess) return e;
    if (occ_s < 1 || occ_spread < 1 || occ_leader < 1) return cudaErrorInvalidConfiguration;
    const long long need_s = ((long long)n + kTh - 1) / kTh;
    const long long need_l = ((long long)m + nchunks + (kTh / kGroup) - 1) / (kTh / kGroup);
    const long long full_spread = (long long)occ_spread * sms;
    const int spread = (long long)m > (long long)kFewLinksPerGroup * full_spread * (kTh / kGroup);
    long long gs = (long long)occ_s * sms, gl = (long long)(spread ? occ_spread : occ_leader) * sms;
    gs = gs < need_s ? gs : need_s;
    gl = gl < need_l ? gl : need_l;
    *grid_s = (int)(gs < kMaxRowsGrid ? gs : kMaxRowsGrid);
    *grid_l = (int)(gl < kMaxRowsGrid ? gl : kMaxRowsGrid);
    *link_spread = spread;
    return cudaSuccess;
}

template <typename T, bool kTape>
void rows_launch(const View<T>& v, cudaStream_t st, cudaEvent_t* evs) {
    if (v.nlong > 0)
        k_stream_rows<T, true, kTape><<<v.grid_s, kTh, 0, st>>>(v);
    else
        k_stream_rows<T, false, kTape><<<v.grid_s, kTh, 0, st>>>(v);
    if (evs) record_kernel_event(evs[0], st);
    if (v.nchunks > 0) {
        if (v.link_spread)
            k_link_rows<T, true, kTape, true><<<v.grid_l, kTh, 0, st>>>(v);
        else
            k_link_rows<T, false, kTape, true><<<v.grid_l, kTh, 0, st>>>(v);
    } else {
        if (v.link_spread)
            k_link_rows<T, true, kTape, false><<<v.grid_l, kTh, 0, st>>>(v);
        else
            k_link_rows<T, false, kTape, false><<<v.grid_l, kTh, 0, st>>>(v);
    }
    if (evs) record_kernel_event(evs[1], st);
}

template <typename T>
cudaError_t rows_iteration(const View<T>& v, cudaStream_t st, cudaEvent_t* evs) {
    if (v.tape_x)
        rows_launch<T, true>(v, st, evs);
    else
        rows_launch<T, false>(v, st, evs);
    return cudaGetLastError();
}
template cudaError_t rows_iteration<float>(const View<float>&, cudaStream_t, cudaEvent_t*);
template cudaError_t rows_iteration<double>(const View<double>&, cudaStream_t, cudaEvent_t*);

}  // namespace pmp
