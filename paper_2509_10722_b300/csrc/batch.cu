// Batched PMP: many independent NUM instances of uneven sizes solved together.
//
// The instances are stacked block-diagonally in one global numbering (instance i owns a
// contiguous range of streams and of links), so one CSC / CSR pair, one state layout and
// the same per-stream / per-link epilogues serve all of them.  What is per instance: the
// penalty rho, the iteration count, the stopping test and rho rule (Sec. III-F, III-G),
// i.e. one control block each.  Two kernels per iteration for the whole batch:
//   - a list of work items (instance, first row, end row) that never cross an instance;
//     a block takes an item, runs the rows of it (a thread per stream / 8 lanes per link,
//     exactly the row-kernel arithmetic) unless that instance has stopped, and writes the
//     item's residual partial sums to the item's own slot;
//   - the block that finishes the last link item of an instance (a per-instance arrival
//     count) finishes that instance's iteration: FP64 sums of its item slots in a fixed
//     order by the whole block, norms, stopping test, rho; an instance that stops takes
//     itself off the count of running instances (the host stops replaying at zero).
//     Instances are finished as their items complete, in parallel with the rest.
// The work partition (fixed-size items taken by the blocks in turn, or balanced: one
// contiguous range of streams / of link entries per block, cut at instance boundaries;
// lanes per link) is a runtime schedule, chosen by the caller or by the autotuner in
// batch_api.cu; the arithmetic of a stream or a link does not depend on it except through
// the lanes per link, which fix the order of the additions of R x.
// No block waits on another; sums are in a fixed order, so runs are deterministic.
#include <algorithm>

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

// kSplit: some stream has a route of more than kLongRoute links (summed by a warp, as in
// the single-instance stream kernel); otherwise compiled without that phase.
template <typename T, bool kSplit>
__global__ void __launch_bounds__(kTh) k_stream_batch(BatchView<T> b) {
    using V = typename Pair<T>::type;
    __shared__ double red[kWarps];
    if (b.glob->running == 0) return;
    // the link kernel of the previous iteration is done: its chunk queue starts over
    if (blockIdx.x == 0 && threadIdx.x == 0) b.glob->chunk_next = 0;
    const View<T>& v = b.v;
    int it0 = blockIdx.x, it1 = b.nsitems, step = gridDim.x;  // items in turn, or
    if (b.sblk) {                                            // this block's range
        it0 = __ldg(b.sblk + blockIdx.x);
        it1 = __ldg(b.sblk + blockIdx.x + 1);
        step = 1;
    }
    for (int it = it0; it < it1; it += step) {
        const int4 item = __ldg(b.sitems + it);
        const Ctl* c = b.ctls + item.x;
        if (c->stop) continue;  // block-uniform
        const T alpha = (T)c->alpha;
        const T inv_rho = (T)(1.0 / c->rho);
        Acc<T> acc;
        for (int j = item.y + threadIdx.x; j < item.z; j += kTh) {
            const int p = __ldg(v.col_ptr + j), pn = __ldg(v.col_ptr + j + 1);
            if (kSplit && pn - p > kLongRoute) continue;  // summed by a warp below
            const T xo = v.x[j], Zo = v.Z[j], wt = __ldg(v.wt + j);
            const T lo = v.box_uniform ? v.lo_u : __ldg(v.lo + j);
            const T hi = v.box_uniform ? v.hi_u : __ldg(v.hi + j);
            const V sum = route_sum<T>(v.row_idx, v.pby, p, pn, v.m, v.dbg);
            stream_epilogue(v, j, sum, (T)(pn - p), xo, Zo, wt, lo, hi, alpha, inv_rho, acc);
        }
        const double s = block_sum(acc.value(), red);
        if (threadIdx.x == 0) b.part_s[it] = s;
    }
    // streams with long routes: one warp each; the residual term goes to the stream's slot
    const int lane = threadIdx.x & 31;
    for (int q = blockIdx.x * kWarps + (int)(threadIdx.x >> 5); kSplit && q < v.nlong;
         q += gridDim.x * kWarps) {
        const Ctl* c = b.ctls + __ldg(b.lr_inst + q);
        if (c->stop) continue;  // warp-uniform
        const int j = __ldg(v.long_routes + q);
        const int p = __ldg(v.col_ptr + j), pn = __ldg(v.col_ptr + j + 1);
        const V sum = warp_route_sum<T>(v.row_idx, v.pby, p, pn, lane, v.m, v.dbg);
        if (lane == 0) {
            const T alpha = (T)c->alpha;
            const T inv_rho = (T)(1.0 / c->rho);
            const T xo = v.x[j], Zo = v.Z[j], wt = __ldg(v.wt + j);
            const T lo = v.box_uniform ? v.lo_u : __ldg(v.lo + j);
            const T hi = v.box_uniform ? v.hi_u : __ldg(v.hi + j);
            Acc<T> acc;
            stream_epilogue(v, j, sum, (T)(pn - p), xo, Zo, wt, lo, hi, alpha, inv_rho, acc);
            b.part_r[q] = acc.value();
        }
    }
}

// End of iteration of instance i, by one warp: FP64 sums of its stream-item, link-item
// and chunked-link slots (lane-strided, then the shuffle tree: a fixed order), then the
// single-thread step of Sec. III-F / III-G.
template <typename T>
__device__ void finish_instance(const BatchView<T>& b, int i, int lane) {
    double ss = 0.0, rr = 0.0, sl = 0.0;
    const int s0 = b.sitem_off[i], s1 = b.sitem_off[i + 1];
    const int q0 = b.litem_off[i], q1 = b.litem_off[i + 1];
    for (int q = s0 + lane; q < s1; q += 32) ss += __ldcg(b.part_s + q);
    for (int q = q0 + lane; q < q1; q += 32) {
        rr += __ldcg(b.part_l + 2 * q);
        sl += __ldcg(b.part_l + 2 * q + 1);
    }
    if (b.v.nlong > 0)
        for (int q = b.lroff[i] + lane; q < b.lroff[i + 1]; q += 32) ss += __ldcg(b.part_r + q);
    if (b.nchunks > 0)
        for (int q = b.coff[i] + lane; q < b.coff[i + 1]; q += 32) {
            rr += __ldcg(b.part_c + 2 * q);  // zero except at a link's first chunk
            sl += __ldcg(b.part_c + 2 * q + 1);
        }
    ss = warp_sum(ss);
    rr = warp_sum(rr);
    sl = warp_sum(sl);
    if (lane == 0) {
        Ctl* c = b.ctls + i;
        finalize_iteration(c, rr, ss + sl,
                           b.hist + (size_t)i * 3 * (c->hist_len > 0 ? c->hist_len : 1),
                           b.sched + (size_t)i * b.sched_stride);
        b.arrive[i] = 0;
        if (c->stop != RUNNING) atomicSub(&b.glob->running, 1);
    }
}

// Count one finished part (a link item or a chunked link) of instance i; true for the
// part that completes the instance.  Single thread.
template <typename T>
__device__ __forceinline__ bool instance_done(const BatchView<T>& b, int i) {
    const int parts = b.litem_off[i + 1] - b.litem_off[i] + (b.nchunks > 0 ? b.crows[i] : 0);
    return atomicAdd(b.arrive + i, 1u) == (unsigned)(parts - 1);
}

template <typename T, int G>
__global__ void __launch_bounds__(kTh) k_link_batch(BatchView<T> b) {
    __shared__ double red[kWarps];
    __shared__ int fin;
    if (b.glob->running == 0) return;
    const View<T>& v = b.v;
    auto g = cg::tiled_partition<G>(cg::this_thread_block());
    const bool leader = g.thread_rank() == 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kGroups = kTh / G;
    int it0 = blockIdx.x, it1 = b.nlitems, step = gridDim.x;  // items in turn, or
    if (b.lblk) {                                            // this block's range
        it0 = __ldg(b.lblk + blockIdx.x);
        it1 = __ldg(b.lblk + blockIdx.x + 1);
        step = 1;
    }
    for (int it = it0; it < it1; it += step) {
        const int4 item = __ldg(b.litems + it);
        const Ctl* c = b.ctls + item.x;
        if (c->stop) continue;  // block-uniform
        const T alpha = (T)c->alpha, rho = (T)c->rho, inv_rho = (T)(1.0 / c->rho);
        Acc<T> r2, s2;
        for (int l = item.y + (int)(threadIdx.x / G); l < item.z; l += kGroups) {
            const int p0 = __ldg(v.row_ptr + l), p1 = __ldg(v.row_ptr + l + 1);
            if (b.nchunks > 0 && p1 - p0 > kLongRow) continue;  // done by its chunks
            LinkState<T> st;
            if (leader) st = load_link(v, l);
            const T s = group_gather_sum<G>(g, v.col_idx, v.x, p0, p1, v.n, v.dbg);
            if (leader) link_epilogue(v, l, st, s, p1 - p0, alpha, rho, inv_rho, r2, s2);
        }
        const double R2 = block_sum(r2.value(), red);
        const double S2 = block_sum(s2.value(), red);
        if (threadIdx.x == 0) {
            b.part_l[2 * it] = R2;
            b.part_l[2 * it + 1] = S2;
            __threadfence();
            fin = instance_done(b, item.x);
        }
        __syncthreads();
        if (fin && warp == 0) {  // every part of this instance is in
            __threadfence();
            finish_instance(b, item.x, lane);
        }
    }
    // chunks of the longer links: one warp each, taken from a queue shared by the grid,
    // longest first, each warp taking its next chunk before it sums the current one, as in
    // the single-instance row kernel (the iteration's stream kernel resets the queue)
    if (b.nchunks > 0) {
        int t = 0;  // queue position
        if (lane == 0) t = (int)atomicAdd(&b.glob->chunk_next, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        while (t < b.nchunks) {
            int tn = 0;
            if (lane == 0) tn = (int)atomicAdd(&b.glob->chunk_next, 1u);
            const int q = __ldg(v.chunk_queue + t);
            const int i = __ldg(b.chunk_inst + q);
            const Ctl* c = b.ctls + i;
            if (!c->stop) {  // warp-uniform
                const int4 ch = __ldg(b.chunks + q);
                const T s = warp_gather_sum(v.col_idx, v.x, ch.y, ch.z, lane, v.n, v.dbg);
                int done = 0;
                if (lane == 0) {
                    b.carry[q] = s;
                    __threadfence();
                    const int p0 = __ldg(v.row_ptr + ch.x), p1 = __ldg(v.row_ptr + ch.x + 1);
                    const int nch = (p1 - p0 + kChunk - 1) / kChunk;
                    done = atomicAdd(b.arrive_c + ch.w, 1) == nch - 1;
                }
                done = __shfl_sync(0xffffffffu, done, 0);
                if (done) {
                    __threadfence();
                    const int p0 = __ldg(v.row_ptr + ch.x), p1 = __ldg(v.row_ptr + ch.x + 1);
                    const int nch = (p1 - p0 + kChunk - 1) / kChunk;
                    const T tot = warp_sum_slots(b.carry + ch.w, nch, lane);
                    int whole = 0;
                    if (lane == 0) {
                        const T alpha = (T)c->alpha, rho = (T)c->rho, inv_rho = (T)(1.0 / c->rho);
                        Acc<T> r2, s2;
                        b.arrive_c[ch.w] = 0;
                        const LinkState<T> st = load_link(v, ch.x);
                        link_epilogue(v, ch.x, st, tot, p1 - p0, alpha, rho, inv_rho, r2, s2);
                        b.part_c[2 * ch.w] = r2.value();
                        b.part_c[2 * ch.w + 1] = s2.value();
                        __threadfence();
                        whole = instance_done(b, i);
                    }
                    whole = __shfl_sync(0xffffffffu, whole, 0);
                    if (whole) {
                        __threadfence();
                        finish_instance(b, i, lane);
                    }
                }
            }
            t = __shfl_sync(0xffffffffu, tn, 0);
        }
    }
}

// x and prices to FP64 in the caller's order, and sum U_j(x_j) per instance (one block per
// stream item, FP64, then the last block sums each instance's items in item order).
template <typename T>
__global__ void __launch_bounds__(kTh) k_export_batch(BatchView<T> b, double* x_out,
                                                      double* y_out, double* part) {
    __shared__ double red[kWarps];
    __shared__ int last;
    const View<T>& v = b.v;
    for (int it = blockIdx.x; it < b.nsitems; it += gridDim.x) {
        const int4 item = __ldg(b.sitems + it);
        double obj = 0.0;
        for (int j = item.y + threadIdx.x; j < item.z; j += kTh) {
            const double xj = (double)v.x[j];
            const double wt = (double)v.wt[j];
            if (x_out) x_out[v.perm ? v.perm[j] : j] = xj;
            if (v.ut && v.ut[j] == 2)
                obj += -wt / xj;
            else
                obj += wt > 0.0 ? wt * log(xj) : -wt * xj;
        }
        const double s = block_sum(obj, red);
        if (threadIdx.x == 0) part[it] = s;
    }
    if (y_out)
        for (int l = blockIdx.x * kTh + threadIdx.x; l < v.m; l += gridDim.x * kTh)
            y_out[l] = (double)v.pby[l].y;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&b.glob->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < b.count; i += kTh) {
        double s = 0.0;
        for (int q = b.sitem_off[i]; q < b.sitem_off[i + 1]; ++q) s += __ldcg(part + q);
        b.ctls[i].objective = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) b.glob->ticket = 0;
}

// Every route of instance i must use only links of instance i (block-diagonal R).
__global__ void k_check_blocks(int count, const int64_t* __restrict__ stream_off,
                               const int64_t* __restrict__ link_off,
                               const int64_t* __restrict__ route_ptr,
                               const int* __restrict__ route_links, int* err) {
    const long long n = stream_off[count];
    bool bad = false;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = count - 1;  // instance of stream j
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (stream_off[mid] <= j)
                lo = mid;
            else
                hi = mid - 1;
        }
        const long long l0 = link_off[lo], l1 = link_off[lo + 1];
        for (long long e = route_ptr[j]; e < route_ptr[j + 1]; ++e) {
            const int l = route_links[e];
            bad |= l < l0 || l >= l1;
        }
    }
    if (bad) atomicOr(err, VB_BLOCKS);
}

// The largest i in [0, count) with off[i] <= pos (off increasing, off[0] <= pos).
__device__ __forceinline__ int block_of(const int64_t* __restrict__ off, int count, long long pos) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= pos)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Shift the instances' own numbering to the stacked one, in place: route_ptr[p] of instance
// i (p in (so[i], so[i+1]]) gains the entries of instances 0..i-1, eo[i]; its link ids gain
// the links before it, lo[i].  A link id that leaves the int32 range becomes -1, which the
// validation rejects.
__global__ void k_stack_offsets(int count, const int64_t* __restrict__ so,
                                const int64_t* __restrict__ lo, const int64_t* __restrict__ eo,
                                int64_t* route_ptr, int* route_links, long long n, long long nnz) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n + nnz;
         q += (long long)gridDim.x * blockDim.x) {
        if (q < n) {
            const long long p = q + 1;
            route_ptr[p] += eo[block_of(so, count, p - 1)];
        } else {
            const long long e = q - n;
            const long long l = (long long)route_links[e] + lo[block_of(eo, count, e)];
            route_links[e] = (l >= 0 && l <= 2147483647LL) ? (int)l : -1;
        }
    }
}

__global__ void k_batch_arm(Ctl* ctls, BatchGlobal* glob, int count, long long max_iters,
                            double eps_abs, const double* eps_scale) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        Ctl* c = ctls + i;
        c->k_limit = c->k + max_iters;
        c->eps_tol = eps_abs > 0.0 ? eps_abs * eps_scale[i] : 0.0;
        c->stop = RUNNING;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        glob->running = max_iters > 0 ? count : 0;  // instances still running
        glob->ticket = 0;
        glob->chunk_next = 0;
    }
}

__global__ void k_batch_reset(Ctl* ctls, BatchGlobal* glob, int count, double rho0,
                              double alpha, double mu, double gamma, int period, int hist_len,
                              int sched_len) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        Ctl c;
        memset(&c, 0, sizeof(c));
        c.rho = rho0;
        c.alpha = alpha;
        c.mu = mu;
        c.gamma = gamma;
        c.period = period;
        c.hist_len = hist_len;
        c.sched_len = sched_len;
        ctls[i] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        glob->running = 0;
        glob->ticket = 0;
        glob->chunk_next = 0;
    }
}

template <typename T>
cudaError_t link_occupancy(int lanes, int* occ) {
    switch (lanes) {
        case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_link_batch<T, 4>, kTh, 0);
        case 8: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_link_batch<T, 8>, kTh, 0);
        case 16: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_link_batch<T, 16>, kTh, 0);
        case 32: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_link_batch<T, 32>, kTh, 0);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t batch_occupancy(int lanes, int* occ_s, int* occ_l, int* occ_e) {
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_s, k_stream_batch<T, true>, kTh, 0);
    if (e != cudaSuccess) return e;
    e = link_occupancy<T>(lanes, occ_l);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_e, k_export_batch<T>, kTh, 0);
}

int blocks_for(long long count) {
    long long b = (count + kTh - 1) / kTh;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

cudaError_t batch_resident(int precision, int lanes, int* blocks_s, int* blocks_l) {
    int dev = 0, sms = 0, os = 0, ol = 0, oe = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = precision == 0 ? batch_occupancy<float>(lanes, &os, &ol, &oe)
                       : batch_occupancy<double>(lanes, &os, &ol, &oe);
    if (e != cudaSuccess) return e;
    if (os < 1 || ol < 1) return cudaErrorInvalidConfiguration;
    *blocks_s = os * sms;
    *blocks_l = ol * sms;
    return cudaSuccess;
}

cudaError_t batch_grids(int precision, int lanes, int nsitems, int nlitems, int nchunks,
                        int* grid_s, int* grid_l, int* grid_e) {
    int dev = 0, sms = 0, os = 0, ol = 0, oe = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = precision == 0 ? batch_occupancy<float>(lanes, &os, &ol, &oe)
                       : batch_occupancy<double>(lanes, &os, &ol, &oe);
    if (e != cudaSuccess) return e;
    if (os < 1 || ol < 1 || oe < 1) return cudaErrorInvalidConfiguration;
    const long long gs = (long long)os * sms, gl = (long long)ol * sms, ge = (long long)oe * sms;
    *grid_s = (int)(gs < nsitems ? gs : nsitems);
    const long long need_l = std::max<long long>(nlitems, ((long long)nchunks + kWarps - 1) / kWarps);
    *grid_l = (int)(gl < need_l ? gl : need_l);
    *grid_e = (int)(ge < nsitems ? ge : nsitems);
    return cudaSuccess;
}

cudaError_t check_blocks(int count, const int64_t* stream_off, const int64_t* link_off,
                         long long n, const int64_t* route_ptr, const int* route_links, int* err,
                         cudaStream_t st) {
    k_check_blocks<<<blocks_for(n), kTh, 0, st>>>(count, stream_off, link_off, route_ptr,
                                                  route_links, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t stack_offsets(int count, const int64_t* so, const int64_t* lo, const int64_t* eo,
                          int64_t* route_ptr, int* route_links, long long n, long long nnz,
                          cudaStream_t st) {
    k_stack_offsets<<<blocks_for(n + nnz), kTh, 0, st>>>(count, so, lo, eo, route_ptr,
                                                        route_links, n, nnz);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t batch_iteration(const BatchView<T>& b, int grid_s, int grid_l, cudaStream_t st,
                            cudaEvent_t* evs) {
    if (b.v.nlong > 0)
        k_stream_batch<T, true><<<grid_s, kTh, 0, st>>>(b);
    else
        k_stream_batch<T, false><<<grid_s, kTh, 0, st>>>(b);
    if (evs) record_kernel_event(evs[0], st);
    switch (b.lanes) {
        case 4: k_link_batch<T, 4><<<grid_l, kTh, 0, st>>>(b); break;
        case 8: k_link_batch<T, 8><<<grid_l, kTh, 0, st>>>(b); break;
        case 16: k_link_batch<T, 16><<<grid_l, kTh, 0, st>>>(b); break;
        case 32: k_link_batch<T, 32><<<grid_l, kTh, 0, st>>>(b); break;
        default: return cudaErrorInvalidValue;
    }
    if (evs) record_kernel_event(evs[1], st);
    return cudaGetLastError();
}
template cudaError_t batch_iteration<float>(const BatchView<float>&, int, int, cudaStream_t,
                                            cudaEvent_t*);
template cudaError_t batch_iteration<double>(const BatchView<double>&, int, int, cudaStream_t,
                                             cudaEvent_t*);

template <typename T>
cudaError_t batch_export(const BatchView<T>& b, int grid_e, double* x_out, double* y_out,
                         double* part, cudaStream_t st) {
    k_export_batch<T><<<grid_e, kTh, 0, st>>>(b, x_out, y_out, part);
    note_launches(1);
    return cudaGetLastError();
}
template cudaError_t batch_export<float>(const BatchView<float>&, int, double*, double*, double*,
                                         cudaStream_t);
template cudaError_t batch_export<double>(const BatchView<double>&, int, double*, double*, double*,
                                          cudaStream_t);

cudaError_t batch_arm(Ctl* ctls, BatchGlobal* glob, int count, long long max_iters,
                      double eps_abs, const double* eps_scale, cudaStream_t st) {
    k_batch_arm<<<blocks_for(count), kTh, 0, st>>>(ctls, glob, count, max_iters, eps_abs,
                                                   eps_scale);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_reset(Ctl* ctls, BatchGlobal* glob, int count, double rho0, double alpha,
                        double mu, double gamma, int period, int hist_len, int sched_len,
                        cudaStream_t st) {
    k_batch_reset<<<blocks_for(count), kTh, 0, st>>>(ctls, glob, count, rho0, alpha, mu, gamma,
                                                     period, hist_len, sched_len);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pmp
