// Persistent form of the batched solve: one cooperative launch runs up to `iters` PMP
// iterations (Sec. III-D..G) of every instance of the batch.
//
// The host plans each launch: an instance with more work per iteration than the plan's
// load bound per block owns a team of consecutive blocks; smaller instances are packed
// several to a block, which runs one iteration of each in turn (a team of one block).  A
// team runs its instance's iterations on its own, with no grid-wide barrier: per iteration
//   1. stream pass: the team's blocks take the instance's streams in turn (one thread per
//      stream, one warp per stream of more than kLongRoute links), exactly the arithmetic
//      of the row and batch kernels; each block writes its residual partial to its slot;
//   2. team barrier: every rate of the instance is written;
//   3. link pass: a group of G lanes per link (links of more than kLongRow streams by whole
//      warps in chunks, the warp that completes a link running its epilogue), again the
//      batch kernel's arithmetic; residual partials to the block's slots;
//   4. team barrier with the end of the iteration: the team's first block waits for the
//      others, sums the team's slots in a fixed order (FP64), runs the stopping test and
//      rho rule of the instance (Sec. III-F, III-G), and then releases the team.
// An instance that stops is left by its team at the top of the next iteration (every block
// of the team reads the same control block after the same barrier, so all leave together).
//
// Values written by other blocks of the launch (rates, link averages and prices, chunk
// sums, partials, the control block) are read from L2 (ld.cg or volatile), never through
// the read-only path.  Blocks of a team wait on each other, so all blocks must be resident
// at once: the host launches the kernel cooperatively (the launch fails rather than run a
// grid that does not fit).  Every wait is bounded: after `wait_polls` polls a waiting block
// records a timeout in the batch's global record and returns, and so, in turn, does every
// other block of its team (their own waits run out); no wait is unbounded.
// Iterates do not depend on the team sizes (the arithmetic of a stream or a link is that
// of the batch kernels); the grouping of the FP64 residual sums does.
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

__device__ __forceinline__ unsigned int ld_volatile(const unsigned int* p) {
    return *(const volatile unsigned int*)p;
}

// A link's state written by another block of the launch (the chunk path: the warp that
// completes a long link changes from one iteration to the next).
template <typename T>
__device__ __forceinline__ LinkState<T> load_link_l2(const View<T>& v, int l) {
    LinkState<T> s;
    s.py = __ldcg(v.pby + l);
    s.Rxo = __ldcg(v.Rx + l);
    s.pso = __ldcg(v.ps + l);
    s.zso = __ldcg(v.zs + l);
    s.cl = __ldg(v.c + l);
    return s;
}

// Record the first timeout of the launch.
__device__ __forceinline__ void note_timeout(BatchGlobal* glob) {
    if (atomicCAS(&glob->timeout, 0, 1) == 0) glob->timeout_block = (int)blockIdx.x;
}

// Barrier of the g blocks of one team; bar = (arrivals, generation).  The last block to
// arrive resets the count and releases the others.  Returns false if this block's wait
// ran out (it then records the timeout).  Called by every thread of the block.
__device__ bool team_barrier(unsigned int* bar, int g, long long polls, BatchGlobal* glob) {
    __shared__ int s_ok;
    __syncthreads();  // the block's work of this phase is done
    if (threadIdx.x == 0) {
        const unsigned int gen = ld_volatile(bar + 1);  // cannot move until this block arrives
        __threadfence();                                // the block's writes before its arrival
        int ok = 1;
        if (atomicAdd(bar, 1u) == (unsigned int)(g - 1)) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);  // release
        } else {
            for (long long k = 0; ld_volatile(bar + 1) == gen; ++k) {
                if (k >= polls) {
                    ok = 0;
                    note_timeout(glob);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// End-of-iteration barrier: every block arrives; the team's first block (master) waits
// for all g arrivals, runs `finish` with the whole block, then resets the count and
// releases the team.  The control block is therefore only ever updated by the master's
// threads.  Returns false if this block's wait ran out.
template <class F>
__device__ bool team_finish_barrier(unsigned int* bar, int g, bool master, long long polls,
                                    BatchGlobal* glob, F&& finish) {
    __shared__ int s_ok;
    __shared__ unsigned int s_gen;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int gen = ld_volatile(bar + 1);
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        if (master) {
            for (long long k = 0; ld_volatile(bar) < (unsigned int)g; ++k) {
                if (k >= polls) {
                    ok = 0;
                    note_timeout(glob);
                    break;
                }
                __nanosleep(64);
            }
        } else {
            for (long long k = 0; ld_volatile(bar + 1) == gen; ++k) {
                if (k >= polls) {
                    ok = 0;
                    note_timeout(glob);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
        s_gen = gen;
    }
    __syncthreads();
    if (!s_ok) return false;
    if (master) {
        finish();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);  // release the team
        }
    }
    return true;
}

// The master block's end of iteration of instance i: FP64 sums of the team's block slots,
// of the instance's long-route slots and chunked-link slots (lane-strided, then the
// shuffle tree: a fixed order), then the single-thread step of Sec. III-F / III-G.
template <typename T>
__device__ void finish_team(const BatchView<T>& b, int i, int first, int g, int lane) {
    double ss = 0.0, rr = 0.0, sl = 0.0;
    for (int q = first + lane; q < first + g; q += 32) {
        ss += __ldcg(b.part_t + 3 * (size_t)q);
        rr += __ldcg(b.part_t + 3 * (size_t)q + 1);
        sl += __ldcg(b.part_t + 3 * (size_t)q + 2);
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
        if (c->stop != RUNNING) atomicSub(&b.glob->running, 1);
        __threadfence();
    }
}

// One PMP iteration of instance tm.x by this block, member tm.y of a team of tm.z blocks
// starting at block tm.w.  False if a wait of this block ran out.
template <typename T, int G, bool kSplit>
__device__ __forceinline__ bool team_iteration(const BatchView<T>& b, int4 tm, double* red) {
    using V = typename Pair<T>::type;
    const View<T>& v = b.v;
    const int i = tm.x, r = tm.y, g = tm.z, first = tm.w;
    const bool master = r == 0;
    Ctl* c = b.ctls + i;
    unsigned int* bar = b.bar + 2 * (size_t)i;
    const int s0 = __ldg(b.soff + i), s1 = __ldg(b.soff + i + 1);
    const int l0 = __ldg(b.loff + i), l1 = __ldg(b.loff + i + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto grp = cg::tiled_partition<G>(cg::this_thread_block());
    const bool leader = grp.thread_rank() == 0;
    constexpr int kGroups = kTh / G;
    const T alpha = (T)__ldcg(&c->alpha);
    const double rho_d = *(const volatile double*)&c->rho;
    const T rho = (T)rho_d, inv_rho = (T)(1.0 / rho_d);

    // 1. streams of the instance, the team's blocks in turn
    {
        Acc<T> acc;
        for (int j = s0 + r * kTh + (int)threadIdx.x; j < s1; j += g * kTh) {
            const int p = __ldg(v.col_ptr + j), pn = __ldg(v.col_ptr + j + 1);
            if (kSplit && pn - p > kLongRoute) continue;  // summed by a warp below
            const T xo = v.x[j], Zo = v.Z[j], wt = __ldg(v.wt + j);
            const T lo = v.box_uniform ? v.lo_u : __ldg(v.lo + j);
            const T hi = v.box_uniform ? v.hi_u : __ldg(v.hi + j);
            const V sum = route_sum<T, true>(v.row_idx, v.pby, p, pn, v.m, v.dbg);
            stream_epilogue(v, j, sum, (T)(pn - p), xo, Zo, wt, lo, hi, alpha, inv_rho, acc);
        }
        const double s = block_sum(acc.value(), red);
        if (threadIdx.x == 0) b.part_t[3 * (size_t)blockIdx.x] = s;
        if (kSplit) {
            const int q1 = __ldg(b.lroff + i + 1);
            for (int q = __ldg(b.lroff + i) + r * kWarps + warp; q < q1; q += g * kWarps) {
                const int j = __ldg(v.long_routes + q);
                const int p = __ldg(v.col_ptr + j), pn = __ldg(v.col_ptr + j + 1);
                const V sum = warp_route_sum<T, true>(v.row_idx, v.pby, p, pn, lane, v.m, v.dbg);
                if (lane == 0) {
                    const T xo = v.x[j], Zo = v.Z[j], wt = __ldg(v.wt + j);
                    const T lo = v.box_uniform ? v.lo_u : __ldg(v.lo + j);
                    const T hi = v.box_uniform ? v.hi_u : __ldg(v.hi + j);
                    Acc<T> a1;
                    stream_epilogue(v, j, sum, (T)(pn - p), xo, Zo, wt, lo, hi, alpha, inv_rho, a1);
                    b.part_r[q] = a1.value();
                }
            }
        }
    }
    // 2. every rate of the instance is written
    if (!team_barrier(bar, g, b.wait_polls, b.glob)) return false;

    // 3. links of the instance
    {
        Acc<T> r2, s2;
        for (int l = l0 + r * kGroups + (int)(threadIdx.x / G); l < l1; l += g * kGroups) {
            const int p0 = __ldg(v.row_ptr + l), p1 = __ldg(v.row_ptr + l + 1);
            if (b.nchunks > 0 && p1 - p0 > kLongRow) continue;  // done by its chunks
            LinkState<T> st;
            if (leader) st = load_link(v, l);  // written by this thread last iteration
            const T s = group_gather_sum<G, 1, true>(grp, v.col_idx, v.x, p0, p1, v.n, v.dbg);
            if (leader) link_epilogue(v, l, st, s, p1 - p0, alpha, rho, inv_rho, r2, s2);
        }
        double rs[2] = {r2.value(), s2.value()};
        block_sum_n<2>(rs, red);
        if (threadIdx.x == 0) {
            b.part_t[3 * (size_t)blockIdx.x + 1] = rs[0];
            b.part_t[3 * (size_t)blockIdx.x + 2] = rs[1];
        }
        if (b.nchunks > 0) {
            const int q1 = __ldg(b.coff + i + 1);
            for (int q = __ldg(b.coff + i) + r * kWarps + warp; q < q1; q += g * kWarps) {
                const int4 ch = __ldg(v.chunks + q);  // (link, first, end, first chunk)
                const T s = warp_gather_sum<T, true>(v.col_idx, v.x, ch.y, ch.z, lane, v.n, v.dbg);
                const int p0 = __ldg(v.row_ptr + ch.x), p1 = __ldg(v.row_ptr + ch.x + 1);
                const int nch = (p1 - p0 + kChunk - 1) / kChunk;
                int done = 0;
                if (lane == 0) {
                    b.carry[q] = s;
                    __threadfence();
                    done = atomicAdd(b.arrive_c + ch.w, 1) == nch - 1;
                }
                done = __shfl_sync(0xffffffffu, done, 0);
                if (!done) continue;
                __threadfence();
                const T t = warp_sum_slots(b.carry + ch.w, nch, lane);
                if (lane == 0) {
                    Acc<T> a, bb;
                    b.arrive_c[ch.w] = 0;
                    const LinkState<T> st = load_link_l2(v, ch.x);
                    link_epilogue(v, ch.x, st, t, p1 - p0, alpha, rho, inv_rho, a, bb);
                    b.part_c[2 * ch.w] = a.value();
                    b.part_c[2 * ch.w + 1] = bb.value();
                }
            }
        }
    }
    // 4. the end of the iteration, by the master
    return team_finish_barrier(bar, g, master, b.wait_polls, b.glob, [&] {
        if (warp == 0) finish_team(b, i, first, g, lane);
    });
}

// Block b runs the tasks tasks[btasks[b].x .. + btasks[b].y): either its place in one
// team of several blocks, or several instances of one block each (small instances packed
// together, each run in turn).  Every iteration, each task whose instance still runs gets
// one iteration; the block leaves when all of its instances have stopped.
// Six resident blocks per SM (40 registers, a few spilled): measured faster than the four
// that the unconstrained 64 registers allow (c4 solve 528 against 585 ms).
template <typename T, int G, bool kSplit>
__global__ void __launch_bounds__(kTh, 6) k_batch_persistent(BatchView<T> b) {
    __shared__ double red[3 * kWarps];
    const int2 bt = __ldg(b.btasks + blockIdx.x);
    for (int it = 0; it < b.iters; ++it) {
        bool any = false;
        for (int t = bt.x; t < bt.x + bt.y; ++t) {
            const int4 tm = __ldg(b.teams + t);  // (instance, rank, team size, first block)
            // written by the instance's master after its last barrier: the same value in
            // every block of the team
            if (*(const volatile int*)&b.ctls[tm.x].stop != RUNNING) continue;
            any = true;
            if (!team_iteration<T, G, kSplit>(b, tm, red)) return;
        }
        if (!any) break;
    }
}

template <typename T, int G>
const void* persistent_kernel(bool split) {
    return split ? (const void*)k_batch_persistent<T, G, true>
                 : (const void*)k_batch_persistent<T, G, false>;
}

template <typename T>
const void* persistent_kernel(int lanes, bool split) {
    switch (lanes) {
        case 4: return persistent_kernel<T, 4>(split);
        case 8: return persistent_kernel<T, 8>(split);
        case 16: return persistent_kernel<T, 16>(split);
        case 32: return persistent_kernel<T, 32>(split);
        default: return nullptr;
    }
}

}  // namespace

cudaError_t batch_persistent_capacity(int precision, int lanes, bool split, int* blocks) {
    const void* k = precision == 0 ? persistent_kernel<float>(lanes, split)
                                   : persistent_kernel<double>(lanes, split);
    if (!k) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kTh, 0);
    if (e != cudaSuccess) return e;
    *blocks = occ * sms;
    return cudaSuccess;
}

template <typename T>
cudaError_t batch_persistent_launch(const BatchView<T>& b, int grid, cudaStream_t st) {
    const void* k = persistent_kernel<T>(b.lanes, b.v.nlong > 0);
    if (!k) return cudaErrorInvalidValue;
    BatchView<T> arg = b;
    void* args[] = {&arg};
    cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kTh), args, 0, st);
    note_launches(1);
    return e;
}
template cudaError_t batch_persistent_launch<float>(const BatchView<float>&, int, cudaStream_t);
template cudaError_t batch_persistent_launch<double>(const BatchView<double>&, int, cudaStream_t);

}  // namespace pmp
