// C ABI of the PMP solver: batches of independent instances (num_batch_*), their work
// partition and its autotuner (the kernels are in batch.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "handle.cuh"
#include "num_pmp.h"
#include "pmp_internal.cuh"

using namespace pmp::host;
using pmp::Ctl;
using pmp::View;

struct num_batch {
    num_problem* p = nullptr;  // the stacked problem; owns every device array below
    int count = 0;
    std::vector<int64_t> soff, loff;
    pmp::Ctl* ctls = nullptr;
    pmp::Ctl* ctls_host = nullptr;  // pinned [count]
    pmp::BatchGlobal* glob = nullptr;
    pmp::BatchGlobal* glob_host = nullptr;  // pinned
    int4 *sitems = nullptr, *litems = nullptr;
    int nsitems = 0, nlitems = 0;
    int *sitem_off = nullptr, *litem_off = nullptr;
    double *part_s = nullptr, *part_l = nullptr, *part_e = nullptr;
    double* hist = nullptr;
    signed char* sched = nullptr;
    int sched_stride = 0;
    double* eps_scale = nullptr;
    int grid_s = 0, grid_l = 0, grid_e = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    double kernel_ms[2] = {0.0, 0.0};
    long long kernel_runs[2] = {0, 0};
    std::vector<double> J;  // terminals nnz_i + m_i of each instance
    num_batch_schedule cfg{};          // the work partition in use
    int cap_sitems = 0, cap_litems = 0;  // item capacity (the smallest item sizes)
    unsigned int* arrive = nullptr;    // [count] per-instance arrivals of finished parts
    int* chunk_inst = nullptr;         // [nchunks] instance of each long-link chunk
    int* coff = nullptr;               // [count + 1] chunk range of each instance
    int* crows = nullptr;              // [count] chunked links of each instance
    double* part_c = nullptr;          // [2 nchunks] residual terms of chunked links
    int* lr_inst = nullptr;            // [nlong] instance of each long-route stream
    int* lroff = nullptr;              // [count + 1] long-route range of each instance
    double* part_r = nullptr;          // [nlong] residual terms of long-route streams
    // persistent form (num_batch_set_persistent)
    bool persistent = false;
    long long wait_polls = 0;          // polls of a team wait before it gives up
    bool broken = false;               // a wait ran out: the iterates are undefined until reset
    int* soff_d = nullptr;             // [count + 1] stream / link ranges of the instances
    int* loff_d = nullptr;
    unsigned int* bar = nullptr;       // [2 count] team barriers
    int4* teams = nullptr;             // [cap_teams + count] tasks (instance, rank, size, first)
    int2* btasks = nullptr;            // [cap_teams] each block's range of tasks
    double* part_t = nullptr;          // [3 cap_teams] per-block residual partials
    int cap_teams = 0;
    int grid_p = 0;                    // blocks of the current team plan
    // balanced partitions (stream_item / link_item = 0): each block's item range
    int* sblk = nullptr;               // [kMaxBalancedBlocks + 1]
    int* lblk = nullptr;
    bool sbal = false, lbal = false;
    std::vector<int> link_deg;         // entries of each link (host copy, for the weights)
};

namespace {

// Work partition of a batch: defaults, limits and the autotuner's candidates.
constexpr num_batch_schedule kBatchDefault = {0, 0, 8};  // balanced ranges, 8 lanes
constexpr int kMaxBalancedBlocks = 4096;  // above any resident grid of the batch kernels
constexpr int kBalancedMinWork = 256;     // streams (or link entries) per block at least
constexpr int kLinkEpilogueWeight = 4;    // a link's epilogue, in route entries
constexpr int kStreamItemMin = 256, kStreamItemMax = 65536;
constexpr int kLinkItemMin = 32, kLinkItemMax = 8192;
constexpr int kTuneStreamItems[] = {0, 512, 1024, 2048, 4096, 8192};  // 0: balanced
constexpr int kTuneLinkItems[] = {0, 64, 128, 256, 512, 1024};
constexpr int kTuneLanes[] = {4, 8, 16, 32};

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

bool valid_schedule(const num_batch_schedule& c) {
    return (c.stream_item == 0 || pow2_in(c.stream_item, kStreamItemMin, kStreamItemMax)) &&
           (c.link_item == 0 || pow2_in(c.link_item, kLinkItemMin, kLinkItemMax)) &&
           (c.link_lanes == 4 || c.link_lanes == 8 || c.link_lanes == 16 || c.link_lanes == 32);
}

template <typename T>
pmp::BatchView<T> make_batch_view(const num_batch* b) {
    pmp::BatchView<T> v;
    std::memset(&v, 0, sizeof(v));
    v.v = make_view<T>(b->p);
    v.ctls = b->ctls;
    v.glob = b->glob;
    v.sitems = b->sitems;
    v.litems = b->litems;
    v.nsitems = b->nsitems;
    v.nlitems = b->nlitems;
    v.sitem_off = b->sitem_off;
    v.litem_off = b->litem_off;
    v.sblk = b->sbal ? b->sblk : nullptr;
    v.lblk = b->lbal ? b->lblk : nullptr;
    v.count = b->count;
    v.part_s = b->part_s;
    v.part_l = b->part_l;
    v.hist = b->hist;
    v.sched = b->sched;
    v.sched_stride = b->sched_stride;
    v.arrive = b->arrive;
    v.lanes = b->cfg.link_lanes;
    const num_problem* h = b->p;
    v.chunks = h->chunks;
    v.nchunks = h->nchunks;
    v.chunk_inst = b->chunk_inst;
    v.coff = b->coff;
    v.crows = b->crows;
    v.carry = (T*)h->carry_l;
    v.arrive_c = h->arrive_l;
    v.part_c = b->part_c;
    v.lr_inst = b->lr_inst;
    v.lroff = b->lroff;
    v.part_r = b->part_r;
    v.soff = b->soff_d;
    v.loff = b->loff_d;
    v.teams = b->teams;
    v.btasks = b->btasks;
    v.part_t = b->part_t;
    v.bar = b->bar;
    v.wait_polls = b->wait_polls;
    v.iters = h->prm.check_every;
    return v;
}

cudaError_t batch_run(num_batch* b, int count) {
    num_problem* h = b->p;
    const bool prof = h->prm.profile != 0;
    if (prof) {
        cudaError_t e = pmp::record_kernel_event(h->evs[0], h->stream);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < count; ++i) {
        cudaEvent_t* ev = prof && i < profiled_iterations(h) ? h->evs.data() + 1 + (size_t)i * 2 : nullptr;
        cudaError_t e = h->prec == NUM_FUSED_FP32
                            ? pmp::batch_iteration<float>(make_batch_view<float>(b), b->grid_s,
                                                          b->grid_l, h->stream, ev)
                            : pmp::batch_iteration<double>(make_batch_view<double>(b), b->grid_s,
                                                           b->grid_l, h->stream, ev);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void batch_destroy(num_batch* b) {
    if (!b) return;
    if (b->p && b->p->stream) cudaStreamSynchronize(b->p->stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ctls_host) cudaFreeHost(b->ctls_host);
    if (b->glob_host) cudaFreeHost(b->glob_host);
    destroy_handle(b->p);
    delete b;
}

int batch_reset_all(num_batch* b) {
    const num_params& q = b->p->prm;
    cudaError_t e = pmp::batch_reset(b->ctls, b->glob, b->count, q.rho0, q.alpha, q.mu, q.gamma,
                                     q.rho_period, q.history, 0, b->p->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->arrive, 0, sizeof(unsigned int) * (size_t)b->count, b->p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "resetting the instances");
    return NUM_OK;
}

// Cut the rows [0, off[count]) into `blocks` consecutive ranges of equal weight and each
// range again at instance boundaries (off): items (instance, first row, end row) in row
// order, blk[b] = first item of block b.  pre (prefix sums of the row weights, pre[r] =
// weight of the rows before r) may be NULL for unit weights.
void balanced_items(const std::vector<int64_t>& off, const std::vector<double>* pre,
                    int blocks, std::vector<int4>& items, std::vector<int>& blk) {
    const int count = (int)off.size() - 1;
    const int64_t rows = off[count];
    const double W = pre ? (*pre)[rows] : (double)rows;
    items.clear();
    blk.assign((size_t)blocks + 1, 0);
    int64_t r = 0;
    int inst = 0;
    for (int q = 0; q < blocks; ++q) {
        blk[q] = (int)items.size();
        // the first row whose prefix weight reaches the block's share
        const double target = W * (double)(q + 1) / (double)blocks;
        int64_t end;
        if (q == blocks - 1)
            end = rows;
        else if (pre)
            end = (int64_t)(std::lower_bound(pre->begin() + r, pre->begin() + rows + 1, target) -
                            pre->begin());
        else
            end = (int64_t)std::ceil(target);
        end = std::min<int64_t>(std::max<int64_t>(end, r), rows);
        while (r < end) {
            while (off[inst + 1] <= r) ++inst;
            const int64_t cut = std::min<int64_t>(end, off[inst + 1]);
            items.push_back(make_int4(inst, (int)r, (int)cut, 0));
            r = cut;
        }
    }
    blk[blocks] = (int)items.size();
}

// Build the work items of schedule `cfg` (instance, first row, end row) and size the grids;
// a captured graph of the old partition is dropped.  Streams keep their instance's range
// after the first-link ordering because an instance's links are a contiguous id range.
// stream_item / link_item = 0: balanced, one range of equal work per block (streams; link
// entries plus an epilogue weight per link, chunked links counting their epilogue only).
int batch_apply_schedule(num_batch* b, const num_batch_schedule& cfg) {
    num_problem* h = b->p;
    cudaStream_t st = h->stream;
    const int prec = h->prec == NUM_FUSED_FP32 ? 0 : 1;
    std::vector<int4> si, li;
    std::vector<int> so(b->count + 1), lo_(b->count + 1), sblk, lblk;
    int res_s = 0, res_l = 0;
    cudaError_t e = pmp::batch_resident(prec, cfg.link_lanes, &res_s, &res_l);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy of the batch kernels");
    res_s = std::min(res_s, kMaxBalancedBlocks);
    res_l = std::min(res_l, kMaxBalancedBlocks);
    int grid_s_bal = 0, grid_l_bal = 0;
    if (cfg.stream_item == 0) {
        const int64_t N = b->soff[b->count];
        grid_s_bal = (int)std::max<int64_t>(
            1, std::min<int64_t>(res_s, (N + kBalancedMinWork - 1) / kBalancedMinWork));
        balanced_items(b->soff, nullptr, grid_s_bal, si, sblk);
    } else {
        for (int i = 0; i < b->count; ++i)
            for (int64_t r = b->soff[i]; r < b->soff[i + 1]; r += cfg.stream_item)
                si.push_back(make_int4(i, (int)r, (int)std::min<int64_t>(r + cfg.stream_item,
                                                                         b->soff[i + 1]), 0));
    }
    if (cfg.link_item == 0) {
        const int64_t M = b->loff[b->count];
        if (b->link_deg.empty()) {  // entries of every link, once
            std::vector<int> rp((size_t)M + 1);
            e = cudaMemcpyAsync(rp.data(), h->row_ptr, sizeof(int) * rp.size(),
                                cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "reading the link degrees");
            b->link_deg.resize((size_t)M);
            for (int64_t l = 0; l < M; ++l) b->link_deg[l] = rp[l + 1] - rp[l];
        }
        std::vector<double> pre((size_t)M + 1, 0.0);
        const bool chunked = h->nchunks > 0;
        for (int64_t l = 0; l < M; ++l) {
            const int d = b->link_deg[l];
            pre[l + 1] = pre[l] + (chunked && d > pmp::kLongRow ? 0.0 : (double)d) +
                         (double)kLinkEpilogueWeight;
        }
        grid_l_bal = (int)std::max<int64_t>(
            1, std::min<int64_t>(res_l, (int64_t)(pre[M] / kBalancedMinWork) + 1));
        // blocks beyond the ranges still sum the chunks of the long links
        const int grid_chunks = (int)std::min<int64_t>(res_l, (h->nchunks + 7) / 8);
        balanced_items(b->loff, &pre, grid_l_bal, li, lblk);
        if (grid_chunks > grid_l_bal) {
            lblk.resize((size_t)grid_chunks + 1, lblk.back());
            grid_l_bal = grid_chunks;
        }
    } else {
        for (int i = 0; i < b->count; ++i)
            for (int64_t r = b->loff[i]; r < b->loff[i + 1]; r += cfg.link_item)
                li.push_back(make_int4(i, (int)r, (int)std::min<int64_t>(r + cfg.link_item,
                                                                         b->loff[i + 1]), 0));
    }
    // the first item of each instance (items are in row order, instances contiguous)
    std::fill(so.begin(), so.end(), -1);
    std::fill(lo_.begin(), lo_.end(), -1);
    for (int q = (int)si.size() - 1; q >= 0; --q) so[si[q].x] = q;
    for (int q = (int)li.size() - 1; q >= 0; --q) lo_[li[q].x] = q;
    so[b->count] = (int)si.size();
    lo_[b->count] = (int)li.size();
    for (int i = b->count - 1; i >= 0; --i) {
        if (so[i] < 0) so[i] = so[i + 1];
        if (lo_[i] < 0) lo_[i] = lo_[i + 1];
    }
    if ((int)si.size() > b->cap_sitems || (int)li.size() > b->cap_litems)
        return fail(NUM_ERR_STATE, "work items exceed their capacity");
    e = cudaStreamSynchronize(st);  // no kernel may still read the old items
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->sitems, si.data(), sizeof(int4) * si.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->litems, li.data(), sizeof(int4) * li.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->sitem_off, so.data(), sizeof(int) * (b->count + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->litem_off, lo_.data(), sizeof(int) * (b->count + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !sblk.empty())
        e = cudaMemcpyAsync(b->sblk, sblk.data(), sizeof(int) * sblk.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !lblk.empty())
        e = cudaMemcpyAsync(b->lblk, lblk.data(), sizeof(int) * lblk.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
    if (e != cudaSuccess) return cuda_fail(e, "copying the work items");
    b->nsitems = (int)si.size();
    b->nlitems = (int)li.size();
    e = pmp::batch_grids(prec, cfg.link_lanes, b->nsitems, b->nlitems, h->nchunks, &b->grid_s,
                         &b->grid_l, &b->grid_e);
    if (e != cudaSuccess) return cuda_fail(e, "sizing the batch grids");
    b->sbal = cfg.stream_item == 0;
    b->lbal = cfg.link_item == 0;
    if (b->sbal) b->grid_s = grid_s_bal;
    if (b->lbal) b->grid_l = grid_l_bal;
    b->cfg = cfg;
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    return NUM_OK;
}

// The instance of every long-link chunk of the stacked problem, each instance's chunk range
// and number of chunked links, and zeroed residual slots for the chunked links.  Chunks are
// in link order and an instance's links are a contiguous id range, so an instance's chunks
// are contiguous.
int batch_chunk_tables(num_batch* b) {
    num_problem* h = b->p;
    const int nc = h->nchunks;
    if (nc <= 0) return NUM_OK;
    cudaStream_t st = h->stream;
    std::vector<int4> ch((size_t)nc);
    cudaError_t e = cudaMemcpyAsync(ch.data(), h->chunks, sizeof(int4) * (size_t)nc,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the chunk table");
    std::vector<int> inst((size_t)nc), coff(b->count + 1, 0), crows(b->count, 0);
    for (int q = 0; q < nc; ++q) {
        const int64_t link = ch[q].x;
        const int i = (int)(std::upper_bound(b->loff.begin(), b->loff.end(), link) -
                            b->loff.begin()) - 1;
        inst[q] = i;
        coff[i + 1] += 1;
        if (ch[q].w == q) crows[i] += 1;
    }
    for (int i = 0; i < b->count; ++i) coff[i + 1] += coff[i];
    b->chunk_inst = (int*)dev_alloc(h, sizeof(int) * (size_t)nc);
    b->coff = (int*)dev_alloc(h, sizeof(int) * (size_t)(b->count + 1));
    b->crows = (int*)dev_alloc(h, sizeof(int) * (size_t)b->count);
    b->part_c = (double*)dev_alloc(h, sizeof(double) * 2 * (size_t)nc);
    if (!b->chunk_inst || !b->coff || !b->crows || !b->part_c)
        return fail(NUM_ERR_OOM, "device allocation failed");
    e = cudaMemcpyAsync(b->chunk_inst, inst.data(), sizeof(int) * (size_t)nc,
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->coff, coff.data(), sizeof(int) * (size_t)(b->count + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->crows, crows.data(), sizeof(int) * (size_t)b->count,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->part_c, 0, sizeof(double) * 2 * (size_t)nc, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
    if (e != cudaSuccess) return cuda_fail(e, "copying the chunk tables");
    return NUM_OK;
}

// The instance of every long-route stream of the stacked problem (the list is in stream
// order and an instance's streams are a contiguous range, so each instance has a contiguous
// part of it), and zeroed residual slots for those streams.
int batch_long_route_tables(num_batch* b) {
    num_problem* h = b->p;
    const int nl = h->nlong;
    if (nl <= 0) return NUM_OK;
    cudaStream_t st = h->stream;
    std::vector<int> js((size_t)nl);
    cudaError_t e = cudaMemcpyAsync(js.data(), h->long_routes, sizeof(int) * (size_t)nl,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the long-route list");
    std::vector<int> inst((size_t)nl), off(b->count + 1, 0);
    for (int q = 0; q < nl; ++q) {
        const int i = (int)(std::upper_bound(b->soff.begin(), b->soff.end(), (int64_t)js[q]) -
                            b->soff.begin()) - 1;
        inst[q] = i;
        off[i + 1] += 1;
    }
    for (int i = 0; i < b->count; ++i) off[i + 1] += off[i];
    b->lr_inst = (int*)dev_alloc(h, sizeof(int) * (size_t)nl);
    b->lroff = (int*)dev_alloc(h, sizeof(int) * (size_t)(b->count + 1));
    b->part_r = (double*)dev_alloc(h, sizeof(double) * (size_t)nl);
    if (!b->lr_inst || !b->lroff || !b->part_r)
        return fail(NUM_ERR_OOM, "device allocation failed");
    e = cudaMemcpyAsync(b->lr_inst, inst.data(), sizeof(int) * (size_t)nl, cudaMemcpyHostToDevice,
                        st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->lroff, off.data(), sizeof(int) * (size_t)(b->count + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->part_r, 0, sizeof(double) * (size_t)nl, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
    if (e != cudaSuccess) return cuda_fail(e, "copying the long-route tables");
    return NUM_OK;
}

// Device time of the stream kernel and of the link kernel, summed over `iters` iterations
// of schedule `cfg` (after two untimed ones), with no stopping test.
int batch_time_schedule(num_batch* b, const num_batch_schedule& cfg, int iters, double* ms_s,
                        double* ms_l) {
    int rc = batch_apply_schedule(b, cfg);
    if (rc != NUM_OK) return rc;
    num_problem* h = b->p;
    cudaStream_t st = h->stream;
    cudaError_t e = pmp::batch_arm(b->ctls, b->glob, b->count, (long long)iters + 2, 0.0,
                                   b->eps_scale, st);
    if (e != cudaSuccess) return cuda_fail(e, "arming the instances");
    std::vector<cudaEvent_t> ev(2 * (size_t)iters + 1, nullptr);
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    auto run = [&](cudaEvent_t* evs) {
        return h->prec == NUM_FUSED_FP32
                   ? pmp::batch_iteration<float>(make_batch_view<float>(b), b->grid_s, b->grid_l, st, evs)
                   : pmp::batch_iteration<double>(make_batch_view<double>(b), b->grid_s, b->grid_l, st, evs);
    };
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = run(nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    for (int i = 0; i < iters && e == cudaSuccess; ++i) e = run(ev.data() + 1 + 2 * (size_t)i);
    pmp::note_launches(2 * ((long long)iters + 2));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    double ts = 0.0, tl = 0.0;
    for (int i = 0; i < iters && e == cudaSuccess; ++i) {
        float a = 0.f, c = 0.f;
        e = cudaEventElapsedTime(&a, ev[2 * i], ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&c, ev[2 * i + 1], ev[2 * i + 2]);
        ts += a;
        tl += c;
    }
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(e, "timing a schedule");
    *ms_s = ts;
    *ms_l = tl;
    return NUM_OK;
}

// Persistent form: the plan of one launch.  Each running instance's work per iteration is
// estimated as two gathers per route entry plus its streams and links.  With a load bound
// B per block, an instance of more work than B gets a team of ceil(w / B) blocks (at most
// one per 256 streams or per 256 lanes of links: more would have nothing to do), and the
// others are packed several to a block, first-fit by decreasing work, each run in turn by
// its block.  B is the smallest bound (bisection) whose plan fits in `cap` resident
// blocks.  Fills tasks (instance, rank, team size, first block) and the per-block task
// ranges; returns the number of blocks (0: nothing runs).
constexpr int kPersistTh = 256;            // threads per block of the persistent kernel
constexpr long long kDefaultWaitPolls = 1LL << 22;  // about a second of polling per wait

int plan_teams(const num_batch* b, const std::vector<char>& live, int cap,
               std::vector<int4>& tasks, std::vector<int2>& btasks) {
    std::vector<int> ids;
    std::vector<double> w(b->count, 0.0);
    std::vector<int64_t> useful(b->count, 1);
    double W = 0.0;
    for (int i = 0; i < b->count; ++i) {
        if (!live[i]) continue;
        const int64_t n_i = b->soff[i + 1] - b->soff[i], m_i = b->loff[i + 1] - b->loff[i];
        const double nnz_i = b->J[i] - (double)m_i;
        w[i] = 2.0 * nnz_i + (double)n_i + (double)m_i;
        useful[i] = std::max<int64_t>(
            1, std::max<int64_t>((n_i + kPersistTh - 1) / kPersistTh,
                                 (m_i * b->cfg.link_lanes + kPersistTh - 1) / kPersistTh));
        W += w[i];
        ids.push_back(i);
    }
    tasks.clear();
    btasks.clear();
    if (ids.empty()) return 0;
    std::sort(ids.begin(), ids.end(), [&](int a, int c) { return w[a] > w[c] || (w[a] == w[c] && a < c); });
    // blocks of the plan under bound B; with `build`, the plan itself
    auto plan = [&](double B, bool build) -> long long {
        long long blocks = 0;
        std::vector<double> load;        // packed blocks: work so far
        std::vector<std::vector<int>> members;
        for (int i : ids) {
            if (w[i] > B) {
                const int64_t g = std::min<int64_t>((int64_t)std::ceil(w[i] / B), useful[i]);
                if (build) {
                    const int first = (int)btasks.size();
                    for (int64_t r = 0; r < g; ++r) {
                        btasks.push_back(make_int2((int)tasks.size(), 1));
                        tasks.push_back(make_int4(i, (int)r, (int)g, first));
                    }
                }
                blocks += g;
            } else {
                size_t k = 0;
                while (k < load.size() && load[k] + w[i] > B) ++k;  // first fit
                if (k == load.size()) {
                    load.push_back(0.0);
                    members.emplace_back();
                }
                load[k] += w[i];
                members[k].push_back(i);
            }
        }
        blocks += (long long)load.size();
        if (build)
            for (auto& mem : members) {
                const int blk = (int)btasks.size();
                btasks.push_back(make_int2((int)tasks.size(), (int)mem.size()));
                for (int i : mem) tasks.push_back(make_int4(i, 0, 1, blk));
            }
        return blocks;
    };
    // at B = W everything fits in one block; at B = W / cap no plan uses fewer blocks
    double lo = std::max(W / cap, 1.0), hi = std::max(W, lo);
    if (plan(lo, false) > cap) {
        for (int it = 0; it < 60 && hi > lo * (1.0 + 1e-3); ++it) {
            const double mid = 0.5 * (lo + hi);
            if (plan(mid, false) <= cap)
                hi = mid;
            else
                lo = mid;
        }
    } else {
        hi = lo;
    }
    plan(hi, true);
    return (int)btasks.size();
}

// Runs the armed instances of the batch with cooperative launches of the persistent
// kernel, check_every iterations per launch, re-planning the teams over the instances
// still running before each launch, until none runs.  NUM_ERR_TIMEOUT if a team wait ran
// out (the batch is then marked broken).
int batch_solve_persistent(num_batch* b, int64_t max_iters) {
    num_problem* h = b->p;
    cudaStream_t st = h->stream;
    int cap = 0;
    cudaError_t e = pmp::batch_persistent_capacity(h->prec == NUM_FUSED_FP32 ? 0 : 1,
                                                   b->cfg.link_lanes, h->nlong > 0, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy of the persistent kernel");
    if (cap < 1) return fail(NUM_ERR_STATE, "the persistent kernel cannot be resident");
    // tasks: at most one per block of a team, or one per instance
    const int ntask_cap = cap + b->count;
    if (cap > b->cap_teams) {
        if (b->teams) dev_free(h, b->teams);
        if (b->btasks) dev_free(h, b->btasks);
        if (b->part_t) dev_free(h, b->part_t);
        b->teams = (int4*)dev_alloc(h, sizeof(int4) * (size_t)ntask_cap);
        b->btasks = (int2*)dev_alloc(h, sizeof(int2) * (size_t)cap);
        b->part_t = (double*)dev_alloc(h, sizeof(double) * 3 * (size_t)cap);
        b->cap_teams = b->teams && b->btasks && b->part_t ? cap : 0;
        if (!b->cap_teams) return fail(NUM_ERR_OOM, "device allocation failed");
    }
    const int K = h->prm.check_every;
    const long long max_launches = (max_iters + K - 1) / K + 1;
    std::vector<char> live(b->count), planned;
    std::vector<int4> teams;
    std::vector<int2> btasks;
    for (long long it = 0;; ++it) {
        if (it >= max_launches) return fail(NUM_ERR_STATE, "the iteration limit was not honoured");
        e = cudaMemcpyAsync(b->ctls_host, b->ctls, sizeof(pmp::Ctl) * b->count,
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading the control blocks");
        for (int i = 0; i < b->count; ++i) live[i] = b->ctls_host[i].stop == pmp::RUNNING;
        if (live != planned) {  // instances stopped since the last plan (or none yet)
            b->grid_p = plan_teams(b, live, cap, teams, btasks);
            if (b->grid_p == 0) break;
            if (b->grid_p > cap || (int)teams.size() > ntask_cap)
                return fail(NUM_ERR_STATE, "the team plan does not fit");
            e = cudaMemcpyAsync(b->teams, teams.data(), sizeof(int4) * teams.size(),
                                cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->btasks, btasks.data(), sizeof(int2) * btasks.size(),
                                    cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the vectors are reused
            if (e != cudaSuccess) return cuda_fail(e, "copying the team plan");
            planned = live;
        }
        e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned int) * 2 * (size_t)b->count, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(&b->glob->timeout, 0, 2 * sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "arming the team barriers");
        TraceRange launch("num_batch_solve: persistent launch of check_every iterations");
        e = h->prec == NUM_FUSED_FP32
                ? pmp::batch_persistent_launch<float>(make_batch_view<float>(b), b->grid_p, st)
                : pmp::batch_persistent_launch<double>(make_batch_view<double>(b), b->grid_p, st);
        if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the persistent kernel");
        e = cudaMemcpyAsync(b->glob_host, b->glob, sizeof(pmp::BatchGlobal),
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "persistent iterations");
        if (b->glob_host->timeout) {
            b->broken = true;
            return fail(NUM_ERR_TIMEOUT,
                        "a wait between the blocks of an instance's team ran out (block " +
                            std::to_string(b->glob_host->timeout_block) +
                            "); the iterates are undefined until num_batch_reset");
        }
        if (b->glob_host->running == 0) break;
    }
    return NUM_OK;
}

// The batch over a stacked problem (host or device arrays, as create_impl takes them);
// inst_nnz[count] (host) holds each instance's route entries.  The offsets are checked.
int batch_create_impl(num_batch** out, int32_t count, const int64_t* stream_off,
                      const int64_t* link_off, const int64_t* inst_nnz, const int64_t* route_ptr,
                      const int32_t* route_links, const double* c, const uint8_t* utype,
                      const double* w, const double* lo, const double* hi, const num_params* p,
                      void* cuda_stream, bool on_device) {
    if (stream_off[0] != 0 || link_off[0] != 0)
        return fail(NUM_ERR_INVALID, "stream_off[0] and link_off[0] must be 0");
    for (int i = 0; i < count; ++i)
        if (stream_off[i + 1] <= stream_off[i] || link_off[i + 1] <= link_off[i])
            return fail(NUM_ERR_INVALID, "every instance needs >= 1 stream and >= 1 link");
    num_params prm;
    if (p)
        prm = *p;
    else
        num_default_params(&prm);
    if (prm.precision == NUM_PLAIN_FP64)
        return fail(NUM_ERR_INVALID, "batches run the fused row kernels (FP32 or FP64)");
    const int64_t n = stream_off[count], m = link_off[count];
    if (n > INT32_MAX - 1 || m > INT32_MAX - 1)
        return fail(NUM_ERR_INVALID, "total n and m must be < 2^31 - 1");
    num_batch* b = new (std::nothrow) num_batch();
    if (!b) return fail(NUM_ERR_OOM, "host allocation failed");
    b->count = count;
    b->soff.assign(stream_off, stream_off + count + 1);
    b->loff.assign(link_off, link_off + count + 1);
    BatchSpec spec{count, stream_off, link_off};
    int rc = create_impl(&b->p, n, m, route_ptr, route_links, c, utype, w, lo, hi, &prm,
                         cuda_stream, on_device, &spec);
    if (rc != NUM_OK) {
        delete b;
        return rc;
    }
    num_problem* h = b->p;
    // work items are built by batch_apply_schedule; room for the smallest item sizes
    std::vector<double> scale(count);
    int64_t cap_s = 0, cap_l = 0;
    for (int i = 0; i < count; ++i) {
        cap_s += (stream_off[i + 1] - stream_off[i] + kStreamItemMin - 1) / kStreamItemMin;
        cap_l += (link_off[i + 1] - link_off[i] + kLinkItemMin - 1) / kLinkItemMin;
        b->J.push_back((double)(inst_nnz[i] + link_off[i + 1] - link_off[i]));
        scale[i] = std::sqrt(b->J.back());
    }
    if (cap_s > INT32_MAX / 4 || cap_l > INT32_MAX / 4) {
        batch_destroy(b);
        return fail(NUM_ERR_INVALID, "too many work items");
    }
    // balanced partitions make at most one item per block plus one per instance
    cap_s = std::max<int64_t>(cap_s, (int64_t)kMaxBalancedBlocks + count);
    cap_l = std::max<int64_t>(cap_l, (int64_t)kMaxBalancedBlocks + count);
    b->cap_sitems = (int)cap_s;
    b->cap_litems = (int)cap_l;
    const int H = prm.history > 0 ? prm.history : 1;
    b->ctls = (pmp::Ctl*)dev_alloc(h, sizeof(pmp::Ctl) * count);
    b->glob = (pmp::BatchGlobal*)dev_alloc(h, sizeof(pmp::BatchGlobal));
    b->sitems = (int4*)dev_alloc(h, sizeof(int4) * (size_t)cap_s);
    b->litems = (int4*)dev_alloc(h, sizeof(int4) * (size_t)cap_l);
    b->sitem_off = (int*)dev_alloc(h, sizeof(int) * (count + 1));
    b->litem_off = (int*)dev_alloc(h, sizeof(int) * (count + 1));
    b->part_s = (double*)dev_alloc(h, sizeof(double) * (size_t)cap_s);
    b->part_l = (double*)dev_alloc(h, sizeof(double) * 2 * (size_t)cap_l);
    b->part_e = (double*)dev_alloc(h, sizeof(double) * (size_t)cap_s);
    b->arrive = (unsigned int*)dev_alloc(h, sizeof(unsigned int) * (size_t)count);
    b->hist = (double*)dev_alloc(h, sizeof(double) * 3 * (size_t)H * count);
    b->eps_scale = (double*)dev_alloc(h, sizeof(double) * count);
    b->soff_d = (int*)dev_alloc(h, sizeof(int) * (count + 1));
    b->loff_d = (int*)dev_alloc(h, sizeof(int) * (count + 1));
    b->bar = (unsigned int*)dev_alloc(h, sizeof(unsigned int) * 2 * (size_t)count);
    b->sblk = (int*)dev_alloc(h, sizeof(int) * (kMaxBalancedBlocks + 1));
    b->lblk = (int*)dev_alloc(h, sizeof(int) * (kMaxBalancedBlocks + 1));
    if (!b->ctls || !b->glob || !b->sitems || !b->litems || !b->sitem_off || !b->litem_off ||
        !b->part_s || !b->part_l || !b->part_e || !b->hist || !b->eps_scale || !b->arrive ||
        !b->soff_d || !b->loff_d || !b->bar || !b->sblk || !b->lblk) {
        batch_destroy(b);
        return fail(NUM_ERR_OOM, "device allocation failed");
    }
    cudaStream_t st = h->stream;
    cudaError_t e;
#define BK(call, what)                  \
    do {                                \
        e = (call);                     \
        if (e != cudaSuccess) {         \
            batch_destroy(b);           \
            return cuda_fail(e, what);  \
        }                               \
    } while (0)
    BK(cudaHostAlloc((void**)&b->ctls_host, sizeof(pmp::Ctl) * count, cudaHostAllocDefault),
       "cudaHostAlloc");
    BK(cudaHostAlloc((void**)&b->glob_host, sizeof(pmp::BatchGlobal), cudaHostAllocDefault),
       "cudaHostAlloc");
    BK(cudaMemcpyAsync(b->eps_scale, scale.data(), sizeof(double) * count, cudaMemcpyHostToDevice,
                       st), "copy scales");
    BK(cudaMemsetAsync(b->hist, 0, sizeof(double) * 3 * (size_t)H * count, st), "memset");
    {
        std::vector<int> so32(count + 1), lo32(count + 1);
        for (int i = 0; i <= count; ++i) {
            so32[i] = (int)stream_off[i];
            lo32[i] = (int)link_off[i];
        }
        BK(cudaMemcpyAsync(b->soff_d, so32.data(), sizeof(int) * (count + 1),
                           cudaMemcpyHostToDevice, st), "copy ranges");
        BK(cudaMemcpyAsync(b->loff_d, lo32.data(), sizeof(int) * (count + 1),
                           cudaMemcpyHostToDevice, st), "copy ranges");
        BK(cudaMemsetAsync(b->bar, 0, sizeof(unsigned int) * 2 * (size_t)count, st), "memset");
        BK(cudaStreamSynchronize(st), "copy ranges");  // the host vectors go out of scope
    }
    rc = batch_chunk_tables(b);
    if (rc == NUM_OK) rc = batch_long_route_tables(b);
    if (rc != NUM_OK) {
        batch_destroy(b);
        return rc;
    }
    rc = batch_apply_schedule(b, kBatchDefault);
    if (rc != NUM_OK) {
        batch_destroy(b);
        return rc;
    }
    rc = batch_reset_all(b);
    if (rc != NUM_OK) {
        batch_destroy(b);
        return rc;
    }
    BK(cudaStreamSynchronize(st), "batch setup");
#undef BK
    *out = b;
    return NUM_OK;
}

}  // namespace

extern "C" {

int num_batch_create(num_batch** out, int32_t count, const int64_t* stream_off,
                     const int64_t* link_off, const int64_t* route_ptr,
                     const int32_t* route_links, const double* c, const uint8_t* utype,
                     const double* w, const double* lo, const double* hi, const num_params* p,
                     void* cuda_stream) {
    TraceRange trace("num_batch_create");
    g_last_error.clear();
    if (!out) return fail(NUM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (count < 1 || !stream_off || !link_off || !route_ptr)
        return fail(NUM_ERR_INVALID, "count must be >= 1 and the offsets non-NULL");
    const int64_t n = stream_off[count];
    if (n < 1 || n > INT32_MAX - 1) return fail(NUM_ERR_INVALID, "total n must be in [1, 2^31 - 1)");
    std::vector<int64_t> nnz(count);
    for (int i = 0; i < count; ++i) {
        if (stream_off[i + 1] <= stream_off[i] || stream_off[i + 1] > n)
            return fail(NUM_ERR_INVALID, "every instance needs >= 1 stream");
        nnz[i] = route_ptr[stream_off[i + 1]] - route_ptr[stream_off[i]];
    }
    return batch_create_impl(out, count, stream_off, link_off, nnz.data(), route_ptr,
                             route_links, c, utype, w, lo, hi, p, cuda_stream, false);
}

int num_batch_create_instances(num_batch** out, int32_t count, const num_instance* insts,
                               const num_params* p, void* cuda_stream) {
    TraceRange trace("num_batch_create_instances");
    g_last_error.clear();
    if (!out) return fail(NUM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (count < 1 || !insts) return fail(NUM_ERR_INVALID, "count must be >= 1 and insts non-NULL");
    std::vector<int64_t> so(count + 1, 0), lo(count + 1, 0), eo(count + 1, 0), nnz(count);
    bool any_lo = false;
    for (int i = 0; i < count; ++i) {
        const num_instance& t = insts[i];
        if (t.n < 1 || t.m < 1) return fail(NUM_ERR_INVALID, "every instance needs n, m >= 1");
        if (!t.route_ptr || !t.route_links || !t.c || !t.utype || !t.w || !t.hi)
            return fail(NUM_ERR_INVALID, "an instance has a required array NULL");
        if (t.route_ptr[0] != 0) return fail(NUM_ERR_INVALID, "an instance has route_ptr[0] != 0");
        nnz[i] = t.route_ptr[t.n];
        if (nnz[i] < t.n) return fail(NUM_ERR_INVALID, "an instance has an empty route");
        so[i + 1] = so[i] + t.n;
        lo[i + 1] = lo[i] + t.m;
        eo[i + 1] = eo[i] + nnz[i];
        if (so[i + 1] > INT32_MAX - 1 || lo[i + 1] > INT32_MAX - 1 || eo[i + 1] > INT32_MAX - 1)
            return fail(NUM_ERR_INVALID, "the stacked problem exceeds 2^31 - 1 streams, links or entries");
        any_lo = any_lo || t.lo != nullptr;
    }
    num_params prm;
    if (p)
        prm = *p;
    else
        num_default_params(&prm);
    const size_t N = (size_t)so[count], M = (size_t)lo[count], NNZ = (size_t)eo[count];
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the stacked inputs live on the device only for the duration of this call
    std::vector<std::pair<void*, size_t>> bufs;
    auto alloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (prm.allocator) {
            q = prm.allocator->alloc(prm.allocator->ctx, bytes, st);
        } else if (cudaMalloc(&q, bytes) != cudaSuccess) {
            cudaGetLastError();
            q = nullptr;
        }
        if (q) bufs.push_back({q, bytes});
        return q;
    };
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (auto& q : bufs) {
            if (prm.allocator)
                prm.allocator->release(prm.allocator->ctx, q.first, q.second, st);
            else
                cudaFree(q.first);
        }
        bufs.clear();
    };
    int64_t* d_rp = (int64_t*)alloc(8 * (N + 1));
    int32_t* d_rl = (int32_t*)alloc(4 * NNZ);
    double* d_c = (double*)alloc(8 * M);
    uint8_t* d_ut = (uint8_t*)alloc(N);
    double* d_w = (double*)alloc(8 * N);
    double* d_lo = any_lo ? (double*)alloc(8 * N) : nullptr;
    double* d_hi = (double*)alloc(8 * N);
    int64_t* d_off = (int64_t*)alloc(8 * 3 * ((size_t)count + 1));
    if (!d_rp || !d_rl || !d_c || !d_ut || !d_w || (any_lo && !d_lo) || !d_hi || !d_off) {
        release();
        return fail(NUM_ERR_OOM, "device allocation failed");
    }
    cudaError_t e = cudaMemsetAsync(d_rp, 0, 8, st);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const num_instance& t = insts[i];
        const size_t n = (size_t)t.n, m = (size_t)t.m;
        e = cudaMemcpyAsync(d_rp + so[i] + 1, t.route_ptr + 1, 8 * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_rl + eo[i], t.route_links, 4 * (size_t)nnz[i],
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_c + lo[i], t.c, 8 * m, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_ut + so[i], t.utype, n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_w + so[i], t.w, 8 * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_hi + so[i], t.hi, 8 * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && d_lo)
            e = t.lo ? cudaMemcpyAsync(d_lo + so[i], t.lo, 8 * n, cudaMemcpyHostToDevice, st)
                     : cudaMemsetAsync(d_lo + so[i], 0, 8 * n, st);  // +0.0 is all zero bits
    }
    std::vector<int64_t> offs;
    offs.insert(offs.end(), so.begin(), so.end());
    offs.insert(offs.end(), lo.begin(), lo.end());
    offs.insert(offs.end(), eo.begin(), eo.end());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_off, offs.data(), 8 * offs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = pmp::stack_offsets(count, d_off, d_off + count + 1, d_off + 2 * (count + 1), d_rp,
                               d_rl, (long long)N, (long long)NNZ, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // offs is a pageable host vector
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "stacking the instances");
    }
    const int rc = batch_create_impl(out, count, so.data(), lo.data(), nnz.data(), d_rp, d_rl,
                                     d_c, d_ut, d_w, d_lo, d_hi, &prm, cuda_stream, true);
    release();
    return rc;
}

int num_batch_set_rho_schedules(num_batch* b, const int8_t* decisions, int64_t len) {
    g_last_error.clear();
    if (!b) return fail(NUM_ERR_INVALID, "batch is NULL");
    if (len < 0 || len > INT32_MAX || (len > 0 && !decisions))
        return fail(NUM_ERR_INVALID, "bad schedule");
    for (int64_t i = 0; i < len * b->count; ++i)
        if (decisions[i] < -1 || decisions[i] > 1)
            return fail(NUM_ERR_INVALID, "schedule entries must be -1, 0 or +1");
    num_problem* h = b->p;
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    if (b->sched) {
        dev_free(h, b->sched);
        b->sched = nullptr;
    }
    b->sched_stride = 0;
    if (len > 0) {
        b->sched = (signed char*)dev_alloc(h, (size_t)len * b->count);
        if (!b->sched) return fail(NUM_ERR_OOM, "device allocation failed");
        e = cudaMemcpyAsync(b->sched, decisions, (size_t)len * b->count, cudaMemcpyHostToDevice,
                            h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy schedule");
        b->sched_stride = (int)len;
    }
    if (b->graph_exec) {
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    // every instance: sched_len = len (the rest of its control block is kept)
    e = cudaMemcpyAsync(b->ctls_host, b->ctls, sizeof(pmp::Ctl) * b->count,
                        cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "schedule");
    for (int i = 0; i < b->count; ++i) b->ctls_host[i].sched_len = (int)len;
    e = cudaMemcpyAsync(b->ctls, b->ctls_host, sizeof(pmp::Ctl) * b->count,
                        cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return finish_cuda(e, "schedule");
}

int num_batch_solve(num_batch* b, int64_t max_iters, double eps_abs, int64_t* iters_done,
                    int32_t* status) {
    TraceRange trace("num_batch_solve");
    g_last_error.clear();
    if (!b) return fail(NUM_ERR_INVALID, "batch is NULL");
    if (max_iters < 0) return fail(NUM_ERR_INVALID, "max_iters must be >= 0");
    if (std::isnan(eps_abs)) return fail(NUM_ERR_INVALID, "eps_abs is NaN");
    if (b->broken)
        return fail(NUM_ERR_STATE, "a persistent solve timed out: call num_batch_reset first");
    num_problem* h = b->p;
    cudaStream_t st = h->stream;
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ctls_host, b->ctls, sizeof(pmp::Ctl) * b->count,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the control blocks");
    std::vector<long long> k0(b->count);
    for (int i = 0; i < b->count; ++i) k0[i] = b->ctls_host[i].k;
    const double eps = eps_abs > 0.0 ? eps_abs : (eps_abs < 0.0 ? h->prm.eps_abs : 0.0);
    e = pmp::batch_arm(b->ctls, b->glob, b->count, max_iters, eps, b->eps_scale, st);
    if (e != cudaSuccess) return cuda_fail(e, "arming the instances");
    const int K = h->prm.check_every;
    if (max_iters > 0 && b->persistent) {
        const int prc = batch_solve_persistent(b, max_iters);
        if (prc != NUM_OK) return prc;
    } else if (max_iters > 0) {
        if (h->prm.use_graph && !b->graph_exec) {
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
            cudaError_t e2 = batch_run(b, K);
            e = cudaStreamEndCapture(st, &b->graph);
            if (e2 != cudaSuccess) return cuda_fail(e2, "capturing the batch graph");
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        }
        const long long max_launches = (max_iters + K - 1) / K + 1;
        long long done_prev = 0;
        for (long long it = 0;; ++it) {
            if (it >= max_launches) return fail(NUM_ERR_STATE, "the iteration limit was not honoured");
            TraceRange replay("num_batch_solve: replay of check_every iterations");
            e = h->prm.use_graph ? cudaGraphLaunch(b->graph_exec, st) : batch_run(b, K);
            if (e != cudaSuccess) return cuda_fail(e, "launching iterations");
            pmp::note_launches((long long)K * 2);
            e = cudaMemcpyAsync(b->glob_host, b->glob, sizeof(pmp::BatchGlobal),
                                cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "iterations");
            if (h->prm.profile) {
                // kernels of iterations after every instance stopped exit at once; the
                // batch's slowest instance decides how many did work
                e = cudaMemcpyAsync(b->ctls_host, b->ctls, sizeof(pmp::Ctl) * b->count,
                                    cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return cuda_fail(e, "iterations");
                long long most = 0;
                for (int i = 0; i < b->count; ++i)
                    most = std::max(most, b->ctls_host[i].k - k0[i]);
                const long long ran = most - done_prev;
                done_prev = most;
                const long long timed = std::min(ran, (long long)profiled_iterations(h));
                for (long long i = 0; i < timed; ++i)
                    for (int q = 0; q < 2; ++q) {
                        float ms = 0.f;
                        e = cudaEventElapsedTime(&ms, h->evs[i * 2 + q], h->evs[i * 2 + q + 1]);
                        if (e != cudaSuccess) return cuda_fail(e, "reading kernel times");
                        b->kernel_ms[q] += ms;
                        b->kernel_runs[q] += 1;
                    }
            }
            if (b->glob_host->running == 0) break;
        }
    }
    e = cudaMemcpyAsync(b->ctls_host, b->ctls, sizeof(pmp::Ctl) * b->count,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the control blocks");
    int rc = NUM_OK;
    for (int i = 0; i < b->count; ++i) {
        const pmp::Ctl& c = b->ctls_host[i];
        if (iters_done) iters_done[i] = c.k - k0[i];
        const int stt = max_iters == 0 ? (int)pmp::LIMIT : c.stop;
        if (status) status[i] = stt == pmp::CONVERGED ? NUM_OK
                                : stt == pmp::NONFINITE ? NUM_ERR_NUMERIC : NUM_NOT_CONVERGED;
        if (stt == pmp::NONFINITE) rc = NUM_ERR_NUMERIC;
        else if (stt != pmp::CONVERGED && rc == NUM_OK) rc = NUM_NOT_CONVERGED;
    }
    const int dbg_rc = check_debug_flag(h);
    if (dbg_rc != NUM_OK) return dbg_rc;
    if (rc == NUM_ERR_NUMERIC) return fail(rc, "a residual of some instance became non-finite");
    return rc;
}

int num_batch_get(const num_batch* bc, double* x, double* prices, double* info) {
    TraceRange trace("num_batch_get");
    g_last_error.clear();
    if (!bc) return fail(NUM_ERR_INVALID, "batch is NULL");
    num_batch* b = const_cast<num_batch*>(bc);
    num_problem* h = b->p;
    cudaStream_t st = h->stream;
    cudaError_t e = order_after_legacy(h);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    double* xo = x ? h->x64 : nullptr;
    double* yo = prices ? h->y64 : nullptr;
    e = h->prec == NUM_FUSED_FP32
            ? pmp::batch_export<float>(make_batch_view<float>(b), b->grid_e, xo, yo, b->part_e, st)
            : pmp::batch_export<double>(make_batch_view<double>(b), b->grid_e, xo, yo, b->part_e,
                                        st);
    if (e != cudaSuccess) return cuda_fail(e, "exporting the solutions");
    if (x) e = cudaMemcpyAsync(x, h->x64, 8 * (size_t)h->n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && prices)
        e = cudaMemcpyAsync(prices, h->y64, 8 * (size_t)h->m, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ctls_host, b->ctls, sizeof(pmp::Ctl) * b->count,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the results");
    if (info) {
        for (int i = 0; i < b->count; ++i) {
            const pmp::Ctl& c = b->ctls_host[i];
            double* o = info + (size_t)i * NUM_INFO_LEN;
            o[NUM_INFO_PRIMAL] = c.rnorm;
            o[NUM_INFO_DUAL] = c.snorm;
            o[NUM_INFO_EPS_TOL] = c.eps_tol;
            o[NUM_INFO_RHO] = c.rho;
            o[NUM_INFO_OBJECTIVE] = c.objective;
            o[NUM_INFO_ITERS] = (double)c.k;
            o[NUM_INFO_STATUS] = (double)c.stop;
            o[NUM_INFO_J] = b->J[i];
        }
    }
    return NUM_OK;
}

int num_batch_get_kernel_times(const num_batch* b, double* ms, int64_t* launches,
                               int32_t max_kernels, int32_t* nkernels) {
    g_last_error.clear();
    if (!b) return fail(NUM_ERR_INVALID, "batch is NULL");
    if (max_kernels < 0 || (max_kernels > 0 && (!ms || !launches)))
        return fail(NUM_ERR_INVALID, "bad buffers");
    if (nkernels) *nkernels = 2;
    for (int q = 0; q < 2 && q < max_kernels; ++q) {
        ms[q] = b->kernel_ms[q];
        launches[q] = b->kernel_runs[q];
    }
    return NUM_OK;
}

int num_batch_get_schedule(const num_batch* b, num_batch_schedule* out) {
    g_last_error.clear();
    if (!b || !out) return fail(NUM_ERR_INVALID, "batch or out is NULL");
    *out = b->cfg;
    return NUM_OK;
}

int num_batch_set_schedule(num_batch* b, const num_batch_schedule* cfg) {
    g_last_error.clear();
    if (!b || !cfg) return fail(NUM_ERR_INVALID, "batch or schedule is NULL");
    if (!valid_schedule(*cfg))
        return fail(NUM_ERR_INVALID, "stream_item must be a power of two in [256, 65536], "
                                     "link_item a power of two in [32, 8192], link_lanes 4, 8, "
                                     "16 or 32");
    cudaError_t e = order_after_legacy(b->p);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    return batch_apply_schedule(b, *cfg);
}

int num_batch_autotune(num_batch* b, int32_t trial_iters, num_batch_schedule* chosen,
                       double* trial_ms, int32_t max_trials, int32_t* ntrials) {
    TraceRange trace("num_batch_autotune");
    g_last_error.clear();
    if (!b) return fail(NUM_ERR_INVALID, "batch is NULL");
    if (trial_iters < 1 || trial_iters > 500)
        return fail(NUM_ERR_INVALID, "trial_iters must be in [1, 500]");
    if (max_trials < 0 || (max_trials > 0 && !trial_ms))
        return fail(NUM_ERR_INVALID, "bad trial buffer");
    num_problem* h = b->p;
    cudaError_t e = order_after_legacy(h);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    num_batch_schedule best = b->cfg;
    int t = 0;
    auto record = [&](const num_batch_schedule& c, double ms) {
        if (t < max_trials) {
            trial_ms[4 * t] = c.stream_item;
            trial_ms[4 * t + 1] = c.link_item;
            trial_ms[4 * t + 2] = c.link_lanes;
            trial_ms[4 * t + 3] = ms;
        }
        ++t;
    };
    // stage 1: streams per stream item (the stream kernel's time), link side as it is
    double best_s = 0.0;
    for (int si : kTuneStreamItems) {
        num_batch_schedule c{si, best.link_item, best.link_lanes};
        double ts = 0.0, tl = 0.0;
        const int rc = batch_time_schedule(b, c, trial_iters, &ts, &tl);
        if (rc != NUM_OK) return rc;
        record(c, ts);
        if (si == kTuneStreamItems[0] || ts < best_s) {
            best_s = ts;
            best.stream_item = si;
        }
    }
    // stage 2: links per link item and lanes per link (the link kernel's time)
    double best_l = 0.0;
    bool first = true;
    const int stream_item = best.stream_item;
    for (int li : kTuneLinkItems)
        for (int ln : kTuneLanes) {
            num_batch_schedule c{stream_item, li, ln};
            double ts = 0.0, tl = 0.0;
            const int rc = batch_time_schedule(b, c, trial_iters, &ts, &tl);
            if (rc != NUM_OK) return rc;
            record(c, tl);
            if (first || tl < best_l) {
                best_l = tl;
                best.link_item = li;
                best.link_lanes = ln;
                first = false;
            }
        }
    int rc = batch_apply_schedule(b, best);
    if (rc != NUM_OK) return rc;
    // the trials moved the iterates: start over from zero
    e = zero_state(h);
    if (e != cudaSuccess) return cuda_fail(e, "zeroing the state");
    rc = batch_reset_all(b);
    if (rc != NUM_OK) return rc;
    e = cudaMemsetAsync(b->hist, 0,
                        sizeof(double) * 3 * (size_t)(h->prm.history > 0 ? h->prm.history : 1) *
                            b->count, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "resetting after the trials");
    b->kernel_ms[0] = b->kernel_ms[1] = 0.0;
    b->kernel_runs[0] = b->kernel_runs[1] = 0;
    if (chosen) *chosen = best;
    if (ntrials) *ntrials = t;
    return NUM_OK;
}

int num_batch_set_persistent(num_batch* b, int32_t enable, int64_t wait_polls) {
    g_last_error.clear();
    if (!b) return fail(NUM_ERR_INVALID, "batch is NULL");
    if (enable != 0 && enable != 1) return fail(NUM_ERR_INVALID, "enable must be 0 or 1");
    if (wait_polls < 0) return fail(NUM_ERR_INVALID, "wait_polls must be >= 0");
    num_problem* h = b->p;
    if (enable) {
        int cap = 0;
        cudaError_t e = pmp::batch_persistent_capacity(h->prec == NUM_FUSED_FP32 ? 0 : 1,
                                                       b->cfg.link_lanes, h->nlong > 0, &cap);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy of the persistent kernel");
        if (cap < 1) return fail(NUM_ERR_STATE, "the persistent kernel cannot be resident");
    }
    b->persistent = enable != 0;
    b->wait_polls = wait_polls > 0 ? wait_polls : kDefaultWaitPolls;
    return NUM_OK;
}

int num_batch_reset(num_batch* b) {
    TraceRange trace("num_batch_reset");
    g_last_error.clear();
    if (!b) return fail(NUM_ERR_INVALID, "batch is NULL");
    num_problem* h = b->p;
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = zero_state(h);
    if (e != cudaSuccess) return cuda_fail(e, "zeroing the state");
    int rc = batch_reset_all(b);
    if (rc != NUM_OK) return rc;
    e = cudaMemsetAsync(b->hist, 0,
                        sizeof(double) * 3 * (size_t)(h->prm.history > 0 ? h->prm.history : 1) *
                            b->count, h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned int) * 2 * (size_t)b->count, h->stream);
    if (e == cudaSuccess && h->nchunks > 0)
        e = cudaMemsetAsync(h->arrive_l, 0, sizeof(int) * (size_t)h->nchunks, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "resetting the batch");
    b->broken = false;
    return NUM_OK;
}

void num_batch_destroy(num_batch* b) { batch_destroy(b); }

}  // extern "C"
