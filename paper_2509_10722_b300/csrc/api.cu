// C ABI of the PMP solver (declared in include/num_pmp.h): handle lifetime, device memory,
// input validation, the CUDA-graph iteration loop and result export.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "num_pmp.h"
#include "pmp_internal.cuh"

using pmp::Ctl;
using pmp::View;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(NUM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                                  cudaGetErrorString(e) + ")");
}

constexpr int kMaxGrid = 8192;
constexpr int kExportBlocksMax = 1024;

std::atomic<long long> g_launches{0};

}  // namespace

namespace pmp {
void note_launches(long long count) { g_launches.fetch_add(count, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }
int report_error(int code, const std::string& msg) { return fail(code, msg); }
int report_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }
void clear_error() { g_last_error.clear(); }
}  // namespace pmp

struct num_problem {
    int64_t n = 0, m = 0, nnz = 0;
    int Js = 0, Jl = 0;
    num_params prm{};
    num_allocator alloc{};
    bool custom_alloc = false;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;  // where the work goes
    bool own_stream = false;
    cudaEvent_t legacy_ev = nullptr;
    int device = 0;
    int prec = 0;
    std::vector<std::pair<void*, size_t>> blocks;

    int *col_ptr = nullptr, *row_idx = nullptr, *row_ptr = nullptr, *col_idx = nullptr;
    int2 *tiles_s = nullptr, *tiles_l = nullptr;
    int ntiles_s = 0, ntiles_l = 0, tile_s = 0, tile_l = 0, grid_s = 0, grid_l = 0;
    int sched_kind = NUM_SCHEDULE_ROWS;  // fused paths: row kernels or merge-path tiles
    int* perm = nullptr;                 // caller's index of the stream at each position
    uint8_t* ut = nullptr;               // utility types, only if some stream has U = -w / x
    int4* chunks = nullptr;              // row kernels: chunks of the long links
    int nchunks = 0;
    int narrive_l = 0;                   // entries of arrive_l
    void *wt = nullptr, *lo = nullptr, *hi = nullptr, *c = nullptr;
    void *x = nullptr, *Z = nullptr, *pby = nullptr, *zs = nullptr, *Rx = nullptr, *ps = nullptr;
    void *carry_s = nullptr, *carry_l = nullptr;
    int *arrive_s = nullptr, *arrive_l = nullptr;
    double *part_s = nullptr, *part_l = nullptr;
    int plain_nb = 0;
    void *A = nullptr, *B = nullptr, *tS = nullptr, *tR = nullptr, *tL = nullptr, *RxN = nullptr,
         *pbar = nullptr, *y = nullptr;
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;  // pinned
    double* hist = nullptr;
    signed char* sched = nullptr;
    int sched_len = 0;
    double* x64 = nullptr;
    double* y64 = nullptr;
    double* part_exp = nullptr;
    int exp_blocks = 0;
    int box_uniform = 0;
    double lo_u = 0.0, hi_u = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    double last_eps_tol = 0.0;
    // profiling: evs[0] before the first kernel of a batch of iterations, then one event
    // after every kernel; per-kernel totals
    std::vector<cudaEvent_t> evs;
    double kernel_ms[pmp::kPlainKernelsPerIter] = {};
    long long kernel_runs[pmp::kPlainKernelsPerIter] = {};
    int kpi = 0;  // kernels per iteration
};

namespace {

void* dev_alloc(num_problem* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (h->custom_alloc) {
        p = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->user_stream);
    } else {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (p) h->blocks.emplace_back(p, bytes);
    return p;
}

void dev_free(num_problem* h, void* p) {
    if (!p) return;
    for (size_t i = 0; i < h->blocks.size(); ++i) {
        if (h->blocks[i].first == p) {
            if (h->custom_alloc)
                h->alloc.release(h->alloc.ctx, p, h->blocks[i].second, (void*)h->stream);
            else
                cudaFree(p);
            h->blocks.erase(h->blocks.begin() + i);
            return;
        }
    }
}

void destroy_handle(num_problem* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    while (!h->blocks.empty()) dev_free(h, h->blocks.back().first);
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    for (cudaEvent_t ev : h->evs) cudaEventDestroy(ev);
    if (h->legacy_ev) cudaEventDestroy(h->legacy_ev);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Work submitted by the caller to the legacy default stream before this call must finish
// before the handle's own stream runs (the handle's stream is a non-blocking one then).
cudaError_t order_after_legacy(num_problem* h) {
    if (!h->own_stream) return cudaSuccess;
    cudaError_t e = cudaEventRecord(h->legacy_ev, cudaStreamLegacy);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(h->stream, h->legacy_ev, 0);
}

template <typename T>
View<T> make_view(const num_problem* h) {
    View<T> v;
    std::memset(&v, 0, sizeof(v));
    v.n = (int)h->n;
    v.m = (int)h->m;
    v.nnz = (int)h->nnz;
    v.Js = h->Js;
    v.Jl = h->Jl;
    v.col_ptr = h->col_ptr;
    v.row_idx = h->row_idx;
    v.row_ptr = h->row_ptr;
    v.col_idx = h->col_idx;
    v.tiles_s = h->tiles_s;
    v.tiles_l = h->tiles_l;
    v.ntiles_s = h->ntiles_s;
    v.ntiles_l = h->ntiles_l;
    v.tile_s = h->tile_s;
    v.tile_l = h->tile_l;
    v.wt = (const T*)h->wt;
    v.lo = (const T*)h->lo;
    v.hi = (const T*)h->hi;
    v.lo_u = (T)h->lo_u;
    v.hi_u = (T)h->hi_u;
    v.box_uniform = h->box_uniform;
    v.c = (const T*)h->c;
    v.x = (T*)h->x;
    v.Z = (T*)h->Z;
    v.pby = (typename View<T>::T2*)h->pby;
    v.zs = (T*)h->zs;
    v.Rx = (T*)h->Rx;
    v.ps = (T*)h->ps;
    v.carry_s = (typename View<T>::T2*)h->carry_s;
    v.carry_l = (T*)h->carry_l;
    v.arrive_s = h->arrive_s;
    v.arrive_l = h->arrive_l;
    v.part_s = h->part_s;
    v.part_l = h->part_l;
    v.grid_s = h->grid_s;
    v.grid_l = h->grid_l;
    v.chunks = h->chunks;
    v.nchunks = h->nchunks;
    v.perm = h->perm;
    v.ut = h->ut;
    v.ctl = h->ctl;
    v.hist = h->hist;
    v.sched = h->sched;
    v.A = (T*)h->A;
    v.B = (T*)h->B;
    v.tS = (T*)h->tS;
    v.tR = (T*)h->tR;
    v.tL = (T*)h->tL;
    v.RxN = (T*)h->RxN;
    v.pbar = (T*)h->pbar;
    v.y = (T*)h->y;
    return v;
}

// Enqueue `count` iterations (count <= check_every when profiling).  Not counted as
// launches here: the caller counts what actually executes.
cudaError_t run_iterations(num_problem* h, int count) {
    const bool prof = h->prm.profile != 0;
    if (prof) {
        cudaError_t e = pmp::record_kernel_event(h->evs[0], h->stream);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < count; ++i) {
        cudaEvent_t* ev = prof ? h->evs.data() + 1 + (size_t)i * h->kpi : nullptr;
        cudaError_t e;
        const bool rows = h->sched_kind == NUM_SCHEDULE_ROWS;
        if (h->prec == NUM_FUSED_FP32)
            e = rows ? pmp::rows_iteration<float>(make_view<float>(h), h->stream, ev)
                     : pmp::fused_iteration<float>(make_view<float>(h), h->stream, ev);
        else if (h->prec == NUM_FUSED_FP64)
            e = rows ? pmp::rows_iteration<double>(make_view<double>(h), h->stream, ev)
                     : pmp::fused_iteration<double>(make_view<double>(h), h->stream, ev);
        else
            e = pmp::plain_iteration(make_view<double>(h), h->plain_nb, h->stream, ev);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// After a batch of iterations completed (stream synchronized): add the per-kernel times of
// the first `ran` iterations of the batch (the later ones exited at the stop flag).
cudaError_t accumulate_kernel_times(num_problem* h, long long ran) {
    for (long long i = 0; i < ran; ++i) {
        for (int q = 0; q < h->kpi; ++q) {
            const size_t cur = 1 + (size_t)i * h->kpi + q;
            float ms = 0.f;
            cudaError_t e = cudaEventElapsedTime(&ms, h->evs[cur - 1], h->evs[cur]);
            if (e != cudaSuccess) return e;
            h->kernel_ms[q] += ms;
            h->kernel_runs[q] += 1;
        }
    }
    return cudaSuccess;
}

cudaError_t zero_state(num_problem* h) {
    const size_t ts = h->prec == NUM_FUSED_FP32 ? 4 : 8;
    cudaStream_t st = h->stream;
    cudaError_t e = cudaSuccess;
    auto z = [&](void* p, size_t bytes) {
        if (p && e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, st);
    };
    z(h->x, ts * h->n);
    z(h->Z, ts * h->n);
    z(h->pby, 2 * ts * h->m);
    z(h->zs, ts * h->m);
    z(h->Rx, ts * h->m);
    z(h->ps, ts * h->m);
    z(h->pbar, ts * h->m);
    z(h->y, ts * h->m);
    z(h->arrive_s, sizeof(int) * (size_t)h->ntiles_s);
    z(h->arrive_l, sizeof(int) * (size_t)h->narrive_l);
    if (h->hist && h->prm.history > 0) z(h->hist, sizeof(double) * 3 * (size_t)h->prm.history);
    if (e != cudaSuccess) return e;
    e = pmp::ctl_reset(h->ctl, h->prm.rho0, h->prm.alpha, h->prm.mu, h->prm.gamma,
                       h->prm.rho_period, h->prm.history, st);
    if (e != cudaSuccess) return e;
    if (h->sched_len > 0) e = pmp::ctl_set_schedule_len(h->ctl, h->sched_len, st);
    return e;
}

bool is_pow2_tile(int t) { return t >= 256 && t <= 8192 && (t & (t - 1)) == 0; }

int check_params(const num_params& p) {
    if (!(p.rho0 > 0.0) || !std::isfinite(p.rho0))
        return fail(NUM_ERR_INVALID, "rho0 must be finite and > 0");
    if (!(p.alpha > 0.0 && p.alpha < 2.0)) return fail(NUM_ERR_INVALID, "alpha must be in (0, 2)");
    if (!(p.mu >= 1.0) || !std::isfinite(p.mu)) return fail(NUM_ERR_INVALID, "mu must be >= 1");
    if (!(p.gamma >= 1.0) || !std::isfinite(p.gamma))
        return fail(NUM_ERR_INVALID, "gamma must be >= 1");
    if (std::isnan(p.eps_abs)) return fail(NUM_ERR_INVALID, "eps_abs is NaN");
    if (p.rho_period < 0) return fail(NUM_ERR_INVALID, "rho_period must be >= 0");
    if (p.precision < 0 || p.precision > 2) return fail(NUM_ERR_INVALID, "unknown precision");
    if (p.check_every < 1) return fail(NUM_ERR_INVALID, "check_every must be >= 1");
    if (p.tile_items != 0 && !is_pow2_tile(p.tile_items))
        return fail(NUM_ERR_INVALID, "tile_items must be 0 or a power of two in [256, 8192]");
    if (p.history < 0) return fail(NUM_ERR_INVALID, "history must be >= 0");
    if (p.profile != 0 && p.profile != 1) return fail(NUM_ERR_INVALID, "profile must be 0 or 1");
    if (p.schedule < 0 || p.schedule > NUM_SCHEDULE_TILES)
        return fail(NUM_ERR_INVALID, "unknown schedule");
    if (p.reorder != 0 && p.reorder != 1) return fail(NUM_ERR_INVALID, "reorder must be 0 or 1");
    if (p.allocator && (!p.allocator->alloc || !p.allocator->release))
        return fail(NUM_ERR_INVALID, "allocator needs alloc and release");
    return NUM_OK;
}

std::string describe_bits(int bits) {
    std::string s;
    auto add = [&](int b, const char* t) {
        if (bits & b) s += (s.empty() ? "" : "; ") + std::string(t);
    };
    add(pmp::VB_ROUTE, "route_ptr must start at 0 and increase (every route nonempty)");
    add(pmp::VB_LINK_ID, "a link id is outside [0, m)");
    add(pmp::VB_DUPLICATE, "a link appears twice in one route");
    add(pmp::VB_CAPACITY, "a capacity is not finite and > 0");
    add(pmp::VB_WEIGHT, "a weight is not finite and > 0");
    add(pmp::VB_UTYPE, "a utility type is not NUM_LOG, NUM_LINEAR or NUM_ALPHA2");
    add(pmp::VB_BOX, "a box is not finite with lo <= hi (and hi > 0 for log and alpha = 2)");
    add(pmp::VB_BLOCKS, "a route uses a link of another instance of the batch");
    return s;
}

// Instances of a batch: host arrays of count + 1 offsets into the stacked numbering.
struct BatchSpec {
    int count;
    const int64_t* stream_off;
    const int64_t* link_off;
};

int create_impl(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
                const int32_t* route_links, const double* c, const uint8_t* utype,
                const double* w, const double* lo, const double* hi, const num_params* p,
                void* cuda_stream, bool on_device, const BatchSpec* batch = nullptr) {
    g_last_error.clear();
    if (!out) return fail(NUM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!route_ptr || !route_links || !c || !utype || !w || !hi)
        return fail(NUM_ERR_INVALID, "a required array is NULL");
    if (n < 1 || m < 1) return fail(NUM_ERR_INVALID, "n and m must be >= 1");
    if (n > INT32_MAX - 1 || m > INT32_MAX - 1)
        return fail(NUM_ERR_INVALID, "n and m must be < 2^31 - 1");
    num_params prm;
    if (p)
        prm = *p;
    else
        num_default_params(&prm);
    int rc = check_params(prm);
    if (rc != NUM_OK) return rc;

    int64_t p0 = 0, nnz = 0;
    if (on_device) {
        cudaError_t e = cudaMemcpy(&p0, route_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(&nnz, route_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "reading route_ptr");
    } else {
        p0 = route_ptr[0];
        nnz = route_ptr[n];
    }
    if (p0 != 0) return fail(NUM_ERR_INVALID, "route_ptr[0] must be 0");
    if (nnz < n) return fail(NUM_ERR_INVALID, "route_ptr[n] < n: some route is empty");
    if (nnz + (n > m ? n : m) > (int64_t)INT32_MAX - 1)
        return fail(NUM_ERR_INVALID, "nnz + max(n, m) must be < 2^31 - 1");

    num_problem* h = new (std::nothrow) num_problem();
    if (!h) return fail(NUM_ERR_OOM, "host allocation failed");
    h->n = n;
    h->m = m;
    h->nnz = nnz;
    h->Js = (int)(nnz + n);
    h->Jl = (int)(nnz + m);
    h->prm = prm;
    h->prec = prm.precision;
    h->user_stream = (cudaStream_t)cuda_stream;
    if (prm.allocator) {
        h->alloc = *prm.allocator;
        h->custom_alloc = true;
    }
    h->prm.allocator = nullptr;

    const bool fp32 = h->prec == NUM_FUSED_FP32;
    const bool plain = h->prec == NUM_PLAIN_FP64;
    const size_t ts = fp32 ? 4 : 8;
    const size_t N = (size_t)n, M = (size_t)m, NNZ = (size_t)nnz;
    h->tile_s = prm.tile_items ? prm.tile_items : pmp::fused_tile_items_stream(fp32 ? 0 : 1);
    h->tile_l = prm.tile_items ? prm.tile_items : pmp::fused_tile_items_link(fp32 ? 0 : 1);
    h->ntiles_s = (int)((h->Js + (int64_t)h->tile_s - 1) / h->tile_s);
    h->ntiles_l = (int)((h->Jl + (int64_t)h->tile_l - 1) / h->tile_l);
    h->plain_nb = pmp::plain_partial_blocks((int)n, (int)m);
    h->sched_kind = prm.schedule == NUM_SCHEDULE_TILES ? NUM_SCHEDULE_TILES : NUM_SCHEDULE_ROWS;
    const bool tiles = !plain && h->sched_kind == NUM_SCHEDULE_TILES;
    const bool rowk = !plain && h->sched_kind == NUM_SCHEDULE_ROWS;
    h->exp_blocks = pmp::export_partial_blocks((int)n);

    // ---- device memory: the handle's arrays, then the transient build buffers ----
    bool ok = true;
    auto A = [&](size_t bytes) -> void* {
        if (!ok) return nullptr;
        void* q = dev_alloc(h, bytes);
        if (!q) ok = false;
        return q;
    };
    h->col_ptr = (int*)A(4 * (N + 1));
    h->row_idx = (int*)A(4 * NNZ);
    h->row_ptr = (int*)A(4 * (M + 1));
    h->col_idx = (int*)A(4 * NNZ);
    h->wt = A(ts * N);
    h->lo = A(ts * N);
    h->hi = A(ts * N);
    h->c = A(ts * M);
    h->x = A(ts * N);
    h->Z = A(ts * N);
    h->zs = A(ts * M);
    h->Rx = A(ts * M);
    h->ps = A(ts * M);
    if (plain) {
        h->pbar = A(ts * M);
        h->y = A(ts * M);
        h->A = A(ts * N);
        h->B = A(ts * N);
        h->tS = A(ts * N);
        h->tR = A(ts * M);
        h->tL = A(ts * M);
        h->RxN = A(ts * M);
    } else {
        h->pby = A(2 * ts * M);
    }
    if (tiles) {
        h->tiles_s = (int2*)A(sizeof(int2) * (size_t)h->ntiles_s);
        h->tiles_l = (int2*)A(sizeof(int2) * (size_t)h->ntiles_l);
        h->carry_s = A(2 * ts * 2 * (size_t)h->ntiles_s);
        h->carry_l = A(ts * 2 * (size_t)h->ntiles_l);
        h->arrive_s = (int*)A(sizeof(int) * (size_t)h->ntiles_s);
        h->arrive_l = (int*)A(sizeof(int) * (size_t)h->ntiles_l);
        h->narrive_l = h->ntiles_l;
    }
    const size_t npart = (size_t)(kMaxGrid > h->plain_nb ? kMaxGrid : h->plain_nb);
    h->part_s = (double*)A(sizeof(double) * npart);
    h->part_l = (double*)A(sizeof(double) * 2 * npart);
    h->ctl = (Ctl*)A(sizeof(Ctl));
    h->hist = (double*)A(sizeof(double) * 3 * (size_t)(prm.history > 0 ? prm.history : 1));
    h->x64 = (double*)A(8 * N);
    h->y64 = (double*)A(8 * M);
    h->part_exp = (double*)A(sizeof(double) * kExportBlocksMax);
    // transient
    int64_t* d_rp = nullptr;
    int* d_rl = nullptr;
    double *d_c = nullptr, *d_w = nullptr, *d_lo = nullptr, *d_hi = nullptr;
    uint8_t* d_ut = nullptr;
    if (!on_device) {
        d_rp = (int64_t*)A(8 * (N + 1));
        d_rl = (int*)A(4 * NNZ);
        d_c = (double*)A(8 * M);
        d_w = (double*)A(8 * N);
        d_lo = lo ? (double*)A(8 * N) : nullptr;
        d_hi = (double*)A(8 * N);
        d_ut = (uint8_t*)A(N);
    }
    int* d_err = (int*)A(sizeof(int) * 2);
    int64_t* d_soff = batch ? (int64_t*)A(8 * ((size_t)batch->count + 1)) : nullptr;
    int64_t* d_loff = batch ? (int64_t*)A(8 * ((size_t)batch->count + 1)) : nullptr;
    unsigned long long* d_box = (unsigned long long*)A(sizeof(unsigned long long) * 4);
    pmp::Scratch s{};
    s.keys_a = (int*)A(4 * NNZ);
    s.vals_a = (int*)A(4 * NNZ);
    s.keys_b = (int*)A(4 * NNZ);
    s.vals_b = (int*)A(4 * NNZ);
    s.hist_len = pmp::radix_hist_len((int)nnz);
    s.scan_tmp_len = pmp::scan_tmp_len(s.hist_len);
    s.hist = (int*)A(4 * s.hist_len);
    s.scan_tmp = (int*)A(4 * s.scan_tmp_len);
    const bool reorder = prm.reorder != 0;
    h->perm = reorder ? (int*)A(4 * N) : nullptr;
    int64_t* d_rp2 = reorder ? (int64_t*)A(8 * (N + 1)) : nullptr;
    int* d_rl2 = reorder ? (int*)A(4 * NNZ) : nullptr;
    int* d_lens = reorder ? (int*)A(4 * (N + 1)) : nullptr;
    int* d_ptr32 = reorder ? (int*)A(4 * (N + 1)) : nullptr;
    int* d_ptmp = reorder ? (int*)A(4 * pmp::scan_tmp_len(N + 1)) : nullptr;
    int* d_ccount = rowk ? (int*)A(4 * (M + 1)) : nullptr;
    int* d_coff = rowk ? (int*)A(4 * (M + 1)) : nullptr;
    int* d_ctmp = rowk ? (int*)A(4 * pmp::scan_tmp_len(M + 1)) : nullptr;
    if (!ok) {
        destroy_handle(h);
        return fail(NUM_ERR_OOM, "device allocation failed");
    }

    // ---- from here on: CUDA work ----
    cudaError_t e;
#define CK(call, what)                          \
    do {                                        \
        e = (call);                             \
        if (e != cudaSuccess) {                 \
            destroy_handle(h);                  \
            return cuda_fail(e, what);          \
        }                                       \
    } while (0)
    CK(cudaGetDevice(&h->device), "cudaGetDevice");
    if (h->user_stream == nullptr) {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        h->own_stream = true;
        CK(cudaEventCreateWithFlags(&h->legacy_ev, cudaEventDisableTiming), "cudaEventCreate");
    } else {
        h->stream = h->user_stream;
    }
    CK(cudaHostAlloc((void**)&h->ctl_host, sizeof(Ctl), cudaHostAllocDefault), "cudaHostAlloc");
    h->kpi = plain ? pmp::kPlainKernelsPerIter : pmp::kFusedKernelsPerIter;
    if (prm.profile) {
        h->evs.resize(1 + (size_t)prm.check_every * h->kpi, nullptr);
        for (auto& ev : h->evs) CK(cudaEventCreate(&ev), "cudaEventCreate");
    }
    CK(order_after_legacy(h), "ordering after the default stream");
    cudaStream_t st = h->stream;
    if (!on_device) {
        CK(cudaMemcpyAsync(d_rp, route_ptr, 8 * (N + 1), cudaMemcpyHostToDevice, st), "copy route_ptr");
        CK(cudaMemcpyAsync(d_rl, route_links, 4 * NNZ, cudaMemcpyHostToDevice, st), "copy route_links");
        CK(cudaMemcpyAsync(d_c, c, 8 * M, cudaMemcpyHostToDevice, st), "copy c");
        CK(cudaMemcpyAsync(d_w, w, 8 * N, cudaMemcpyHostToDevice, st), "copy w");
        if (lo) CK(cudaMemcpyAsync(d_lo, lo, 8 * N, cudaMemcpyHostToDevice, st), "copy lo");
        CK(cudaMemcpyAsync(d_hi, hi, 8 * N, cudaMemcpyHostToDevice, st), "copy hi");
        CK(cudaMemcpyAsync(d_ut, utype, N, cudaMemcpyHostToDevice, st), "copy utype");
        route_ptr = d_rp;
        route_links = d_rl;
        c = d_c;
        w = d_w;
        lo = d_lo;
        hi = d_hi;
        utype = d_ut;
    }
    CK(cudaMemsetAsync(d_err, 0, sizeof(int) * 2, st), "memset");
    CK(pmp::validate_inputs((int)n, (int)m, route_ptr, route_links, c, utype, w, lo, hi, d_err,
                            d_box, st),
       "validating the inputs");
    if (batch) {
        CK(cudaMemcpyAsync(d_soff, batch->stream_off, 8 * ((size_t)batch->count + 1),
                           cudaMemcpyHostToDevice, st), "copy offsets");
        CK(cudaMemcpyAsync(d_loff, batch->link_off, 8 * ((size_t)batch->count + 1),
                           cudaMemcpyHostToDevice, st), "copy offsets");
    }
    int err_bits = 0, flags[2] = {0, 0};
    unsigned long long box[4];
    CK(cudaMemcpyAsync(flags, d_err, sizeof(flags), cudaMemcpyDeviceToHost, st), "read flags");
    CK(cudaMemcpyAsync(box, d_box, sizeof(box), cudaMemcpyDeviceToHost, st), "read box");
    CK(cudaStreamSynchronize(st), "validation");
    err_bits = flags[0];
    if (!err_bits && batch) {
        CK(pmp::check_blocks(batch->count, d_soff, d_loff, n, route_ptr, route_links, d_err, st),
           "checking the instance blocks");
        CK(cudaMemcpyAsync(&err_bits, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "read flags");
        CK(cudaStreamSynchronize(st), "validation");
    }
    if (err_bits) {
        destroy_handle(h);
        return fail(NUM_ERR_INVALID, describe_bits(err_bits));
    }
    if (reorder) {
        CK(pmp::relabel_streams((int)n, (int)m, route_ptr, route_links, s, h->perm, d_lens,
                                d_ptr32, d_ptmp, d_rp2, d_rl2, st),
           "ordering the streams");
    }
    CK(pmp::build_operator((int)n, (int)m, (int)nnz, reorder ? d_rp2 : route_ptr,
                           reorder ? d_rl2 : route_links, h->col_ptr, h->row_idx, h->row_ptr,
                           h->col_idx, s, d_err, st),
       "building the operator");
    CK(cudaMemcpyAsync(&err_bits, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "read flags");
    CK(cudaStreamSynchronize(st), "operator build");
    if (err_bits) {
        destroy_handle(h);
        return fail(NUM_ERR_INVALID, describe_bits(err_bits));
    }
    const double lmin = pmp::ordered_key_to_double(box[0]), lmax = pmp::ordered_key_to_double(box[1]);
    const double hmin = pmp::ordered_key_to_double(box[2]), hmax = pmp::ordered_key_to_double(box[3]);
    h->box_uniform = (lmin == lmax && hmin == hmax) ? 1 : 0;
    if (flags[1]) {  // some stream has U = -w / x: keep the types on the device
        h->ut = (uint8_t*)dev_alloc(h, N);
        if (!h->ut) {
            destroy_handle(h);
            return fail(NUM_ERR_OOM, "device allocation failed");
        }
    }
    h->lo_u = lmin;
    h->hi_u = hmin;
    if (fp32)
        CK(pmp::convert_params<float>((int)n, (int)m, c, utype, w, lo, hi, h->perm,
                                      (float*)h->c, (float*)h->wt, (float*)h->lo, (float*)h->hi,
                                      st, h->ut),
           "converting parameters");
    else
        CK(pmp::convert_params<double>((int)n, (int)m, c, utype, w, lo, hi, h->perm,
                                       (double*)h->c, (double*)h->wt, (double*)h->lo,
                                       (double*)h->hi, st, h->ut),
           "converting parameters");
    if (tiles) {
        CK(pmp::build_tiles(h->col_ptr, (int)n, h->Js, h->tile_s, h->ntiles_s, h->tiles_s, st),
           "stream tiles");
        CK(pmp::build_tiles(h->row_ptr, (int)m, h->Jl, h->tile_l, h->ntiles_l, h->tiles_l, st),
           "link tiles");
        CK(pmp::fused_grids(fp32 ? 0 : 1, h->tile_s, h->tile_l, h->ntiles_s, h->ntiles_l,
                            &h->grid_s, &h->grid_l),
           "sizing the fused grids");
    }
    if (rowk) {
        CK(pmp::count_chunks(h->row_ptr, (int)m, d_ccount, d_coff, d_ctmp, &h->nchunks, st),
           "counting long-link chunks");
        const size_t nc = (size_t)(h->nchunks > 0 ? h->nchunks : 1);
        h->chunks = (int4*)dev_alloc(h, sizeof(int4) * nc);
        h->carry_l = dev_alloc(h, ts * nc);
        h->arrive_l = (int*)dev_alloc(h, sizeof(int) * nc);
        h->narrive_l = (int)nc;
        if (!h->chunks || !h->carry_l || !h->arrive_l) {
            destroy_handle(h);
            return fail(NUM_ERR_OOM, "device allocation failed");
        }
        if (h->nchunks > 0)
            CK(pmp::fill_chunks(h->row_ptr, (int)m, d_coff, h->chunks, st), "long-link chunks");
        CK(pmp::rows_grids(fp32 ? 0 : 1, (int)n, (int)m, h->nchunks, &h->grid_s, &h->grid_l),
           "sizing the row-kernel grids");
    }
    CK(zero_state(h), "zeroing the state");
    CK(cudaStreamSynchronize(st), "setup");
    // release the transient buffers
    for (void* q : {(void*)d_rp, (void*)d_rl, (void*)d_c, (void*)d_w, (void*)d_lo, (void*)d_hi,
                    (void*)d_ut, (void*)d_err, (void*)d_box, (void*)s.keys_a, (void*)s.vals_a,
                    (void*)s.keys_b, (void*)s.vals_b, (void*)s.hist, (void*)s.scan_tmp,
                    (void*)d_ccount, (void*)d_coff, (void*)d_ctmp, (void*)d_rp2, (void*)d_rl2,
                    (void*)d_lens, (void*)d_ptr32, (void*)d_ptmp, (void*)d_soff, (void*)d_loff})
        dev_free(h, q);
#undef CK
    *out = h;
    return NUM_OK;
}

int finish_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return cuda_fail(e, what);
    return NUM_OK;
}

}  // namespace

extern "C" {

void num_default_params(num_params* p) {
    if (!p) return;
    p->rho0 = 1.0;
    p->alpha = 1.6;
    p->mu = 2.0;
    p->gamma = 1.1;
    p->eps_abs = 1e-4;
    p->rho_period = 50;
    p->precision = NUM_FUSED_FP32;
    p->check_every = 50;
    p->tile_items = 0;
    p->history = 4096;
    p->use_graph = 1;
    p->schedule = 0;
    p->reorder = 1;
    p->profile = 0;
    p->allocator = nullptr;
}

int num_create(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
               const int32_t* route_links, const double* c, const uint8_t* utype,
               const double* w, const double* lo, const double* hi, const num_params* p,
               void* cuda_stream) {
    return create_impl(out, n, m, route_ptr, route_links, c, utype, w, lo, hi, p, cuda_stream,
                       false);
}

int num_create_device(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
                      const int32_t* route_links, const double* c, const uint8_t* utype,
                      const double* w, const double* lo, const double* hi,
                      const num_params* p, void* cuda_stream) {
    return create_impl(out, n, m, route_ptr, route_links, c, utype, w, lo, hi, p, cuda_stream,
                       true);
}

int num_set_rho_schedule(num_problem* h, const int8_t* decisions, int64_t count) {
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    if (count < 0 || count > INT32_MAX || (count > 0 && !decisions))
        return fail(NUM_ERR_INVALID, "bad schedule");
    for (int64_t i = 0; i < count; ++i)
        if (decisions[i] < -1 || decisions[i] > 1)
            return fail(NUM_ERR_INVALID, "schedule entries must be -1, 0 or +1");
    cudaError_t e = order_after_legacy(h);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    if (h->sched) {
        cudaStreamSynchronize(h->stream);
        dev_free(h, h->sched);
        h->sched = nullptr;
    }
    h->sched_len = 0;
    if (count > 0) {
        h->sched = (signed char*)dev_alloc(h, (size_t)count);
        if (!h->sched) return fail(NUM_ERR_OOM, "device allocation failed");
        e = cudaMemcpyAsync(h->sched, decisions, (size_t)count, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy schedule");
        h->sched_len = (int)count;
    }
    // graphs captured the old schedule pointer
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    if (h->graph) {
        cudaGraphDestroy(h->graph);
        h->graph = nullptr;
    }
    e = pmp::ctl_set_schedule_len(h->ctl, h->sched_len, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "schedule");
    return finish_cuda(cudaStreamSynchronize(h->stream), "schedule");
}

int num_solve(num_problem* h, int64_t max_iters, double eps_abs, int64_t* iters_done) {
    g_last_error.clear();
    if (iters_done) *iters_done = 0;
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    if (max_iters < 0) return fail(NUM_ERR_INVALID, "max_iters must be >= 0");
    if (std::isnan(eps_abs)) return fail(NUM_ERR_INVALID, "eps_abs is NaN");
    cudaStream_t st = h->stream;
    cudaError_t e = order_after_legacy(h);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the control block");
    const long long k0 = h->ctl_host->k;
    if (max_iters == 0) return NUM_NOT_CONVERGED;
    const double eps = eps_abs > 0.0 ? eps_abs : (eps_abs < 0.0 ? h->prm.eps_abs : 0.0);
    const double eps_tol = eps > 0.0 ? eps * std::sqrt((double)(h->nnz + h->m)) : 0.0;
    h->last_eps_tol = eps_tol;
    e = pmp::ctl_arm(h->ctl, k0 + max_iters, eps_tol, st);
    if (e != cudaSuccess) return cuda_fail(e, "arming the control block");
    const int K = h->prm.check_every;
    if (h->prm.use_graph && !h->graph_exec) {
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t e2 = run_iterations(h, K);
        e = cudaStreamEndCapture(st, &h->graph);
        if (e2 != cudaSuccess) return cuda_fail(e2, "capturing the iteration graph");
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&h->graph_exec, h->graph, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
    const long long max_launches = (max_iters + K - 1) / K + 1;
    for (long long it = 0;; ++it) {
        if (it >= max_launches) return fail(NUM_ERR_STATE, "the iteration limit was not honoured");
        const long long k_before = h->ctl_host->k;
        if (h->prm.use_graph)
            e = cudaGraphLaunch(h->graph_exec, st);
        else
            e = run_iterations(h, K);
        if (e != cudaSuccess) return cuda_fail(e, "launching iterations");
        pmp::note_launches((long long)K * h->kpi);
        e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "iterations");
        if (h->prm.profile) {
            e = accumulate_kernel_times(h, h->ctl_host->k - k_before);
            if (e != cudaSuccess) return cuda_fail(e, "reading kernel times");
        }
        if (h->ctl_host->stop != pmp::RUNNING) break;
    }
    if (iters_done) *iters_done = h->ctl_host->k - k0;
    switch (h->ctl_host->stop) {
        case pmp::CONVERGED: return NUM_OK;
        case pmp::LIMIT: return NUM_NOT_CONVERGED;
        default: return fail(NUM_ERR_NUMERIC, "a residual became non-finite");
    }
}

static int get_impl(const num_problem* hc, double* x, double* prices, double* info, bool dev) {
    g_last_error.clear();
    if (!hc) return fail(NUM_ERR_INVALID, "handle is NULL");
    num_problem* h = const_cast<num_problem*>(hc);
    cudaStream_t st = h->stream;
    cudaError_t e = order_after_legacy(h);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    double* xo = dev ? x : (x ? h->x64 : nullptr);
    double* yo = dev ? prices : (prices ? h->y64 : nullptr);
    if (h->prec == NUM_FUSED_FP32)
        e = pmp::export_solution<float>(make_view<float>(h), xo, yo, h->part_exp, h->exp_blocks, st);
    else
        e = pmp::export_solution<double>(make_view<double>(h), xo, yo, h->part_exp,
                                         h->exp_blocks, st);
    if (e != cudaSuccess) return cuda_fail(e, "exporting the solution");
    if (!dev) {
        if (x) e = cudaMemcpyAsync(x, h->x64, 8 * (size_t)h->n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && prices)
            e = cudaMemcpyAsync(prices, h->y64, 8 * (size_t)h->m, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "copying the solution");
    }
    e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the results");
    if (info) {
        const Ctl& c = *h->ctl_host;
        info[NUM_INFO_PRIMAL] = c.rnorm;
        info[NUM_INFO_DUAL] = c.snorm;
        info[NUM_INFO_EPS_TOL] = h->last_eps_tol;
        info[NUM_INFO_RHO] = c.rho;
        info[NUM_INFO_OBJECTIVE] = c.objective;
        info[NUM_INFO_ITERS] = (double)c.k;
        info[NUM_INFO_STATUS] = (double)c.stop;
        info[NUM_INFO_J] = (double)(h->nnz + h->m);
    }
    return NUM_OK;
}

int num_get(const num_problem* h, double* x, double* prices, double* info) {
    return get_impl(h, x, prices, info, false);
}

int num_get_device(const num_problem* h, double* x, double* prices, double* info) {
    return get_impl(h, x, prices, info, true);
}

int num_get_history(const num_problem* hc, double* hist, int64_t max_rows, int64_t* rows) {
    g_last_error.clear();
    if (rows) *rows = 0;
    if (!hc) return fail(NUM_ERR_INVALID, "handle is NULL");
    if (max_rows < 0 || (max_rows > 0 && !hist)) return fail(NUM_ERR_INVALID, "bad buffer");
    num_problem* h = const_cast<num_problem*>(hc);
    const int H = h->prm.history;
    std::vector<double> ring((size_t)3 * (H > 0 ? H : 1));
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && H > 0)
        e = cudaMemcpyAsync(ring.data(), h->hist, sizeof(double) * 3 * (size_t)H,
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the history");
    const long long k = h->ctl_host->k;
    long long have = H > 0 ? (k < H ? k : H) : 0;
    if (have > max_rows) have = max_rows;
    for (long long i = 0; i < have; ++i) {
        const long long it = k - have + i;  // 0-based iteration index
        const double* src = ring.data() + 3 * (it % H);
        hist[3 * i] = src[0];
        hist[3 * i + 1] = src[1];
        hist[3 * i + 2] = src[2];
    }
    if (rows) *rows = have;
    return NUM_OK;
}

int num_get_operator(const num_problem* hc, int64_t* row_ptr, int32_t* col_idx) {
    g_last_error.clear();
    if (!hc || !row_ptr || !col_idx) return fail(NUM_ERR_INVALID, "NULL argument");
    num_problem* h = const_cast<num_problem*>(hc);
    std::vector<int> rp((size_t)h->m + 1);
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rp.data(), h->row_ptr, 4 * rp.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(col_idx, h->col_idx, 4 * (size_t)h->nnz, cudaMemcpyDeviceToHost,
                            h->stream);
    std::vector<int> perm(h->perm ? (size_t)h->n : 0);
    if (e == cudaSuccess && h->perm)
        e = cudaMemcpyAsync(perm.data(), h->perm, 4 * perm.size(), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the operator");
    for (size_t i = 0; i < rp.size(); ++i) row_ptr[i] = rp[i];
    if (h->perm) {  // the device works on relabeled streams: report the caller's ids
        for (int64_t q = 0; q < h->nnz; ++q) col_idx[q] = perm[col_idx[q]];
        for (int64_t l = 0; l < h->m; ++l) std::sort(col_idx + rp[l], col_idx + rp[l + 1]);
    }
    return NUM_OK;
}

int num_reset(num_problem* h) {
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess) e = zero_state(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return finish_cuda(e, "reset");
}

int num_set_capacity(num_problem* h, const double* c) {
    g_last_error.clear();
    if (!h || !c) return fail(NUM_ERR_INVALID, "NULL argument");
    for (int64_t l = 0; l < h->m; ++l)
        if (!(c[l] > 0.0) || !std::isfinite(c[l]))
            return fail(NUM_ERR_INVALID, "a capacity is not finite and > 0");
    cudaStream_t st = h->stream;
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->y64, c, 8 * (size_t)h->m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = h->prec == NUM_FUSED_FP32
                ? pmp::convert_params<float>(0, (int)h->m, h->y64, nullptr, nullptr, nullptr,
                                             nullptr, nullptr, (float*)h->c, nullptr, nullptr,
                                             nullptr, st)
                : pmp::convert_params<double>(0, (int)h->m, h->y64, nullptr, nullptr, nullptr,
                                              nullptr, nullptr, (double*)h->c, nullptr, nullptr,
                                              nullptr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return finish_cuda(e, "setting the capacities");
}

static int state_io(num_problem* h, double** arrays, double* rho, bool out) {
    cudaStream_t st = h->stream;
    cudaError_t e = order_after_legacy(h);
    if (e != cudaSuccess) return cuda_fail(e, "ordering");
    if (!out) {
        // a fresh run from the given iterate: iteration 0, the given rho, no history
        e = pmp::ctl_reset(h->ctl, *rho, h->prm.alpha, h->prm.mu, h->prm.gamma,
                           h->prm.rho_period, h->prm.history, st);
        if (e == cudaSuccess && h->sched_len > 0)
            e = pmp::ctl_set_schedule_len(h->ctl, h->sched_len, st);
        if (e != cudaSuccess) return cuda_fail(e, "resetting the control block");
    }
    for (int which = 0; which < 7; ++which) {
        double* host = arrays[which];
        if (!host) continue;
        double* buf = which < 2 ? h->x64 : h->y64;
        const size_t bytes = 8 * (size_t)(which < 2 ? h->n : h->m);
        if (!out) e = cudaMemcpyAsync(buf, host, bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = h->prec == NUM_FUSED_FP32
                    ? pmp::state_transfer<float>(make_view<float>(h), which, buf, out, st)
                    : pmp::state_transfer<double>(make_view<double>(h), which, buf, out, st);
        if (e == cudaSuccess && out) e = cudaMemcpyAsync(host, buf, bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the staging buffer is reused
        if (e != cudaSuccess) return cuda_fail(e, "transferring the state");
    }
    if (out) {
        e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading the control block");
        *rho = h->ctl_host->rho;
    }
    return NUM_OK;
}

int num_get_state(const num_problem* hc, double* x, double* Z, double* pbar, double* y,
                  double* zs, double* Rx, double* ps, double* rho) {
    g_last_error.clear();
    if (!hc || !rho) return fail(NUM_ERR_INVALID, "NULL argument");
    double* arrays[7] = {x, Z, pbar, y, zs, Rx, ps};
    return state_io(const_cast<num_problem*>(hc), arrays, rho, true);
}

int num_set_state(num_problem* h, const double* x, const double* Z, const double* pbar,
                  const double* y, const double* zs, const double* Rx, const double* ps,
                  double rho) {
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "NULL argument");
    if (!(rho > 0.0) || !std::isfinite(rho)) return fail(NUM_ERR_INVALID, "rho must be > 0");
    double* arrays[7] = {const_cast<double*>(x), const_cast<double*>(Z), const_cast<double*>(pbar),
                         const_cast<double*>(y), const_cast<double*>(zs), const_cast<double*>(Rx),
                         const_cast<double*>(ps)};
    return state_io(h, arrays, &rho, false);
}

int num_set_weights(num_problem* h, const double* w) {
    g_last_error.clear();
    if (!h || !w) return fail(NUM_ERR_INVALID, "NULL argument");
    for (int64_t j = 0; j < h->n; ++j)
        if (!(w[j] > 0.0) || !std::isfinite(w[j]))
            return fail(NUM_ERR_INVALID, "a weight is not finite and > 0");
    cudaStream_t st = h->stream;
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->x64, w, 8 * (size_t)h->n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = h->prec == NUM_FUSED_FP32 ? pmp::set_weights<float>(make_view<float>(h), h->x64, st)
                                      : pmp::set_weights<double>(make_view<double>(h), h->x64, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return finish_cuda(e, "setting the weights");
}

}  // extern "C"

namespace {

// Device pointers of the iterate's arrays, in a fixed order, with their byte sizes.
void state_arrays(num_problem* h, std::vector<std::pair<void*, size_t>>& out) {
    const size_t ts = h->prec == NUM_FUSED_FP32 ? 4 : 8;
    const size_t N = (size_t)h->n, M = (size_t)h->m;
    out.clear();
    out.emplace_back(h->x, ts * N);
    out.emplace_back(h->Z, ts * N);
    if (h->pby) out.emplace_back(h->pby, 2 * ts * M);
    if (h->pbar) out.emplace_back(h->pbar, ts * M);
    if (h->y) out.emplace_back(h->y, ts * M);
    out.emplace_back(h->zs, ts * M);
    out.emplace_back(h->Rx, ts * M);
    out.emplace_back(h->ps, ts * M);
    out.emplace_back(h->ctl, sizeof(Ctl));
}

size_t state_bytes(num_problem* h) {
    std::vector<std::pair<void*, size_t>> a;
    state_arrays(h, a);
    size_t b = 0;
    for (auto& q : a) b += (q.second + 255) / 256 * 256;
    return b;
}

cudaError_t copy_state(num_problem* h, char* slot, bool save) {
    std::vector<std::pair<void*, size_t>> a;
    state_arrays(h, a);
    size_t off = 0;
    for (auto& q : a) {
        cudaError_t e = save ? cudaMemcpyAsync(slot + off, q.first, q.second,
                                               cudaMemcpyDeviceToDevice, h->stream)
                             : cudaMemcpyAsync(q.first, slot + off, q.second,
                                               cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return e;
        off += (q.second + 255) / 256 * 256;
    }
    return cudaSuccess;
}

template <typename T>
int adjoint_impl(num_problem* h, int64_t K, int64_t Kc, const double* xbar, int objective,
                 double* c_grad, double* w_grad, double* objective_out) {
    using T2 = typename pmp::Pair<T>::type;
    cudaStream_t st = h->stream;
    const size_t N = (size_t)h->n, M = (size_t)h->m;
    const int64_t nseg = (K + Kc - 1) / Kc;
    const size_t sb = state_bytes(h);
    std::vector<void*> owned;
    bool ok = true;
    auto A = [&](size_t bytes) -> void* {
        void* q = ok ? dev_alloc(h, bytes) : nullptr;
        if (!q) ok = false;
        else owned.push_back(q);
        return q;
    };
    pmp::AdjView<T> a;
    std::memset(&a, 0, sizeof(a));
    a.alpha = h->prm.alpha;
    a.xb = (T*)A(sizeof(T) * N);
    a.Zb = (T*)A(sizeof(T) * N);
    a.ab = (T2*)A(sizeof(T2) * N);
    a.wb = (T*)A(sizeof(T) * N);
    a.yb = (T*)A(sizeof(T) * M);
    a.zsb = (T*)A(sizeof(T) * M);
    a.Rxb = (T*)A(sizeof(T) * M);
    a.cb = (T*)A(sizeof(T) * M);
    if (h->chunks && h->nchunks > 0) a.abc = (T2*)A(sizeof(T2) * (size_t)h->nchunks);
    T* tape_x = (T*)A(sizeof(T) * N * (size_t)Kc);
    T* tape_ps = (T*)A(sizeof(T) * M * (size_t)Kc);
    double* tape_rho = (double*)A(sizeof(double) * (size_t)Kc);
    char* ckpt = (char*)A(sb * (size_t)(nseg + 1));
    double* xbar_dev = xbar ? (double*)A(8 * N) : nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (void* q : owned) dev_free(h, q);
    };
    if (!ok) {
        release();
        return fail(NUM_ERR_OOM, "device allocation failed (tape and checkpoints)");
    }
    cudaError_t e = cudaSuccess;
#define AK(call, what)                 \
    do {                               \
        e = (call);                    \
        if (e != cudaSuccess) {        \
            release();                 \
            return cuda_fail(e, what); \
        }                              \
    } while (0)
    AK(order_after_legacy(h), "ordering");
    if (xbar) AK(cudaMemcpyAsync(xbar_dev, xbar, 8 * N, cudaMemcpyHostToDevice, st), "copy xbar");
    // run `cnt` iterations one at a time, keeping rho, x and the slack flow of each
    auto tape_segment = [&](int64_t cnt) -> cudaError_t {
        for (int64_t i = 0; i < cnt; ++i) {
            cudaError_t r = pmp::record_rho(h->ctl, tape_rho + i, st);
            if (r == cudaSuccess) r = run_iterations(h, 1);
            pmp::note_launches(h->kpi);
            if (r == cudaSuccess)
                r = cudaMemcpyAsync(tape_x + N * (size_t)i, h->x, sizeof(T) * N,
                                    cudaMemcpyDeviceToDevice, st);
            if (r == cudaSuccess)
                r = cudaMemcpyAsync(tape_ps + M * (size_t)i, h->ps, sizeof(T) * M,
                                    cudaMemcpyDeviceToDevice, st);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    // forward K iterations from the zero state, keeping the state at every segment start;
    // the last segment is taped on the way, so the backward sweep starts without a recompute
    AK(zero_state(h), "zeroing the state");
    for (int64_t s = 0; s < nseg; ++s) {
        const int64_t cnt = std::min<int64_t>(Kc, K - s * Kc);
        AK(copy_state(h, ckpt + sb * (size_t)s, true), "checkpoint");
        AK(pmp::ctl_arm(h->ctl, s * Kc + cnt, 0.0, st), "arming");
        if (s < nseg - 1) {
            AK(run_iterations(h, (int)cnt), "forward iterations");
            pmp::note_launches(cnt * h->kpi);
        } else {
            AK(tape_segment(cnt), "forward iterations of the last segment");
        }
    }
    if (objective_out) {
        AK(h->prec == NUM_FUSED_FP32
               ? pmp::export_solution<float>(make_view<float>(h), nullptr, nullptr, h->part_exp,
                                             h->exp_blocks, st)
               : pmp::export_solution<double>(make_view<double>(h), nullptr, nullptr,
                                              h->part_exp, h->exp_blocks, st),
           "objective");
    }
    // the forward result (with its objective) is restored at the end
    AK(copy_state(h, ckpt + sb * (size_t)nseg, true), "final state");
    a.v = make_view<T>(h);
    AK(pmp::adjoint_init<T>(a, xbar_dev, objective, st), "adjoint init");
    // backward, one segment at a time: recompute its iterates (deterministic; the last
    // segment's are taped already), then sweep
    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int64_t cnt = std::min<int64_t>(Kc, K - s * Kc);
        if (s < nseg - 1) {
            AK(copy_state(h, ckpt + sb * (size_t)s, false), "restore checkpoint");
            AK(pmp::ctl_arm(h->ctl, s * Kc + cnt, 0.0, st), "arming");
            AK(tape_segment(cnt), "recomputing a segment");
        }
        for (int64_t i = cnt - 1; i >= 0; --i)
            AK(pmp::adjoint_step<T>(a, tape_x + N * (size_t)i, tape_ps + M * (size_t)i,
                                    tape_rho + i, st),
               "adjoint iteration");
    }
    // dJ/dw (n values, caller order) through the n-sized staging buffer, dJ/dc (m values)
    // through the m-sized one
    if (w_grad) {
        AK(pmp::adjoint_export<T>(a, /*c_grad=*/nullptr, /*w_grad=*/h->x64, st), "export dJ/dw");
        AK(cudaMemcpyAsync(w_grad, h->x64, 8 * N, cudaMemcpyDeviceToHost, st), "dJ/dw");
    }
    if (c_grad) {
        AK(pmp::adjoint_export<T>(a, /*c_grad=*/h->y64, /*w_grad=*/nullptr, st), "export dJ/dc");
        AK(cudaMemcpyAsync(c_grad, h->y64, 8 * M, cudaMemcpyDeviceToHost, st), "dJ/dc");
    }
    // leave the handle at the forward result
    AK(copy_state(h, ckpt + sb * (size_t)nseg, false), "restore the final state");
    AK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st), "ctl");
    AK(cudaStreamSynchronize(st), "adjoint");
#undef AK
    if (objective_out) *objective_out = h->ctl_host->objective;
    release();
    return NUM_OK;
}

}  // namespace

extern "C" {

int num_adjoint(num_problem* h, int64_t iters, int32_t checkpoint_every, const double* xbar,
                int32_t objective, double* c_grad, double* w_grad, double* objective_out) {
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    if (iters < 1) return fail(NUM_ERR_INVALID, "iters must be >= 1");
    if (objective != 0 && objective != 1) return fail(NUM_ERR_INVALID, "objective must be 0 or 1");
    if (!xbar && !objective) return fail(NUM_ERR_INVALID, "nothing to differentiate");
    if (checkpoint_every < 0) return fail(NUM_ERR_INVALID, "checkpoint_every must be >= 0");
    const int64_t Kc = checkpoint_every == 0 ? iters : std::min<int64_t>(checkpoint_every, iters);
    return h->prec == NUM_FUSED_FP32
               ? adjoint_impl<float>(h, iters, Kc, xbar, objective, c_grad, w_grad, objective_out)
               : adjoint_impl<double>(h, iters, Kc, xbar, objective, c_grad, w_grad,
                                      objective_out);
}

int num_iteration_bytes(const num_problem* h, double* out) {
    g_last_error.clear();
    if (!h || !out) return fail(NUM_ERR_INVALID, "NULL argument");
    const double ts = h->prec == NUM_FUSED_FP32 ? 4.0 : 8.0;
    const double n = (double)h->n, m = (double)h->m, nnz = (double)h->nnz;
    const double box = h->box_uniform ? 0.0 : 2.0 * ts * n;
    // stream kernel: col_ptr, route entries, x and Z read + written, weights, box,
    // the (pbar, y) vector gathered once
    out[0] = 4.0 * (n + 1) + 4.0 * nnz + ts * (4.0 * n + n) + box + 2.0 * ts * m;
    // link kernel: row_ptr, link entries, x gathered once, link state read
    // (pbar, y, zs, Rx, ps, c) and written (pbar, y, zs, Rx, ps)
    out[1] = 4.0 * (m + 1) + 4.0 * nnz + ts * n + ts * 11.0 * m;
    return NUM_OK;
}

int num_get_kernel_times(const num_problem* h, double* ms, int64_t* launches,
                         int32_t max_kernels, int32_t* nkernels) {
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    if (max_kernels < 0 || (max_kernels > 0 && (!ms || !launches)))
        return fail(NUM_ERR_INVALID, "bad buffers");
    if (nkernels) *nkernels = h->kpi;
    for (int q = 0; q < h->kpi && q < max_kernels; ++q) {
        ms[q] = h->kernel_ms[q];
        launches[q] = h->kernel_runs[q];
    }
    return NUM_OK;
}

int64_t num_kernel_launches(void) { return pmp::launches(); }

void num_destroy(num_problem* h) { destroy_handle(h); }

const char* num_strerror(int code) {
    switch (code) {
        case NUM_OK: return "ok";
        case NUM_NOT_CONVERGED: return "iteration limit reached before the stopping test passed";
        case NUM_ERR_INVALID: return "invalid argument or instance";
        case NUM_ERR_OOM: return "device allocation failed";
        case NUM_ERR_CUDA: return "CUDA runtime error";
        case NUM_ERR_NUMERIC: return "non-finite residual";
        case NUM_ERR_STATE: return "call not valid in this state";
        default: return "unknown status code";
    }
}

const char* num_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---- batches of independent instances ----------------------------------------------------------

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
};

namespace {

// Work partition of a batch: defaults, limits and the autotuner's candidates.
constexpr num_batch_schedule kBatchDefault = {2048, 256, 8};
constexpr int kStreamItemMin = 256, kStreamItemMax = 65536;
constexpr int kLinkItemMin = 32, kLinkItemMax = 8192;
constexpr int kTuneStreamItems[] = {512, 1024, 2048, 4096, 8192};
constexpr int kTuneLinkItems[] = {64, 128, 256, 512, 1024};
constexpr int kTuneLanes[] = {4, 8, 16, 32};

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

bool valid_schedule(const num_batch_schedule& c) {
    return pow2_in(c.stream_item, kStreamItemMin, kStreamItemMax) &&
           pow2_in(c.link_item, kLinkItemMin, kLinkItemMax) &&
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
        cudaEvent_t* ev = prof ? h->evs.data() + 1 + (size_t)i * 2 : nullptr;
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

// Build the work items of schedule `cfg` (instance, first row, end row) and size the grids;
// a captured graph of the old partition is dropped.  Streams keep their instance's range
// after the first-link ordering because an instance's links are a contiguous id range.
int batch_apply_schedule(num_batch* b, const num_batch_schedule& cfg) {
    num_problem* h = b->p;
    cudaStream_t st = h->stream;
    std::vector<int4> si, li;
    std::vector<int> so(b->count + 1), lo_(b->count + 1);
    for (int i = 0; i < b->count; ++i) {
        so[i] = (int)si.size();
        for (int64_t r = b->soff[i]; r < b->soff[i + 1]; r += cfg.stream_item)
            si.push_back(make_int4(i, (int)r, (int)std::min<int64_t>(r + cfg.stream_item,
                                                                     b->soff[i + 1]), 0));
        lo_[i] = (int)li.size();
        for (int64_t r = b->loff[i]; r < b->loff[i + 1]; r += cfg.link_item)
            li.push_back(make_int4(i, (int)r, (int)std::min<int64_t>(r + cfg.link_item,
                                                                     b->loff[i + 1]), 0));
    }
    so[b->count] = (int)si.size();
    lo_[b->count] = (int)li.size();
    if ((int)si.size() > b->cap_sitems || (int)li.size() > b->cap_litems)
        return fail(NUM_ERR_STATE, "work items exceed their capacity");
    cudaError_t e = cudaStreamSynchronize(st);  // no kernel may still read the old items
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
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
    if (e != cudaSuccess) return cuda_fail(e, "copying the work items");
    b->nsitems = (int)si.size();
    b->nlitems = (int)li.size();
    e = pmp::batch_grids(h->prec == NUM_FUSED_FP32 ? 0 : 1, cfg.link_lanes, b->nsitems,
                         b->nlitems, h->nchunks, &b->grid_s, &b->grid_l, &b->grid_e);
    if (e != cudaSuccess) return cuda_fail(e, "sizing the batch grids");
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

}  // namespace

extern "C" {

int num_batch_create(num_batch** out, int32_t count, const int64_t* stream_off,
                     const int64_t* link_off, const int64_t* route_ptr,
                     const int32_t* route_links, const double* c, const uint8_t* utype,
                     const double* w, const double* lo, const double* hi, const num_params* p,
                     void* cuda_stream) {
    g_last_error.clear();
    if (!out) return fail(NUM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (count < 1 || !stream_off || !link_off || !route_ptr)
        return fail(NUM_ERR_INVALID, "count must be >= 1 and the offsets non-NULL");
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
    if (prm.precision == NUM_PLAIN_FP64 || prm.schedule == NUM_SCHEDULE_TILES)
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
                         cuda_stream, false, &spec);
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
        const int64_t nnz_i = route_ptr[stream_off[i + 1]] - route_ptr[stream_off[i]];
        b->J.push_back((double)(nnz_i + link_off[i + 1] - link_off[i]));
        scale[i] = std::sqrt(b->J.back());
    }
    if (cap_s > INT32_MAX / 4 || cap_l > INT32_MAX / 4) {
        batch_destroy(b);
        return fail(NUM_ERR_INVALID, "too many work items");
    }
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
    if (!b->ctls || !b->glob || !b->sitems || !b->litems || !b->sitem_off || !b->litem_off ||
        !b->part_s || !b->part_l || !b->part_e || !b->hist || !b->eps_scale || !b->arrive) {
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
    rc = batch_chunk_tables(b);
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
    g_last_error.clear();
    if (!b) return fail(NUM_ERR_INVALID, "batch is NULL");
    if (max_iters < 0) return fail(NUM_ERR_INVALID, "max_iters must be >= 0");
    if (std::isnan(eps_abs)) return fail(NUM_ERR_INVALID, "eps_abs is NaN");
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
    if (max_iters > 0) {
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
                for (long long i = 0; i < ran; ++i)
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
    if (rc == NUM_ERR_NUMERIC) return fail(rc, "a residual of some instance became non-finite");
    return rc;
}

int num_batch_get(const num_batch* bc, double* x, double* prices, double* info) {
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

void num_batch_destroy(num_batch* b) { batch_destroy(b); }

}  // extern "C"
