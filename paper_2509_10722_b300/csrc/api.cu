// C ABI of the PMP solver (declared in include/num_pmp.h), single instances: handle
// lifetime, device memory, input validation, the CUDA-graph iteration loop, result export,
// state import and export.  The adjoint is in adjoint_api.cu, batches in batch_api.cu;
// what they share with this file is declared in handle.cuh.
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

#include "handle.cuh"
#include "num_pmp.h"
#include "pmp_internal.cuh"

using pmp::Ctl;
using pmp::View;

namespace pmp {
namespace host {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(NUM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                                  cudaGetErrorString(e) + ")");
}

std::atomic<long long> g_launches{0};

}  // namespace host
}  // namespace pmp

using namespace pmp::host;

namespace pmp {
void note_launches(long long count) { g_launches.fetch_add(count, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }
int report_error(int code, const std::string& msg) { return fail(code, msg); }
int report_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }
void clear_error() { g_last_error.clear(); }
}  // namespace pmp

namespace pmp {
namespace host {

// Device memory of the handle.  The kernels read pairs of values (and the chunk table) as
// 16-byte loads, so every block must start on a 16-byte boundary: cudaMalloc's always do;
// a block from the caller's allocator that does not is asked 16 bytes larger and used from
// its first 16-byte boundary.
void* dev_alloc(num_problem* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (h->custom_alloc) {
        p = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->user_stream);
        if (p && ((uintptr_t)p & 15u) != 0) {
            h->alloc.release(h->alloc.ctx, p, bytes, (void*)h->user_stream);
            bytes += 16;
            void* raw = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->user_stream);
            if (!raw) return nullptr;
            void* q = (void*)(((uintptr_t)raw + 15u) & ~(uintptr_t)15u);
            h->blocks.push_back({q, raw, bytes});
            return q;
        }
    } else {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (p) h->blocks.push_back({p, p, bytes});
    return p;
}

void dev_free(num_problem* h, void* p) {
    if (!p) return;
    for (size_t i = 0; i < h->blocks.size(); ++i) {
        if (h->blocks[i].ptr == p) {
            const auto b = h->blocks[i];
            if (h->custom_alloc)
                h->alloc.release(h->alloc.ctx, b.raw, b.bytes, (void*)h->stream);
            else
                cudaFree(b.raw);
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
    adjoint_tape_free(h);
    while (!h->blocks.empty()) dev_free(h, h->blocks.back().ptr);
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


// Enqueue `count` iterations (count <= check_every when profiling).  Not counted as
// launches here: the caller counts what actually executes.
cudaError_t run_iterations(num_problem* h, int count) {
    const bool prof = h->prm.profile != 0;
    if (prof) {
        cudaError_t e = pmp::record_kernel_event(h->evs[0], h->stream);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < count; ++i) {
        cudaEvent_t* ev =
            prof && i < profiled_iterations(h) ? h->evs.data() + 1 + (size_t)i * h->kpi : nullptr;
        cudaError_t e;
        if (h->prec == NUM_FUSED_FP32)
            e = pmp::rows_iteration<float>(make_view<float>(h), h->stream, ev);
        else if (h->prec == NUM_FUSED_FP64)
            e = pmp::rows_iteration<double>(make_view<double>(h), h->stream, ev);
        else
            e = pmp::plain_iteration(make_view<double>(h), h->plain_nb, h->stream, ev);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// After a batch of iterations completed (stream synchronized): add the per-kernel times of
// the profiled ones among the first `ran` iterations of the batch (the later ones exited
// at the stop flag).
cudaError_t accumulate_kernel_times(num_problem* h, long long ran) {
    const long long timed = std::min(ran, (long long)profiled_iterations(h));
    for (long long i = 0; i < timed; ++i) {
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
    z(h->dbg, sizeof(unsigned int));
    z(h->x, ts * h->n);
    z(h->Z, ts * h->n);
    z(h->pby, 2 * ts * h->m);
    z(h->zs, ts * h->m);
    z(h->Rx, ts * h->m);
    z(h->ps, ts * h->m);
    z(h->pbar, ts * h->m);
    z(h->y, ts * h->m);
    z(h->arrive_l, sizeof(int) * (size_t)h->narrive_l);
    if (h->hist && h->prm.history > 0) z(h->hist, sizeof(double) * 3 * (size_t)h->prm.history);
    if (e != cudaSuccess) return e;
    e = pmp::ctl_reset(h->ctl, h->prm.rho0, h->prm.alpha, h->prm.mu, h->prm.gamma,
                       h->prm.rho_period, h->prm.history, st);
    if (e != cudaSuccess) return e;
    if (h->sched_len > 0) e = pmp::ctl_set_schedule_len(h->ctl, h->sched_len, st);
    return e;
}


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
    if (p.history < 0) return fail(NUM_ERR_INVALID, "history must be >= 0");
    if (p.profile < 0 || p.profile > 2) return fail(NUM_ERR_INVALID, "profile must be 0, 1 or 2");
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


int create_impl(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
                const int32_t* route_links, const double* c, const uint8_t* utype,
                const double* w, const double* lo, const double* hi, const num_params* p,
                void* cuda_stream, bool on_device, const BatchSpec* batch) {
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
        // on the caller's stream, so that work it queued there (which may be what fills
        // route_ptr) comes first; NULL is the legacy default stream
        cudaStream_t us = (cudaStream_t)cuda_stream;
        cudaError_t e = cudaMemcpyAsync(&p0, route_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, us);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&nnz, route_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, us);
        if (e == cudaSuccess) e = cudaStreamSynchronize(us);
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
    h->plain_nb = pmp::plain_partial_blocks((int)n, (int)m);
    const bool rowk = !plain;
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
    const size_t npart = (size_t)(kMaxGrid > h->plain_nb ? kMaxGrid : h->plain_nb);
    h->part_s = (double*)A(sizeof(double) * npart);
    h->part_l = (double*)A(sizeof(double) * 2 * npart);
    h->ctl = (Ctl*)A(sizeof(Ctl));
    h->dbg = (unsigned int*)A(sizeof(unsigned int));
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
    const size_t NM = (N > M ? N : M) + 1;  // the chunk and long-route tables share these
    int* d_ccount = rowk ? (int*)A(4 * NM) : nullptr;
    int* d_coff = rowk ? (int*)A(4 * NM) : nullptr;
    int* d_ctmp = rowk ? (int*)A(4 * pmp::scan_tmp_len(NM)) : nullptr;
    if (!ok) {
        destroy_handle(h);
        return fail(NUM_ERR_OOM, "device allocation failed");
    }

    // ---- from here on: CUDA work ----
    cudaError_t e;
    // Host inputs are copied on a second stream, `cs`: the routes first, then the other
    // arrays, which arrive while the routes are validated and the operator is built.  Any
    // early return waits for those copies before the memory they target is released.
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_start = nullptr, ev_routes = nullptr, ev_values = nullptr;
    auto end_copies = [&]() {
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        for (cudaEvent_t ev : {ev_start, ev_routes, ev_values})
            if (ev) cudaEventDestroy(ev);
        cs = nullptr;
        ev_start = ev_routes = ev_values = nullptr;
    };
    auto drop = [&]() {
        end_copies();
        destroy_handle(h);
    };
#define CK(call, what)                          \
    do {                                        \
        e = (call);                             \
        if (e != cudaSuccess) {                 \
            drop();                             \
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
        h->evs.resize(1 + (size_t)profiled_iterations(h) * h->kpi, nullptr);
        for (auto& ev : h->evs) CK(cudaEventCreate(&ev), "cudaEventCreate");
    }
    CK(order_after_legacy(h), "ordering after the default stream");
    cudaStream_t st = h->stream;
    if (!on_device) {
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
        for (cudaEvent_t* ev : {&ev_start, &ev_routes, &ev_values})
            CK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming), "cudaEventCreate");
        CK(cudaEventRecord(ev_start, st), "cudaEventRecord");
        CK(cudaStreamWaitEvent(cs, ev_start, 0), "cudaStreamWaitEvent");
        CK(cudaMemcpyAsync(d_rp, route_ptr, 8 * (N + 1), cudaMemcpyHostToDevice, cs), "copy route_ptr");
        CK(cudaMemcpyAsync(d_rl, route_links, 4 * NNZ, cudaMemcpyHostToDevice, cs), "copy route_links");
        CK(cudaEventRecord(ev_routes, cs), "cudaEventRecord");
        CK(cudaMemcpyAsync(d_c, c, 8 * M, cudaMemcpyHostToDevice, cs), "copy c");
        CK(cudaMemcpyAsync(d_w, w, 8 * N, cudaMemcpyHostToDevice, cs), "copy w");
        if (lo) CK(cudaMemcpyAsync(d_lo, lo, 8 * N, cudaMemcpyHostToDevice, cs), "copy lo");
        CK(cudaMemcpyAsync(d_hi, hi, 8 * N, cudaMemcpyHostToDevice, cs), "copy hi");
        CK(cudaMemcpyAsync(d_ut, utype, N, cudaMemcpyHostToDevice, cs), "copy utype");
        CK(cudaEventRecord(ev_values, cs), "cudaEventRecord");
        CK(cudaStreamWaitEvent(st, ev_routes, 0), "cudaStreamWaitEvent");
        route_ptr = d_rp;
        route_links = d_rl;
        c = d_c;
        w = d_w;
        lo = d_lo;
        hi = d_hi;
        utype = d_ut;
    }
    // the routes first: the ordering and the operator build index with them
    CK(cudaMemsetAsync(d_err, 0, sizeof(int) * 2, st), "memset");
    CK(pmp::validate_routes((int)n, (int)m, (long long)nnz, route_ptr, route_links, d_err, st),
       "validating the routes");
    if (batch) {
        CK(cudaMemcpyAsync(d_soff, batch->stream_off, 8 * ((size_t)batch->count + 1),
                           cudaMemcpyHostToDevice, st), "copy offsets");
        CK(cudaMemcpyAsync(d_loff, batch->link_off, 8 * ((size_t)batch->count + 1),
                           cudaMemcpyHostToDevice, st), "copy offsets");
    }
    int err_bits = 0, flags[2] = {0, 0};
    unsigned long long box[4];
    CK(cudaMemcpyAsync(&err_bits, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "read flags");
    CK(cudaStreamSynchronize(st), "validation");
    if (!err_bits && batch) {
        CK(pmp::check_blocks(batch->count, d_soff, d_loff, n, route_ptr, route_links, d_err, st),
           "checking the instance blocks");
        CK(cudaMemcpyAsync(&err_bits, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "read flags");
        CK(cudaStreamSynchronize(st), "validation");
    }
    if (err_bits) {
        drop();
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
        drop();
        return fail(NUM_ERR_INVALID, describe_bits(err_bits));
    }
    // then the values, once their copies are in
    if (cs) CK(cudaStreamWaitEvent(st, ev_values, 0), "cudaStreamWaitEvent");
    CK(pmp::validate_values((int)n, (int)m, c, utype, w, lo, hi, d_err, d_box, st),
       "validating the values");
    CK(cudaMemcpyAsync(flags, d_err, sizeof(flags), cudaMemcpyDeviceToHost, st), "read flags");
    CK(cudaMemcpyAsync(box, d_box, sizeof(box), cudaMemcpyDeviceToHost, st), "read box");
    CK(cudaStreamSynchronize(st), "validation");
    if (flags[0]) {
        drop();
        return fail(NUM_ERR_INVALID, describe_bits(flags[0]));
    }
    const double lmin = pmp::ordered_key_to_double(box[0]), lmax = pmp::ordered_key_to_double(box[1]);
    const double hmin = pmp::ordered_key_to_double(box[2]), hmax = pmp::ordered_key_to_double(box[3]);
    h->box_uniform = (lmin == lmax && hmin == hmax) ? 1 : 0;
    if (flags[1]) {  // some stream has U = -w / x: keep the types on the device
        h->ut = (uint8_t*)dev_alloc(h, N);
        if (!h->ut) {
            drop();
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
    if (rowk) {
        CK(pmp::count_chunks(h->row_ptr, (int)m, d_ccount, d_coff, d_ctmp, &h->nchunks, st),
           "counting long-link chunks");
        const size_t nc = (size_t)(h->nchunks > 0 ? h->nchunks : 1);
        h->chunks = (int4*)dev_alloc(h, sizeof(int4) * nc);
        h->chunk_queue = (int*)dev_alloc(h, sizeof(int) * nc);
        h->carry_l = dev_alloc(h, ts * nc);
        h->arrive_l = (int*)dev_alloc(h, sizeof(int) * nc);
        h->narrive_l = (int)nc;
        if (!h->chunks || !h->chunk_queue || !h->carry_l || !h->arrive_l) {
            drop();
            return fail(NUM_ERR_OOM, "device allocation failed");
        }
        if (h->nchunks > 0) {
            CK(pmp::fill_chunks(h->row_ptr, (int)m, d_coff, h->chunks, st), "long-link chunks");
            CK(pmp::order_chunks(h->chunks, h->nchunks, s, h->chunk_queue, st),
               "ordering the chunk queue");
        }
        CK(pmp::count_long_routes(h->col_ptr, (int)n, d_ccount, d_coff, d_ctmp, &h->nlong, st),
           "counting long routes");
        h->long_routes = (int*)dev_alloc(h, sizeof(int) * (size_t)(h->nlong > 0 ? h->nlong : 1));
        if (!h->long_routes) {
            drop();
            return fail(NUM_ERR_OOM, "device allocation failed");
        }
        if (h->nlong > 0)
            CK(pmp::fill_long_routes(h->col_ptr, (int)n, d_coff, h->long_routes, st),
               "long routes");
        CK(pmp::rows_grids(fp32 ? 0 : 1, (int)n, (int)m, h->nchunks, &h->grid_s, &h->grid_l,
                           &h->link_spread),
           "sizing the row-kernel grids");
    }
    CK(zero_state(h), "zeroing the state");
    CK(cudaStreamSynchronize(st), "setup");
    end_copies();
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

int check_debug_flag(num_problem* h) {
#ifdef PMP_DEBUG_BOUNDS
    unsigned int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, h->dbg, sizeof(flag), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the debug flag");
    if (flag) return fail(NUM_ERR_STATE, "debug build: a kernel gathered at an index out of range");
#else
    (void)h;
#endif
    return NUM_OK;
}

int finish_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return cuda_fail(e, what);
    return NUM_OK;
}

}  // namespace host
}  // namespace pmp

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
    p->history = 4096;
    p->use_graph = 1;
    p->reorder = 1;
    p->profile = 0;
    p->allocator = nullptr;
}

int num_create(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
               const int32_t* route_links, const double* c, const uint8_t* utype,
               const double* w, const double* lo, const double* hi, const num_params* p,
               void* cuda_stream) {
    TraceRange trace("num_create");
    return create_impl(out, n, m, route_ptr, route_links, c, utype, w, lo, hi, p, cuda_stream,
                       false);
}

int num_create_device(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
                      const int32_t* route_links, const double* c, const uint8_t* utype,
                      const double* w, const double* lo, const double* hi,
                      const num_params* p, void* cuda_stream) {
    TraceRange trace("num_create_device");
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
    TraceRange trace("num_solve");
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
        TraceRange replay("num_solve: replay of check_every iterations");
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
    const int dbg_rc = check_debug_flag(h);
    if (dbg_rc != NUM_OK) return dbg_rc;
    switch (h->ctl_host->stop) {
        case pmp::CONVERGED: return NUM_OK;
        case pmp::LIMIT: return NUM_NOT_CONVERGED;
        default: return fail(NUM_ERR_NUMERIC, "a residual became non-finite");
    }
}

static int get_impl(const num_problem* hc, double* x, double* prices, double* info, bool dev) {
    TraceRange trace("num_get");
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
    h->param_gen += 1;
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
    h->param_gen += 1;
    return finish_cuda(e, "setting the weights");
}

// The device-array forms of the two setters: the values are checked on the device (finite
// and > 0) before they replace the handle's.
static int set_values_device(num_problem* h, const double* a, bool capacity) {
    const int count = (int)(capacity ? h->m : h->n);
    cudaStream_t st = h->stream;
    if (!h->err_d) {
        h->err_d = (int*)dev_alloc(h, sizeof(int));
        if (!h->err_d) return fail(NUM_ERR_OOM, "device allocation failed");
    }
    int bad = 0;
    cudaError_t e = order_after_legacy(h);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err_d, 0, sizeof(int), st);
    if (e == cudaSuccess) e = pmp::validate_positive(count, a, h->err_d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, h->err_d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "checking the values");
    if (bad)
        return fail(NUM_ERR_INVALID, capacity ? "a capacity is not finite and > 0"
                                              : "a weight is not finite and > 0");
    double* stage = capacity ? h->y64 : h->x64;
    e = cudaMemcpyAsync(stage, a, 8 * (size_t)count, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        if (capacity)
            e = h->prec == NUM_FUSED_FP32
                    ? pmp::convert_params<float>(0, count, stage, nullptr, nullptr, nullptr,
                                                 nullptr, nullptr, (float*)h->c, nullptr,
                                                 nullptr, nullptr, st)
                    : pmp::convert_params<double>(0, count, stage, nullptr, nullptr, nullptr,
                                                  nullptr, nullptr, (double*)h->c, nullptr,
                                                  nullptr, nullptr, st);
        else
            e = h->prec == NUM_FUSED_FP32 ? pmp::set_weights<float>(make_view<float>(h), stage, st)
                                          : pmp::set_weights<double>(make_view<double>(h), stage, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    h->param_gen += 1;
    return finish_cuda(e, capacity ? "setting the capacities" : "setting the weights");
}

int num_set_capacity_device(num_problem* h, const double* c) {
    g_last_error.clear();
    if (!h || !c) return fail(NUM_ERR_INVALID, "NULL argument");
    return set_values_device(h, c, true);
}

int num_set_weights_device(num_problem* h, const double* w) {
    g_last_error.clear();
    if (!h || !w) return fail(NUM_ERR_INVALID, "NULL argument");
    return set_values_device(h, w, false);
}

}  // extern "C"

extern "C" {

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
        case NUM_ERR_TIMEOUT: return "a bounded wait between blocks ran out";
        default: return "unknown status code";
    }
}

const char* num_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

