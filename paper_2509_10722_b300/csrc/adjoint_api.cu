// C ABI of the PMP solver: num_adjoint, the reverse-mode derivative of unrolled
// iterations (forward with checkpoints, per-segment recompute to a tape, backward sweep;
// the kernels are in adjoint.cu).
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
    const int dbg_rc = check_debug_flag(h);
    if (dbg_rc != NUM_OK) {
        release();
        return dbg_rc;
    }
    release();
    return NUM_OK;
}

}  // namespace

extern "C" {

int num_adjoint(num_problem* h, int64_t iters, int32_t checkpoint_every, const double* xbar,
                int32_t objective, double* c_grad, double* w_grad, double* objective_out) {
    TraceRange trace("num_adjoint");
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

}  // extern "C"
