// C ABI of the PMP solver: the reverse-mode derivative of unrolled iterations (kernels in
// adjoint.cu).
//
//   num_adjoint_forward   K iterations from the zero state, keeping the iterate every Kc
//                         iterations (checkpoints) and the last segment's tape (x, the
//                         slack flows and the rho of each iteration) in the handle;
//   num_adjoint_backward  the backward sweep from what the forward kept: per segment, last
//                         first, the segment's tape (recomputed from its checkpoint unless
//                         it is the one in the tape already), then the transposed
//                         iterations; cotangents and gradients are caller DEVICE arrays;
//   num_adjoint           both, with HOST arrays (the tape is released at the end);
//   num_adjoint_release   frees what the forward kept.
// In the fused paths the tape is written by the forward kernels themselves; in the plain
// FP64 path one iteration at a time is copied out.
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

// What num_adjoint_forward keeps (device memory through the handle's allocator).
struct AdjTape {
    int64_t K = 0, Kc = 0, nseg = 0;
    size_t sb = 0;              // bytes of one checkpoint
    char* ckpt = nullptr;       // nseg + 1 checkpoints (segment starts, then the final state)
    void* tape_x = nullptr;     // Kc x n iterates of one segment
    void* tape_ps = nullptr;    // Kc x m slack flows
    double* tape_rho = nullptr; // Kc rho values
    int64_t tape_seg = -1;      // the segment whose iterations are in the tape
    long long gen = 0;          // the handle's param_gen at the forward
    int prec = 0;
    void *xb = nullptr, *Zb = nullptr, *ab = nullptr, *wb = nullptr, *yb = nullptr,
         *zsb = nullptr, *Rxb = nullptr, *cb = nullptr, *abc = nullptr;
    std::vector<void*> owned;
};

namespace pmp {
namespace host {

void adjoint_tape_free(num_problem* h) {
    if (!h || !h->adj) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* q : h->adj->owned) dev_free(h, q);
    delete h->adj;
    h->adj = nullptr;
}

}  // namespace host
}  // namespace pmp

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

// A new tape for K iterations with checkpoints every Kc (the old one is freed).
int tape_alloc(num_problem* h, int64_t K, int64_t Kc) {
    adjoint_tape_free(h);
    AdjTape* t = new (std::nothrow) AdjTape();
    if (!t) return fail(NUM_ERR_OOM, "host allocation failed");
    h->adj = t;
    const size_t ts = h->prec == NUM_FUSED_FP32 ? 4 : 8;
    const size_t N = (size_t)h->n, M = (size_t)h->m;
    t->K = K;
    t->Kc = Kc;
    t->nseg = (K + Kc - 1) / Kc;
    t->sb = state_bytes(h);
    t->prec = h->prec;
    bool ok = true;
    auto A = [&](size_t bytes) -> void* {
        void* q = ok ? dev_alloc(h, bytes) : nullptr;
        if (!q)
            ok = false;
        else
            t->owned.push_back(q);
        return q;
    };
    t->ckpt = (char*)A(t->sb * (size_t)(t->nseg + 1));
    t->tape_x = A(ts * N * (size_t)Kc);
    t->tape_ps = A(ts * M * (size_t)Kc);
    t->tape_rho = (double*)A(sizeof(double) * (size_t)Kc);
    t->xb = A(ts * N);
    t->Zb = A(ts * N);
    t->ab = A(2 * ts * N);
    t->wb = A(ts * N);
    t->yb = A(ts * M);
    t->zsb = A(ts * M);
    t->Rxb = A(ts * M);
    t->cb = A(ts * M);
    if (h->chunks && h->nchunks > 0) t->abc = A(2 * ts * (size_t)h->nchunks);
    if (!ok) {
        adjoint_tape_free(h);
        return fail(NUM_ERR_OOM, "device allocation failed (adjoint tape and checkpoints)");
    }
    return NUM_OK;
}

// Run iterations k0 + 1 .. k0 + cnt from the current state, writing each one's x, slack
// flows and rho to the tape.
cudaError_t taped_run(num_problem* h, int64_t k0, int64_t cnt) {
    AdjTape* t = h->adj;
    cudaStream_t st = h->stream;
    cudaError_t e = pmp::ctl_arm(h->ctl, k0 + cnt, 0.0, st);
    if (e != cudaSuccess) return e;
    if (h->prec != NUM_PLAIN_FP64) {
        // the fused row kernels write the tape themselves
        h->tape_x = t->tape_x;
        h->tape_ps = t->tape_ps;
        h->tape_rho = t->tape_rho;
        h->tape_k0 = k0;
        h->tape_len = (int)cnt;
        e = run_iterations(h, (int)cnt);
        h->tape_x = h->tape_ps = nullptr;
        h->tape_rho = nullptr;
        h->tape_k0 = 0;
        h->tape_len = 0;
        pmp::note_launches(cnt * h->kpi);
        return e;
    }
    const size_t ts = h->prec == NUM_FUSED_FP32 ? 4 : 8;
    const size_t N = (size_t)h->n, M = (size_t)h->m;
    for (int64_t i = 0; i < cnt && e == cudaSuccess; ++i) {
        e = pmp::record_rho(h->ctl, t->tape_rho + i, st);
        if (e == cudaSuccess) e = run_iterations(h, 1);
        pmp::note_launches(h->kpi);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)t->tape_x + ts * N * (size_t)i, h->x, ts * N,
                                cudaMemcpyDeviceToDevice, st);
        const void* ps = h->ps;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)t->tape_ps + ts * M * (size_t)i, ps, ts * M,
                                cudaMemcpyDeviceToDevice, st);
    }
    return e;
}

int forward_impl(num_problem* h, int64_t K, int64_t Kc) {
    cudaStream_t st = h->stream;
    int rc = tape_alloc(h, K, Kc);
    if (rc != NUM_OK) return rc;
    AdjTape* t = h->adj;
    cudaError_t e = cudaSuccess;
#define FK(call, what)                  \
    do {                                \
        e = (call);                     \
        if (e != cudaSuccess) {         \
            adjoint_tape_free(h);       \
            return cuda_fail(e, what);  \
        }                               \
    } while (0)
    FK(order_after_legacy(h), "ordering");
    FK(zero_state(h), "zeroing the state");
    for (int64_t s = 0; s < t->nseg; ++s) {
        const int64_t cnt = std::min<int64_t>(Kc, K - s * Kc);
        FK(copy_state(h, t->ckpt + t->sb * (size_t)s, true), "checkpoint");
        if (s < t->nseg - 1) {
            FK(pmp::ctl_arm(h->ctl, s * Kc + cnt, 0.0, st), "arming");
            FK(run_iterations(h, (int)cnt), "forward iterations");
            pmp::note_launches(cnt * h->kpi);
        } else {
            FK(taped_run(h, s * Kc, cnt), "forward iterations of the last segment");
        }
    }
    // the objective of the final state (num_get reports it), then the final state itself
    FK(h->prec == NUM_FUSED_FP32
           ? pmp::export_solution<float>(make_view<float>(h), nullptr, nullptr, h->part_exp,
                                         h->exp_blocks, st)
           : pmp::export_solution<double>(make_view<double>(h), nullptr, nullptr, h->part_exp,
                                          h->exp_blocks, st),
       "objective");
    FK(copy_state(h, t->ckpt + t->sb * (size_t)t->nseg, true), "final state");
    FK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st), "ctl");
    FK(cudaStreamSynchronize(st), "adjoint forward");
#undef FK
    t->tape_seg = t->nseg - 1;
    t->gen = h->param_gen;
    return check_debug_flag(h);
}

template <typename T>
int backward_impl(num_problem* h, const double* xbar, double ubar, double* c_grad,
                  double* w_grad) {
    using T2 = typename pmp::Pair<T>::type;
    AdjTape* t = h->adj;
    cudaStream_t st = h->stream;
    const size_t N = (size_t)h->n, M = (size_t)h->m;
    pmp::AdjView<T> a;
    std::memset(&a, 0, sizeof(a));
    a.alpha = h->prm.alpha;
    a.xb = (T*)t->xb;
    a.Zb = (T*)t->Zb;
    a.ab = (T2*)t->ab;
    a.wb = (T*)t->wb;
    a.yb = (T*)t->yb;
    a.zsb = (T*)t->zsb;
    a.Rxb = (T*)t->Rxb;
    a.cb = (T*)t->cb;
    a.abc = (T2*)t->abc;
    cudaError_t e = cudaSuccess;
#define BK(call, what)                 \
    do {                               \
        e = (call);                    \
        if (e != cudaSuccess) {        \
            t->tape_seg = -1;          \
            return cuda_fail(e, what); \
        }                              \
    } while (0)
    BK(order_after_legacy(h), "ordering");
    // the cotangents start from the final state
    BK(copy_state(h, t->ckpt + t->sb * (size_t)t->nseg, false), "restore the final state");
    a.v = make_view<T>(h);
    BK(pmp::adjoint_grids<T>(a), "sizing the adjoint grids");
    BK(pmp::adjoint_init<T>(a, xbar, ubar, st), "adjoint init");
    const T* tx = (const T*)t->tape_x;
    const T* tp = (const T*)t->tape_ps;
    for (int64_t s = t->nseg - 1; s >= 0; --s) {
        const int64_t cnt = std::min<int64_t>(t->Kc, t->K - s * t->Kc);
        if (t->tape_seg != s) {  // recompute the segment's iterations into the tape
            t->tape_seg = -1;
            BK(copy_state(h, t->ckpt + t->sb * (size_t)s, false), "restore checkpoint");
            BK(taped_run(h, s * t->Kc, cnt), "recomputing a segment");
            t->tape_seg = s;
        }
        for (int64_t i = cnt - 1; i >= 0; --i)
            BK(pmp::adjoint_step<T>(a, tx + N * (size_t)i, tp + M * (size_t)i, t->tape_rho + i,
                                    st),
               "adjoint iteration");
    }
    BK(pmp::adjoint_export<T>(a, c_grad, w_grad, st), "exporting the gradients");
    // leave the handle at the forward result
    BK(copy_state(h, t->ckpt + t->sb * (size_t)t->nseg, false), "restore the final state");
    BK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st), "ctl");
    BK(cudaStreamSynchronize(st), "adjoint");
#undef BK
    return check_debug_flag(h);
}

int backward(num_problem* h, const double* xbar, double ubar, double* c_grad, double* w_grad) {
    if (!h->adj) return fail(NUM_ERR_STATE, "no adjoint forward to differentiate (call num_adjoint_forward)");
    if (h->adj->gen != h->param_gen || h->adj->prec != h->prec)
        return fail(NUM_ERR_STATE, "the capacities or weights changed since num_adjoint_forward");
    return h->prec == NUM_FUSED_FP32 ? backward_impl<float>(h, xbar, ubar, c_grad, w_grad)
                                     : backward_impl<double>(h, xbar, ubar, c_grad, w_grad);
}

int checkpoint_interval(int64_t iters, int32_t checkpoint_every, int64_t* Kc) {
    if (iters < 1) return fail(NUM_ERR_INVALID, "iters must be >= 1");
    if (checkpoint_every < 0) return fail(NUM_ERR_INVALID, "checkpoint_every must be >= 0");
    *Kc = checkpoint_every == 0 ? iters : std::min<int64_t>(checkpoint_every, iters);
    return NUM_OK;
}

}  // namespace

extern "C" {

int num_adjoint_forward(num_problem* h, int64_t iters, int32_t checkpoint_every) {
    TraceRange trace("num_adjoint_forward");
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    int64_t Kc = 0;
    const int rc = checkpoint_interval(iters, checkpoint_every, &Kc);
    if (rc != NUM_OK) return rc;
    return forward_impl(h, iters, Kc);
}

int num_adjoint_backward(num_problem* h, const double* xbar, double ubar, double* c_grad,
                         double* w_grad) {
    TraceRange trace("num_adjoint_backward");
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    if (!xbar && ubar == 0.0) return fail(NUM_ERR_INVALID, "nothing to differentiate");
    if (!std::isfinite(ubar)) return fail(NUM_ERR_INVALID, "ubar is not finite");
    return backward(h, xbar, ubar, c_grad, w_grad);
}

int num_adjoint_release(num_problem* h) {
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    adjoint_tape_free(h);
    return NUM_OK;
}

int num_adjoint(num_problem* h, int64_t iters, int32_t checkpoint_every, const double* xbar,
                int32_t objective, double* c_grad, double* w_grad, double* objective_out) {
    TraceRange trace("num_adjoint");
    g_last_error.clear();
    if (!h) return fail(NUM_ERR_INVALID, "handle is NULL");
    if (objective != 0 && objective != 1) return fail(NUM_ERR_INVALID, "objective must be 0 or 1");
    if (!xbar && !objective) return fail(NUM_ERR_INVALID, "nothing to differentiate");
    int64_t Kc = 0;
    int rc = checkpoint_interval(iters, checkpoint_every, &Kc);
    if (rc != NUM_OK) return rc;
    rc = forward_impl(h, iters, Kc);
    if (rc != NUM_OK) return rc;
    const double objective_value = h->ctl_host->objective;
    // host arrays: the cotangent through a device copy, the gradients through the n- and
    // m-sized staging buffers (exported one at a time)
    cudaStream_t st = h->stream;
    double* xbar_dev = nullptr;
    if (xbar) {
        xbar_dev = (double*)dev_alloc(h, 8 * (size_t)h->n);
        if (!xbar_dev) {
            adjoint_tape_free(h);
            return fail(NUM_ERR_OOM, "device allocation failed");
        }
    }
    cudaError_t e = cudaSuccess;
    if (xbar_dev) {
        e = cudaMemcpyAsync(xbar_dev, xbar, 8 * (size_t)h->n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) {
        // dJ/dw to x64 and dJ/dc to y64 in one sweep: x64 / y64 are not used by the sweep
        rc = backward(h, xbar_dev, objective ? 1.0 : 0.0, c_grad ? h->y64 : nullptr,
                      w_grad ? h->x64 : nullptr);
        if (rc == NUM_OK && w_grad)
            e = cudaMemcpyAsync(w_grad, h->x64, 8 * (size_t)h->n, cudaMemcpyDeviceToHost, st);
        if (rc == NUM_OK && c_grad && e == cudaSuccess)
            e = cudaMemcpyAsync(c_grad, h->y64, 8 * (size_t)h->m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (xbar_dev) dev_free(h, xbar_dev);
    adjoint_tape_free(h);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint gradients");
    if (rc != NUM_OK) return rc;
    if (objective_out) *objective_out = objective_value;
    return NUM_OK;
}

}  // extern "C"
