// The plain FP64 GPU path: the same iteration as the fused kernels, written the way a
// tensor library runs it, one kernel per step with every intermediate in global memory:
//   SpMV-transpose (A = R' pbar, B = R' y), stream prox, SpMV (R x), link update,
//   three reductions and a one-block finalize.  It is the baseline the fused FP32 path is
//   measured against (and a second, independently written route to the same numbers).
#include <cuda_runtime.h>

#include "pmp_device.cuh"
#include "pmp_internal.cuh"

namespace pmp {

namespace {

constexpr int kTh = 256;
constexpr int kMaxPartials = 1024;

// A_j = sum over route j of pbar_l, B_j = sum of y_l: one thread per stream
__global__ void k_plain_spmvT(View<double> v) {
    if (v.ctl->stop) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int e = v.col_ptr[j]; e < v.col_ptr[j + 1]; ++e) {
            const int l = checked_index(v.row_idx[e], v.m, v.dbg);
            a += v.pbar[l];
            b += v.y[l];
        }
        v.A[j] = a;
        v.B[j] = b;
    }
}

// z update and prox of every stream (Sec. III-E, III-G)
__global__ void k_plain_stream(View<double> v) {
    const Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    const double alpha = ctl->alpha, inv_rho = 1.0 / ctl->rho;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += gridDim.x * blockDim.x) {
        const double L = (double)(v.col_ptr[j + 1] - v.col_ptr[j]);
        const double xo = v.x[j];
        const double Zn = alpha * L * xo + (1.0 - alpha) * v.Z[j] - alpha * v.A[j];
        const double S = Zn - v.B[j] * inv_rho;
        const double lo = v.box_uniform ? v.lo_u : v.lo[j];
        const double hi = v.box_uniform ? v.hi_u : v.hi[j];
        const double xn = stream_prox<double>(S, L, v.wt[j], inv_rho, lo, hi,
                                              v.ut && v.ut[j] == 2);
        v.Z[j] = Zn;
        v.x[j] = xn;
        v.tS[j] = L * (xn - xo) * (xn - xo);
    }
}

// RxN = R x: one warp per link
__global__ void k_plain_spmv(View<double> v) {
    if (v.ctl->stop) return;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long l = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; l < v.m; l += warps) {
        double s = 0.0;
        for (int e = v.row_ptr[l] + lane; e < v.row_ptr[l + 1]; e += 32)
            s += v.x[checked_index(v.col_idx[e], v.n, v.dbg)];
        s = warp_sum(s);
        if (lane == 0) v.RxN[l] = s;
    }
}

// slack prox, link average, z and price updates, residual terms of every link
__global__ void k_plain_link(View<double> v) {
    const Ctl* ctl = v.ctl;
    if (ctl->stop) return;
    const double alpha = ctl->alpha, rho = ctl->rho, inv_rho = 1.0 / rho;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < v.m; l += gridDim.x * blockDim.x) {
        const double deg = (double)(v.row_ptr[l + 1] - v.row_ptr[l]);
        const double Rxn = v.RxN[l], Rxo = v.Rx[l];
        const double pbo = v.pbar[l], y = v.y[l], pso = v.ps[l], zso = v.zs[l];
        double psn = zso - y * inv_rho;
        psn = psn < -v.c[l] ? -v.c[l] : psn;
        const double pbn = (Rxn + psn) / (deg + 1.0);
        v.zs[l] = alpha * (psn - pbn) + (1.0 - alpha) * zso;
        v.y[l] = y + alpha * rho * pbn;
        v.pbar[l] = pbn;
        v.Rx[l] = Rxn;
        v.ps[l] = psn;
        const double dpb = pbn - pbo, dd = (psn - pbn) - (pso - pbo);
        v.tR[l] = (deg + 1.0) * pbn * pbn;
        v.tL[l] = deg * dpb * dpb - 2.0 * dpb * (Rxn - Rxo) + dd * dd;
    }
}

// block partial sums of one term array
__global__ void k_plain_reduce(const Ctl* ctl, const double* a, int count, double* part) {
    __shared__ double red[kTh / 32];
    if (ctl->stop) return;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        s += a[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_plain_finalize(View<double> v, const double* partS, const double* partR,
                                 const double* partL, int nb) {
    __shared__ double red[kTh / 32];
    if (v.ctl->stop) return;
    double s = 0.0, r = 0.0, l = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        s += partS[i];
        r += partR[i];
        l += partL[i];
    }
    s = block_sum(s, red);
    r = block_sum(r, red);
    l = block_sum(l, red);
    if (threadIdx.x == 0) finalize_iteration(v.ctl, r, s + l, v.hist, v.sched);
}

int blocks(long long count, int cap) {
    long long b = (count + kTh - 1) / kTh;
    b = b < 1 ? 1 : b;
    return (int)(b < cap ? b : cap);
}

}  // namespace

int plain_partial_blocks(int n, int m) { return blocks(n > m ? n : m, kMaxPartials); }

cudaError_t plain_iteration(const View<double>& v, int nb, cudaStream_t st, cudaEvent_t* evs) {
    double* partS = v.part_s;
    double* partR = v.part_l;
    double* partL = v.part_l + nb;
    int q = 0;
    auto mark = [&]() {
        if (evs) record_kernel_event(evs[q], st);
        ++q;
    };
    k_plain_spmvT<<<blocks(v.n, 1 << 16), kTh, 0, st>>>(v);
    mark();
    k_plain_stream<<<blocks(v.n, 1 << 16), kTh, 0, st>>>(v);
    mark();
    k_plain_spmv<<<blocks(32LL * v.m, 1 << 16), kTh, 0, st>>>(v);
    mark();
    k_plain_link<<<blocks(v.m, 1 << 16), kTh, 0, st>>>(v);
    mark();
    k_plain_reduce<<<nb, kTh, 0, st>>>(v.ctl, v.tS, v.n, partS);
    mark();
    k_plain_reduce<<<nb, kTh, 0, st>>>(v.ctl, v.tR, v.m, partR);
    mark();
    k_plain_reduce<<<nb, kTh, 0, st>>>(v.ctl, v.tL, v.m, partL);
    mark();
    k_plain_finalize<<<1, kTh, 0, st>>>(v, partS, partR, partL, nb);
    mark();
    return cudaGetLastError();
}

}  // namespace pmp
