// Reverse-mode derivative of K unrolled PMP iterations (the reduced recurrence of rows.cu,
// Sec. III-D..G) with respect to the capacities c and the weights w, for a cotangent on
// the final rates x_K.  The rho of every iteration is held fixed (the forward run's own
// decisions), which makes the K-step map piecewise smooth.
//
// Forward iteration k (rho = rho_k):
//   stream j:  Z'_k = a L x_{k-1} + (1-a) Z'_{k-1} - a (R' pbar_{k-1})_j
//              S_k  = Z'_k - (R' y_{k-1})_j / rho;   x_k = clip(prox(S_k; L, w, rho))
//   link l:    ps_k = max(zs_{k-1} - y_{k-1} / rho, -c);   pbar_k = ((R x_k)_l + ps_k) / (deg+1)
//              zs_k = a (ps_k - pbar_k) + (1-a) zs_{k-1};   y_k = y_{k-1} + a rho pbar_k
// Backward iteration k, given the cotangents of the state after it:
//   link pass (per link, gathering (Abar, Bbar) of the streams of the link from the stream
//   pass of iteration k+1): pbar_bar_k = R Abar, y_bar_k += R Bbar; then
//     t = pbar_bar_k + a rho y_bar_k - a zs_bar_k;  ps_bar = t / (deg+1) + a zs_bar_k;
//     Rx_bar = t / (deg+1);  zs_bar_{k-1} = (1-a) zs_bar_k + [ps_k > -c] ps_bar;
//     y_bar_{k-1} = y_bar_k - [ps_k > -c] ps_bar / rho;  c_bar -= [ps_k = -c] ps_bar
//   stream pass (per stream, gathering Rx_bar over its route):
//     x_bar_k += R' Rx_bar;  S_bar = x_bar_k dx/dS;  w_bar += x_bar_k dx/dw;
//     t = Z'_bar_k + S_bar;  x_bar_{k-1} = a L t;  Z'_bar_{k-1} = (1-a) t;
//     Abar = -a t;  Bbar = -S_bar / rho
// with the prox Jacobian from x_k alone: unclipped log stream, sqrt(D) = L x + w / (rho x),
// dx/dS = x / sqrt(D), dx/dw = 1 / (rho sqrt(D)); unclipped linear stream, dx/dS = 1/L,
// dx/dw = 1 / (rho L); a stream at a bound of its box, 0.  Only x_k and ps_k of every
// iteration are needed; they are recomputed segment by segment from checkpoints.
// Links of more than kLongRow streams are summed by whole warps in chunks,
// and streams with more than kLongRoute links by one warp each, as in the forward kernels
// (the chunks dealt out to the warps in turn, not from the forward link kernels' queue).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "pmp_device.cuh"
#include "pmp_internal.cuh"
#include "pmp_rows.cuh"

namespace cg = cooperative_groups;

namespace pmp {

namespace {

constexpr int kTh = 256;
constexpr int kGroup = 8;

// The inputs of a link's transpose step that do not depend on the gathers.
template <typename T>
struct AdjLinkState {
    T yb, zsb, ps, c;
};

template <typename T>
__device__ __forceinline__ AdjLinkState<T> adj_load_link(const AdjView<T>& a, int l,
                                                         const T* __restrict__ ps_k) {
    AdjLinkState<T> st;
    st.yb = a.yb[l];
    st.zsb = a.zsb[l];
    st.ps = ps_k[l];
    st.c = a.v.c[l];
    return st;
}

// Transpose of the link step of one link, given sa = (R Abar)_l and sb = (R Bbar)_l.
template <typename T>
__device__ __forceinline__ void adj_link_epilogue(const AdjView<T>& a, int l,
                                                  const AdjLinkState<T>& st, T sa, T sb, int deg,
                                                  T alpha, T rho) {
    const T yb = st.yb + sb;
    const T zsb = st.zsb;
    const T deg1 = (T)(deg + 1);
    const T t = sa + alpha * rho * yb - alpha * zsb;
    const T psb = t / deg1 + alpha * zsb;
    a.Rxb[l] = t / deg1;
    const bool open = st.ps > -st.c;  // slack prox not at its bound
    a.zsb[l] = (T(1) - alpha) * zsb + (open ? psb : T(0));
    a.yb[l] = yb - (open ? psb / rho : T(0));
    if (!open) a.cb[l] -= psb;
}

template <typename T>
__global__ void __launch_bounds__(kTh) k_adj_link(AdjView<T> a, const T* __restrict__ ps_k,
                                                 const double* __restrict__ rho_ptr) {
    using T2 = typename Pair<T>::type;
    auto g = cg::tiled_partition<kGroup>(cg::this_thread_block());
    const bool leader = g.thread_rank() == 0;
    const View<T>& v = a.v;
    const T alpha = (T)a.alpha, rho = (T)*rho_ptr;
    constexpr int kGroups = kTh / kGroup;
    const int m = v.m;
    // one group per link, links in turn over the grid; the bounds of the group's
    // next link are loaded before the current link is summed, and the leader loads the
    // link's own inputs before the gathers
    int l = blockIdx.x * kGroups + (int)(threadIdx.x / kGroup);
    int p0 = 0, p1 = 0;
    if (l < m) {
        p0 = __ldg(v.row_ptr + l);
        p1 = __ldg(v.row_ptr + l + 1);
    }
    while (l < m) {
        const int ln = l + gridDim.x * kGroups;
        int q0 = 0, q1 = 0;
        if (ln < m) {
            q0 = __ldg(v.row_ptr + ln);
            q1 = __ldg(v.row_ptr + ln + 1);
        }
        if (!a.abc || p1 - p0 <= kLongRow) {  // longer links are done by their chunks
            AdjLinkState<T> st;
            if (leader) st = adj_load_link(a, l, ps_k);
            // R Abar, R Bbar: lane k adds entries p0 + k, p0 + k + kGroup, ... in that
            // order, four gathers in flight
            T sa = T(0), sb = T(0);
            for (int e = p0 + g.thread_rank(); e < p1; e += 4 * kGroup) {
                int ix[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    ix[k] = (k == 0 || e + k * kGroup < p1)
                                ? checked_index(__ldg(v.col_idx + e + k * kGroup), v.n, v.dbg)
                                : -1;
                T2 u[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    u[k] = ix[k] >= 0 ? __ldg(a.ab + ix[k]) : T2{T(0), T(0)};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (ix[k] >= 0) {
                        sa += u[k].x;
                        sb += u[k].y;
                    }
            }
#pragma unroll
            for (int o = kGroup / 2; o > 0; o >>= 1) {
                sa += g.shfl_down(sa, o);
                sb += g.shfl_down(sb, o);
            }
            if (leader) adj_link_epilogue(a, l, st, sa, sb, p1 - p0, alpha, rho);
        }
        l = ln;
        p0 = q0;
        p1 = q1;
    }
    if (!a.abc) return;
    // chunks of the longer links: one warp each; the warp that completes a link sums its
    // chunk slots in a fixed order and runs the link's transpose step
    const int lane = threadIdx.x & 31;
    for (int q = blockIdx.x * (kTh / 32) + (int)(threadIdx.x >> 5); q < v.nchunks;
         q += gridDim.x * (kTh / 32)) {
        const int4 ch = __ldg(v.chunks + q);  // (link, first entry, end entry, first chunk)
        T sa = T(0), sb = T(0);
        for (int e = ch.y + lane; e < ch.z; e += 64) {
            const T2 u = a.ab[checked_index(__ldg(v.col_idx + e), v.n, v.dbg)];
            const T2 w = e + 32 < ch.z ? a.ab[checked_index(__ldg(v.col_idx + e + 32), v.n, v.dbg)]
                                       : T2{T(0), T(0)};
            sa += u.x + w.x;
            sb += u.y + w.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_down_sync(0xffffffffu, sa, o);
            sb += __shfl_down_sync(0xffffffffu, sb, o);
        }
        const int p0 = __ldg(v.row_ptr + ch.x), p1 = __ldg(v.row_ptr + ch.x + 1);
        const int nch = (p1 - p0 + kChunk - 1) / kChunk;
        int done = 0;
        if (lane == 0) {
            a.abc[q] = T2{sa, sb};
            __threadfence();
            done = atomicAdd(v.arrive_l + ch.w, 1) == nch - 1;
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        if (!done) continue;
        __threadfence();
        T ta = T(0), tb = T(0);
        for (int k = lane; k < nch; k += 32) {
            const T2 u = __ldcg(a.abc + ch.w + k);
            ta += u.x;
            tb += u.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ta += __shfl_down_sync(0xffffffffu, ta, o);
            tb += __shfl_down_sync(0xffffffffu, tb, o);
        }
        if (lane == 0) {
            v.arrive_l[ch.w] = 0;
            const AdjLinkState<T> st = adj_load_link(a, ch.x, ps_k);
            adj_link_epilogue(a, ch.x, st, ta, tb, p1 - p0, alpha, rho);
        }
    }
}

// The inputs of a stream's transpose step that do not depend on the gathers.
template <typename T>
struct AdjStreamState {
    T xb, x, wt, lo, hi, Zb, wb;
    bool a2;  // U = -w / x
};

template <typename T>
__device__ __forceinline__ AdjStreamState<T> adj_load_stream(const AdjView<T>& a, int j,
                                                             const T* __restrict__ x_k) {
    const View<T>& v = a.v;
    AdjStreamState<T> st;
    st.xb = a.xb[j];
    st.x = x_k[j];
    st.wt = v.wt[j];
    st.lo = v.box_uniform ? v.lo_u : v.lo[j];
    st.hi = v.box_uniform ? v.hi_u : v.hi[j];
    st.Zb = a.Zb[j];
    st.wb = a.wb[j];
    st.a2 = v.ut && v.ut[j] == 2;
    return st;
}

// Transpose of the stream step of stream j, given r = (R' Rx_bar)_j.
template <typename T>
__device__ __forceinline__ void adj_stream_epilogue(const AdjView<T>& a, int j,
                                                    const AdjStreamState<T>& st, T r, int len,
                                                    T alpha, T rho) {
    using T2 = typename Pair<T>::type;
    const T xbk = st.xb + r;
    const T x = st.x, L = (T)len, wt = st.wt;
    T dS = T(0), dw = T(0);
    if (x > st.lo && x < st.hi) {
        if (st.a2) {
            // rho L x^3 - rho S x^2 - w = 0 with S = L x - w / (rho x^2):
            // f_x = rho L x^2 + 2 w / x, dx/dS = rho x^2 / f_x, dx/dw = 1 / f_x
            const T fx = rho * L * x * x + T(2) * wt / x;
            dS = rho * x * x / fx;
            dw = T(1) / fx;
        } else if (wt > T(0)) {
            const T sqD = L * x + wt / (rho * x);
            dS = x / sqD;
            dw = T(1) / (rho * sqD);
        } else {
            dS = T(1) / L;
            dw = T(1) / (rho * L);
        }
    }
    const T Sb = xbk * dS;
    a.wb[j] = st.wb + xbk * dw;
    const T t = st.Zb + Sb;
    a.xb[j] = alpha * L * t;
    a.Zb[j] = (T(1) - alpha) * t;
    T2 ab;
    ab.x = -alpha * t;
    ab.y = -Sb / rho;
    a.ab[j] = ab;
}

template <typename T>
__global__ void __launch_bounds__(kTh) k_adj_stream(AdjView<T> a, const T* __restrict__ x_k,
                                                   const double* __restrict__ rho_ptr) {
    const View<T>& v = a.v;
    const T alpha = (T)a.alpha, rho = (T)*rho_ptr;
    const bool split = v.nlong > 0;
    // one thread per stream, streams in turn over the grid; the stream's own inputs are loaded
    // before its gathers
    for (int j = blockIdx.x * kTh + threadIdx.x; j < v.n; j += gridDim.x * kTh) {
        const int p = __ldg(v.col_ptr + j), pn = __ldg(v.col_ptr + j + 1);
        if (split && pn - p > kLongRoute) continue;  // summed by a warp below
        const AdjStreamState<T> st = adj_load_stream(a, j, x_k);
        T r = T(0);  // (R' Rx_bar)_j in route order, four gathers in flight
        int e = p;
        for (; e + 4 <= pn; e += 4) {
            const int l0 = checked_index(__ldg(v.row_idx + e), v.m, v.dbg);
            const int l1 = checked_index(__ldg(v.row_idx + e + 1), v.m, v.dbg);
            const int l2 = checked_index(__ldg(v.row_idx + e + 2), v.m, v.dbg);
            const int l3 = checked_index(__ldg(v.row_idx + e + 3), v.m, v.dbg);
            const T g0 = __ldg(a.Rxb + l0), g1 = __ldg(a.Rxb + l1);
            const T g2 = __ldg(a.Rxb + l2), g3 = __ldg(a.Rxb + l3);
            r += g0;
            r += g1;
            r += g2;
            r += g3;
        }
        for (; e < pn; ++e) r += __ldg(a.Rxb + checked_index(__ldg(v.row_idx + e), v.m, v.dbg));
        adj_stream_epilogue(a, j, st, r, pn - p, alpha, rho);
    }
    // streams with more than kLongRoute links: one warp each, as in the forward kernel
    const int lane = threadIdx.x & 31;
    for (int q = blockIdx.x * (kTh / 32) + (int)(threadIdx.x >> 5); q < v.nlong;
         q += gridDim.x * (kTh / 32)) {
        const int j = __ldg(v.long_routes + q);
        const int p = __ldg(v.col_ptr + j), pn = __ldg(v.col_ptr + j + 1);
        T r = T(0);
        for (int e = p + lane; e < pn; e += 32)
            r += a.Rxb[checked_index(__ldg(v.row_idx + e), v.m, v.dbg)];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        if (lane == 0) adj_stream_epilogue(a, j, adj_load_stream(a, j, x_k), r, pn - p, alpha, rho);
    }
}

// Initial cotangents for the final rates: x_bar = xbar_in (caller order) plus, for a
// cotangent ubar of the total utility, ubar U'(x) (U' = w / x, w / x^2 or w); the direct
// ubar dU/dw (log x, -1 / x or x) starts w_bar.
template <typename T>
__global__ void k_adj_init(AdjView<T> a, const double* __restrict__ xbar_in, double ubar) {
    using T2 = typename Pair<T>::type;
    const View<T>& v = a.v;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += gridDim.x * blockDim.x) {
        const int o = v.perm ? v.perm[j] : j;
        T xb = xbar_in ? (T)xbar_in[o] : T(0);
        T wb = T(0);
        if (ubar != 0.0) {
            const T x = v.x[j], wt = v.wt[j], u = (T)ubar;
            if (v.ut && v.ut[j] == 2) {
                xb += u * (wt / (x * x));  // U = -w / x
                wb = u * (-T(1) / x);
            } else if (wt > T(0)) {
                xb += u * (wt / x);
                wb = u * log(x);
            } else {
                xb += u * (-wt);
                wb = u * x;
            }
        }
        a.xb[j] = xb;
        a.wb[j] = wb;
        a.Zb[j] = T(0);
        T2 z;
        z.x = T(0);
        z.y = T(0);
        a.ab[j] = z;
    }
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < v.m; l += gridDim.x * blockDim.x) {
        a.yb[l] = T(0);
        a.zsb[l] = T(0);
        a.Rxb[l] = T(0);
        a.cb[l] = T(0);
    }
}

template <typename T>
__global__ void k_adj_export(AdjView<T> a, double* c_grad, double* w_grad) {
    const View<T>& v = a.v;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += gridDim.x * blockDim.x)
        if (w_grad) w_grad[v.perm ? v.perm[j] : j] = (double)a.wb[j];
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < v.m; l += gridDim.x * blockDim.x)
        if (c_grad) c_grad[l] = (double)a.cb[l];
}

__global__ void k_record_rho(const Ctl* ctl, double* out) { *out = ctl->rho; }

template <typename T>
__global__ void k_set_weights(View<T> v, const double* __restrict__ w) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += gridDim.x * blockDim.x) {
        const T wj = (T)w[v.perm ? v.perm[j] : j];
        T* wt = const_cast<T*>(v.wt);
        wt[j] = wt[j] > T(0) ? wj : -wj;  // the utility type rides on the sign
    }
}

int grid_for(long long count) {
    long long b = (count + kTh - 1) / kTh;
    return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

// With a few links or streams per thread slot of a resident grid (c5: 1e5 links, 1e6
// streams), a resident grid that loops was fastest; with tens (ten times c5), one block
// per 256 items up to 8192 blocks.  The switch sits between the two.
constexpr long long kFewBlocksPerSlot = 16;

template <typename K>
cudaError_t pass_grid(K kernel, long long items, long long blocks_needed, int* grid) {
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kTh, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const long long resident = (long long)occ * sms;
    if (blocks_needed > kFewBlocksPerSlot * resident) {
        *grid = grid_for(items);
        return cudaSuccess;
    }
    const long long g = resident < blocks_needed ? resident : blocks_needed;
    *grid = (int)(g < 1 ? 1 : g);
    return cudaSuccess;
}

}  // namespace

template <typename T>
cudaError_t adjoint_grids(AdjView<T>& a) {
    constexpr int kGroups = kTh / kGroup;
    cudaError_t e = pass_grid(k_adj_link<T>, (long long)a.v.m * kGroup,
                              ((long long)a.v.m + kGroups - 1) / kGroups, &a.grid_l);
    if (e != cudaSuccess) return e;
    return pass_grid(k_adj_stream<T>, a.v.n, ((long long)a.v.n + kTh - 1) / kTh, &a.grid_s);
}

template <typename T>
cudaError_t adjoint_init(const AdjView<T>& a, const double* xbar, double ubar, cudaStream_t st) {
    k_adj_init<T><<<grid_for(a.v.n > a.v.m ? a.v.n : a.v.m), kTh, 0, st>>>(a, xbar, ubar);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_step(const AdjView<T>& a, const T* x_k, const T* ps_k, const double* rho,
                         cudaStream_t st) {
    k_adj_link<T><<<a.grid_l > 0 ? a.grid_l : grid_for((long long)a.v.m * kGroup), kTh, 0, st>>>(
        a, ps_k, rho);
    k_adj_stream<T><<<a.grid_s > 0 ? a.grid_s : grid_for(a.v.n), kTh, 0, st>>>(a, x_k, rho);
    note_launches(2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_export(const AdjView<T>& a, double* c_grad, double* w_grad, cudaStream_t st) {
    k_adj_export<T><<<grid_for(a.v.n > a.v.m ? a.v.n : a.v.m), kTh, 0, st>>>(a, c_grad, w_grad);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t record_rho(const Ctl* ctl, double* out, cudaStream_t st) {
    k_record_rho<<<1, 1, 0, st>>>(ctl, out);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t set_weights(const View<T>& v, const double* w, cudaStream_t st) {
    k_set_weights<T><<<grid_for(v.n), kTh, 0, st>>>(v, w);
    note_launches(1);
    return cudaGetLastError();
}

#define PMP_ADJ_INST(T)                                                                        \
    template cudaError_t adjoint_grids<T>(AdjView<T>&);                                        \
    template cudaError_t adjoint_init<T>(const AdjView<T>&, const double*, double, cudaStream_t); \
    template cudaError_t adjoint_step<T>(const AdjView<T>&, const T*, const T*, const double*,  \
                                         cudaStream_t);                                        \
    template cudaError_t adjoint_export<T>(const AdjView<T>&, double*, double*, cudaStream_t);  \
    template cudaError_t set_weights<T>(const View<T>&, const double*, cudaStream_t);
PMP_ADJ_INST(float)
PMP_ADJ_INST(double)
#undef PMP_ADJ_INST

}  // namespace pmp
