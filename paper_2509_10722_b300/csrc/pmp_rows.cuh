// Device pieces shared by the row kernels (rows.cu) and the batched kernels (batch.cu):
// the per-stream and per-link epilogues of one PMP iteration and the group gather-sum.
#pragma once

#include <cuda_runtime.h>

#include "pmp_device.cuh"
#include "pmp_internal.cuh"

namespace pmp {

// Per-thread residual partial sum, in FP64 in both precisions (the FP32 path forms each
// term from its FP32 iterates in FP32 and adds it in FP64; block and grid sums are FP64).
template <typename T>
struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

// Load of a gathered value: through the read-only path (kCg = false), or from L2 (kCg =
// true) when the value may have been written by another block of the same launch (the
// persistent batch kernel); the read-only path is only valid for data that no block of
// the launch writes.
template <bool kCg, typename V>
__device__ __forceinline__ V gload(const V* p) {
    if constexpr (kCg)
        return __ldcg(p);
    else
        return __ldg(p);
}

// Sum of (pbar, y) over the route entries [p, pn) of one stream, in entry order, with
// four gathers in flight.
template <typename T, bool kCg = false>
__device__ __forceinline__ typename Pair<T>::type route_sum(const int* __restrict__ row_idx,
                                                           const typename Pair<T>::type* __restrict__ pby,
                                                           int p, int pn, int m, unsigned int* dbg) {
    using V = typename Pair<T>::type;
    V sum = vzero(V());
    int e = p;
    for (; e + 4 <= pn; e += 4) {
        const int l0 = checked_index(__ldg(row_idx + e), m, dbg);
        const int l1 = checked_index(__ldg(row_idx + e + 1), m, dbg);
        const int l2 = checked_index(__ldg(row_idx + e + 2), m, dbg);
        const int l3 = checked_index(__ldg(row_idx + e + 3), m, dbg);
        const V g0 = gload<kCg>(pby + l0), g1 = gload<kCg>(pby + l1);
        const V g2 = gload<kCg>(pby + l2), g3 = gload<kCg>(pby + l3);
        sum = vadd(sum, g0);
        sum = vadd(sum, g1);
        sum = vadd(sum, g2);
        sum = vadd(sum, g3);
    }
    for (; e < pn; ++e) sum = vadd(sum, gload<kCg>(pby + checked_index(__ldg(row_idx + e), m, dbg)));
    return sum;
}

// Sum of (pbar, y) over the route entries [p, pn) of one long route, by one warp: lane k
// takes p + k, p + k + 32, ... four at a time, then a shuffle tree (a fixed order); the sum
// is complete in lane 0.
template <typename T, bool kCg = false>
__device__ __forceinline__ typename Pair<T>::type warp_route_sum(
    const int* __restrict__ row_idx, const typename Pair<T>::type* __restrict__ pby, int p, int pn,
    int lane, int m, unsigned int* dbg) {
    using V = typename Pair<T>::type;
    V s = vzero(V());
    for (int e = p + lane; e < pn; e += 128) {
        const int l0 = checked_index(__ldg(row_idx + e), m, dbg);
        const int l1 = e + 32 < pn ? checked_index(__ldg(row_idx + e + 32), m, dbg) : -1;
        const int l2 = e + 64 < pn ? checked_index(__ldg(row_idx + e + 64), m, dbg) : -1;
        const int l3 = e + 96 < pn ? checked_index(__ldg(row_idx + e + 96), m, dbg) : -1;
        const V g0 = gload<kCg>(pby + l0);
        const V g1 = l1 >= 0 ? gload<kCg>(pby + l1) : vzero(V());
        const V g2 = l2 >= 0 ? gload<kCg>(pby + l2) : vzero(V());
        const V g3 = l3 >= 0 ? gload<kCg>(pby + l3) : vzero(V());
        s = vadd(s, vadd(vadd(g0, g1), vadd(g2, g3)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, o);
        s.y += __shfl_down_sync(0xffffffffu, s.y, o);
    }
    return s;
}

// ---- stream kernel -------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T stream_epilogue(const View<T>& v, int j, typename Pair<T>::type sum,
                                             T L, T xo, T Zo, T wt, T lo, T hi, T alpha,
                                             T inv_rho, Acc<T>& acc) {
    const T Zn = alpha * L * xo + (T(1) - alpha) * Zo - alpha * sum.x;
    const T S = Zn - sum.y * inv_rho;
    const T xn = stream_prox<T>(S, L, wt, inv_rho, lo, hi, v.ut && v.ut[j] == 2);
    v.Z[j] = Zn;
    v.x[j] = xn;
    // |sigma| (x - x_prev)^2: formed in T, added in FP64
    const T dx = xn - xo;
    acc.add((double)(L * dx * dx));
    return xn;
}

template <typename T>
struct LinkState {
    typename Pair<T>::type py;
    T Rxo, pso, zso, cl;
};

template <typename T>
__device__ __forceinline__ LinkState<T> load_link(const View<T>& v, int l) {
    LinkState<T> s;
    s.py = v.pby[l];
    s.Rxo = v.Rx[l];
    s.pso = v.ps[l];
    s.zso = v.zs[l];
    s.cl = __ldg(v.c + l);
    return s;
}

// Link epilogue (slack prox, average, z and price updates) and its residual terms.
template <typename T>
__device__ __forceinline__ T link_epilogue(const View<T>& v, int l, const LinkState<T>& st,
                                           T Rxn, int deg, T alpha, T rho, T inv_rho,
                                           Acc<T>& r2, Acc<T>& s2) {
    using T2 = typename Pair<T>::type;
    const T pbo = st.py.x, y = st.py.y;
    T psn = st.zso - y * inv_rho;
    psn = psn < -st.cl ? -st.cl : psn;
    const T degf = (T)deg;
    const T pbn = (Rxn + psn) / (degf + T(1));
    T2 out;
    out.x = pbn;
    out.y = y + alpha * rho * pbn;
    v.pby[l] = out;
    v.zs[l] = alpha * (psn - pbn) + (T(1) - alpha) * st.zso;
    v.Rx[l] = Rxn;
    v.ps[l] = psn;
    // residual terms in FP64 from the iterates (the same operations as in T when T is
    // double): the three terms of the dual residual cancel as the iterates settle, so in
    // the FP32 path they are not rounded to FP32 before they are added
    // the terms in T, their sums in FP64 (forming them in FP64 as well changed the
    // residual norms by less than the FP32 rounding of the iterates does, and cost up to a
    // quarter of the link kernel's time where one lane in four or eight runs the epilogue:
    // FP64 is slow on this GPU)
    const T dpb = pbn - pbo, dRx = Rxn - st.Rxo, dd = (psn - pbn) - (st.pso - pbo);
    r2.add((double)((degf + T(1)) * pbn * pbn));
    s2.add((double)(degf * dpb * dpb - T(2) * dpb * dRx + dd * dd));
    return psn;
}

// Sum of x over entries [e0, e1) of the link-major index array, by one group of G lanes,
// in a fixed order: lane k adds the pairs (e, e + G) for e = e0 + k, e0 + k + 2G, ..., each
// pair summed first, then the shuffle tree.  kPairs pairs of gathers are in flight per
// lane; the additions keep the same order whatever kPairs is, so the result is too.
template <int G, int kPairs = 1, bool kCg = false, typename T, class Group>
__device__ __forceinline__ T group_gather_sum(const Group& g, const int* __restrict__ col_idx,
                                              const T* __restrict__ x, int e0, int e1, int n,
                                              unsigned int* dbg) {
    const int sl = g.thread_rank();
    T s = T(0);
    for (int e = e0 + sl; e < e1; e += 2 * kPairs * G) {
        int ix[2 * kPairs];
#pragma unroll
        for (int k = 0; k < 2 * kPairs; ++k)
            ix[k] = (k == 0 || e + k * G < e1) ? checked_index(__ldg(col_idx + e + k * G), n, dbg)
                                               : -1;
        T v[2 * kPairs];
#pragma unroll
        for (int k = 0; k < 2 * kPairs; ++k) v[k] = ix[k] >= 0 ? gload<kCg>(x + ix[k]) : T(0);
#pragma unroll
        for (int q = 0; q < kPairs; ++q)
            if (q == 0 || e + 2 * q * G < e1) s += v[2 * q] + v[2 * q + 1];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += g.shfl_down(s, o);
    return s;
}

// Sum of x over entries [e0, e1) by one warp: lane k takes e0 + k, e0 + k + 32, ... four
// at a time, then a shuffle tree (a fixed order).
template <typename T, bool kCg = false>
__device__ __forceinline__ T warp_gather_sum(const int* __restrict__ col_idx,
                                             const T* __restrict__ x, int e0, int e1, int lane,
                                             int n, unsigned int* dbg) {
    T s = T(0);
    for (int e = e0 + lane; e < e1; e += 128) {
        const int i0 = checked_index(__ldg(col_idx + e), n, dbg);
        const int i1 = e + 32 < e1 ? checked_index(__ldg(col_idx + e + 32), n, dbg) : -1;
        const int i2 = e + 64 < e1 ? checked_index(__ldg(col_idx + e + 64), n, dbg) : -1;
        const int i3 = e + 96 < e1 ? checked_index(__ldg(col_idx + e + 96), n, dbg) : -1;
        const T a = gload<kCg>(x + i0);
        const T b = i1 >= 0 ? gload<kCg>(x + i1) : T(0);
        const T c = i2 >= 0 ? gload<kCg>(x + i2) : T(0);
        const T d = i3 >= 0 ? gload<kCg>(x + i3) : T(0);
        s += (a + b) + (c + d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}

// Sum of the n chunk slots of one row by one warp, in a fixed order; the slots were
// written by other blocks of this launch, so they are read from L2.
template <typename T>
__device__ __forceinline__ T warp_sum_slots(const T* slots, int n, int lane) {
    T s = T(0);
    int q = lane;
    for (; q + 96 < n; q += 128)
        s += (__ldcg(slots + q) + __ldcg(slots + q + 32)) +
             (__ldcg(slots + q + 64) + __ldcg(slots + q + 96));
    for (; q < n; q += 32) s += __ldcg(slots + q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}

}  // namespace pmp
