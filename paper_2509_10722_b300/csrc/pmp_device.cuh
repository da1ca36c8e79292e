// Inline device helpers shared by the kernels of the PMP solver (header-only so that each
// translation unit gets its own copy without relocatable device code).
#pragma once

#include <cuda_runtime.h>

#include "pmp_internal.cuh"

namespace pmp {

// ---- small vector arithmetic on the gathered types --------------------------------------------
__device__ __forceinline__ float vzero(float) { return 0.f; }
__device__ __forceinline__ double vzero(double) { return 0.0; }
__device__ __forceinline__ float2 vzero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 vzero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}

// ---- reductions --------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block, valid in thread 0.  Fixed order (deterministic).  `red` holds
// at least blockDim.x / 32 doubles.  Contains __syncthreads.
__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

// Sums of K values over the block at once, valid in thread 0: each value reduced exactly
// as block_sum would (the same order, so the same bits), with two barriers in all instead
// of two per value.  `red` holds at least K * blockDim.x / 32 doubles.
template <int K>
__device__ __forceinline__ void block_sum_n(double (&v)[K], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * nw + warp] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        if (threadIdx.x == 0)
            for (int i = 0; i < nw; ++i) s += red[k * nw + i];
        v[k] = s;
    }
}

// Sum over the block of a[0..count) of a global array (strided per thread, then a block
// reduction), bypassing L1 so values written by other blocks of the same launch are seen.
__device__ __forceinline__ double block_sum_global(const double* a, int count, int stride,
                                                   double* red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += __ldcg(a + (size_t)i * stride);
    return block_sum(s, red);
}

// The grid's residual sums at the end of an iteration, in one pass: the link blocks'
// (r2, s2) pairs part_l[2 * grid_l] and the stream blocks' s2 part_s[grid_s].  Each sum
// takes the same per-thread order as block_sum_global, so the same bits.  Results valid
// in thread 0; `red` holds at least 3 * blockDim.x / 32 doubles.
__device__ __forceinline__ void grid_residual_sums(const double* part_l, int grid_l,
                                                   const double* part_s, int grid_s,
                                                   double* red, double& r2, double& s2l,
                                                   double& s2s) {
    double v[3] = {0.0, 0.0, 0.0};
    const int count = grid_l > grid_s ? grid_l : grid_s;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        if (i < grid_l) {
            v[0] += __ldcg(part_l + 2 * (size_t)i);
            v[1] += __ldcg(part_l + 2 * (size_t)i + 1);
        }
        if (i < grid_s) v[2] += __ldcg(part_s + i);
    }
    block_sum_n<3>(v, red);
    r2 = v[0];
    s2l = v[1];
    s2s = v[2];
}

// ---- the end-of-iteration step -----------------------------------------------------------------
// Given the complete sums r2 = ||r||^2 and s2 = ||s||^2 / rho^2 of this iteration: the
// residual norms of Sec. III-F, the stopping test ||r|| < eps_tol and ||s|| < eps_tol,
// and every `period` iterations the residual balancing of Eq. rho-update (or the forced
// schedule); the dual rescale of Eq. dual-rescale is implicit because prices are stored
// unscaled (y = rho u).  Single thread.
__device__ __forceinline__ void finalize_iteration(Ctl* ctl, double r2, double s2,
                                                   double* hist, const signed char* sched) {
    const double rho = ctl->rho;
    const long long k = ctl->k + 1;
    const double rn = sqrt(r2 > 0.0 ? r2 : 0.0);
    const double sn = rho * sqrt(s2 > 0.0 ? s2 : 0.0);
    ctl->rnorm = rn;
    ctl->snorm = sn;
    ctl->k = k;
    if (ctl->hist_len > 0) {
        double* h = hist + 3 * ((k - 1) % ctl->hist_len);
        h[0] = rn;
        h[1] = sn;
        h[2] = rho;
    }
    int stop = RUNNING;
    if (!isfinite(rn) || !isfinite(sn)) {
        stop = NONFINITE;
    } else if (ctl->eps_tol > 0.0 && rn < ctl->eps_tol && sn < ctl->eps_tol) {
        stop = CONVERGED;
    } else {
        if (ctl->period > 0 && k % ctl->period == 0) {
            int dec;
            if (ctl->n_updates < ctl->sched_len)
                dec = sched[ctl->n_updates];
            else
                dec = rn > ctl->mu * sn ? 1 : (sn > ctl->mu * rn ? -1 : 0);
            ctl->n_updates += 1;
            if (dec > 0)
                ctl->rho = rho * ctl->gamma;
            else if (dec < 0)
                ctl->rho = rho / ctl->gamma;
        }
        if (k >= ctl->k_limit) stop = LIMIT;
    }
    ctl->stop = stop;
}

// ---- proximal operators of Sec. III-E in the iteration precision --------------------------------
// Stream prox: the minimizer over [lo, hi] of -U(x) + (rho/2) sum_t (x - zeta_t)^2, which
// depends on zeta only through S = sum_t zeta_t.  wt > 0: U = wt log x, the positive root
// of rho L x^2 - rho S x - wt = 0 (evaluated without cancellation for S < 0); wt < 0:
// U = |wt| x, x = (S + |wt| / rho) / L; alpha2: U = -wt / x (alpha = 2 fairness), the one
// positive root of L x^3 - S x^2 - wt / rho = 0.  inv_rho = 1 / rho.
template <typename T>
__device__ __forceinline__ T alpha2_root(T S, T L, T c0) {
    // Newton from the right end of the bracket (0, max(S, 0)/L + cbrt(c0 / L)]: f is convex
    // and increasing to the right of the root, so the iterates decrease monotonically to
    // it; stop when they stop decreasing (at most 64 steps)
    T x = (S > T(0) ? S / L : T(0)) + cbrt(c0 / L);
    for (int it = 0; it < 64; ++it) {
        const T f = (L * x - S) * x * x - c0;
        const T fp = (T(3) * L * x - T(2) * S) * x;
        const T xn = x - f / fp;
        if (!(xn < x)) break;
        x = xn;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T stream_prox(T S, T L, T wt, T inv_rho, T lo, T hi,
                                         bool alpha2 = false) {
    T xn;
    if (alpha2) {
        xn = alpha2_root<T>(S, L, wt * inv_rho);
    } else if (wt > T(0)) {
        const T wr = wt * inv_rho;
        const T D = S * S + T(4) * wr * L;
        const T sq = sqrt(D);
        xn = S >= T(0) ? (S + sq) / (T(2) * L) : (T(2) * wr) / (sq - S);
    } else {
        xn = (S - wt * inv_rho) / L;
    }
    xn = xn < lo ? lo : xn;  // comparisons (not fmin/fmax) so that a NaN propagates
    return xn > hi ? hi : xn;
}

}  // namespace pmp
