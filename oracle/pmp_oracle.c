/*
 * Plain FP64 CPU oracle of proximal message passing (PMP) for network utility maximization.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this file's library.  The product (the CUDA path) never calls it and shares
 * no code, header, table or helper with it.
 *
 * It is deliberately the slow, literal form of the method: it stores one flow p_t, one
 * link-side copy z_t and one scaled dual u_t for EVERY terminal t of the bipartite
 * stream/link graph (Sec. III, J = nnz(R) + m terminals), and runs the ADMM steps of
 * Sec. III-D with the residual balancing and over-relaxation of Sec. III-G, in the order
 * the paper states them:
 *
 *   1. stream prox      p_sigma = prox_{f_sigma,rho}(z_sigma - u_sigma)   (Sec. III-D, III-E)
 *   2. link average     pbar_l  = mean of p over the terminals of l       (Sec. III-D)
 *   3. relaxation       p+      = alpha p + (1 - alpha) z                 (Sec. III-G)
 *   4. z update         z_l     = projection of (p+ + u)_l onto 1'z_l = 0 (argmin of g_l, Sec. III-D)
 *   5. u update         u_l    += p+_l - z_l                              (Sec. III-D)
 *   6. residuals        r = pbar, s = rho ((p - pbar) - (p - pbar)_prev)  (Sec. III-F)
 *   7. stopping test    ||r|| < eps_abs sqrt(J) and ||s|| < eps_abs sqrt(J)   (Sec. III-F)
 *   8. every `period` iterations: Eq. (rho-update), then u <- (rho_old / rho_new) u
 *                                                                        (Eq. dual-rescale)
 *
 * Readings where the paper is silent or ambiguous:
 *   - the prox argument is z - u (the ADMM form); the paper's "p - pbar - u" is the same
 *     thing without over-relaxation;
 *   - log and linear prox are clipped to the stream's box [lo, hi] (the utility includes an
 *     indicator of a convex set, Sec. II); clipping the unconstrained 1-D minimizer is exact
 *     for a convex 1-D problem;
 *   - the log root is evaluated as (S + sqrt(D)) / (2|sigma|) when S >= 0 and as
 *     (2 w / rho) / (sqrt(D) - S) when S < 0 (the same number, without cancellation);
 *   - all state starts at zero; p_prev and pbar_prev are zero before the first iteration;
 *   - the rho step uses the residuals of the iteration just finished and is taken only if
 *     the stopping test failed.
 *
 * Compile-time ORACLE_PLANT = k (k >= 1) plants one known mistake in this file; the test
 * suite compiles those variants to show that its pins catch each of them.  A normal build
 * leaves ORACLE_PLANT undefined.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

typedef struct {
    double rho0;       /* initial penalty (not stated by the paper; 1.0 by default) */
    double alpha;      /* over-relaxation, Sec. III-G: 1.6 */
    double mu;         /* residual-balancing threshold, Eq. (rho-update): 2 */
    double gamma;      /* residual-balancing factor, Eq. (rho-update): 1.1 */
    double eps_abs;    /* absolute tolerance, Sec. III-F; <= 0 disables the stopping test */
    int64_t period;    /* iterations between rho updates: 50 */
    int64_t max_iters;
    int32_t debug;     /* 1: check the ADMM identities after every iteration */
    int64_t switch_iter;     /* > 0: capacities become c_switch after this many iterations */
    const double* c_switch;  /* new capacities (a degraded network, Sec. V-D), or NULL */
} oracle_params;

/* ---- proximal operators, Sec. III-E ---------------------------------------------------- */

static double clip(double v, double lo, double hi) {
    if (v < lo) v = lo;
    if (v > hi) v = hi;
    return v;
}

/* argmin_x  -w log x + (rho/2) sum_t (x - zeta_t)^2 over the box, with S = sum_t zeta_t and
 * L = number of terminals: the positive root of rho L x^2 - rho S x - w = 0, clipped. */
double oracle_prox_log(double S, double L, double w, double rho, double lo, double hi) {
#if ORACLE_PLANT == 18
    L = 1.0;
#endif
    double D = S * S + 4.0 * w * L / rho;
    double x;
#if ORACLE_PLANT == 1
    x = (S - sqrt(D)) / (2.0 * L);
#else
    if (S >= 0.0)
        x = (S + sqrt(D)) / (2.0 * L);
    else
        x = (2.0 * w / rho) / (sqrt(D) - S);
#endif
#if ORACLE_PLANT == 13
    return x;
#else
    return clip(x, lo, hi);
#endif
}

/* argmin_x  -w x + (rho/2) sum_t (x - zeta_t)^2 over the box: (S + w / rho) / L, clipped. */
double oracle_prox_linear(double S, double L, double w, double rho, double lo, double hi) {
#if ORACLE_PLANT == 2
    double x = (S - w / rho) / L;
#else
    double x = (S + w / rho) / L;
#endif
    return clip(x, lo, hi);
}

/* argmin_x  w / x + (rho/2) sum_t (x - zeta_t)^2 over x > 0 and the box: the utility
 * U = -w / x of alpha = 2 fairness ("minimum potential delay", named in Sec. II as a
 * utility with a simple prox, Sec. III-B).  The stationarity condition is the cubic
 * f(x) = rho L x^3 - rho S x^2 - w = 0, which has exactly one positive root; it lies in
 * (0, max(S, 0) / L + cbrt(w / (rho L))] (f is negative at 0 and non-negative at the right
 * end), and is found here by bisection down to the last representable bracket. */
double oracle_prox_alpha2(double S, double L, double w, double rho, double lo, double hi) {
    double a = 0.0, b = (S > 0.0 ? S / L : 0.0) + cbrt(w / (rho * L));
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (a + b);
        if (mid <= a || mid >= b) break;
#if ORACLE_PLANT == 14
        const double f = rho * L * mid * mid * mid + rho * S * mid * mid - w;
#else
        const double f = rho * L * mid * mid * mid - rho * S * mid * mid - w;
#endif
        if (f > 0.0)
            b = mid;
        else
            a = mid;
    }
#if ORACLE_PLANT == 17
    (void)lo;
    (void)hi;
    return 0.5 * (a + b);
#else
    return clip(0.5 * (a + b), lo, hi);
#endif
}

/* argmin_p  I{p + c >= 0} + (rho/2)(p - zeta)^2 = max(zeta, -c). */
double oracle_prox_slack(double zeta, double c) {
#if ORACLE_PLANT == 3
    return zeta < -c ? zeta : -c;
#else
    return zeta > -c ? zeta : -c;
#endif
}

/* ---- the solver ------------------------------------------------------------------------ */

/*
 * Inputs follow the problem statement of Sec. II: R given by its routes (CSC, stream-major),
 * capacities c, utility type (0 log, 1 linear, 2 alpha = 2 fairness), weight w and box
 * [lo, hi] per stream.
 * rho_replay (optional, length rho_replay_len) forces the decision of the i-th rho update
 * (-1 divide by gamma, 0 keep, +1 multiply by gamma) instead of Eq. (rho-update).
 *
 * Outputs: x[n], slack[m] (s = p + c of each slack stream, Sec. III-D), lambda[m] = rho u,
 * hist[3 * max_iters] = (||r||, ||s||, rho used in the iteration) per iteration,
 * decisions[max_iters / period] (the rho decision taken at each update point),
 * *iters (iterations run), *converged (1 if the stopping test passed),
 * *identity_violation (debug: the largest violation of the ADMM identities).
 * Returns 0, or -1 on bad input / allocation failure.
 */
int oracle_solve(int64_t n, int64_t m, const int64_t* route_ptr, const int32_t* route_links,
                 const double* c, const uint8_t* utype, const double* w, const double* lo,
                 const double* hi, const oracle_params* prm, const int8_t* rho_replay,
                 int64_t rho_replay_len, double* x_out, double* slack_out, double* lambda_out,
                 double* hist, int8_t* decisions, int64_t* iters, int32_t* converged,
                 double* identity_violation) {
    if (n < 1 || m < 1 || route_ptr[0] != 0) return -1;
    const int64_t nnz = route_ptr[n];
    const int64_t J = nnz + m;                 /* terminals: traffic ones, then one slack per link */

    /* link of every terminal; terminals of every link (counting sort, link-major) */
    int64_t* link_of = (int64_t*)malloc(sizeof(int64_t) * J);
    int64_t* link_cnt = (int64_t*)calloc(m + 1, sizeof(int64_t));
    int64_t* link_start = (int64_t*)malloc(sizeof(int64_t) * (m + 1));
    int64_t* link_terms = (int64_t*)malloc(sizeof(int64_t) * J);
    double* p = (double*)calloc(J, sizeof(double));
    double* z = (double*)calloc(J, sizeof(double));
    double* u = (double*)calloc(J, sizeof(double));
    double* pplus = (double*)calloc(J, sizeof(double));
    double* p_prev = (double*)calloc(J, sizeof(double));
    double* pbar = (double*)calloc(m, sizeof(double));
    double* pbar_prev = (double*)calloc(m, sizeof(double));
    int64_t* fill = (int64_t*)calloc(m, sizeof(int64_t));
    if (!link_of || !link_cnt || !link_start || !link_terms || !p || !z || !u || !pplus ||
        !p_prev || !pbar || !pbar_prev || !fill) {
        free(link_of); free(link_cnt); free(link_start); free(link_terms); free(p); free(z);
        free(u); free(pplus); free(p_prev); free(pbar); free(pbar_prev); free(fill);
        return -1;
    }
    for (int64_t t = 0; t < nnz; ++t) link_of[t] = route_links[t];
    for (int64_t l = 0; l < m; ++l) link_of[nnz + l] = l;
    for (int64_t t = 0; t < J; ++t) link_cnt[link_of[t]]++;
    link_start[0] = 0;
    for (int64_t l = 0; l < m; ++l) link_start[l + 1] = link_start[l] + link_cnt[l];
    for (int64_t t = 0; t < J; ++t) {
        int64_t l = link_of[t];
        link_terms[link_start[l] + fill[l]++] = t;
    }

    const double alpha = prm->alpha;
    const double tol = prm->eps_abs * sqrt((double)J);
    double rho = prm->rho0;
    int64_t k = 0, n_updates = 0;
    int32_t conv = 0;
    double worst = 0.0;

    for (k = 1; k <= prm->max_iters; ++k) {
        /* capacity change between two iterations (warm start after degradation, Sec. V-D):
         * the slack streams' cost uses the new c from here on, the iterate is kept */
        if (prm->c_switch && prm->switch_iter > 0 && k == prm->switch_iter + 1) c = prm->c_switch;
        /* 1. stream prox: traffic streams, then slack streams */
        for (int64_t s = 0; s < n; ++s) {
            double S = 0.0;
            for (int64_t t = route_ptr[s]; t < route_ptr[s + 1]; ++t) S += z[t] - u[t];
            double L = (double)(route_ptr[s + 1] - route_ptr[s]);
            double xs = utype[s] == 0   ? oracle_prox_log(S, L, w[s], rho, lo[s], hi[s])
                        : utype[s] == 2 ? oracle_prox_alpha2(S, L, w[s], rho, lo[s], hi[s])
                                        : oracle_prox_linear(S, L, w[s], rho, lo[s], hi[s]);
            for (int64_t t = route_ptr[s]; t < route_ptr[s + 1]; ++t) p[t] = xs;
        }
        for (int64_t l = 0; l < m; ++l) {
            int64_t t = nnz + l;
            p[t] = oracle_prox_slack(z[t] - u[t], c[l]);
        }
        /* 2. link averages over all |l| = deg_l + 1 terminals */
        for (int64_t l = 0; l < m; ++l) {
            double sum = 0.0;
            for (int64_t i = link_start[l]; i < link_start[l + 1]; ++i) sum += p[link_terms[i]];
#if ORACLE_PLANT == 4
            double cnt = (double)(link_cnt[l] > 1 ? link_cnt[l] - 1 : 1);
#else
            double cnt = (double)link_cnt[l];
#endif
            pbar[l] = sum / cnt;
        }
        /* 3. over-relaxation */
        for (int64_t t = 0; t < J; ++t) {
#if ORACLE_PLANT == 5
            pplus[t] = (1.0 - alpha) * p[t] + alpha * z[t];
#else
            pplus[t] = alpha * p[t] + (1.0 - alpha) * z[t];
#endif
        }
        /* 4. z update: project v = p+ + u of each link onto {sum of the link's entries = 0} */
        for (int64_t l = 0; l < m; ++l) {
            double sum = 0.0;
            int64_t cnt = 0;
            for (int64_t i = link_start[l]; i < link_start[l + 1]; ++i) {
                int64_t t = link_terms[i];
#if ORACLE_PLANT == 12
                if (t >= nnz) continue;
#endif
                sum += pplus[t] + u[t];
                cnt++;
            }
            double mean = cnt ? sum / (double)cnt : 0.0;
            for (int64_t i = link_start[l]; i < link_start[l + 1]; ++i) {
                int64_t t = link_terms[i];
                z[t] = pplus[t] + u[t] - mean;
            }
        }
        /* 5. scaled dual update */
        for (int64_t t = 0; t < J; ++t) {
#if ORACLE_PLANT == 6
            u[t] += p[t] - z[t];
#else
            u[t] += pplus[t] - z[t];
#endif
        }
        /* 6. residuals over all J terminals */
        double r2 = 0.0, s2 = 0.0;
        for (int64_t t = 0; t < J; ++t) {
            double pb = pbar[link_of[t]];
#if ORACLE_PLANT == 8
            if (t < nnz) continue;
#endif
            r2 += pb * pb;
        }
        for (int64_t t = 0; t < J; ++t) {
            int64_t l = link_of[t];
#if ORACLE_PLANT == 15
            double d = p[t] - pbar[l];
#else
            double d = (p[t] - pbar[l]) - (p_prev[t] - pbar_prev[l]);
#endif
            s2 += d * d;
        }
        double rnorm = sqrt(r2);
#if ORACLE_PLANT == 7
        double snorm = sqrt(s2);
#else
        double snorm = rho * sqrt(s2);
#endif
        if (hist) {
            hist[3 * (k - 1) + 0] = rnorm;
            hist[3 * (k - 1) + 1] = snorm;
            hist[3 * (k - 1) + 2] = rho;
        }
        if (prm->debug) {
            /* u constant over each link's terminals; z sums to zero over each link */
            for (int64_t l = 0; l < m; ++l) {
                double u0 = u[link_terms[link_start[l]]];
                double zs = 0.0, scale = 1.0;
                for (int64_t i = link_start[l]; i < link_start[l + 1]; ++i) {
                    int64_t t = link_terms[i];
                    double du = fabs(u[t] - u0);
                    if (du > worst) worst = du;
                    zs += z[t];
                    if (fabs(z[t]) > scale) scale = fabs(z[t]);
                }
                double dz = fabs(zs) / scale;
                if (dz > worst) worst = dz;
            }
        }
        /* 7. stopping test */
#if ORACLE_PLANT == 11
        const double tol_used = prm->eps_abs;
#else
        const double tol_used = tol;
#endif
        if (prm->eps_abs > 0.0 && rnorm < tol_used && snorm < tol_used) {
            conv = 1;
            break;
        }
        /* 8. residual balancing every `period` iterations, then the dual rescale */
#if ORACLE_PLANT == 16
        if (prm->period > 0 && k > 1 && (k - 1) % prm->period == 0) {
#else
        if (prm->period > 0 && k % prm->period == 0) {
#endif
            int8_t dec;
            if (rho_replay && n_updates < rho_replay_len) {
                dec = rho_replay[n_updates];
            } else {
#if ORACLE_PLANT == 9
                dec = (snorm > prm->mu * rnorm) ? 1 : (rnorm > prm->mu * snorm) ? -1 : 0;
#else
                dec = (rnorm > prm->mu * snorm) ? 1 : (snorm > prm->mu * rnorm) ? -1 : 0;
#endif
            }
            if (decisions) decisions[n_updates] = dec;
            n_updates++;
            double rho_new = dec > 0 ? rho * prm->gamma : dec < 0 ? rho / prm->gamma : rho;
            if (rho_new != rho) {
#if ORACLE_PLANT == 10
                double ratio = rho_new / rho;
#else
                double ratio = rho / rho_new;
#endif
                for (int64_t t = 0; t < J; ++t) u[t] *= ratio;
                rho = rho_new;
            }
        }
        /* 9. keep this iterate for the next dual residual */
        memcpy(p_prev, p, sizeof(double) * J);
        memcpy(pbar_prev, pbar, sizeof(double) * m);
    }
    if (k > prm->max_iters) k = prm->max_iters;

    /* recover the NUM solution: x from any terminal of the stream, s = p + c of the slack
     * stream (Sec. III-D), lambda = rho u of any terminal of the link (y = rho u) */
    for (int64_t s = 0; s < n; ++s) x_out[s] = p[route_ptr[s]];
    for (int64_t l = 0; l < m; ++l) {
        if (slack_out) slack_out[l] = p[nnz + l] + c[l];
        if (lambda_out) lambda_out[l] = rho * u[nnz + l];
    }
    *iters = k;
    *converged = conv;
    if (identity_violation) *identity_violation = worst;

    free(link_of); free(link_cnt); free(link_start); free(link_terms); free(p); free(z);
    free(u); free(pplus); free(p_prev); free(pbar); free(pbar_prev); free(fill);
    return 0;
}
