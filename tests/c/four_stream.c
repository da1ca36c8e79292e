/* The C ABI from plain C: the four-stream example of Sec. III-A (c = 1, w = 1, log
 * utilities) solved on the device, checked against its closed-form optimum
 * x = (1, 1/3, 2/3, 2/3), prices (1, 3/2, 3/2) (KKT of Sec. II, stationarity of Sec. VI-B).
 * Then the same network twice in one batch, the second copy with doubled capacities.
 * Built by tests/test_c_abi.py with gcc against include/num_pmp.h and the library only.
 * Exit status 0 on success; a message on stderr otherwise.
 * With the argument "--no-gpu" it only exercises calls that need no device. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "num_pmp.h"

static int check(int rc, const char* what) {
    if (rc < 0) {
        fprintf(stderr, "%s: %s (%d): %s\n", what, num_strerror(rc), rc, num_last_error());
        return 1;
    }
    return 0;
}

int main(int argc, char** argv) {
    num_params p;
    num_default_params(&p);
    if (p.alpha != 1.6 || p.mu != 2.0 || p.gamma != 1.1 || p.rho_period != 50) {
        fprintf(stderr, "unexpected defaults\n");
        return 1;
    }
    if (strcmp(num_strerror(NUM_ERR_INVALID), num_strerror(NUM_OK)) == 0) {
        fprintf(stderr, "num_strerror does not tell codes apart\n");
        return 1;
    }
    /* a NULL output pointer is refused on the host, before any CUDA call */
    if (num_create(NULL, 1, 1, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL) !=
        NUM_ERR_INVALID) {
        fprintf(stderr, "NULL out accepted\n");
        return 1;
    }
    if (argc > 1 && strcmp(argv[1], "--no-gpu") == 0) return 0;

    const int64_t route_ptr[5] = {0, 1, 3, 4, 5};
    const int32_t route_links[5] = {0, 1, 2, 1, 2};
    const double c[3] = {1.0, 1.0, 1.0};
    const uint8_t utype[4] = {NUM_LOG, NUM_LOG, NUM_LOG, NUM_LOG};
    const double w[4] = {1.0, 1.0, 1.0, 1.0};
    const double hi[4] = {50.0, 50.0, 50.0, 50.0};
    num_problem* h = NULL;
    p.precision = NUM_FUSED_FP64;
    if (check(num_create(&h, 4, 3, route_ptr, route_links, c, utype, w, NULL, hi, &p, NULL),
              "num_create"))
        return 1;
    int64_t done = 0;
    const int rc = num_solve(h, 100000, 1e-10, &done);
    if (check(rc, "num_solve")) return 1;
    double x[4], lam[3], info[NUM_INFO_LEN];
    if (check(num_get(h, x, lam, info), "num_get")) return 1;
    num_destroy(h);
    const double xr[4] = {1.0, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0};
    const double lr[3] = {1.0, 1.5, 1.5};
    double err = 0.0;
    for (int j = 0; j < 4; ++j) err = fmax(err, fabs(x[j] - xr[j]));
    for (int l = 0; l < 3; ++l) err = fmax(err, fabs(lam[l] - lr[l]));
    const double obj = log(1.0) + log(1.0 / 3.0) + 2.0 * log(2.0 / 3.0);
    printf("status %d after %lld iterations, max error %.3e, objective %.12f (exact %.12f)\n",
           rc, (long long)done, err, info[NUM_INFO_OBJECTIVE], obj);
    if (rc != NUM_OK || err > 1e-8 || fabs(info[NUM_INFO_OBJECTIVE] - obj) > 1e-8) {
        fprintf(stderr, "wrong solution\n");
        return 1;
    }

    /* The same network twice in one batch, the second with every capacity doubled: with
     * log utilities its rates double and its prices halve.  The instances are passed one
     * by one (num_batch_create_instances); the first without lo, the second with lo = 0. */
    const double c2[3] = {2.0, 2.0, 2.0};
    const double lo0[4] = {0.0, 0.0, 0.0, 0.0};
    num_instance insts[2] = {
        {4, 3, route_ptr, route_links, c, utype, w, NULL, hi},
        {4, 3, route_ptr, route_links, c2, utype, w, lo0, hi},
    };
    num_batch* b = NULL;
    if (check(num_batch_create_instances(&b, 2, insts, &p, NULL), "num_batch_create_instances"))
        return 1;
    int64_t its[2];
    int32_t st[2];
    if (check(num_batch_solve(b, 100000, 1e-10, its, st), "num_batch_solve")) return 1;
    double bx[8], bl[6], binfo[2 * NUM_INFO_LEN];
    if (check(num_batch_get(b, bx, bl, binfo), "num_batch_get")) return 1;
    num_batch_destroy(b);
    double berr = 0.0;
    for (int k = 0; k < 2; ++k) {
        const double s = k == 0 ? 1.0 : 2.0;
        for (int j = 0; j < 4; ++j) berr = fmax(berr, fabs(bx[4 * k + j] - s * xr[j]));
        for (int l = 0; l < 3; ++l) berr = fmax(berr, fabs(bl[3 * k + l] - lr[l] / s));
    }
    printf("batch: status %d %d after %lld %lld iterations, max error %.3e\n", st[0], st[1],
           (long long)its[0], (long long)its[1], berr);
    if (st[0] != NUM_OK || st[1] != NUM_OK || berr > 1e-8) {
        fprintf(stderr, "wrong batch solution\n");
        return 1;
    }
    return 0;
}
