/*
 * num_pmp.h -- C ABI of the B300 (sm_103a) proximal message passing (PMP) solver for
 * network utility maximization.
 *
 * Problem (Sec. II, Eq. vanilla_num):   maximize  sum_j U_j(x_j)
 *                                       subject to R x <= c,  lo_j <= x_j <= hi_j,
 * with the 0/1 link-route matrix R (R_lj = 1 iff stream j uses link l), capacities c > 0,
 * and U_j(x) = w_j log x (NUM_LOG), w_j x (NUM_LINEAR) or -w_j / x (NUM_ALPHA2), w_j > 0.
 * The box is the
 * "indicator of a convex set" of Sec. II; lo = 0 gives the paper's x >= 0.
 *
 * Method: the ADMM form of Sec. III-D (prox device updates, link averages, scaled price
 * updates) with the residuals and stopping test of Sec. III-F and the residual balancing
 * (Eq. rho-update, Eq. dual-rescale) and over-relaxation of Sec. III-G.  The library runs
 * it on one GPU in hand-written CUDA kernels; the per-terminal state of the paper is kept
 * in the exactly equivalent per-stream / per-link form (Z_j = sum of the link-side copies
 * over stream j's terminals; one price y_l = rho u_l per link).
 *
 * Conventions for every function below:
 *   - return value: NUM_OK (0) on success, NUM_NOT_CONVERGED (1) from num_solve when the
 *     iteration limit came first (the state is valid), or a negative NUM_ERR_* code;
 *     num_last_error() then holds a one-line message for the calling thread;
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of
 *     the device that was current when the handle was created;
 *   - the caller owns every array it passes; the library copies what it keeps during
 *     num_create* and never retains a caller pointer;
 *   - one handle must not be used from two threads at once; separate handles are
 *     independent.  All work of a handle is ordered on the CUDA stream given at creation.
 */
#ifndef NUM_PMP_H
#define NUM_PMP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NUM_API __attribute__((visibility("default")))
#else
#define NUM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define NUM_OK 0
#define NUM_NOT_CONVERGED 1
#define NUM_ERR_INVALID (-1) /* bad argument or malformed instance (see num_create) */
#define NUM_ERR_OOM (-2)     /* a device allocation failed */
#define NUM_ERR_CUDA (-3)    /* a CUDA runtime call failed; num_last_error() names it */
#define NUM_ERR_NUMERIC (-4) /* a residual became non-finite; iteration stopped */
#define NUM_ERR_STATE (-5)   /* call not valid for this handle's state */
#define NUM_ERR_TIMEOUT (-6) /* persistent batch: a bounded wait between blocks ran out */

/* ---- utility types (Sec. III-B) ------------------------------------------------------------ */
#define NUM_LOG 0    /* U(x) = w log x, the log-utility stream */
#define NUM_LINEAR 1 /* U(x) = w x, the linear-utility stream */
#define NUM_ALPHA2 2 /* U(x) = -w / x, alpha = 2 fairness ("minimum potential delay", the
                        example of Sec. II of a utility with a simple prox) */

/* ---- kernel path / precision --------------------------------------------------------------- */
#define NUM_FUSED_FP32 0 /* two fused kernels per iteration; FP32 iterates, FP64 residuals,
                            FP64 stopping test and rho */
#define NUM_FUSED_FP64 1 /* the same fused kernels with FP64 iterates */
#define NUM_PLAIN_FP64 2 /* unfused baseline: one kernel per step (SpMV, elementwise prox,
                            SpMV-transpose, reductions), all FP64 */

/* Optional device allocator.  alloc returns device memory of `bytes` bytes usable on
 * `stream` (NULL on failure, which num_create reports as NUM_ERR_OOM); release frees it.
 * The kernels need 16-byte aligned blocks: a block that is not is handed back at once and
 * asked again 16 bytes larger (release then receives that block and size). */
typedef struct {
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void (*release)(void* ctx, void* ptr, size_t bytes, void* stream);
    void* ctx;
} num_allocator;

/* Solver parameters; num_default_params() fills the paper's values.
 *   rho0        initial penalty rho (the paper does not state it; default 1.0)
 *   alpha       over-relaxation parameter, Sec. III-G (default 1.6)
 *   mu, gamma   residual-balancing threshold and factor, Eq. rho-update (2.0, 1.1)
 *   eps_abs     absolute tolerance; the run stops when ||r||_2 and ||s||_2 are both below
 *               eps_abs * sqrt(J), J = nnz(R) + m terminals, Sec. III-F (default 1e-4)
 *   rho_period  iterations between rho updates (default 50; 0 = never update)
 *   precision   NUM_FUSED_FP32 (default), NUM_FUSED_FP64 or NUM_PLAIN_FP64; FP32
 *               iterates reach eps_abs down to about 1e-7 (measured at n = 1e7), tighter
 *               tolerances need an FP64 path
 *   check_every iterations per CUDA-graph replay between two host reads of the stop flag
 *               (default 50); iterations after the stop inside a replay do nothing
 *   history     length of the on-device ring buffer of (||r||, ||s||, rho) per iteration
 *               (default 4096; 0 = none)
 *   use_graph   1 (default): replay captured CUDA graphs; 0: plain launches
 *   reorder     1 (default): place streams in the order of the first link of their route
 *               (stable), so that streams sharing that link are adjacent and the gathers
 *               of both kernels share L2 sectors; results are reported in the caller's
 *               order; 0: keep the caller's order
 *   profile     1: record a CUDA event on the handle's stream after every kernel of every
 *               iteration (inside the replayed graphs) and accumulate per-kernel device
 *               times, read with num_get_kernel_times; 2: the same for the first
 *               iteration of every replay of check_every iterations only (a sample that
 *               costs 1 / check_every of the events); 0 (default): no events
 *   allocator   NULL (default): cudaMalloc / cudaFree */
typedef struct {
    double rho0;
    double alpha;
    double mu;
    double gamma;
    double eps_abs;
    int32_t rho_period;
    int32_t precision;
    int32_t check_every;
    int32_t history;
    int32_t use_graph;
    int32_t reorder;
    int32_t profile;
    const num_allocator* allocator;
} num_params;

typedef struct num_problem num_problem; /* opaque; owns all of its device memory */

/* Fill *p with the defaults listed above.  Never fails. */
NUM_API void num_default_params(num_params* p);

/* Create a solver handle for one NUM instance, from HOST arrays.
 *   n, m         number of traffic streams and of links, both >= 1
 *   route_ptr    int64[n+1], route_ptr[0] = 0, nondecreasing: stream j uses the links
 *                route_links[route_ptr[j] .. route_ptr[j+1]-1] (R in CSC form, Sec. II)
 *   route_links  int32[nnz], nnz = route_ptr[n] < 2^31 - m; link ids in [0, m), no link
 *                twice in one route, every route nonempty (a stream has >= 1 terminal)
 *   c            double[m], capacities, finite and > 0
 *   utype        uint8[n], NUM_LOG, NUM_LINEAR or NUM_ALPHA2
 *   w            double[n], weights, finite and > 0
 *   lo, hi       double[n] box of each rate, finite, lo <= hi, hi > 0 for log and alpha2;
 *                lo may be NULL (all zero)
 *   p            parameters (NULL = defaults)
 *   cuda_stream  cudaStream_t to order all work on (NULL = the legacy default stream)
 * Scalar and pointer checks happen on the host before any CUDA call (NUM_ERR_INVALID);
 * the per-element checks run on the device and are reported as NUM_ERR_INVALID too.
 * Copies the arrays host-to-device, builds the link-major (CSR) copy of R on the device,
 * and zeroes the iteration state (x = z = u = 0, rho = rho0).  Synchronizes the stream.
 * On success *out owns the handle (free it with num_destroy); on failure *out = NULL. */
NUM_API int num_create(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
               const int32_t* route_links, const double* c, const uint8_t* utype,
               const double* w, const double* lo, const double* hi, const num_params* p,
               void* cuda_stream);

/* As num_create, with every array argument a DEVICE pointer (same layout, same rules).
 * The arrays are read in the order of cuda_stream: work the caller queued on that stream
 * before the call (for example, what fills the arrays) completes first.  The arrays of
 * num_create are host memory and are read when the call is made. */
NUM_API int num_create_device(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
                      const int32_t* route_links, const double* c, const uint8_t* utype,
                      const double* w, const double* lo, const double* hi,
                      const num_params* p, void* cuda_stream);

/* Force the rho decision of the first `count` update points (host array, copied):
 * decisions[i] = +1 (rho *= gamma), 0 (keep) or -1 (rho /= gamma) at iteration
 * (i+1) * rho_period; later update points follow Eq. rho-update again.  count = 0 clears
 * the schedule.  Used to compare runs of different precision along one trajectory. */
NUM_API int num_set_rho_schedule(num_problem* h, const int8_t* decisions, int64_t count);

/* Run at most max_iters (>= 0) further PMP iterations, stopping at the first iteration
 * whose residuals pass the test of Sec. III-F with tolerance eps_abs:
 *   eps_abs > 0   use it;   eps_abs < 0   use the handle's parameter;
 *   eps_abs == 0  never stop on the test (run exactly max_iters iterations).
 * *iters_done (may be NULL) receives the iterations run by this call.  Returns NUM_OK when
 * the test passed, NUM_NOT_CONVERGED when max_iters came first, NUM_ERR_NUMERIC on a
 * non-finite residual.  Continues from the current state; synchronizes the stream. */
NUM_API int num_solve(num_problem* h, int64_t max_iters, double eps_abs, int64_t* iters_done);

/* Copy the current solution to HOST buffers (each may be NULL):
 *   x       double[n]  stream rates
 *   prices  double[m]  link prices lambda = rho u = y (Sec. III-D: u = y / rho)
 *   info    double[NUM_INFO_LEN], see NUM_INFO_* (objective sum_j U_j(x_j) in FP64) */
NUM_API int num_get(const num_problem* h, double* x, double* prices, double* info);

/* As num_get with x and prices DEVICE pointers (info stays a host pointer). */
NUM_API int num_get_device(const num_problem* h, double* x, double* prices, double* info);

#define NUM_INFO_PRIMAL 0    /* ||r||_2 of the last iteration */
#define NUM_INFO_DUAL 1      /* ||s||_2 of the last iteration */
#define NUM_INFO_EPS_TOL 2   /* eps_abs * sqrt(J) of the last solve */
#define NUM_INFO_RHO 3       /* current rho */
#define NUM_INFO_OBJECTIVE 4 /* sum_j U_j(x_j) at the current x, FP64 */
#define NUM_INFO_ITERS 5     /* iterations run since creation / reset */
#define NUM_INFO_STATUS 6    /* 0 running, 1 converged, 2 iteration limit, 3 non-finite */
#define NUM_INFO_J 7         /* number of terminals nnz + m */
#define NUM_INFO_LEN 8

/* Copy up to max_rows rows (||r||, ||s||, rho) of the residual history, oldest first, into
 * the HOST array hist[3 * max_rows]; *rows receives the count (<= the history length). */
NUM_API int num_get_history(const num_problem* h, double* hist, int64_t max_rows, int64_t* rows);

/* Copy the device-built link-major form of R to HOST arrays: row_ptr int64[m+1] and
 * col_idx int32[nnz] (each row's stream ids ascending).  For checking the device build. */
NUM_API int num_get_operator(const num_problem* h, int64_t* row_ptr, int32_t* col_idx);

/* Replace the link capacities (HOST double[m], finite and > 0) and keep the iterate, so
 * that the next num_solve continues from the current point: the warm start after a
 * capacity degradation of Sec. V-D.  num_reset first for a cold start instead. */
NUM_API int num_set_capacity(num_problem* h, const double* c);

/* The iterate, as HOST doubles (each pointer may be NULL): per stream, in the caller's
 * order, x[n] and Z[n] (sum over the stream's terminals of the link-side copies z); per
 * link pbar[m] (link average), y[m] (price = rho u), zs[m] (the slack terminal's z),
 * Rx[m] (R x of the last iteration), ps[m] (the slack terminal's flow); *rho. */
NUM_API int num_get_state(const num_problem* h, double* x, double* Z, double* pbar, double* y,
                          double* zs, double* Rx, double* ps, double* rho);

/* Start a fresh run (iteration 0, empty history) from the given iterate and rho (> 0);
 * arrays as in num_get_state, a NULL array leaves that part of the current iterate as is.
 * Used to warm-start a modified instance (for example one pruned after link failures,
 * Sec. V-D) from another instance's solution. */
NUM_API int num_set_state(num_problem* h, const double* x, const double* Z, const double* pbar,
                          const double* y, const double* zs, const double* Rx, const double* ps,
                          double rho);

/* Replace the utility weights (HOST double[n], caller order, finite and > 0); the utility
 * types and the iterate are kept. */
NUM_API int num_set_weights(num_problem* h, const double* w);

/* num_set_capacity and num_set_weights with DEVICE arrays (double[m], double[n] in the
 * caller's order), read on the handle's stream after the caller's prior work on the legacy
 * default stream; the values are checked on the device (NUM_ERR_INVALID, nothing changed,
 * if one is not finite and > 0).  Synchronizes the handle's stream. */
NUM_API int num_set_capacity_device(num_problem* h, const double* c);
NUM_API int num_set_weights_device(num_problem* h, const double* w);

/* Reverse-mode derivative of `iters` PMP iterations run from the zero state (the map from
 * (c, w) to the rates x after exactly `iters` iterations, each iteration's rho fixed at the
 * value this forward run takes): for the cotangent xbar (HOST double[n], caller order, or
 * NULL) plus, if objective = 1, the total utility J = sum_j U_j(x_j) (its gradient in x
 * and its direct dependence on w), writes dJ/dc to c_grad (HOST double[m]) and dJ/dw to
 * w_grad (HOST double[n], caller order), each may be NULL, and the total utility
 * sum_j U_j(x_j) at the final rates (whatever `objective` is) to *objective_out (may be
 * NULL).  The derivative runs the adjoint of every step backwards: transposed gathers over
 * R and the Jacobians of the stream prox (zero at the box bounds) and of the slack prox.
 * It keeps the full iterate every checkpoint_every iterations (0: only at the start) and
 * recomputes each segment but the last (the iteration is deterministic; the last one is
 * recorded by the forward run itself), storing x and the slack flow of each iteration of
 * the segment: device memory about checkpoint_every * (n + m) values +
 * (iters / checkpoint_every) iterates.  checkpoint_every = 0 (one segment) recomputes
 * nothing, at the cost of iters * (n + m) stored values.  A set rho
 * schedule applies to the forward run.  The handle is left at the forward result. */
NUM_API int num_adjoint(num_problem* h, int64_t iters, int32_t checkpoint_every,
                        const double* xbar, int32_t objective, double* c_grad, double* w_grad,
                        double* objective_out);

/* The two halves of num_adjoint, for callers that run the forward map once and
 * differentiate it later (an autograd framework's forward and backward).
 * num_adjoint_forward runs `iters` iterations from the zero state exactly as num_adjoint
 * does (checkpoints every checkpoint_every iterations, the last segment recorded on the
 * way) and keeps what the derivative needs in device memory owned by the handle, until
 * num_adjoint_release, the next num_adjoint_forward or num_adjoint, or num_destroy.  The
 * handle is left at the result of the run (num_get / num_get_device read x and the total
 * utility).  Synchronizes the handle's stream. */
NUM_API int num_adjoint_forward(num_problem* h, int64_t iters, int32_t checkpoint_every);

/* dJ/dc and dJ/dw of the kept forward run for J = <xbar, x> + ubar * sum_j U_j(x_j):
 * xbar (DEVICE double[n], caller order, or NULL) and ubar (a finite scalar, 0 for no
 * utility term; not both absent) are the cotangents of the final rates and of the total
 * utility; c_grad (DEVICE double[m]) and w_grad (DEVICE double[n], caller order) receive
 * the gradients (each may be NULL).  Runs on the handle's stream after the caller's prior
 * work on the legacy default stream and synchronizes it.  Each segment but the one held
 * in memory is recomputed from its checkpoint; the call may be repeated (each repeat
 * recomputes every segment but the first).  NUM_ERR_STATE if no forward is kept or if the
 * capacities or weights changed since it ran.  The handle is left at the forward
 * result. */
NUM_API int num_adjoint_backward(num_problem* h, const double* xbar, double ubar,
                                 double* c_grad, double* w_grad);

/* Free the device memory kept by num_adjoint_forward (nothing kept: no effect). */
NUM_API int num_adjoint_release(num_problem* h);

/* Zero the iteration state and history (x = z = u = 0, rho = rho0, iteration 0). */
NUM_API int num_reset(num_problem* h);

/* Algorithmic bytes of one iteration, for roofline accounting: what the two fused kernels
 * must move (every index array once, every state array read and written once, each
 * gathered vector once).  out[0] = stream kernel, out[1] = link kernel (host doubles). */
NUM_API int num_iteration_bytes(const num_problem* h, double* out);

/* Per-kernel device time of the profiled iterations run so far (profile = 1 or 2).
 * Kernel q of an iteration (fused paths: 0 = stream kernel, 1 = link kernel; plain path:
 * 0 SpMV-transpose, 1 stream prox, 2 SpMV, 3 link update, 4-6 reductions, 7 finalize):
 * ms[q] = total milliseconds between the event before and the event after it,
 * launches[q] = how many of its timed launches did work (launches after the stop flag
 * was set are not counted).
 * Fills min(max_kernels, kernels per iteration) entries of the HOST arrays; *nkernels
 * receives the number of kernels per iteration. */
NUM_API int num_get_kernel_times(const num_problem* h, double* ms, int64_t* launches,
                                 int32_t max_kernels, int32_t* nkernels);

/* Number of kernel launches this library has made in this process so far (every kernel
 * node of a replayed graph counts as one launch). */
NUM_API int64_t num_kernel_launches(void);

/* Total utility sum_j U_j(x_j) (U = w log x for utype 0, -w / x for 2, w x otherwise) of
 * caller DEVICE arrays x[n], utype[n], w[n], written in FP64 to the caller's DEVICE double
 * *objective; no handle, and NO ALLOCATION of any kind.  The paper has no counterpart.
 * For callers that cannot allocate device memory when they need the number (allocation
 * locked by a host framework's memory pool, a real-time loop where cudaMalloc's implicit
 * synchronization is not allowed, a fixed memory budget): the block partials live in a
 * static device array of the library (32 KB, held on every GPU that loads the library
 * until the process exits), so n is limited to 33,554,432; larger n is rejected with
 * NUM_ERR_INVALID and a message.  The first call on each device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  The address is kept for the life of the process: it assumes
 * one CUDA context per device throughout (after cudaDeviceReset and a new context, this
 * entry point would launch into the old context's address).  Work is enqueued on
 * cuda_stream (NULL = the legacy default stream) without synchronizing.  All calls share
 * the array: calls that overlap on the GPU (other streams or host threads) race and give
 * wrong sums; calls ordered on one stream are safe.  Inputs are not validated on the
 * device: a utype other than NUM_LOG (0) or NUM_ALPHA2 (2) counts as NUM_LINEAR here
 * (num_create rejects such values).  A non-sticky CUDA error left on this host thread by
 * an earlier runtime call is cleared on entry, so an error reported by this call is its
 * own. */
NUM_API int num_objective_noalloc(int64_t n, const double* x, const uint8_t* utype,
                                  const double* w, double* objective, void* cuda_stream);

/* Measured rate of uniformly random reads on the current device, in reads per second,
 * written to the HOST double *gathers_per_s.  Both passes of an iteration (Sec. III-D) read
 * one value per route entry at positions set by the routes (x per stream in the link pass,
 * the (pbar, y) pair per link in the stream pass); on random routes these reads, one
 * 32-byte memory sector each, bound the iteration more tightly than HBM bandwidth.  This
 * call measures that ceiling: `count` reads (1 .. 2e9) of 4-byte (vec_bytes = 4) or
 * 8-byte (vec_bytes = 8) elements at uniformly random positions of a vector of vec_len
 * elements (1 .. 2^31 - 1), four independent reads in flight per thread at full
 * occupancy, repeated `repeats` times (1 .. 1000) after one warm-up pass, timed with CUDA
 * events.  Allocates count * 4 + vec_len * vec_bytes bytes of device memory with
 * cudaMalloc for the duration of the call (NUM_ERR_OOM if that fails) and synchronizes its
 * own stream.  The paper has no counterpart; it is a measurement service. */
NUM_API int num_measure_gather_rate(int64_t count, int64_t vec_len, int32_t vec_bytes,
                                    int32_t repeats, double* gathers_per_s);

/* As num_measure_gather_rate, with plain stores of 4- or 8-byte values to the random
 * positions instead of reads: the rate at which a kernel could push each value to a
 * permuted copy (to be read back contiguously) instead of gathering it.  Written to the
 * HOST double *stores_per_s.  The paper has no counterpart; it is a measurement service. */
NUM_API int num_measure_scatter_rate(int64_t count, int64_t vec_len, int32_t vec_bytes,
                                     int32_t repeats, double* stores_per_s);

/* Free every resource of the handle.  NULL is ignored. */
NUM_API void num_destroy(num_problem* h);

/* ---- batches of independent instances --------------------------------------------------- */
/* Many NUM instances of uneven sizes solved together on one GPU: two kernel launches per
 * iteration for the whole batch, each instance with its own rho, iteration count and
 * stopping test (Sec. III-F, III-G); an instance that stops is skipped by later
 * iterations.  Batches are a service of this library (the paper solves one instance at a
 * time). */
typedef struct num_batch num_batch; /* opaque; owns all of its device memory */

/* Create a batch from HOST arrays.  The instances are stacked in one numbering: instance i
 * owns streams [stream_off[i], stream_off[i+1]) and links [link_off[i], link_off[i+1])
 * (int64[count+1] each, starting at 0, strictly increasing: every instance has >= 1 stream
 * and >= 1 link).  route_ptr / route_links / c / utype / w / lo / hi describe the stacked
 * problem exactly as for num_create, with GLOBAL link ids; every route of instance i must
 * use links of instance i only (else NUM_ERR_INVALID).  p->precision must be
 * NUM_FUSED_FP32 or NUM_FUSED_FP64 and p->schedule the row kernels; all instances share
 * the other parameters.  Synchronizes the stream. */
NUM_API int num_batch_create(num_batch** out, int32_t count, const int64_t* stream_off,
                             const int64_t* link_off, const int64_t* route_ptr,
                             const int32_t* route_links, const double* c,
                             const uint8_t* utype, const double* w, const double* lo,
                             const double* hi, const num_params* p, void* cuda_stream);

/* One instance of a batch, as HOST arrays in the layout of num_create (its own link ids
 * 0..m-1; lo may be NULL for lo = 0). */
typedef struct {
    int64_t n, m;
    const int64_t* route_ptr; /* n + 1, route_ptr[0] = 0 */
    const int32_t* route_links;
    const double* c;
    const uint8_t* utype;
    const double* w;
    const double* lo; /* or NULL */
    const double* hi;
} num_instance;

/* Create a batch from `count` separate instances (HOST array insts[count]), as
 * num_batch_create would from their block-diagonal stack, without the caller stacking
 * them: the arrays of each instance are copied to their place in the stacked device arrays
 * and the link ids and route offsets are shifted there, on the device.  Instance i then
 * owns the streams and links that follow those of instances 0..i-1.  The same checks,
 * parameters and results as num_batch_create; the caller keeps ownership of every array.
 * Synchronizes the stream. */
NUM_API int num_batch_create_instances(num_batch** out, int32_t count, const num_instance* insts,
                                       const num_params* p, void* cuda_stream);

/* Force the first len rho decisions of every instance: decisions[i * len + q] is the
 * decision of instance i at its q-th update point (-1, 0, +1; host array, copied). */
NUM_API int num_batch_set_rho_schedules(num_batch* b, const int8_t* decisions, int64_t len);

/* Work partition of a batch's two kernels.  stream_item = 0 (balanced): the stacked
 * streams are cut into one range of equal length per resident block of the stream
 * kernel, and each range again where an instance ends; otherwise every instance's
 * streams are cut into work items of stream_item consecutive streams, which the blocks
 * take in turn.  link_item likewise for the links, where a balanced range holds an equal
 * share of route entries (plus a fixed weight per link for its epilogue).  In the link
 * kernel link_lanes lanes sum R x of one link.  The default is {0, 0, 8}.  The partition
 * does not change the arithmetic of a stream or a link, except that link_lanes fixes the
 * order of the additions of (R x)_l; the residual norms are summed per item, so their
 * last bits follow the partition as well. */
typedef struct {
    int32_t stream_item; /* 0, or a power of two in [256, 65536] */
    int32_t link_item;   /* 0, or a power of two in [32, 8192] */
    int32_t link_lanes;  /* 4, 8, 16 or 32 */
} num_batch_schedule;

/* The partition in use (HOST struct). */
NUM_API int num_batch_get_schedule(const num_batch* b, num_batch_schedule* out);

/* Use partition *s from the next solve on (NUM_ERR_INVALID outside the ranges above).  The
 * iterates are kept; a captured graph is rebuilt.  Synchronizes the stream. */
NUM_API int num_batch_set_schedule(num_batch* b, const num_batch_schedule* s);

/* Autotuner of the partition: times candidate partitions on this batch and keeps the
 * fastest.  Stage 1 tries stream_item in {0, 512, 1024, 2048, 4096, 8192} with the link
 * side unchanged and keeps the one with the least stream-kernel time; stage 2 tries
 * link_item in {0, 64, 128, 256, 512, 1024} times link_lanes in {4, 8, 16, 32} and keeps the least
 * link-kernel time (ties: the earlier candidate).  Each candidate runs 2 untimed and
 * trial_iters (1 .. 500) timed iterations of every instance without a stopping test;
 * kernel times are CUDA events around each kernel.  Afterwards the chosen partition is in
 * use and the batch is RESET (state zero, iteration counts zero, rho = rho0, history
 * cleared): call it after num_batch_create and before solving.  *chosen (HOST, may be
 * NULL) receives the partition.  trial_ms (HOST, 4 * max_trials doubles, may be NULL with
 * max_trials = 0) receives, per candidate in the order tried, (stream_item, link_item,
 * link_lanes, milliseconds of the kernel that stage compares); *ntrials (may be NULL) the
 * number of candidates tried (30).  Synchronizes the stream.  The choice follows measured
 * times, so two calls can choose differently, and with a different link_lanes the
 * results differ in the last bits (see num_batch_schedule); pass the chosen partition to
 * num_batch_set_schedule to reproduce a run. */
NUM_API int num_batch_autotune(num_batch* b, int32_t trial_iters, num_batch_schedule* chosen,
                               double* trial_ms, int32_t max_trials, int32_t* ntrials);

/* Run at most max_iters further iterations of every instance (eps_abs as in num_solve,
 * with eps_tol = eps_abs sqrt(J_i) per instance).  iters_done[count] and status[count]
 * (host arrays, may be NULL) receive each instance's iterations and NUM_OK /
 * NUM_NOT_CONVERGED / NUM_ERR_NUMERIC.  Returns NUM_OK if every instance converged,
 * NUM_NOT_CONVERGED if some hit the limit, NUM_ERR_NUMERIC if some residual became
 * non-finite.  Synchronizes the stream. */
NUM_API int num_batch_solve(num_batch* b, int64_t max_iters, double eps_abs,
                            int64_t* iters_done, int32_t* status);

/* Host copies of the stacked solution: x[total n], prices[total m] (each may be NULL) and
 * info[count * NUM_INFO_LEN], one NUM_INFO_* record per instance (may be NULL). */
NUM_API int num_batch_get(const num_batch* b, double* x, double* prices, double* info);

/* As num_get_kernel_times, for the batch's two kernels (profile = 1 or 2). */
NUM_API int num_batch_get_kernel_times(const num_batch* b, double* ms, int64_t* launches,
                                       int32_t max_kernels, int32_t* nkernels);

/* Persistent form of num_batch_solve (enable = 1; 0 returns to the default form of two
 * launches per iteration replayed from a CUDA graph).  Each num_batch_solve then runs the
 * instances with cooperative launches of one persistent kernel, check_every iterations per
 * launch.  Before each launch the instances still running are planned onto the GPU's
 * resident blocks: with the smallest load bound per block that fits, an instance of more
 * work owns a team of blocks and smaller ones are packed several to a block (run in turn).
 * A team steps through its instance's iterations on its own, its blocks meeting at two
 * barriers per iteration (after the stream pass, and at the end of the iteration, where
 * the team's first block runs the stopping test and rho rule of Sec. III-F / III-G).  The iterates equal those of the
 * default form for the same rho decisions (the arithmetic of a stream or a link is the
 * same); the FP64 residual sums are grouped differently.  Every wait is bounded: a block
 * gives up after wait_polls polls of its barrier (wait_polls = 0: about 2^22 polls, roughly
 * a second), records it, and returns, as do in turn the other blocks of its team;
 * num_batch_solve then returns NUM_ERR_TIMEOUT, the iterates are undefined, and every
 * further solve returns NUM_ERR_STATE until num_batch_reset.  Per-kernel times (profile)
 * are not recorded in this form.  The
 * paper solves one instance at a time; batches are a service of this library. */
NUM_API int num_batch_set_persistent(num_batch* b, int32_t enable, int64_t wait_polls);

/* Every instance back to the zero state of creation (rho0, no iterations, empty residual
 * history); clears the broken state left by a NUM_ERR_TIMEOUT.  Synchronizes the stream. */
NUM_API int num_batch_reset(num_batch* b);

/* Free every resource of the batch.  NULL is ignored. */
NUM_API void num_batch_destroy(num_batch* b);

/* Static text for a status code. */
NUM_API const char* num_strerror(int code);

/* Message of the last failing call on this thread ("" if none). */
NUM_API const char* num_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NUM_PMP_H */
