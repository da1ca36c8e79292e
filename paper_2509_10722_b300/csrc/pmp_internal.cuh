// Internal declarations shared by the CUDA translation units of the PMP solver.
//
// State layout (the exact per-stream / per-link form of the per-terminal ADMM of
// Sec. III-D..G; see the derivation in fused.cu):
//   streams (n):  x_j rate, Z_j = sum of the link-side copies z over stream j's terminals,
//                 wt_j = +w_j (log utility) or -w_j (linear utility), box lo_j / hi_j
//   links   (m):  (pbar_l, y_l) interleaved (link average and price y = rho u),
//                 zs_l (slack terminal's z), Rx_l and ps_l of the previous iteration, c_l
// The operator R is kept twice, as 32-bit index arrays without values: CSC (routes,
// stream-major) for the stream kernel and CSR (link-major, stream ids ascending in a row)
// for the link kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace pmp {

// Iteration control block, one per handle, in device memory.  Written by the finalize step
// at the end of every iteration and read by every kernel at entry (stop flag, rho).
struct Ctl {
    double rho;        // penalty used by the next iteration
    double rnorm;      // ||r||_2 of the last iteration
    double snorm;      // ||s||_2 of the last iteration
    double eps_tol;    // stop when both norms are below it; <= 0 disables the test
    double alpha, mu, gamma;
    double objective;  // sum U_j(x_j), written by the objective reduction
    long long k;       // iterations done since creation / reset
    long long k_limit; // the run stops when k reaches it
    long long n_updates;  // rho update points passed
    int stop;          // 0 running, 1 converged, 2 iteration limit, 3 non-finite residual
    int period;        // rho update period (0 = never)
    int sched_len;     // entries of the forced rho schedule
    int hist_len;      // entries of the residual ring buffer
    unsigned int ticket;  // last-block-done counter of the link kernel
    unsigned int ticket2; // last-block-done counter of the reductions
    unsigned int chunk_next;  // the link kernel's queue of long-link chunks: next to take
};

enum Stop { RUNNING = 0, CONVERGED = 1, LIMIT = 2, NONFINITE = 3 };

// Debug builds (-DPMP_DEBUG_BOUNDS, `build.py --debug`): every gathered index is checked
// against the length of the vector it indexes; one out of range is recorded in *dbg (the
// solve then returns NUM_ERR_STATE) and replaced by 0, so the access stays inside the
// vector.  Release builds compile the check away.
__device__ __forceinline__ int checked_index(int i, int bound, unsigned int* dbg) {
#ifdef PMP_DEBUG_BOUNDS
    if ((unsigned)i >= (unsigned)bound) {
        atomicOr(dbg, 1u);
        return 0;
    }
#else
    (void)bound;
    (void)dbg;
#endif
    return i;
}

// Row kernels (rows.cu): a link with more than kLongRow streams is summed by whole warps
// in chunks of kChunk entries (one chunk per warp; 256 and 2048 measured best on a
// Zipf(1.1) instance); persistent grids are capped at kMaxRowsGrid blocks.
constexpr int kLongRow = 256;
constexpr int kChunk = 2048;
// Row kernels: a stream whose route has more than kLongRoute links is summed by a whole warp
// (a list built at setup), so that a few long routes do not hold up the stream kernel.
constexpr int kLongRoute = 32;
constexpr int kMaxRowsGrid = 8192;

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// Everything a fused or plain kernel needs, passed by value.
template <typename T>
struct View {
    using T2 = typename Pair<T>::type;
    int n, m, nnz;
    const int* col_ptr;         // CSC [n+1]
    const int* row_idx;         // CSC [nnz] link of each route entry
    const int* row_ptr;         // CSR [m+1]
    const int* col_idx;         // CSR [nnz] stream of each link entry
    const T* wt;                // signed weights
    const T* lo;                // per-stream box (unused when box_uniform)
    const T* hi;
    T lo_u, hi_u;
    int box_uniform;
    const T* c;
    T* x;
    T* Z;
    T2* pby;                    // (pbar, y)
    T* zs;
    T* Rx;
    T* ps;
    T* carry_l;                 // row kernels: chunk sums of the long links
    int* arrive_l;              // row kernels: chunks done per long link
    double* part_s;             // per-block residual partials of the stream kernel [grid_s]
    double* part_l;             // ... of the link kernel [2 * grid_l]
    int grid_s, grid_l;
    int link_spread;            // row link kernel: 1 (many links per group: the epilogues of a
                                // group's links spread over its lanes) or 0 (few: one group
                                // per link, its leader runs the epilogue)
    const int4* chunks;         // row kernels: (link, first entry, end entry, first chunk)
    const int* chunk_queue;     // row link kernel: chunk indices in the order its queue hands
                                // them out (the longest first)
    int nchunks;
    const int* perm;            // caller's index of the stream at each position (or NULL)
    const uint8_t* ut;          // utility type per stream, only when some stream has type 2
    Ctl* ctl;
    double* hist;
    const signed char* sched;
    // plain FP64 path only
    T* A;                       // sum of pbar over each route
    T* B;                       // sum of y over each route
    T* tS;                      // per-stream dual-residual term
    T* tR;                      // per-link primal-residual term
    T* tL;                      // per-link dual-residual term
    T* RxN;                     // this iteration's R x
    T* pbar;                    // split arrays of the plain path
    T* y;
    unsigned int* dbg;  // debug builds: set when a gathered index was out of range
    const int* long_routes;  // row kernels: streams with more than kLongRoute links
    int nlong;
    // adjoint tape (row kernels; NULL tape_x: not taping): iteration k0 + i + 1 writes its
    // x to tape_x[i n ..], its slack flows to tape_ps[i m ..] and the rho it used to
    // tape_rho[i], for 0 <= i < tape_len
    T* tape_x;
    T* tape_ps;
    double* tape_rho;
    long long tape_k0;
    int tape_len;
};

// ---- launchers ---------------------------------------------------------------------------------
// One iteration on stream st (rows.cu: the fused FP32 / FP64 kernels; plain.cu: the FP64
// baseline).  If evs is not NULL, evs[q] is recorded on st right after the q-th kernel of
// the iteration (for per-kernel timing), as an external event so that it is a real
// event-record node when the launch is captured into a graph.
cudaError_t plain_iteration(const View<double>& v, int plain_blocks, cudaStream_t st,
                            cudaEvent_t* evs);
constexpr int kFusedKernelsPerIter = 2;

// ---- batched kernels (batch.cu) ---------------------------------------------------------------
struct BatchGlobal {
    unsigned int ticket;  // last-block-done counter of the export kernel
    int running;          // number of instances still running
    int timeout;          // persistent kernel: 1 once a bounded wait of some block ran out
    int timeout_block;    // the block whose wait ran out first
    unsigned int chunk_next;  // batch link kernel: next position in the chunk queue
};

// Work items are (instance, first row, end row, 0); item ranges of instance i are
// [sitem_off[i], sitem_off[i+1]) and [litem_off[i], litem_off[i+1]).
template <typename T>
struct BatchView {
    View<T> v;  // the stacked (block-diagonal) problem's arrays
    Ctl* ctls;  // one control block per instance
    BatchGlobal* glob;
    const int4* sitems;
    const int4* litems;
    int nsitems, nlitems;
    // balanced partitions: block b takes items [sblk[b], sblk[b+1]) (and lblk for the link
    // kernel); NULL: block b takes items b, b + gridDim.x, ...
    const int* sblk;
    const int* lblk;
    const int* sitem_off;
    const int* litem_off;
    int count;
    double* part_s;  // [nsitems]
    double* part_l;  // [2 nlitems]
    double* hist;    // [count][max(hist_len, 1)][3]
    const signed char* sched;  // [count][sched_stride]
    int sched_stride;
    unsigned int* arrive;  // [count] link items (and chunked links) of the instance done
    int lanes;             // lanes per link in the link kernel: 4, 8, 16 or 32
    // links of more than kLongRow streams, summed by whole warps in chunks (the stacked
    // problem's chunk table; chunks never cross an instance)
    const int4* chunks;    // [nchunks] (link, first entry, end entry, first chunk of link)
    int nchunks;
    const int* chunk_inst; // [nchunks] instance of each chunk
    const int* coff;       // [count + 1] chunk range of each instance
    const int* crows;      // [count] chunked links of each instance
    T* carry;              // [nchunks] chunk sums
    int* arrive_c;         // [nchunks] chunks of a link done (at its first chunk)
    double* part_c;        // [2 nchunks] residual terms of a chunked link (at its first chunk)
    // streams with more than kLongRoute links (v.long_routes, in stream order), one warp each
    const int* lr_inst;    // [v.nlong] instance of each
    const int* lroff;      // [count + 1] range of each instance in the list
    double* part_r;        // [v.nlong] residual term of each
    // persistent form (batch_persistent.cu): each instance has a team of blocks
    const int* soff;       // [count + 1] stream range of each instance
    const int* loff;       // [count + 1] link range of each instance
    const int4* teams;     // [tasks] (instance, rank in its team, team size, team's first block)
    const int2* btasks;    // [grid] each block's range of tasks (first, count)
    double* part_t;        // [3 grid] per-block residual partials: s2 of streams, r2, s2 of links
    unsigned int* bar;     // [2 count] per-instance team barrier: arrivals, generation
    long long wait_polls;  // polls of a barrier wait before it gives up
    int iters;             // iterations per launch
};

// Profiling event after a kernel: an external event node while the stream is being
// captured into a graph (so that replays record it), a plain record otherwise.
inline cudaError_t record_kernel_event(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
               : cudaEventRecord(ev, st);
}

cudaError_t batch_grids(int precision, int lanes, int nsitems, int nlitems, int nchunks,
                        int* grid_s, int* grid_l, int* grid_e);
// Resident blocks of the two batch kernels (occupancy x SMs), the grids of a balanced
// partition.
cudaError_t batch_resident(int precision, int lanes, int* blocks_s, int* blocks_l);
// Persistent form: the most blocks of the persistent kernel that can be resident at once
// (the bound of a cooperative launch), and one cooperative launch of it.
cudaError_t batch_persistent_capacity(int precision, int lanes, bool split, int* blocks);
template <typename T>
cudaError_t batch_persistent_launch(const BatchView<T>& b, int grid, cudaStream_t st);
cudaError_t check_blocks(int count, const int64_t* stream_off, const int64_t* link_off,
                         long long n, const int64_t* route_ptr, const int* route_links, int* err,
                         cudaStream_t st);
// In place on the device: route_ptr[1..n] and route_links[0..nnz) of instances copied
// one after the other, each in its own numbering, shifted to the stacked numbering (so,
// lo, eo: device int64[count + 1] offsets of the streams, links and entries).
cudaError_t stack_offsets(int count, const int64_t* so, const int64_t* lo, const int64_t* eo,
                          int64_t* route_ptr, int* route_links, long long n, long long nnz,
                          cudaStream_t st);
template <typename T>
cudaError_t batch_iteration(const BatchView<T>& b, int grid_s, int grid_l, cudaStream_t st,
                            cudaEvent_t* evs);
template <typename T>
cudaError_t batch_export(const BatchView<T>& b, int grid_e, double* x_out, double* y_out,
                         double* part, cudaStream_t st);
cudaError_t batch_arm(Ctl* ctls, BatchGlobal* glob, int count, long long max_iters,
                      double eps_abs, const double* eps_scale, cudaStream_t st);
cudaError_t batch_reset(Ctl* ctls, BatchGlobal* glob, int count, double rho0, double alpha,
                        double mu, double gamma, int period, int hist_len, int sched_len,
                        cudaStream_t st);

// ---- adjoint (adjoint.cu) -----------------------------------------------------------------------
template <typename T>
struct AdjView {
    View<T> v;
    double alpha;
    T* xb;                        // x_bar [n]
    T* Zb;                        // Z'_bar [n]
    typename Pair<T>::type* ab;   // (Abar, Bbar) per stream [n]
    T* yb;                        // y_bar [m]
    T* zsb;                       // zs_bar [m]
    T* Rxb;                       // Rx_bar [m]
    T* cb;                        // dJ/dc [m]
    T* wb;                        // dJ/dw [n]
    typename Pair<T>::type* abc;  // [v.nchunks] chunk sums of (Abar, Bbar) of long links
    int grid_l, grid_s;           // grids of the two passes (by adjoint_grids)
};
// Grids of the backward link and stream passes (their blocks loop over links and streams):
// the blocks that fit on the GPU at once when each thread slot has a few items, else one
// block per 256 items up to 8192.
template <typename T>
cudaError_t adjoint_grids(AdjView<T>& a);
template <typename T>
// x_bar = xbar (caller order, may be NULL) + ubar U'(x); w_bar = ubar dU/dw; others zero.
cudaError_t adjoint_init(const AdjView<T>& a, const double* xbar, double ubar, cudaStream_t st);
template <typename T>
cudaError_t adjoint_step(const AdjView<T>& a, const T* x_k, const T* ps_k, const double* rho,
                         cudaStream_t st);
template <typename T>
cudaError_t adjoint_export(const AdjView<T>& a, double* c_grad, double* w_grad, cudaStream_t st);
cudaError_t record_rho(const Ctl* ctl, double* out, cudaStream_t st);
template <typename T>
cudaError_t set_weights(const View<T>& v, const double* w, cudaStream_t st);

// ---- row kernels (rows.cu) ------------------------------------------------------------------
// Grids of the two row kernels, and the link kernel's variant: link_spread = 0 when each
// group has few links to sum (one group per link, the leader runs the epilogue), else 1
// (a group sums 8 consecutive links and each lane runs one epilogue); the sums are the
// same either way.
cudaError_t rows_grids(int precision, int n, int m, int nchunks, int* grid_s, int* grid_l,
                       int* link_spread);
template <typename T>
cudaError_t rows_iteration(const View<T>& v, cudaStream_t st, cudaEvent_t* evs);
// Chunk table of the links with more than kLongRow streams: counts[m+1] and offs[m+1] are
// caller scratch, tmp is scan scratch of scan_tmp_len(m + 1) ints; *nchunks (host) is the
// number of chunks; chunks (may be NULL on the counting call) receives them.
cudaError_t count_chunks(const int* row_ptr, int m, int* counts, int* offs, int* tmp,
                         int* nchunks, cudaStream_t st);
cudaError_t count_long_routes(const int* col_ptr, int n, int* flags, int* offs, int* tmp,
                              int* nlong, cudaStream_t st);
cudaError_t fill_long_routes(const int* col_ptr, int n, const int* offs, int* list,
                             cudaStream_t st);
cudaError_t fill_chunks(const int* row_ptr, int m, const int* offs, int4* chunks,
                        cudaStream_t st);
constexpr int kPlainKernelsPerIter = 8;

// Process-wide count of kernel launches made by this library (graph replays count every
// kernel node they run).
void note_launches(long long count);
long long launches();

// Set the calling thread's num_last_error() message; returns code.
int report_error(int code, const std::string& msg);
int report_cuda_error(cudaError_t e, const char* what);  // NUM_ERR_CUDA
void clear_error();
int plain_partial_blocks(int n, int m);

// ---- operator and state (operator.cu) -------------------------------------------------------
// Error bits of the device-side validation.
enum ValidationBits {
    VB_ROUTE = 1,     // route_ptr not increasing (an empty route) or not starting at 0
    VB_LINK_ID = 2,   // link id outside [0, m)
    VB_DUPLICATE = 4, // a link twice in one route
    VB_CAPACITY = 8,  // c not finite or <= 0
    VB_WEIGHT = 16,   // w not finite or <= 0
    VB_UTYPE = 32,    // utility type not 0 or 1
    VB_BOX = 64,      // lo / hi not finite, lo > hi, or hi <= 0 for a log stream
    VB_BLOCKS = 128,  // batch: a route uses a link of another instance
};

struct Scratch {  // transient buffers of the operator build, caller-allocated
    int* keys_a; int* vals_a; int* keys_b; int* vals_b;
    int* hist;     // radix histogram / scan buffer
    int* scan_tmp; // block sums of the scans
    size_t hist_len, scan_tmp_len;
};

size_t radix_hist_len(int nnz);
size_t scan_tmp_len(size_t len);
// Order of the long-link chunk queue: queue[nchunks] receives the chunk indices by
// decreasing chunk length, equal lengths in chunk order (a stable radix sort in s).
cudaError_t order_chunks(const int4* chunks, int nchunks, const Scratch& s, int* queue,
                         cudaStream_t st);

// Validate the inputs in two parts, so that the routes can be checked and the operator
// built while the other arrays are still being copied: the routes (route_ptr increasing
// from 0, link ids in [0, m); nnz = route_ptr[n], read on the host), then the values
// (weights, types, boxes, capacities).  *err_bits (device int) accumulates
// ValidationBits, err_bits[1] is set when some stream has U = -w / x, and box_minmax
// (device unsigned long long[4]) receives order-preserving keys of min lo, max lo, min hi,
// max hi.
cudaError_t validate_routes(int n, int m, long long nnz, const int64_t* route_ptr,
                            const int* route_links, int* err_bits, cudaStream_t st);
// *err |= 1 if some a[i], i < count, is not finite and > 0 (device array).
cudaError_t validate_positive(int count, const double* a, int* err, cudaStream_t st);
cudaError_t validate_values(int n, int m, const double* c, const uint8_t* utype,
                            const double* w, const double* lo, const double* hi, int* err_bits,
                            unsigned long long* box_minmax, cudaStream_t st);
// Order the streams by the first link of their route (stable): perm[j] = caller's index of
// the stream placed at position j; route_ptr_new / route_links_new receive the routes in
// that order.  lens and ptr32 are int[n+1] scratch, scan_tmp holds scan_tmp_len(n + 1).
cudaError_t relabel_streams(int n, int m, const int64_t* route_ptr, const int* route_links,
                            const Scratch& s, int* perm, int* lens, int* ptr32, int* scan_tmp,
                            int64_t* route_ptr_new, int* route_links_new, cudaStream_t st);
// Build the CSC int32 pointer, and the CSR (row_ptr, col_idx) by a stable device radix sort.
// Also flags duplicates (VB_DUPLICATE) into err_bits.
cudaError_t build_operator(int n, int m, int nnz, const int64_t* route_ptr,
                           const int* route_links, int* col_ptr, int* row_idx, int* row_ptr,
                           int* col_idx, const Scratch& s, int* err_bits, cudaStream_t st);
// Convert parameters to the iteration precision (stream arrays in relabeled order).
template <typename T>
cudaError_t convert_params(int n, int m, const double* c, const uint8_t* utype,
                           const double* w, const double* lo, const double* hi, const int* perm,
                           T* c_t, T* wt_t, T* lo_t, T* hi_t, cudaStream_t st,
                           uint8_t* ut_out = nullptr);
double ordered_key_to_double(unsigned long long k);
// x (T) -> double copies; objective partials and its FP64 reduction into ctl->objective.
template <typename T>
cudaError_t export_solution(const View<T>& v, double* x_out, double* y_out, double* part,
                            int part_blocks, cudaStream_t st);
int export_partial_blocks(int n);
// One state array between the device iterate and an FP64 device buffer in the caller's
// order: which = 0 x, 1 Z (streams), 2 pbar, 3 y, 4 zs, 5 Rx, 6 ps (links).
template <typename T>
cudaError_t state_transfer(const View<T>& v, int which, double* buf, bool out, cudaStream_t st);

// Small control kernels.
cudaError_t ctl_arm(Ctl* ctl, long long k_limit, double eps_tol, cudaStream_t st);
cudaError_t ctl_reset(Ctl* ctl, double rho0, double alpha, double mu, double gamma, int period,
                      int hist_len, cudaStream_t st);
cudaError_t ctl_set_schedule_len(Ctl* ctl, int len, cudaStream_t st);

}  // namespace pmp
