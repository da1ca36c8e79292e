// Host-side internals shared by the C-ABI sources (api.cu, adjoint_api.cu, batch_api.cu):
// the problem handle, error reporting, device allocation through the handle, the view of a
// handle's arrays that the kernels take, and handle creation.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "num_pmp.h"
#include "pmp_internal.cuh"

struct num_problem {
    int64_t n = 0, m = 0, nnz = 0;
    num_params prm{};
    num_allocator alloc{};
    bool custom_alloc = false;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;  // where the work goes
    bool own_stream = false;
    cudaEvent_t legacy_ev = nullptr;
    int device = 0;
    int prec = 0;
    struct Block {
        void* ptr;     // what the library uses: 16-byte aligned
        void* raw;     // what the allocator returned
        size_t bytes;  // what was asked of the allocator
    };
    std::vector<Block> blocks;

    int *col_ptr = nullptr, *row_idx = nullptr, *row_ptr = nullptr, *col_idx = nullptr;
    int grid_s = 0, grid_l = 0;
    int link_spread = 0;
    int* perm = nullptr;                 // caller's index of the stream at each position
    uint8_t* ut = nullptr;               // utility types, only if some stream has U = -w / x
    int4* chunks = nullptr;              // row kernels: chunks of the long links
    int* chunk_queue = nullptr;          // row kernels: the chunks, longest first
    int* long_routes = nullptr;          // row kernels: streams with long routes
    int nlong = 0;
    int nchunks = 0;
    int narrive_l = 0;                   // entries of arrive_l
    void *wt = nullptr, *lo = nullptr, *hi = nullptr, *c = nullptr;
    void *x = nullptr, *Z = nullptr, *pby = nullptr, *zs = nullptr, *Rx = nullptr, *ps = nullptr;
    void* carry_l = nullptr;   // chunk sums of the long links
    int* arrive_l = nullptr;   // chunks done per long link
    double *part_s = nullptr, *part_l = nullptr;
    int plain_nb = 0;
    void *A = nullptr, *B = nullptr, *tS = nullptr, *tR = nullptr, *tL = nullptr, *RxN = nullptr,
         *pbar = nullptr, *y = nullptr;
    pmp::Ctl* ctl = nullptr;
    pmp::Ctl* ctl_host = nullptr;
    unsigned int* dbg = nullptr;  // out-of-range gather flag of debug builds (device)  // pinned
    double* hist = nullptr;
    signed char* sched = nullptr;
    int sched_len = 0;
    double* x64 = nullptr;
    double* y64 = nullptr;
    double* part_exp = nullptr;
    int exp_blocks = 0;
    int box_uniform = 0;
    double lo_u = 0.0, hi_u = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    double last_eps_tol = 0.0;
    // profiling: evs[0] before the first kernel of a batch of iterations, then one event
    // after every kernel; per-kernel totals
    std::vector<cudaEvent_t> evs;
    double kernel_ms[pmp::kPlainKernelsPerIter] = {};
    long long kernel_runs[pmp::kPlainKernelsPerIter] = {};
    int kpi = 0;  // kernels per iteration
    // adjoint: what num_adjoint_forward keeps for num_adjoint_backward (adjoint_api.cu)
    struct AdjTape* adj = nullptr;
    long long param_gen = 0;  // changes whenever c or w change
    int* err_d = nullptr;     // device flag of the setters that take device arrays
    // set only while a taped forward run is enqueued (see View::tape_x)
    void* tape_x = nullptr;
    void* tape_ps = nullptr;
    double* tape_rho = nullptr;
    long long tape_k0 = 0;
    int tape_len = 0;
};

namespace pmp {
namespace host {

extern thread_local std::string g_last_error;  // the message num_last_error() returns

int fail(int code, const std::string& msg);           // sets the message, returns code
int cuda_fail(cudaError_t e, const char* what);        // NUM_ERR_CUDA with the CUDA error
int finish_cuda(cudaError_t e, const char* what);      // NUM_OK or cuda_fail

// NVTX range for the life of a scope: names the library's phases (create, solve, each
// replay of a graph of iterations, export, adjoint, batch calls) in profiler traces.  With
// no tool attached a range costs a pointer check.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

constexpr int kMaxGrid = 8192;
constexpr int kExportBlocksMax = 1024;

void* dev_alloc(num_problem* h, size_t bytes);  // through the handle's allocator; NULL on failure
void dev_free(num_problem* h, void* p);
void destroy_handle(num_problem* h);
void adjoint_tape_free(num_problem* h);  // the adjoint tape's host record (adjoint_api.cu)
cudaError_t order_after_legacy(num_problem* h);  // order the handle's stream after the legacy one
cudaError_t run_iterations(num_problem* h, int count);
// Iterations of each replay of check_every iterations that carry kernel events: all of
// them (profile = 1), the first (profile = 2) or none.
inline int profiled_iterations(const num_problem* h) {
    return h->prm.profile == 1 ? h->prm.check_every : (h->prm.profile == 2 ? 1 : 0);
}
cudaError_t zero_state(num_problem* h);
// NUM_OK, or in a debug build NUM_ERR_STATE if a kernel recorded an out-of-range gather
int check_debug_flag(num_problem* h);

template <typename T>
View<T> make_view(const num_problem* h) {
    View<T> v;
    std::memset(&v, 0, sizeof(v));
    v.n = (int)h->n;
    v.m = (int)h->m;
    v.nnz = (int)h->nnz;
    v.col_ptr = h->col_ptr;
    v.row_idx = h->row_idx;
    v.row_ptr = h->row_ptr;
    v.col_idx = h->col_idx;
    v.wt = (const T*)h->wt;
    v.lo = (const T*)h->lo;
    v.hi = (const T*)h->hi;
    v.lo_u = (T)h->lo_u;
    v.hi_u = (T)h->hi_u;
    v.box_uniform = h->box_uniform;
    v.c = (const T*)h->c;
    v.x = (T*)h->x;
    v.Z = (T*)h->Z;
    v.pby = (typename View<T>::T2*)h->pby;
    v.zs = (T*)h->zs;
    v.Rx = (T*)h->Rx;
    v.ps = (T*)h->ps;
    v.carry_l = (T*)h->carry_l;
    v.arrive_l = h->arrive_l;
    v.part_s = h->part_s;
    v.part_l = h->part_l;
    v.grid_s = h->grid_s;
    v.grid_l = h->grid_l;
    v.link_spread = h->link_spread;
    v.chunks = h->chunks;
    v.chunk_queue = h->chunk_queue;
    v.nchunks = h->nchunks;
    v.perm = h->perm;
    v.ut = h->ut;
    v.ctl = h->ctl;
    v.dbg = h->dbg;
    v.long_routes = h->long_routes;
    v.nlong = h->nlong;
    v.hist = h->hist;
    v.sched = h->sched;
    v.A = (T*)h->A;
    v.B = (T*)h->B;
    v.tS = (T*)h->tS;
    v.tR = (T*)h->tR;
    v.tL = (T*)h->tL;
    v.RxN = (T*)h->RxN;
    v.pbar = (T*)h->pbar;
    v.y = (T*)h->y;
    v.tape_x = (T*)h->tape_x;
    v.tape_ps = (T*)h->tape_ps;
    v.tape_rho = h->tape_rho;
    v.tape_k0 = h->tape_k0;
    v.tape_len = h->tape_len;
    return v;
}

// Instances of a batch: host arrays of count + 1 offsets into the stacked numbering.
struct BatchSpec {
    int count;
    const int64_t* stream_off;
    const int64_t* link_off;
};

int create_impl(num_problem** out, int64_t n, int64_t m, const int64_t* route_ptr,
                const int32_t* route_links, const double* c, const uint8_t* utype,
                const double* w, const double* lo, const double* hi, const num_params* p,
                void* cuda_stream, bool on_device, const BatchSpec* batch = nullptr);

}  // namespace host
}  // namespace pmp
