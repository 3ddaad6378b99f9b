// Host side and kernels of the C ABI declared in include/tabsimplex.h: the
// dense full-tableau simplex of arXiv 2211.10979 (Section III), one GPU.
//
// Kernels:
//   k_validate       checks the device inputs (finite, b >= 0) before a build
//   k_build          Initialization Step: tableau of Table I with the slack basis
//   k_pivot_persistent  Steps 1-3 iterated inside one cooperative launch
//   k_ml_*           the same phases, one launch each (fallback / profiling)
//   k_extract_*      solution read-out (x, y, objective)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "tabsimplex.h"
#include "tsx_device.cuh"

using namespace tsx;

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

static void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

#define CUDA_TRY(call, ret)                                                            \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                       \
            return ret;                                                                \
        }                                                                              \
    } while (0)

// ------------------------------------------------------------- allocator
static std::mutex g_alloc_mu;
static lp_alloc_fn g_alloc = nullptr;
static lp_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

struct Block {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// ---------------------------------------------------------------- handle
struct lp_handle {
    int m = 0, n = 0, W = 0, ld = 0;
    int device = 0;
    cudaStream_t stream = nullptr;   // handle stream
    bool own_stream = false;
    cudaEvent_t ready = nullptr;     // last work of the handle
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    lp_alloc_fn alloc = nullptr;     // allocator captured at create
    lp_free_fn dealloc = nullptr;
    void* alloc_ctx = nullptr;
    const double *A = nullptr, *b = nullptr, *c = nullptr;
    Block inputs;                    // owned copy of (A, b, c) for lp_create
    Block work;                      // tableau + work buffers
    double* T = nullptr;
    double* F = nullptr;
    double* R = nullptr;
    int* act = nullptr;
    ArgPart* cpart = nullptr;
    RatPart* rpart = nullptr;
    DevState* st = nullptr;
    int* basis = nullptr;
    double* sol = nullptr;           // x (n), y (m), obj (1)
    Block logs;
    long long log_cap = 0;
    int max_grid = 0;                // rpart capacity
    bool solved = false;
    int last_status = LP_ERR_STATE;
    long long iters = 0;
    lp_stats stats{};
};

static void* dev_alloc(lp_handle* h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (h->alloc) return h->alloc(bytes, (void*)h->stream, h->alloc_ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dev_free(lp_handle* h, Block& blk) {
    if (!blk.ptr) return;
    if (h->dealloc)
        h->dealloc(blk.ptr, blk.bytes, (void*)h->stream, h->alloc_ctx);
    else
        cudaFreeAsync(blk.ptr, h->stream);
    blk.ptr = nullptr;
    blk.bytes = 0;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------- kernels
__global__ void k_reset_state(DevState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->status = kRunning;
        st->q = -1;
        st->p = -1;
        st->bland = 0;
        st->degen_run = 0;
        st->bad = 0;
        st->iters = 0;
        st->active_sectors = 0;
        st->nact = 0;
        st->next_slot = 0;
        st->theta = 0.0;
        st->bar_count = 0;
        st->bar_gen = 0;
        for (int k = 0; k < 6; ++k) st->phase_ns[k] = 0;
    }
}

// Input check for device-created LPs: every entry finite, b >= 0.
__global__ void k_validate(int m, int n, const double* __restrict__ A, const double* __restrict__ b,
                           const double* __restrict__ c, DevState* st) {
    const size_t mn = (size_t)m * (size_t)n;
    const size_t total = mn + (size_t)m + (size_t)n;
    int bad = 0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        double v;
        if (k < mn) {
            v = A[k];
            bad |= !isfinite(v);
        } else if (k < mn + m) {
            v = b[k - mn];
            bad |= !isfinite(v) || !(v >= 0.0);
        } else {
            v = c[k - mn - m];
            bad |= !isfinite(v);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->bad, 1);
}

// Initialization Step (Section III, Table I): row 0 = [-c, 0 | 0],
// row i = [A_i, e_i | b_i]; padding columns [W, ld) are zero.  One thread per
// 32-byte group of 4 columns.  Also seeds the slack basis.
__global__ void k_build(int m, int n, int W, int ld, const double* __restrict__ A,
                        const double* __restrict__ b, const double* __restrict__ c,
                        double* __restrict__ T, int* __restrict__ basis) {
    const size_t groups_per_row = (size_t)ld / 4;
    const size_t total = (size_t)(m + 1) * groups_per_row;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / groups_per_row);
        const int j0 = (int)(g - (size_t)i * groups_per_row) * 4;
        double out[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = j0 + e;
            double v = 0.0;
            if (i == 0) {
                if (j < n) v = -c[j];
            } else {
                if (j < n)
                    v = A[(size_t)(i - 1) * (size_t)n + j];
                else if (j == n + i - 1)
                    v = 1.0;
                else if (j == W - 1)
                    v = b[i - 1];
            }
            out[e] = v;
        }
        st_sector(T + (size_t)i * (size_t)ld + j0, make_sec4(out[0], out[1], out[2], out[3]));
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)m;
         i += (size_t)gridDim.x * blockDim.x)
        basis[i] = n + (int)i;
}

// Pivot bookkeeping shared by both paths (one thread): basis update, pivot log.
__device__ __forceinline__ void record_pivot(const Params& P, long long it, int q, int p) {
    P.basis[p - 1] = q;
    if (it < P.log_cap) {
        P.qlog[it] = q;
        P.plog[it] = p;
    }
}

// Cycling guard: a pivot with minimum ratio <= 0 does not move the objective;
// k_cyc of them in a row switch to Bland's rule until a positive-ratio pivot.
__device__ __forceinline__ void degeneracy_step(const Params& P, double theta, int& bland, int& degen) {
    if (P.rule != 0) return;
    if (theta <= 0.0) {
        ++degen;
        if (P.k_cyc > 0 && degen >= P.k_cyc) bland = 1;
    } else {
        degen = 0;
        bland = 0;
    }
}

__device__ __forceinline__ void finish(const Params& P, int status, long long it, int bland, int degen,
                                       const long long* ph) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicCAS(&P.st->status, kRunning, status);
        P.st->iters = it;
        P.st->bland = bland;
        P.st->degen_run = degen;
        for (int k = 0; k < 6; ++k) P.st->phase_ns[k] = ph[k];
    }
}

// Phase timer of block 0, thread 0 (other threads keep it at zero).
struct PhaseClock {
    long long acc[6] = {0, 0, 0, 0, 0, 0};
    long long t = 0;
    bool on = false;
    __device__ void start() {
        on = blockIdx.x == 0 && threadIdx.x == 0;
        if (on) t = global_ns();
    }
    __device__ void lap(int k) {   // closes interval k, opens the next one
        if (on) {
            const long long now = global_ns();
            acc[k] += now - t;
            t = now;
        }
    }
};

// Steps 1-3 iterated inside one cooperative launch; three grid barriers per
// pivot (after P2, after P3, after P4).  Every block takes the same decisions
// from the same reduced values, so all leave the loop together.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_pivot_persistent(Params P) {
    __shared__ BlockScratch s;
    PhaseClock clk;
    phase_init_argmin(P);
    if (!grid_barrier(P.st, P.timeout_ns, s)) return;
    long long it = 0;
    int bland = P.rule == 1 ? 1 : 0;
    int degen = 0;
    clk.start();
    for (;;) {
        const ArgPart e = phase_entering(P, s);           // Step 1
        const int q = bland ? e.jfirst : e.j;
        if (q == INT_MAX) { finish(P, kOptimal, it, bland, degen, clk.acc); return; }
        if (it >= P.max_iters) { finish(P, kIterLimit, it, bland, degen, clk.acc); return; }
        phase_ratio(P, q, bland, s);                      // Step 2 (block partials)
        clk.lap(0);
        if (!grid_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(3);
        const RatPart l = phase_leaving(P, s);            // Step 2 (global)
        if (l.i == INT_MAX) { finish(P, kUnbounded, it, bland, degen, clk.acc); return; }
        const double piv = __ldcg(P.F + l.i);
        if (!isfinite(piv) || !isfinite(l.r)) { finish(P, kNumeric, it, bland, degen, clk.acc); return; }
        phase_stage_row(P, l.i, piv, s);                  // Step 3 (pivot row)
        if (blockIdx.x == 0 && threadIdx.x == 0) record_pivot(P, it, q, l.i);
        clk.lap(1);
        if (!grid_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(4);
        phase_update(P, l.i);                             // Step 3 (rank-1 update)
        ++it;
        degeneracy_step(P, l.r, bland, degen);
        clk.lap(2);
        if (!grid_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(5);
    }
}

// ---- one launch per phase (same device functions; state in DevState)
__global__ void k_ml_init(Params P) {
    if (blockIdx.x == 0 && threadIdx.x == 0) P.st->bland = P.rule == 1 ? 1 : 0;
    phase_init_argmin(P);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_ml_select(Params P) {
    __shared__ BlockScratch s;
    if (P.st->status != kRunning) return;
    const int bland = P.st->bland;
    const long long it = P.st->iters;
    const ArgPart e = phase_entering(P, s);
    const int q = bland ? e.jfirst : e.j;
    if (q == INT_MAX || it >= P.max_iters) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicCAS(&P.st->status, kRunning, q == INT_MAX ? kOptimal : kIterLimit);
        return;
    }
    phase_ratio(P, q, bland, s);
    if (blockIdx.x == 0 && threadIdx.x == 0) P.st->q = q;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_ml_stage(Params P) {
    __shared__ BlockScratch s;
    if (P.st->status != kRunning) return;
    const RatPart l = phase_leaving(P, s);
    if (l.i == INT_MAX) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&P.st->status, kRunning, kUnbounded);
        return;
    }
    const double piv = __ldcg(P.F + l.i);
    if (!isfinite(piv) || !isfinite(l.r)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&P.st->status, kRunning, kNumeric);
        return;
    }
    phase_stage_row(P, l.i, piv, s);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        record_pivot(P, P.st->iters, P.st->q, l.i);
        P.st->p = l.i;
        P.st->theta = l.r;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_ml_update(Params P) {
    if (P.st->status != kRunning) return;
    const int p = P.st->p;
    phase_update(P, p);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int bland = P.st->bland, degen = P.st->degen_run;
        degeneracy_step(P, P.st->theta, bland, degen);
        P.st->bland = bland;
        P.st->degen_run = degen;
        P.st->iters += 1;
    }
}

// Solution read-out (Table I layout): y_i = T[0][n+i], obj = T[0][W-1],
// x zeroed, then x[basis[i]] = T[i+1][W-1] for structural basics.
__global__ void k_extract_dense(int m, int n, int W, int ld, const double* __restrict__ T,
                                double* __restrict__ sol) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n + m + 1; k += gridDim.x * blockDim.x) {
        if (k < n)
            sol[k] = 0.0;
        else if (k < n + m)
            sol[k] = T[n + (k - n)];
        else
            sol[k] = T[W - 1];
    }
}

__global__ void k_extract_x(int m, int n, int W, int ld, const double* __restrict__ T,
                            const int* __restrict__ basis, double* __restrict__ sol) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int v = basis[i];
        if (v < n) sol[v] = T[(size_t)(i + 1) * (size_t)ld + (W - 1)];
    }
}

// ------------------------------------------------------------------- API
// (C linkage comes from the declarations in tabsimplex.h)

const char* lp_version(void) { return "tabsimplex 0.1 (sm_103a)"; }

const char* lp_last_error(void) { return g_last_error.c_str(); }

int lp_set_allocator(lp_alloc_fn alloc_fn, lp_free_fn free_fn, void* ctx) {
    if ((alloc_fn == nullptr) != (free_fn == nullptr)) {
        set_error("lp_set_allocator: give both functions or neither");
        return -1;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc_fn;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return 0;
}

void lp_options_init(lp_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->rule = LP_RULE_DANTZIG;
    o->eps_d = 1e-9;
    o->eps_p = 1e-9;
    o->max_iters = -1;
    o->k_cyc = 50;
    o->barrier_timeout_ns = 2000000000LL;
    o->path = LP_PATH_AUTO;
    o->skip_zero_columns = 1;
    o->threads = 0;
    o->blocks = 0;
    o->log_capacity = 0;
    o->stream = nullptr;
}

static void destroy_impl(lp_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    dev_free(h, h->logs);
    dev_free(h, h->work);
    dev_free(h, h->inputs);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->ready) cudaEventDestroy(h->ready);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

void lp_destroy(lp_t h) { destroy_impl(h); }

// Common part of the two create calls: sizes, stream, events, work buffers.
static lp_handle* create_common(int m, int n, cudaStream_t stream, bool own_stream) {
    if (m <= 0 || n <= 0) {
        set_error("lp_create: need m > 0 and n > 0 (got m=%d, n=%d)", m, n);
        return nullptr;
    }
    if ((long long)n + m + 1 > (long long)INT_MAX - 256) {
        set_error("lp_create: n + m + 1 too large");
        return nullptr;
    }
    lp_handle* h = new lp_handle();
    h->m = m;
    h->n = n;
    h->W = n + m + 1;
    h->ld = (int)align_up((size_t)h->W, 16);
    cudaGetDevice(&h->device);
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        h->alloc = g_alloc;
        h->dealloc = g_free;
        h->alloc_ctx = g_alloc_ctx;
    }
    if (own_stream) {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("lp_create: cudaStreamCreate failed: %s", cudaGetErrorString(cudaGetLastError()));
            delete h;
            return nullptr;
        }
        h->own_stream = true;
    } else {
        h->stream = stream;
    }
    bool ok = cudaEventCreateWithFlags(&h->ready, cudaEventDisableTiming) == cudaSuccess;
    for (auto& e : h->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    if (!ok) {
        set_error("lp_create: cudaEventCreate failed");
        destroy_impl(h);
        return nullptr;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    h->max_grid = std::max(1, nsm) * 32;   // rpart capacity (>= any co-resident grid)
    const int nstrips = (h->ld + kStripCols - 1) / kStripCols;
    // one allocation: T | F | R | act | cpart | rpart | st | basis | sol
    const size_t sz_T = (size_t)(m + 1) * (size_t)h->ld * sizeof(double);
    const size_t off_F = align_up(sz_T, 256);
    const size_t off_R = align_up(off_F + (size_t)(m + 1) * sizeof(double), 256);
    const size_t off_act = align_up(off_R + (size_t)h->ld * sizeof(double), 256);
    const size_t off_cp = align_up(off_act + (size_t)(h->ld / 4) * sizeof(int), 256);
    const size_t off_rp = align_up(off_cp + (size_t)nstrips * sizeof(ArgPart), 256);
    const size_t off_st = align_up(off_rp + (size_t)h->max_grid * sizeof(RatPart), 256);
    const size_t off_bs = align_up(off_st + sizeof(DevState), 256);
    const size_t off_sol = align_up(off_bs + (size_t)m * sizeof(int), 256);
    const size_t total = align_up(off_sol + (size_t)(n + m + 1) * sizeof(double), 256);
    h->work.ptr = dev_alloc(h, total);
    if (!h->work.ptr) {
        set_error("lp_create: device allocation of %zu bytes failed", total);
        destroy_impl(h);
        return nullptr;
    }
    h->work.bytes = total;
    char* base = (char*)h->work.ptr;
    h->T = (double*)base;
    h->F = (double*)(base + off_F);
    h->R = (double*)(base + off_R);
    h->act = (int*)(base + off_act);
    h->cpart = (ArgPart*)(base + off_cp);
    h->rpart = (RatPart*)(base + off_rp);
    h->st = (DevState*)(base + off_st);
    h->basis = (int*)(base + off_bs);
    h->sol = (double*)(base + off_sol);
    return h;
}

// Validates the device-resident inputs; returns false (and sets the error) if bad.
static bool validate_inputs(lp_handle* h) {
    k_reset_state<<<1, 32, 0, h->stream>>>(h->st);
    const size_t total = (size_t)h->m * h->n + h->m + h->n;
    int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
    k_validate<<<grid, 256, 0, h->stream>>>(h->m, h->n, h->A, h->b, h->c, h->st);
    int bad = 0;
    if (cudaMemcpyAsync(&bad, &h->st->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        set_error("lp_create: validation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return false;
    }
    if (bad) {
        set_error("lp_create: inputs must be finite with b >= 0");
        return false;
    }
    return true;
}

lp_t lp_create(int m, int n, const double* A, const double* b, const double* c) {
    if (!A || !b || !c) {
        set_error("lp_create: NULL input array");
        return nullptr;
    }
    lp_handle* h = create_common(m, n, nullptr, true);
    if (!h) return nullptr;
    const size_t mn = (size_t)m * (size_t)n;
    const size_t off_b = align_up(mn * sizeof(double), 256);
    const size_t off_c = align_up(off_b + (size_t)m * sizeof(double), 256);
    const size_t total = align_up(off_c + (size_t)n * sizeof(double), 256);
    h->inputs.ptr = dev_alloc(h, total);
    if (!h->inputs.ptr) {
        set_error("lp_create: device allocation of %zu input bytes failed", total);
        destroy_impl(h);
        return nullptr;
    }
    h->inputs.bytes = total;
    char* base = (char*)h->inputs.ptr;
    h->A = (const double*)base;
    h->b = (const double*)(base + off_b);
    h->c = (const double*)(base + off_c);
    if (cudaMemcpyAsync((void*)h->A, A, mn * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync((void*)h->b, b, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync((void*)h->c, c, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
        set_error("lp_create: host-to-device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
        destroy_impl(h);
        return nullptr;
    }
    if (!validate_inputs(h)) {
        destroy_impl(h);
        return nullptr;
    }
    cudaEventRecord(h->ready, h->stream);
    return h;
}

lp_t lp_create_device(int m, int n, const double* dA, const double* db, const double* dc, void* stream) {
    if (!dA || !db || !dc) {
        set_error("lp_create_device: NULL input pointer");
        return nullptr;
    }
    lp_handle* h = create_common(m, n, (cudaStream_t)stream, false);
    if (!h) return nullptr;
    h->A = dA;
    h->b = db;
    h->c = dc;
    if (!validate_inputs(h)) {
        destroy_impl(h);
        return nullptr;
    }
    cudaEventRecord(h->ready, h->stream);
    return h;
}

template <int NT>
static cudaError_t launch_persistent(const Params& P, int grid, cudaStream_t s) {
    void* args[] = {(void*)&P};
    return cudaLaunchCooperativeKernel((const void*)k_pivot_persistent<NT>, grid, NT, args, 0, s);
}

template <int NT>
static int max_coresident(int device) {
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pivot_persistent<NT>, NT, 0);
    return nsm * per;
}

template <int NT>
static lp_status run_multilaunch(lp_handle* h, const Params& P, int grid, cudaStream_t s, long long& launches) {
    k_ml_init<<<grid, NT, 0, s>>>(P);
    ++launches;
    int status = kRunning;
    int batch = 4;
    for (;;) {
        for (int k = 0; k < batch; ++k) {
            k_ml_select<NT><<<grid, NT, 0, s>>>(P);
            k_ml_stage<NT><<<grid, NT, 0, s>>>(P);
            k_ml_update<NT><<<grid, NT, 0, s>>>(P);
            launches += 3;
        }
        CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
        CUDA_TRY(cudaMemcpyAsync(&status, &h->st->status, sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
        CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
        if (status != kRunning) break;
        batch = std::min(batch * 2, 64);
    }
    return (lp_status)status;
}

template <int NT>
static lp_status solve_nt(lp_handle* h, const lp_options& o, cudaStream_t s) {
    const int m = h->m, n = h->n;
    Params P{};
    P.T = h->T;
    P.ld = h->ld;
    P.m = m;
    P.n = n;
    P.W = h->W;
    P.basis = h->basis;
    P.F = h->F;
    P.R = h->R;
    P.act = h->act;
    P.cpart = h->cpart;
    P.rpart = h->rpart;
    P.st = h->st;
    P.eps_d = o.eps_d;
    P.eps_p = o.eps_p;
    P.max_iters = o.max_iters < 0 ? 50LL * ((long long)m + n) : o.max_iters;
    P.k_cyc = o.k_cyc;
    P.rule = o.rule;
    P.timeout_ns = std::max(0LL, o.barrier_timeout_ns);
    P.nstrips = (h->ld + kStripCols - 1) / kStripCols;
    P.nrc = (m + 1 + kUnitRows - 1) / kUnitRows;
    P.nunits = (long long)P.nstrips * P.nrc;
    P.skip_zero = o.skip_zero_columns ? 1 : 0;

    // pivot log buffers
    if (o.log_capacity > 0 && o.log_capacity != h->log_cap) {
        dev_free(h, h->logs);
        h->log_cap = 0;
        const size_t bytes = (size_t)o.log_capacity * 2 * sizeof(int);
        h->logs.ptr = dev_alloc(h, bytes);
        if (!h->logs.ptr) {
            set_error("lp_solve: allocation of the pivot log failed");
            return LP_ERR_NOMEM;
        }
        h->logs.bytes = bytes;
        h->log_cap = o.log_capacity;
    }
    P.log_cap = o.log_capacity > 0 ? h->log_cap : 0;
    P.qlog = P.log_cap ? (int*)h->logs.ptr : nullptr;
    P.plog = P.log_cap ? (int*)h->logs.ptr + P.log_cap : nullptr;

    // grid: enough warps for the units, at most the co-resident blocks
    const int warps = NT / 32;
    const long long want = (P.nunits + warps - 1) / warps;
    int coresident = max_coresident<NT>(h->device);
    int grid = (int)std::min<long long>(std::max<long long>(1, want), std::max(1, coresident));
    grid = std::min(grid, h->max_grid);
    if (o.blocks > 0) grid = std::min(grid, o.blocks);

    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    int path = o.path;
    if (path == LP_PATH_AUTO) path = (coop && coresident > 0) ? LP_PATH_PERSISTENT : LP_PATH_MULTILAUNCH;
    if (path == LP_PATH_PERSISTENT && (!coop || coresident <= 0)) {
        set_error("lp_solve: persistent path requested but cooperative launch is unavailable");
        return LP_ERR_CUDA;
    }

    // Initialization Step
    cudaEventRecord(h->ev[0], s);
    k_reset_state<<<1, 32, 0, s>>>(h->st);
    {
        const size_t groups = (size_t)(m + 1) * (size_t)(h->ld / 4);
        int g = (int)std::min<size_t>((groups + 255) / 256, 152 * 16);
        k_build<<<g, 256, 0, s>>>(m, n, h->W, h->ld, h->A, h->b, h->c, h->T, h->basis);
    }
    CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    cudaEventRecord(h->ev[1], s);

    long long launches = 2;
    lp_status st;
    if (path == LP_PATH_PERSISTENT) {
        cudaError_t e = launch_persistent<NT>(P, grid, s);
        if (e != cudaSuccess) {
            if (o.path == LP_PATH_AUTO) {   // co-residency refused: fall back
                cudaGetLastError();
                path = LP_PATH_MULTILAUNCH;
            } else {
                set_error("lp_solve: cooperative launch failed: %s", cudaGetErrorString(e));
                return LP_ERR_CUDA;
            }
        } else {
            ++launches;
        }
    }
    if (path == LP_PATH_MULTILAUNCH) {
        if (run_multilaunch<NT>(h, P, grid, s, launches) == LP_ERR_CUDA) return LP_ERR_CUDA;
    }
    cudaEventRecord(h->ev[2], s);
    DevState hs{};
    CUDA_TRY(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    cudaEventRecord(h->ready, s);

    float ms_build = 0.f, ms_pivot = 0.f;
    cudaEventElapsedTime(&ms_build, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&ms_pivot, h->ev[1], h->ev[2]);
    h->stats = lp_stats{};
    h->stats.iters = hs.iters;
    h->stats.build_ms = ms_build;
    h->stats.pivot_ms = ms_pivot;
    h->stats.kernel_launches = launches;
    h->stats.dense_update_bytes = 2.0 * (double)(m + 1) * (double)h->W * sizeof(double) * (double)hs.iters;
    // bytes Step 3 moves: read + write of every listed 32-B group in rows
    // 1..m except p, read + write of the objective row and write of row p over
    // all groups; plus the side traffic of Steps 1-2 and the staging: column q
    // and right-hand-side sectors (m + 1 rows), pivot row read, R write + read.
    {
        const double nsec = (double)(h->ld / 4);
        const double upd = 64.0 * (double)(m - 1) * (double)hs.active_sectors + 96.0 * nsec * (double)hs.iters;
        const double side = (64.0 * (double)(m + 1) + 24.0 * (double)h->ld) * (double)hs.iters;
        h->stats.update_bytes = upd + side;
    }
    h->stats.path = path;
    h->stats.grid = grid;
    h->stats.block = NT;
    h->stats.ld = h->ld;
    for (int k = 0; k < 6; ++k) h->stats.phase_ms[k] = 1e-6 * (double)hs.phase_ns[k];

    h->iters = hs.iters;
    h->solved = true;
    st = (lp_status)hs.status;
    if (hs.status == kRunning) {
        set_error("lp_solve: kernel ended without a status");
        st = LP_ERR_CUDA;
    } else if (hs.status == kTimeout) {
        set_error("lp_solve: a grid barrier wait exceeded %lld ns", (long long)P.timeout_ns);
    }
    h->last_status = st;
    return st;
}

lp_status lp_solve(lp_t h, const lp_options* opt) {
    if (!h) {
        set_error("lp_solve: NULL handle");
        return LP_ERR_INVALID;
    }
    lp_options o;
    if (opt)
        o = *opt;
    else
        lp_options_init(&o);
    if (!(o.eps_d >= 0.0) || !(o.eps_p >= 0.0) || o.rule < 0 || o.rule > 1 || o.path < 0 || o.path > 2 ||
        o.log_capacity < 0) {
        set_error("lp_solve: invalid options");
        return LP_ERR_INVALID;
    }
    CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : h->stream;
    CUDA_TRY(cudaStreamWaitEvent(s, h->ready, 0), LP_ERR_CUDA);
    int nt = o.threads ? o.threads : 256;
    switch (nt) {
        case 128: return solve_nt<128>(h, o, s);
        case 256: return solve_nt<256>(h, o, s);
        case 512: return solve_nt<512>(h, o, s);
        default:
            set_error("lp_solve: threads must be 0, 128, 256 or 512 (got %d)", nt);
            return LP_ERR_INVALID;
    }
}

lp_status lp_get_solution(lp_t h, double* x, double* y, double* obj, int* basis, long long* iters) {
    if (!h) {
        set_error("lp_get_solution: NULL handle");
        return LP_ERR_INVALID;
    }
    if (!h->solved) {
        set_error("lp_get_solution: no solve has run on this handle");
        return LP_ERR_STATE;
    }
    CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
    cudaStream_t s = h->stream;
    CUDA_TRY(cudaStreamWaitEvent(s, h->ready, 0), LP_ERR_CUDA);
    const int m = h->m, n = h->n;
    if (x || y || obj) {
        int g = std::min((n + m + 1 + 255) / 256, 1024);
        k_extract_dense<<<g, 256, 0, s>>>(m, n, h->W, h->ld, h->T, h->sol);
        if (x) k_extract_x<<<std::min((m + 255) / 256, 1024), 256, 0, s>>>(m, n, h->W, h->ld, h->T, h->basis, h->sol);
        CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
        if (x) CUDA_TRY(cudaMemcpyAsync(x, h->sol, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
        if (y) CUDA_TRY(cudaMemcpyAsync(y, h->sol + n, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
        if (obj) CUDA_TRY(cudaMemcpyAsync(obj, h->sol + n + m, sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    }
    if (basis) CUDA_TRY(cudaMemcpyAsync(basis, h->basis, (size_t)m * sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    if (iters) *iters = h->iters;
    return (lp_status)h->last_status;
}

lp_status lp_get_tableau(lp_t h, double* T) {
    if (!h || !T) {
        set_error("lp_get_tableau: NULL argument");
        return LP_ERR_INVALID;
    }
    if (!h->solved) {
        set_error("lp_get_tableau: no solve has run on this handle");
        return LP_ERR_STATE;
    }
    CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ready, 0), LP_ERR_CUDA);
    CUDA_TRY(cudaMemcpy2DAsync(T, (size_t)h->W * sizeof(double), h->T, (size_t)h->ld * sizeof(double),
                               (size_t)h->W * sizeof(double), (size_t)h->m + 1, cudaMemcpyDeviceToHost, h->stream),
             LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(h->stream), LP_ERR_CUDA);
    return LP_OPTIMAL;
}

lp_status lp_get_pivot_log(lp_t h, int* q, int* p, long long cap, long long* count) {
    if (!h || cap < 0) {
        set_error("lp_get_pivot_log: bad argument");
        return LP_ERR_INVALID;
    }
    if (!h->solved) {
        set_error("lp_get_pivot_log: no solve has run on this handle");
        return LP_ERR_STATE;
    }
    long long k = std::min(h->iters, h->log_cap);
    k = std::min(k, cap);
    if (count) *count = k;
    if (k > 0 && h->logs.ptr) {
        CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
        if (q) CUDA_TRY(cudaMemcpyAsync(q, h->logs.ptr, (size_t)k * sizeof(int), cudaMemcpyDeviceToHost, h->stream), LP_ERR_CUDA);
        if (p) CUDA_TRY(cudaMemcpyAsync(p, (int*)h->logs.ptr + h->log_cap, (size_t)k * sizeof(int), cudaMemcpyDeviceToHost, h->stream), LP_ERR_CUDA);
        CUDA_TRY(cudaStreamSynchronize(h->stream), LP_ERR_CUDA);
    }
    return LP_OPTIMAL;
}

lp_status lp_get_stats(lp_t h, lp_stats* stats) {
    if (!h || !stats) {
        set_error("lp_get_stats: NULL argument");
        return LP_ERR_INVALID;
    }
    if (!h->solved) {
        set_error("lp_get_stats: no solve has run on this handle");
        return LP_ERR_STATE;
    }
    *stats = h->stats;
    return LP_OPTIMAL;
}

// ------------------------------------------------------- no-allocation solve
// lp_solve_noalloc: the pivot kernels run on work buffers carved out of one
// file-scope device array instead of allocated memory, for callers that cannot
// allocate device memory (see tabsimplex.h).  The array is a host-side stand-in
// in host code; its device address on each device is looked up once with
// cudaGetSymbolAddress and passed to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LP_NOALLOC_SCRATCH_BYTES];

constexpr int kNoAllocMaxGrid = 1024;   // ratio-partial slots in the array
constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the array on the current device (set up on first use).
static void* noalloc_scratch(int device) {
    if (device < 0 || device >= kNoAllocMaxDevices) {
        set_error("lp_solve_noalloc: device ordinal %d out of range", device);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("lp_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return nullptr;
        }
        g_noalloc_ptr[device] = ptr;
    }
    return g_noalloc_ptr[device];
}

template <int NT>
static lp_status noalloc_nt(int m, int n, const double* dA, const double* db, const double* dc, double* dT,
                            int ld, int* dbasis, const lp_options& o, long long* iters_out, char* base,
                            size_t off_R, size_t off_act, size_t off_cp, size_t off_rp, size_t off_st) {
    cudaStream_t s = (cudaStream_t)o.stream;
    int device = 0;
    CUDA_TRY(cudaGetDevice(&device), LP_ERR_CUDA);
    Params P{};
    P.T = dT;
    P.ld = ld;
    P.m = m;
    P.n = n;
    P.W = n + m + 1;
    P.basis = dbasis;
    P.F = (double*)base;
    P.R = (double*)(base + off_R);
    P.act = (int*)(base + off_act);
    P.cpart = (ArgPart*)(base + off_cp);
    P.rpart = (RatPart*)(base + off_rp);
    P.st = (DevState*)(base + off_st);
    P.qlog = nullptr;
    P.plog = nullptr;
    P.log_cap = 0;
    P.eps_d = o.eps_d;
    P.eps_p = o.eps_p;
    P.max_iters = o.max_iters < 0 ? 50LL * ((long long)m + n) : o.max_iters;
    P.k_cyc = o.k_cyc;
    P.rule = o.rule;
    P.timeout_ns = std::max(0LL, o.barrier_timeout_ns);
    P.nstrips = (ld + kStripCols - 1) / kStripCols;
    P.nrc = (m + 1 + kUnitRows - 1) / kUnitRows;
    P.nunits = (long long)P.nstrips * P.nrc;
    P.skip_zero = o.skip_zero_columns ? 1 : 0;

    // validate the inputs: the state word starts from zero on every call
    k_reset_state<<<1, 32, 0, s>>>(P.st);
    {
        const size_t total = (size_t)m * n + m + n;
        int g = (int)std::min<size_t>((total + 255) / 256, 4096);
        k_validate<<<g, 256, 0, s>>>(m, n, dA, db, dc, P.st);
    }
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, &P.st->bad, sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    if (bad) {
        set_error("lp_solve_noalloc: inputs must be finite with b >= 0");
        return LP_ERR_INVALID;
    }

    const long long want = (P.nunits + NT / 32 - 1) / (NT / 32);
    int coresident = max_coresident<NT>(device);
    int grid = (int)std::min<long long>(std::max<long long>(1, want), std::max(1, coresident));
    grid = std::min(grid, kNoAllocMaxGrid);
    if (o.blocks > 0) grid = std::min(grid, o.blocks);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    int path = o.path;
    if (path == LP_PATH_AUTO) path = (coop && coresident > 0) ? LP_PATH_PERSISTENT : LP_PATH_MULTILAUNCH;
    if (path == LP_PATH_PERSISTENT && (!coop || coresident <= 0)) {
        set_error("lp_solve_noalloc: persistent path requested but cooperative launch is unavailable");
        return LP_ERR_CUDA;
    }

    k_reset_state<<<1, 32, 0, s>>>(P.st);
    {
        const size_t groups = (size_t)(m + 1) * (size_t)(ld / 4);
        int g = (int)std::min<size_t>((groups + 255) / 256, 152 * 16);
        k_build<<<g, 256, 0, s>>>(m, n, n + m + 1, ld, dA, db, dc, dT, dbasis);
    }
    CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    if (path == LP_PATH_PERSISTENT) {
        cudaError_t e = launch_persistent<NT>(P, grid, s);
        if (e != cudaSuccess) {
            if (o.path != LP_PATH_AUTO) {
                set_error("lp_solve_noalloc: cooperative launch failed: %s", cudaGetErrorString(e));
                return LP_ERR_CUDA;
            }
            cudaGetLastError();
            path = LP_PATH_MULTILAUNCH;
        }
    }
    if (path == LP_PATH_MULTILAUNCH) {
        k_ml_init<<<grid, NT, 0, s>>>(P);
        int status = kRunning;
        int batch = 4;
        for (;;) {
            for (int k = 0; k < batch; ++k) {
                k_ml_select<NT><<<grid, NT, 0, s>>>(P);
                k_ml_stage<NT><<<grid, NT, 0, s>>>(P);
                k_ml_update<NT><<<grid, NT, 0, s>>>(P);
            }
            CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
            CUDA_TRY(cudaMemcpyAsync(&status, &P.st->status, sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
            CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
            if (status != kRunning) break;
            batch = std::min(batch * 2, 64);
        }
    }
    DevState hs{};
    CUDA_TRY(cudaMemcpyAsync(&hs, P.st, sizeof(DevState), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    if (iters_out) *iters_out = hs.iters;
    if (hs.status == kRunning) {
        set_error("lp_solve_noalloc: kernel ended without a status");
        return LP_ERR_CUDA;
    }
    if (hs.status == kTimeout) set_error("lp_solve_noalloc: a grid barrier wait exceeded %lld ns", (long long)P.timeout_ns);
    return (lp_status)hs.status;
}

lp_status lp_solve_noalloc(int m, int n, const double* dA, const double* db, const double* dc, double* dT,
                           long long ld, int* dbasis, const lp_options* opt, long long* iters) {
    if (iters) *iters = 0;
    if (!dA || !db || !dc || !dT || !dbasis) {
        set_error("lp_solve_noalloc: NULL pointer argument");
        return LP_ERR_INVALID;
    }
    if (m <= 0 || n <= 0 || (long long)n + m + 1 > (long long)INT_MAX - 256) {
        set_error("lp_solve_noalloc: need m > 0, n > 0 (got m=%d, n=%d)", m, n);
        return LP_ERR_INVALID;
    }
    if (ld < (long long)n + m + 1 || ld % 4 != 0 || ld > (long long)INT_MAX - 256) {
        set_error("lp_solve_noalloc: ld must be >= n + m + 1 = %lld and a multiple of 4 (got %lld)",
                  (long long)n + m + 1, ld);
        return LP_ERR_INVALID;
    }
    if (((uintptr_t)dT & 31u) != 0) {
        set_error("lp_solve_noalloc: dT must be 32-byte aligned");
        return LP_ERR_INVALID;
    }
    lp_options o;
    if (opt)
        o = *opt;
    else
        lp_options_init(&o);
    if (!(o.eps_d >= 0.0) || !(o.eps_p >= 0.0) || o.rule < 0 || o.rule > 1 || o.path < 0 || o.path > 2 ||
        o.log_capacity != 0 || o.blocks < 0 || o.blocks > kNoAllocMaxGrid) {
        set_error("lp_solve_noalloc: invalid options (log_capacity must be 0, blocks <= %d)", kNoAllocMaxGrid);
        return LP_ERR_INVALID;
    }
    // layout of the array: F | R | act | cpart | rpart | state
    const size_t nstrips = ((size_t)ld + kStripCols - 1) / kStripCols;
    const size_t off_R = align_up((size_t)(m + 1) * sizeof(double), 256);
    const size_t off_act = align_up(off_R + (size_t)ld * sizeof(double), 256);
    const size_t off_cp = align_up(off_act + (size_t)(ld / 4) * sizeof(int), 256);
    const size_t off_rp = align_up(off_cp + nstrips * sizeof(ArgPart), 256);
    const size_t off_st = align_up(off_rp + (size_t)kNoAllocMaxGrid * sizeof(RatPart), 256);
    const size_t need = align_up(off_st + sizeof(DevState), 256);
    if (need > (size_t)LP_NOALLOC_SCRATCH_BYTES) {
        set_error("lp_solve_noalloc: m=%d, ld=%lld need %zu bytes of work buffers, more than the %u-byte "
                  "fixed array; use lp_create/lp_solve for this size",
                  m, ld, need, (unsigned)LP_NOALLOC_SCRATCH_BYTES);
        return LP_ERR_INVALID;
    }
    int device = 0;
    CUDA_TRY(cudaGetDevice(&device), LP_ERR_CUDA);
    char* base = (char*)noalloc_scratch(device);
    if (!base) return LP_ERR_CUDA;
    const int nt = o.threads ? o.threads : 256;
    switch (nt) {
        case 128: return noalloc_nt<128>(m, n, dA, db, dc, dT, (int)ld, dbasis, o, iters, base, off_R, off_act, off_cp, off_rp, off_st);
        case 256: return noalloc_nt<256>(m, n, dA, db, dc, dT, (int)ld, dbasis, o, iters, base, off_R, off_act, off_cp, off_rp, off_st);
        case 512: return noalloc_nt<512>(m, n, dA, db, dc, dT, (int)ld, dbasis, o, iters, base, off_R, off_act, off_cp, off_rp, off_st);
        default:
            set_error("lp_solve_noalloc: threads must be 0, 128, 256 or 512 (got %d)", nt);
            return LP_ERR_INVALID;
    }
}
