// Host side of the C ABI declared in include/tabsimplex.h: the dense
// full-tableau simplex of arXiv 2211.10979 (Section III) on one GPU, with a
// double tableau (exact path) or a float tableau followed by an FP64 recovery
// of the final basis.  Kernels live in tsx_kernels.cuh (pivoting) and
// tsx_recover.cuh (FP64 recovery).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tabsimplex.h"
#include "tsx_cluster.cuh"
#include "tsx_host.h"
#include "tsx_hybrid_host.h"
#include "tsx_kernels.cuh"
#include "tsx_recover.cuh"
#include "tsx_team.cuh"

using namespace tsx;

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void tsx::set_error(const char* fmt, ...) {
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

static thread_local bool t_default_alloc = false;

void tsx::use_default_allocator(bool on) { t_default_alloc = on; }

void tsx::current_allocator(lp_alloc_fn* alloc_fn, lp_free_fn* free_fn, void** ctx) {
    if (t_default_alloc) {
        *alloc_fn = nullptr;
        *free_fn = nullptr;
        *ctx = nullptr;
        return;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    *alloc_fn = g_alloc;
    *free_fn = g_free;
    *ctx = g_alloc_ctx;
}

struct Block {
    void* ptr = nullptr;
    size_t bytes = 0;
};

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Sequential carving of one allocation into 256-byte aligned pieces.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t at = align_up(off, 256);
        off = at + bytes;
        return at;
    }
};

// ---------------------------------------------------------------- handle
struct Work {                        // pivot buffers for one precision and layout
    Block blk;
    int elem = 0;                    // bytes per tableau entry (8 or 4), 0 = none
    int cond = -1;                   // 1: condensed tableau, 0: full
    int Ws = 0;                      // stored width: n + 1 (condensed) or n + m + 1
    int ld = 0;
    int* var = nullptr;              // condensed: variable of each column slot (n)
    void* T = nullptr;
    void* F = nullptr;
    void* R = nullptr;
    int* act = nullptr;
    ArgPart* cpart = nullptr;
    RatPart* rpart = nullptr;
};

struct RecBufs {                     // FP64 recovery buffers
    Block vec;                       // m / n sized vectors
    Block kb;                        // k-sized (capacity kcap)
    int kcap = -1;
    double *s = nullptr, *aZ = nullptr, *d = nullptr, *arow = nullptr;
    int *isbasic = nullptr, *inR = nullptr;
    DevState* rst = nullptr;
    RecCheck* chk = nullptr;
    RecChoice* choice = nullptr;
    int* singular = nullptr;
    double *M = nullptr, *inv = nullptr, *xS = nullptr, *yR = nullptr, *bR = nullptr, *cS = nullptr;
    double *rp = nullptr, *rd = nullptr, *aS = nullptr, *rho = nullptr, *venter = nullptr;
    int *pivrow = nullptr, *S = nullptr, *Rr = nullptr;
    int* pivstep = nullptr;          // in-place refactorisation: step of each pivot row
    double* dpiv = nullptr;          // its pivot elements
    void* parts = nullptr;           // its per-block pivot-search posts (2 x kRecMaxGrid)
};

struct lp_handle {
    int m = 0, n = 0, W = 0;
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
    Block common;                    // state, basis, read-out
    DevState* st = nullptr;
    int* basis = nullptr;
    double* sol = nullptr;           // x (n), y (m), obj (1)
    Work work;
    RecBufs rec;
    Block logs;
    long long log_cap = 0;
    int max_grid = 0;                // rpart capacity
    bool solved = false;
    bool checked = true;             // inputs validated (false: create_device_unchecked)
    int last_status = LP_ERR_STATE;
    bool sol_ready = false;          // sol already holds the read-out (float path)
    std::vector<int> final_basis;    // float path: basic variables after the recovery
    long long iters = 0;
    lp_stats stats{};
    double create_ms[3] = {0, 0, 0};   // lp_create: copy and check (device), whole call (host)
};

namespace {
struct Recycled {
    std::mutex mu;
    std::vector<cudaEvent_t> ev[2];   // [0] timing disabled, [1] timing
    std::vector<cudaStream_t> st;
};
constexpr int kMaxRecycleDevices = 64;
Recycled& recycled(int dev) {
    static Recycled r[kMaxRecycleDevices];
    return r[dev];
}
int current_device_index() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxRecycleDevices) return -1;
    return dev;
}
}  // namespace

cudaEvent_t tsx::event_get(bool timing) {
    const int dev = current_device_index();
    if (dev >= 0) {
        Recycled& r = recycled(dev);
        std::lock_guard<std::mutex> lk(r.mu);
        if (!r.ev[timing].empty()) {
            cudaEvent_t e = r.ev[timing].back();
            r.ev[timing].pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, timing ? cudaEventDefault : cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

void tsx::event_put(cudaEvent_t e, bool timing) {
    if (!e) return;
    const int dev = current_device_index();
    if (dev < 0) {
        cudaEventDestroy(e);
        return;
    }
    Recycled& r = recycled(dev);
    std::lock_guard<std::mutex> lk(r.mu);
    r.ev[timing].push_back(e);
}

cudaStream_t tsx::stream_get() {
    const int dev = current_device_index();
    if (dev >= 0) {
        Recycled& r = recycled(dev);
        std::lock_guard<std::mutex> lk(r.mu);
        if (!r.st.empty()) {
            cudaStream_t s = r.st.back();
            r.st.pop_back();
            return s;
        }
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    return s;
}

void tsx::stream_put(cudaStream_t s) {
    if (!s) return;
    const int dev = current_device_index();
    if (dev < 0) {
        cudaStreamDestroy(s);
        return;
    }
    Recycled& r = recycled(dev);
    std::lock_guard<std::mutex> lk(r.mu);
    r.st.push_back(s);
}

cudaError_t tsx::pool_alloc(void** ptr, size_t bytes, cudaStream_t stream) {
    constexpr int kMaxPoolDevices = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxPoolDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaMallocAsync(ptr, bytes, stream);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t p = nullptr;
            e = cudaMemPoolCreate(&p, &props);
            if (e != cudaSuccess) return e;
            unsigned long long keep = ~0ull;   // keep freed memory in the pool
            cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[dev] = p;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, stream);
}

static void* dev_alloc(lp_handle* h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (h->alloc) return h->alloc(bytes, (void*)h->stream, h->alloc_ctx);
    void* p = nullptr;
    if (pool_alloc(&p, bytes, h->stream) != cudaSuccess) {
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

static bool dev_alloc_block(lp_handle* h, Block& blk, size_t bytes) {
    blk.ptr = dev_alloc(h, bytes);
    blk.bytes = blk.ptr ? bytes : 0;
    return blk.ptr != nullptr;
}

static int grid_for(long long work, int nt, int cap) {
    return (int)std::max<long long>(1, std::min<long long>((work + nt - 1) / nt, cap));
}

// ------------------------------------------------------------------- API
// (C linkage comes from the declarations in tabsimplex.h)

const char* lp_version(void) { return "tabsimplex 0.2 (sm_103a)"; }

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
    o->precision = LP_PREC_FP64;
    o->eps_d_fp32 = 1e-5;
    o->eps_p_fp32 = 1e-6;
    o->recover_tol = 1e-9;
    o->cleanup_max = 1000;
    o->layout = LP_LAYOUT_CONDENSED;
    o->gpu_share = 0.95;
    o->cpu_threads = 0;
}

static void destroy_impl(lp_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    dev_free(h, h->logs);
    dev_free(h, h->work.blk);
    dev_free(h, h->rec.vec);
    dev_free(h, h->rec.kb);
    dev_free(h, h->common);
    dev_free(h, h->inputs);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& e : h->ev) event_put(e, true);
    event_put(h->ready, false);
    if (h->own_stream && h->stream) stream_put(h->stream);
    delete h;
}

void lp_destroy(lp_t h) { destroy_impl(h); }

// The handle's timing events, created on first use (a server creates and
// destroys many handles; most never time anything).
static bool ensure_events(lp_handle* h) {
    for (auto& e : h->ev)
        if (!e && !(e = event_get(true))) {
            set_error("cudaEventCreate failed: %s", cudaGetErrorString(cudaGetLastError()));
            return false;
        }
    return true;
}

// Common part of the two create calls: sizes, stream, events, state block.
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
    cudaGetDevice(&h->device);
    current_allocator(&h->alloc, &h->dealloc, &h->alloc_ctx);
    if (own_stream) {
        if (!(h->stream = stream_get())) {
            set_error("lp_create: cudaStreamCreate failed: %s", cudaGetErrorString(cudaGetLastError()));
            delete h;
            return nullptr;
        }
        h->own_stream = true;
    } else {
        h->stream = stream;
    }
    const bool ok = (h->ready = event_get(false)) != nullptr;
    if (!ok) {
        set_error("lp_create: cudaEventCreate failed");
        destroy_impl(h);
        return nullptr;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    h->max_grid = std::max(1, nsm) * 32;   // rpart capacity (>= any co-resident grid)
    Carve cv;
    const size_t o_st = cv.take(sizeof(DevState));
    const size_t o_bs = cv.take((size_t)m * sizeof(int));
    const size_t o_sol = cv.take((size_t)(n + m + 1) * sizeof(double));
    if (!dev_alloc_block(h, h->common, align_up(cv.off, 256))) {
        set_error("lp_create: device allocation of %zu bytes failed", cv.off);
        destroy_impl(h);
        return nullptr;
    }
    char* base = (char*)h->common.ptr;
    h->st = (DevState*)(base + o_st);
    h->basis = (int*)(base + o_bs);
    h->sol = (double*)(base + o_sol);
    return h;
}

// Validates the device-resident inputs; returns false (and sets the error) if
// bad.  `done` (may be null) is recorded on the handle stream after the check.
static bool validate_inputs(lp_handle* h, cudaEvent_t done = nullptr) {
    k_reset_state<<<1, 32, 0, h->stream>>>(h->st);
    const size_t total = (size_t)h->m * h->n + h->m + h->n;
    int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
    k_validate<<<grid, 256, 0, h->stream>>>(h->m, h->n, h->A, h->b, h->c, h->st);
    if (done) cudaEventRecord(done, h->stream);
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

const double* tsx::host_alias(const double* p, size_t count) {
    if (!p || count == 0) return nullptr;
    cudaPointerAttributes a0{}, a1{};
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, p + (count - 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer ||
        !a1.devicePointer)
        return nullptr;
    const char* d0 = static_cast<const char*>(a0.devicePointer);
    if (static_cast<const char*>(a1.devicePointer) - d0 != (ptrdiff_t)((count - 1) * sizeof(double)))
        return nullptr;   // not one mapping
    return reinterpret_cast<const double*>(d0);
}

cudaError_t tsx::launch_ingest(const double* sA, double* dA, size_t mn, const double* sb, double* db, size_t m,
                               const double* sc, double* dc, size_t n, DevState* st, cudaStream_t s) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    k_ingest<<<std::max(1, nsm) * 2, 256, 0, s>>>(sA, dA, mn, sb, db, m, sc, dc, n, st);
    return cudaGetLastError();
}

lp_t lp_create(int m, int n, const double* A, const double* b, const double* c) {
    if (!A || !b || !c) {
        set_error("lp_create: NULL input array");
        return nullptr;
    }
    const auto t_call = std::chrono::steady_clock::now();
    lp_handle* h = create_common(m, n, nullptr, true);
    if (!h) return nullptr;
    if (!ensure_events(h)) {
        destroy_impl(h);
        return nullptr;
    }
    const size_t mn = (size_t)m * (size_t)n;
    Carve cv;
    const size_t o_A = cv.take(mn * sizeof(double));
    const size_t o_b = cv.take((size_t)m * sizeof(double));
    const size_t o_c = cv.take((size_t)n * sizeof(double));
    if (!dev_alloc_block(h, h->inputs, align_up(cv.off, 256))) {
        set_error("lp_create: device allocation of %zu input bytes failed", cv.off);
        destroy_impl(h);
        return nullptr;
    }
    char* base = (char*)h->inputs.ptr;
    h->A = (const double*)(base + o_A);
    h->b = (const double*)(base + o_b);
    h->c = (const double*)(base + o_c);
    const double* gA = host_alias(A, mn);
    const double* gb = gA ? host_alias(b, (size_t)m) : nullptr;
    const double* gc = gb ? host_alias(c, (size_t)n) : nullptr;
    if (gc) {
        // page-locked inputs: one kernel reads them over the host link,
        // stores them and checks them (the check's time is part of the copy)
        cudaEventRecord(h->ev[0], h->stream);
        k_reset_state<<<1, 32, 0, h->stream>>>(h->st);
        cudaError_t e = launch_ingest(gA, (double*)h->A, mn, gb, (double*)h->b, (size_t)m, gc, (double*)h->c, (size_t)n, h->st,
                                      h->stream);
        cudaEventRecord(h->ev[1], h->stream);
        int bad = 0;
        if (e != cudaSuccess || cudaMemcpyAsync(&bad, &h->st->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            set_error("lp_create: reading the inputs failed: %s", cudaGetErrorString(cudaGetLastError()));
            destroy_impl(h);
            return nullptr;
        }
        if (bad) {
            set_error("lp_create: inputs must be finite with b >= 0");
            destroy_impl(h);
            return nullptr;
        }
        float ms_copy = 0.f;
        cudaEventElapsedTime(&ms_copy, h->ev[0], h->ev[1]);
        cudaEventRecord(h->ready, h->stream);
        h->create_ms[0] = ms_copy;
        h->create_ms[1] = 0.0;
        h->create_ms[2] = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t_call).count();
        return h;
    }
    cudaEventRecord(h->ev[0], h->stream);
    if (cudaMemcpyAsync((void*)h->A, A, mn * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync((void*)h->b, b, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync((void*)h->c, c, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
        set_error("lp_create: host-to-device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
        destroy_impl(h);
        return nullptr;
    }
    cudaEventRecord(h->ev[1], h->stream);
    if (!validate_inputs(h, h->ev[2])) {
        destroy_impl(h);
        return nullptr;
    }
    float ms_copy = 0.f, ms_check = 0.f;
    cudaEventElapsedTime(&ms_copy, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&ms_check, h->ev[1], h->ev[2]);
    cudaEventRecord(h->ready, h->stream);
    h->create_ms[0] = ms_copy;
    h->create_ms[1] = ms_check;
    h->create_ms[2] = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t_call).count();
    return h;
}

lp_t tsx::create_device_unchecked(int m, int n, const double* dA, const double* db, const double* dc,
                                 cudaStream_t stream) {
    if (!dA || !db || !dc) {
        set_error("lp_create_device: NULL input pointer");
        return nullptr;
    }
    lp_handle* h = create_common(m, n, stream, false);
    if (!h) return nullptr;
    h->A = dA;
    h->b = db;
    h->c = dc;
    h->checked = false;
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

// Leading dimension of a tableau of `elem`-byte entries: 128-byte rows.
static int tableau_ld(int W, int elem) { return (int)align_up((size_t)W, 128 / elem); }

// (Re)allocates the pivot buffers for a tableau of `elem`-byte entries.
static lp_status ensure_work(lp_handle* h, int elem, int cond) {
    if (h->work.elem == elem && h->work.cond == cond && h->work.blk.ptr) return LP_OPTIMAL;
    dev_free(h, h->work.blk);
    h->work = Work{};
    const int Ws = cond ? h->n + 1 : h->W;
    const int ld = tableau_ld(Ws, elem);
    const int E = 32 / elem;
    const int nstrips = (ld + 32 * E - 1) / (32 * E);
    Carve cv;
    const size_t o_T = cv.take((size_t)(h->m + 1) * (size_t)ld * elem);
    const size_t o_F = cv.take((size_t)(h->m + 1) * elem);
    const size_t o_R = cv.take((size_t)ld * elem);
    const size_t o_act = cv.take((size_t)(ld / E) * sizeof(int));
    const size_t o_cp = cv.take((size_t)nstrips * sizeof(ArgPart));
    const size_t o_rp = cv.take((size_t)h->max_grid * sizeof(RatPart));
    const size_t o_var = cv.take((size_t)h->n * sizeof(int));
    if (!dev_alloc_block(h, h->work.blk, align_up(cv.off, 256))) {
        set_error("lp_solve: device allocation of %zu bytes for the tableau failed", cv.off);
        return LP_ERR_NOMEM;
    }
    char* base = (char*)h->work.blk.ptr;
    h->work.elem = elem;
    h->work.cond = cond;
    h->work.Ws = Ws;
    h->work.ld = ld;
    h->work.var = (int*)(base + o_var);
    h->work.T = base + o_T;
    h->work.F = base + o_F;
    h->work.R = base + o_R;
    h->work.act = (int*)(base + o_act);
    h->work.cpart = (ArgPart*)(base + o_cp);
    h->work.rpart = (RatPart*)(base + o_rp);
    return LP_OPTIMAL;
}

// Dynamic shared memory of the persistent kernel: the update's bulk-copy
// rings (one per warp).
template <int NT>
static size_t persistent_smem() {
    return tma_smem_bytes(NT);
}

// Rows of an update slot of the persistent kernel for an LP with m rows:
// persistent_rows(NT), or 8 below 3072 rows, where 16-row slots are too few
// to spread evenly over the grid's warps (measured against 16: 1024² +17 %,
// 2048² +2.5 %, 4096² -3 %).
template <int NT>
static int persistent_slot_rows(int m) {
    return persistent_rows(NT) > 8 && m < 3072 ? 8 : persistent_rows(NT);
}

template <int NT, typename V>
static const void* persistent_kernel(int m) {
    if constexpr (persistent_rows(NT) > 8) {
        if (persistent_slot_rows<NT>(m) == 8) return (const void*)k_pivot_persistent<NT, V, 8>;
    }
    return (const void*)k_pivot_persistent<NT, V>;
}

template <int NT, typename V>
static void allow_persistent_smem() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(persistent_kernel<NT, V>(1 << 30), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)persistent_smem<NT>());
        cudaFuncSetAttribute(persistent_kernel<NT, V>(1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)persistent_smem<NT>());
    });
}

template <int NT, typename V>
static cudaError_t launch_persistent(const Params<V>& P, int grid, cudaStream_t s) {
    allow_persistent_smem<NT, V>();
    void* args[] = {(void*)&P};
    return cudaLaunchCooperativeKernel(persistent_kernel<NT, V>(P.m), grid, NT, args, persistent_smem<NT>(), s);
}

template <int NT, typename V>
static int max_coresident(int device) {
    allow_persistent_smem<NT, V>();
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pivot_persistent<NT, V>, NT, persistent_smem<NT>());
    return nsm * per;
}

template <int NT, typename V>
static lp_status run_multilaunch(const Params<V>& P, int grid, cudaStream_t s, long long& launches) {
    k_ml_init<V><<<grid, NT, 0, s>>>(P);
    ++launches;
    int status = kRunning;
    int batch = 4;
    for (;;) {
        for (int k = 0; k < batch; ++k) {
            k_ml_select<NT, V><<<grid, NT, 0, s>>>(P);
            k_ml_stage<NT, V><<<grid, NT, 0, s>>>(P);
            k_ml_update<NT, V><<<grid, NT, 0, s>>>(P);
            launches += 3;
        }
        CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
        CUDA_TRY(cudaMemcpyAsync(&status, &P.st->status, sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
        CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
        if (status != kRunning) break;
        batch = std::min(batch * 2, 64);
    }
    return (lp_status)status;
}

// Pivot-kernel parameters over a tableau of V with the given buffers.
template <typename V>
static Params<V> make_params(int m, int n, int ld, V* T, V* F, V* R, int* act, ArgPart* cpart, RatPart* rpart,
                             DevState* st, int* basis, const lp_options& o, double eps_d, double eps_p,
                             int* var = nullptr) {
    constexpr int E = Lanes<V>::E;
    Params<V> P{};
    P.T = T;
    P.ld = ld;
    P.m = m;
    P.n = n;
    P.cond = var ? 1 : 0;
    P.var = var;
    P.W = var ? n + 1 : n + m + 1;
    P.basis = basis;
    P.F = F;
    P.R = R;
    P.act = act;
    P.cpart = cpart;
    P.rpart = rpart;
    P.st = st;
    P.eps_d = eps_d;
    P.eps_p = eps_p;
    P.max_iters = o.max_iters < 0 ? 50LL * ((long long)m + n) : o.max_iters;
    P.k_cyc = o.k_cyc;
    P.rule = o.rule;
    P.timeout_ns = std::max(0LL, o.barrier_timeout_ns);
    P.nstrips = (ld + 32 * E - 1) / (32 * E);
    P.skip_zero = o.skip_zero_columns ? 1 : 0;
    return P;
}

// Grid of the pivot kernels: enough warps for the update slots (`rows` rows
// each), at most `resident` blocks.
template <int NT, typename V>
static int update_grid(int m, int ld, int rows, int resident, int max_grid, int user_blocks) {
    constexpr int E = Lanes<V>::E;
    const long long slots = (long long)((ld / E + 31) / 32) * (((long long)m + rows - 1) / rows);
    const long long want = (slots + NT / 32 - 1) / (NT / 32);
    int grid = (int)std::min<long long>(std::max<long long>(1, want), std::max(1, resident));
    grid = std::min(grid, max_grid);
    if (user_blocks > 0) grid = std::min(grid, user_blocks);
    return grid;
}

template <int NT, typename V>
static int pivot_grid(int device, int m, int ld, int max_grid, int user_blocks, int& coresident) {
    coresident = max_coresident<NT, V>(device);
    return update_grid<NT, V>(m, ld, persistent_slot_rows<NT>(m), coresident, max_grid, user_blocks);
}

// Grid of the one-launch-per-phase path: its update kernel keeps two blocks
// of 256 threads on an SM.
template <int NT, typename V>
static int multilaunch_grid(int device, int m, int ld, int max_grid, int user_blocks) {
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ml_update<NT, V>, NT, 0);
    return update_grid<NT, V>(m, ld, kRowsInFlight, std::max(1, nsm * per), max_grid, user_blocks);
}

// ------------------------------------------------------- cluster path
// An FP64 condensed LP whose tableau fits the shared memory of one cluster of
// up to 16 blocks is solved by k_cluster_solve (tsx_cluster.cuh).  The
// cluster size: the smallest power of two giving each block at most 16
// constraint rows (more blocks add FP64 pipes; fewer cut the barrier's
// reach), raised until the block's rows fit its shared memory, and lowered
// when the device cannot co-schedule that many blocks with that much shared
// memory.  0: the LP does not fit a cluster.
template <int NT>
static size_t cluster_static_smem() {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k_cluster_solve<NT>);
    return fa.sharedSizeBytes;
}

template <int NT>
static cudaError_t cluster_allow(size_t smem) {
    static std::mutex mu;
    static size_t allowed = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (smem <= allowed) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute((const void*)k_cluster_solve<NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_cluster_solve<NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) allowed = smem;
    return e;
}

template <int NT>
static cudaLaunchConfig_t cluster_config(int C, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int NT>
static int cluster_size_for(int device, int m, int n) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t limit = (size_t)std::max(0, optin) > cluster_static_smem<NT>() + 256
                             ? (size_t)optin - cluster_static_smem<NT>() - 256
                             : 0;
    int C = 1;
    while (C < kClusterMax && cluster_rows_per(m, C) > 16) C *= 2;
    while (C <= kClusterMax && cluster_smem_bytes(m, n, C) > limit) C *= 2;
    for (; C >= 1; C /= 2) {
        const size_t smem = cluster_smem_bytes(m, n, C);
        if (smem > limit) return 0;
        if (cluster_allow<NT>(smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config<NT>(C, smem, nullptr, attr);
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, (const void*)k_cluster_solve<NT>, &cfg) == cudaSuccess &&
            nclusters > 0)
            return C;
        cudaGetLastError();
    }
    return 0;
}

template <int NT>
static cudaError_t launch_cluster(const ClusterParams& P, int C, cudaStream_t s) {
    const size_t smem = cluster_smem_bytes(P.m, P.n, C);
    cudaError_t e = cluster_allow<NT>(smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config<NT>(C, smem, s, attr);
    return cudaLaunchKernelEx(&cfg, k_cluster_solve<NT>, P);
}

// ------------------------------------------------------- hybrid path
// The paper's CPU+GPU split (Section IV) on the handle's built condensed
// tableau: the first nG = round(gpu_share n) column slots and a copy of the
// right-hand side go to a GPU tableau for k_pivot_hybrid (tsx_hybrid.cuh), the
// other slots and another copy of the right-hand side to host memory for the
// host team (tsx_hybrid_host.h); both run to the end, then the parts are put
// back into the handle's tableau, var[] and basis, and the GPU's state words
// into the handle's (the caller reads the status from there).
template <int NT>
static lp_status run_hybrid(lp_handle* h, const lp_options& o, cudaStream_t s, const Params<double>& Pf,
                            double eps_d, double eps_p, long long& launches, int& grid_used) {
    const int m = h->m, n = h->n, ld = h->work.ld;
    const int nG = (int)std::min<long long>(n, std::max<long long>(0, std::llround(o.gpu_share * n)));
    const int nC = n - nG;
    const int ldG = tableau_ld(nG + 1, 8), ldC = nC + 1;
    const int nstrips = (ldG + 127) / 128;
    double* T = (double*)h->work.T;
    // the GPU part
    Carve cv;
    const size_t o_T = cv.take((size_t)(m + 1) * ldG * 8), o_F = cv.take((size_t)(m + 1) * 8);
    const size_t o_R = cv.take((size_t)ldG * 8), o_cp = cv.take((size_t)nstrips * sizeof(ArgPart));
    const size_t o_rp = cv.take((size_t)h->max_grid * sizeof(RatPart)), o_var = cv.take((size_t)std::max(1, nG) * 4);
    const size_t o_bas = cv.take((size_t)m * 4), o_st = cv.take(sizeof(DevState));
    Block gblk;
    if (!dev_alloc_block(h, gblk, align_up(cv.off, 256))) {
        set_error("lp_solve: device allocation of the hybrid path's GPU part failed");
        return LP_ERR_NOMEM;
    }
    char* gb = (char*)gblk.ptr;
    double* TG = (double*)(gb + o_T);
    int* varG = (int*)(gb + o_var);
    int* basG = (int*)(gb + o_bas);
    DevState* stG = (DevState*)(gb + o_st);
    // the host part (pageable) and the mailbox with the column buffers (mapped)
    std::vector<double> TC((size_t)(m + 1) * ldC), FC((size_t)m + 1), RC((size_t)ldC);
    std::vector<int> varC(std::max(1, nC)), basC(m);
    const size_t mbytes = sizeof(HybMailbox) + 4 * ((size_t)m + 1) * sizeof(double);
    char* mh = nullptr;
    char* md = nullptr;
    lp_status rc = LP_OPTIMAL;
    auto fail = [&](lp_status st, const char* what) {
        set_error("lp_solve (hybrid): %s", what);
        rc = st;
    };
    if (cudaHostAlloc((void**)&mh, mbytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&md, mh, 0) != cudaSuccess) {
        cudaGetLastError();
        if (mh) cudaFreeHost(mh);
        dev_free(h, gblk);
        set_error("lp_solve (hybrid): mapped host memory for the mailbox failed");
        return LP_ERR_NOMEM;
    }
    memset(mh, 0, mbytes);
    HybMailbox* mb = (HybMailbox*)mh;
    double* gF = (double*)(mh + sizeof(HybMailbox));
    double* cF = gF + 2 * ((size_t)m + 1);
    // split the built tableau
    {
        std::vector<int> iota(std::max(1, nG));
        for (int j = 0; j < nG; ++j) iota[j] = j;
        for (int j = 0; j < nC; ++j) varC[j] = nG + j;
        bool ok = cudaMemsetAsync(TG, 0, (size_t)(m + 1) * ldG * 8, s) == cudaSuccess;
        if (nG > 0)
            ok = ok && cudaMemcpy2DAsync(TG, (size_t)ldG * 8, T, (size_t)ld * 8, (size_t)nG * 8, m + 1,
                                         cudaMemcpyDeviceToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpy2DAsync(TG + nG, (size_t)ldG * 8, T + n, (size_t)ld * 8, 8, m + 1,
                                     cudaMemcpyDeviceToDevice, s) == cudaSuccess;
        if (nC > 0)
            ok = ok && cudaMemcpy2DAsync(TC.data(), (size_t)ldC * 8, T + nG, (size_t)ld * 8, (size_t)nC * 8, m + 1,
                                         cudaMemcpyDeviceToHost, s) == cudaSuccess;
        ok = ok && cudaMemcpy2DAsync(TC.data() + nC, (size_t)ldC * 8, T + n, (size_t)ld * 8, 8, m + 1,
                                     cudaMemcpyDeviceToHost, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(basG, h->basis, (size_t)m * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(basC.data(), h->basis, (size_t)m * 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
        if (nG > 0)
            ok = ok && cudaMemcpyAsync(varG, iota.data(), (size_t)nG * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
        k_reset_state<<<1, 32, 0, s>>>(stG);
        ok = ok && cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
        if (!ok) fail(LP_ERR_CUDA, "splitting the tableau failed");
    }
    if (rc == LP_OPTIMAL) {
        Params<double> P = make_params<double>(m, nG, ldG, TG, (double*)(gb + o_F), (double*)(gb + o_R), nullptr,
                                               (ArgPart*)(gb + o_cp), (RatPart*)(gb + o_rp), stG, basG, o, eps_d,
                                               eps_p, varG);
        P.log_cap = Pf.log_cap;
        P.qlog = Pf.qlog;
        P.plog = Pf.plog;
        int coresident = 0;
        const int grid = pivot_grid<NT, double>(h->device, m, ldG, h->max_grid, o.blocks, coresident);
        HybParams HP{};
        HP.mb = (HybMailbox*)md;
        HP.gF = (double*)(md + sizeof(HybMailbox));
        HP.cF = HP.gF + 2 * ((size_t)m + 1);
        HP.wait_ns = std::max(0LL, o.barrier_timeout_ns);
        void* args[] = {(void*)&P, (void*)&HP};
        if (cudaLaunchCooperativeKernel((const void*)k_pivot_hybrid<NT>, grid, NT, args, 0, s) != cudaSuccess) {
            cudaGetLastError();
            fail(LP_ERR_CUDA, "cooperative launch of the GPU part failed");
        } else {
            ++launches;
            grid_used = grid;
            HybHost H;
            H.m = m;
            H.nC = nC;
            H.ldC = ldC;
            H.T = TC.data();
            H.var = varC.data();
            H.basis = basC.data();
            H.F = FC.data();
            H.R = RC.data();
            H.mb = mb;
            H.gF = gF;
            H.cF = cF;
            H.eps_d = eps_d;
            H.eps_p = eps_p;
            H.max_iters = P.max_iters;
            H.k_cyc = o.k_cyc;
            H.rule = o.rule;
            H.wait_ns = std::max(1LL, o.barrier_timeout_ns);
            const int hw = (int)std::thread::hardware_concurrency();
            H.nthreads = o.cpu_threads > 0 ? o.cpu_threads : std::max(1, hw - 1);
            HybTeam team(H);
            team.run();
            DevState gs{};
            if (cudaMemcpyAsync(&gs, stG, sizeof gs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                cudaGetLastError();
                fail(LP_ERR_CUDA, "the GPU part failed");
            } else if (gs.status == kTimeout || H.status == kTimeout) {
                gs.status = kTimeout;
                set_error("lp_solve (hybrid): a wait for the other side exceeded %lld ns", (long long)HP.wait_ns);
            } else if (gs.status != H.status || gs.iters != H.iters) {
                fail(LP_ERR_CUDA, "the GPU and host parts ended differently");
            }
            if (rc == LP_OPTIMAL) {
                // put the parts back: slots [0, nG) and the right-hand side from the
                // GPU, [nG, n) from the host; var[], basis and the state words
                bool ok = true;
                if (nG > 0) {
                    ok = ok && cudaMemcpy2DAsync(T, (size_t)ld * 8, TG, (size_t)ldG * 8, (size_t)nG * 8, m + 1,
                                                 cudaMemcpyDeviceToDevice, s) == cudaSuccess;
                    ok = ok && cudaMemcpyAsync(h->work.var, varG, (size_t)nG * 4, cudaMemcpyDeviceToDevice, s) ==
                                   cudaSuccess;
                }
                ok = ok && cudaMemcpy2DAsync(T + n, (size_t)ld * 8, TG + nG, (size_t)ldG * 8, 8, m + 1,
                                             cudaMemcpyDeviceToDevice, s) == cudaSuccess;
                if (nC > 0) {
                    ok = ok && cudaMemcpy2DAsync(T + nG, (size_t)ld * 8, TC.data(), (size_t)ldC * 8, (size_t)nC * 8,
                                                 m + 1, cudaMemcpyHostToDevice, s) == cudaSuccess;
                    ok = ok && cudaMemcpyAsync(h->work.var + nG, varC.data(), (size_t)nC * 4, cudaMemcpyHostToDevice,
                                               s) == cudaSuccess;
                }
                ok = ok && cudaMemcpyAsync(h->basis, basG, (size_t)m * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
                ok = ok && cudaMemcpyAsync(h->st, &gs, sizeof gs, cudaMemcpyHostToDevice, s) == cudaSuccess;
                ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
                if (!ok) fail(LP_ERR_CUDA, "reassembling the tableau failed");
            }
        }
    }
    cudaStreamSynchronize(s);
    cudaFreeHost(mh);
    dev_free(h, gblk);
    return rc;
}

// Runs the pivot phase (build + Steps 1-3) on the handle's tableau of V.
template <int NT, typename V>
static lp_status pivot_phase(lp_handle* h, const lp_options& o, cudaStream_t s, double eps_d, double eps_p,
                             DevState& hs, long long& launches, int& path_used, int& grid_used) {
    const int m = h->m, n = h->n;
    const int ld = h->work.ld;
    Params<V> P = make_params<V>(m, n, ld, (V*)h->work.T, (V*)h->work.F, (V*)h->work.R, h->work.act,
                                 h->work.cpart, h->work.rpart, h->st, h->basis, o, eps_d, eps_p,
                                 h->work.cond ? h->work.var : nullptr);
    P.log_cap = o.log_capacity > 0 ? h->log_cap : 0;
    P.qlog = P.log_cap ? (int*)h->logs.ptr : nullptr;
    P.plog = P.log_cap ? (int*)h->logs.ptr + P.log_cap : nullptr;

    int coresident = 0;
    const int grid = pivot_grid<NT, V>(h->device, m, ld, h->max_grid, o.blocks, coresident);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    int path = o.path;
    // the cluster path: FP64, condensed tableau, small enough for one cluster
    int csize = 0;
    const bool cluster_ok = sizeof(V) == 8 && h->work.cond && (path == LP_PATH_AUTO || path == LP_PATH_CLUSTER);
    if (cluster_ok) csize = cluster_size_for<NT>(h->device, m, n);
    if (path == LP_PATH_CLUSTER && !csize) {
        set_error("lp_solve: the cluster path needs an FP64 condensed tableau that fits one cluster's shared memory");
        return LP_ERR_INVALID;
    }
    if (path == LP_PATH_HYBRID && !(sizeof(V) == 8 && h->work.cond)) {
        set_error("lp_solve: the hybrid path needs an FP64 condensed tableau");
        return LP_ERR_INVALID;
    }
    if (path == LP_PATH_HYBRID && (!coop || coresident <= 0)) {
        set_error("lp_solve: the hybrid path needs a cooperative launch");
        return LP_ERR_CUDA;
    }
    if (path == LP_PATH_AUTO && csize) path = LP_PATH_CLUSTER;
    if (path == LP_PATH_AUTO) path = (coop && coresident > 0) ? LP_PATH_PERSISTENT : LP_PATH_MULTILAUNCH;
    if (path == LP_PATH_PERSISTENT && (!coop || coresident <= 0)) {
        set_error("lp_solve: persistent path requested but cooperative launch is unavailable");
        return LP_ERR_CUDA;
    }

    // Initialization Step
    cudaEventRecord(h->ev[0], s);
    k_reset_state<<<1, 32, 0, s>>>(h->st);
    {
        constexpr int E = Lanes<V>::E;
        const size_t groups = (size_t)(m + 1) * (size_t)(ld / E);
        int g = (int)std::min<size_t>((groups + 255) / 256, 152 * 16);
        k_build<V><<<g, 256, 0, s>>>(m, n, h->work.Ws, ld, h->A, h->b, h->c, (V*)h->work.T, h->basis,
                                     h->work.cond ? h->work.var : nullptr);
    }
    CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    cudaEventRecord(h->ev[1], s);
    launches += 2;

    int grid_run = grid;
    if constexpr (sizeof(V) == 8) {
        if (path == LP_PATH_HYBRID) {
            const lp_status hr = run_hybrid<NT>(h, o, s, P, eps_d, eps_p, launches, grid_run);
            if (hr != LP_OPTIMAL) return hr;
        }
    }
    if (path == LP_PATH_CLUSTER) {
        ClusterParams CP{};
        CP.T = (double*)h->work.T;
        CP.ldg = ld;
        CP.m = m;
        CP.n = n;
        CP.basis = h->basis;
        CP.var = h->work.var;
        CP.st = h->st;
        CP.qlog = P.qlog;
        CP.plog = P.plog;
        CP.log_cap = P.log_cap;
        CP.eps_d = eps_d;
        CP.eps_p = eps_p;
        CP.max_iters = o.max_iters;
        CP.k_cyc = o.k_cyc;
        CP.rule = o.rule;
        cudaError_t e = launch_cluster<NT>(CP, csize, s);
        if (e != cudaSuccess) {
            set_error("lp_solve: cluster launch failed: %s", cudaGetErrorString(e));
            return LP_ERR_CUDA;
        }
        ++launches;
        grid_run = csize;
    }
    if (path == LP_PATH_PERSISTENT) {
        cudaError_t e = launch_persistent<NT, V>(P, grid, s);
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
        grid_run = multilaunch_grid<NT, V>(h->device, m, ld, h->max_grid, o.blocks);
        if (run_multilaunch<NT, V>(P, grid_run, s, launches) == LP_ERR_CUDA) return LP_ERR_CUDA;
    }
    cudaEventRecord(h->ev[2], s);
    CUDA_TRY(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    path_used = path;
    grid_used = grid_run;
    if (hs.status == kRunning) {
        set_error("lp_solve: kernel ended without a status");
        return LP_ERR_CUDA;
    }
    if (hs.status == kTimeout) set_error("lp_solve: a grid barrier wait exceeded %lld ns", (long long)P.timeout_ns);
    return (lp_status)hs.status;
}

// ------------------------------------------------------------ FP64 recovery
constexpr int kRecMaxGrid = 152 * 8;   // blocks of the in-place refactorisation, upper bound

static lp_status ensure_recovery(lp_handle* h, int k) {
    RecBufs& r = h->rec;
    const int m = h->m, n = h->n;
    if (!r.vec.ptr) {
        Carve cv;
        const size_t o_s = cv.take((size_t)m * 8), o_aZ = cv.take((size_t)m * 8);
        const size_t o_d = cv.take((size_t)n * 8), o_ar = cv.take((size_t)n * 8);
        const size_t o_ib = cv.take((size_t)(n + m) * 4), o_ir = cv.take((size_t)m * 4);
        const size_t o_rst = cv.take(sizeof(DevState)), o_chk = cv.take(sizeof(RecCheck));
        const size_t o_ch = cv.take(sizeof(RecChoice)), o_sg = cv.take(sizeof(int));
        if (!dev_alloc_block(h, r.vec, align_up(cv.off, 256))) {
            set_error("lp_solve: allocation of the recovery vectors failed");
            return LP_ERR_NOMEM;
        }
        char* b = (char*)r.vec.ptr;
        r.s = (double*)(b + o_s);
        r.aZ = (double*)(b + o_aZ);
        r.d = (double*)(b + o_d);
        r.arow = (double*)(b + o_ar);
        r.isbasic = (int*)(b + o_ib);
        r.inR = (int*)(b + o_ir);
        r.rst = (DevState*)(b + o_rst);
        r.chk = (RecCheck*)(b + o_chk);
        r.choice = (RecChoice*)(b + o_ch);
        r.singular = (int*)(b + o_sg);
    }
    if (k > r.kcap) {
        dev_free(h, r.kb);
        const int kc = std::max(std::max(k, 2 * std::max(r.kcap, 0)), 16);
        const size_t K = (size_t)kc;
        Carve cv;
        const size_t o_M = cv.take(K * 2 * K * 8), o_inv = cv.take(K * K * 8);
        size_t o_v[9];
        for (auto& o : o_v) o = cv.take(K * 8);
        size_t o_i[3];
        for (auto& o : o_i) o = cv.take(K * 4);
        const size_t o_ps = cv.take(K * 4), o_dp = cv.take(K * 8);
        const size_t o_parts = cv.take(2 * (size_t)kRecMaxGrid * sizeof(PivVal));
        if (!dev_alloc_block(h, r.kb, align_up(cv.off, 256))) {
            set_error("lp_solve: allocation of the recovery matrices (k = %d) failed", k);
            r.kcap = -1;
            return LP_ERR_NOMEM;
        }
        char* b = (char*)r.kb.ptr;
        r.M = (double*)(b + o_M);
        r.inv = (double*)(b + o_inv);
        double** vs[9] = {&r.xS, &r.yR, &r.bR, &r.cS, &r.rp, &r.rd, &r.aS, &r.rho, &r.venter};
        for (int t = 0; t < 9; ++t) *vs[t] = (double*)(b + o_v[t]);
        int** is[3] = {&r.pivrow, &r.S, &r.Rr};
        for (int t = 0; t < 3; ++t) *is[t] = (int*)(b + o_i[t]);
        r.pivstep = (int*)(b + o_ps);
        r.dpiv = (double*)(b + o_dp);
        r.parts = b + o_parts;
        r.kcap = kc;
    }
    return LP_OPTIMAL;
}

// Refactorises A_RS for the sets (S, R), solves x_S and y_R (one refinement
// step), computes the slacks and the objective-row entries, and runs the
// checks.  Fills `chk`.  Returns LP_ERR_NUMERIC if A_RS is singular.
static lp_status recover_factor(lp_handle* h, const lp_options& o, cudaStream_t s, const std::vector<int>& S,
                                const std::vector<int>& R, RecCheck& chk, long long& launches) {
    RecBufs& r = h->rec;
    const int m = h->m, n = h->n, k = (int)S.size();
    lp_status st = ensure_recovery(h, k);
    if (st != LP_OPTIMAL) return st;
    if (k > 0) {
        CUDA_TRY(cudaMemcpyAsync(r.S, S.data(), (size_t)k * 4, cudaMemcpyHostToDevice, s), LP_ERR_CUDA);
        CUDA_TRY(cudaMemcpyAsync(r.Rr, R.data(), (size_t)k * 4, cudaMemcpyHostToDevice, s), LP_ERR_CUDA);
    }
    k_rec_flags<<<grid_for(n + m, 256, 4096), 256, 0, s>>>(m, n, r.S, r.Rr, k, r.isbasic, r.inR);
    k_rec_flags2<<<grid_for(k, 256, 4096), 256, 0, s>>>(m, n, r.S, r.Rr, k, r.isbasic, r.inR);
    launches += 2;
    int singular = 0;
    if (k > 0) {
        const size_t kk = (size_t)k;
        CUDA_TRY(cudaMemsetAsync(r.singular, 0, 4, s), LP_ERR_CUDA);
        k_reset_state<<<1, 32, 0, s>>>(r.rst);
        int nsm = 0, per = 0, optin = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        const size_t bits = sizeof(unsigned) * ((kk + 31) / 32);
        int* sg = r.singular;
        int* pv = r.pivrow;
        double* Mx = r.M;
        DevState* rs = r.rst;
        long long to = std::max(0LL, o.barrier_timeout_ns);
        int kv = k;
        const size_t smem_ip = kk * 8 + bits;   // pivot row + used-row bitmap
        static std::once_flag once;
        static size_t ip_limit = 0;             // dynamic shared memory the in-place kernel may use
        std::call_once(once, [optin] {
            cudaFuncAttributes fa{};
            if (cudaFuncGetAttributes(&fa, k_rec_gj_inplace<256>) == cudaSuccess &&
                (size_t)optin > fa.sharedSizeBytes) {
                const size_t lim = (size_t)optin - fa.sharedSizeBytes;
                if (cudaFuncSetAttribute((const void*)k_rec_gj_inplace<256>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) == cudaSuccess)
                    ip_limit = lim;
            }
            cudaGetLastError();   // a refused attribute must not surface as a later launch's error
        });
        if (smem_ip <= ip_limit) {
            // in place on the k x k block (k_rec_gj_inplace)
            k_rec_gather_square<<<grid_for((long long)(kk * kk), 256, 152 * 16), 256, 0, s>>>(n, h->A, r.S, r.Rr, k,
                                                                                            r.M);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rec_gj_inplace<256>, 256, smem_ip);
            int g = std::max(1, std::min(std::min(nsm * std::max(per, 1), kRecMaxGrid),
                                         grid_for(32LL * k, 256, 1 << 20)));
            if (o.blocks > 0) g = std::min(g, o.blocks);   // blocks per LP
            double* dp = r.dpiv;
            PivVal* parts = (PivVal*)r.parts;
            void* args[] = {&Mx, &kv, &pv, &dp, &parts, &sg, &rs, &to};
            CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_rec_gj_inplace<256>, g, 256, args, smem_ip, s),
                     LP_ERR_CUDA);
            k_rec_pivstep<<<grid_for(k, 256, 1024), 256, 0, s>>>(r.pivrow, k, r.pivstep);
            k_rec_finish_inplace<<<grid_for((long long)(kk * kk), 256, 152 * 16), 256, 0, s>>>(r.M, k, r.pivrow,
                                                                                             r.pivstep, r.dpiv, r.inv);
            launches += 2;
        } else {
            // [A_RS | I] (k x 2k), for k beyond the in-place kernel's shared memory
            if (bits > 48 * 1024) {
                set_error("lp_solve: k = %d structural basic variables exceed the refactorisation's limit", k);
                return LP_ERR_INVALID;
            }
            k_rec_gather<<<grid_for((long long)(2 * kk * kk), 256, 152 * 16), 256, 0, s>>>(n, h->A, r.S, r.Rr, k,
                                                                                          r.M);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rec_gauss_jordan<256>, 256, bits);
            int g = std::max(1, std::min(nsm * std::max(per, 1), grid_for((long long)(2 * kk * kk), 256, 1 << 20)));
            if (o.blocks > 0) g = std::min(g, o.blocks);   // blocks per LP
            void* args[] = {&Mx, &kv, &pv, &sg, &rs, &to};
            CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_rec_gauss_jordan<256>, g, 256, args, bits, s),
                     LP_ERR_CUDA);
            k_rec_finish<<<grid_for((long long)(kk * kk), 256, 152 * 16), 256, 0, s>>>(r.M, k, r.pivrow, r.inv);
        }
        k_rec_gather_rhs<<<grid_for(k, 256, 1024), 256, 0, s>>>(h->b, h->c, r.S, r.Rr, k, r.bR, r.cS);
        const int gw = grid_for(32LL * k, 256, 4096);
        k_rec_matvec<<<gw, 256, 0, s>>>(r.inv, k, r.bR, 0, nullptr, r.xS);
        k_rec_matvec<<<grid_for(k, 256, 1024), 256, 0, s>>>(r.inv, k, r.cS, 1, nullptr, r.yR);
        // one step of iterative refinement in FP64
        k_rec_residual<<<grid_for(64LL * k, 256, 4096), 256, 0, s>>>(n, h->A, r.S, r.Rr, k, r.bR, r.cS, r.xS, r.yR,
                                                                       r.rp, r.rd);
        k_rec_matvec<<<gw, 256, 0, s>>>(r.inv, k, r.rp, 0, r.xS, r.xS);
        k_rec_matvec<<<grid_for(k, 256, 1024), 256, 0, s>>>(r.inv, k, r.rd, 1, r.yR, r.yR);
        k_rec_residual<<<grid_for(64LL * k, 256, 4096), 256, 0, s>>>(n, h->A, r.S, r.Rr, k, r.bR, r.cS, r.xS, r.yR,
                                                                       r.rp, r.rd);
        launches += 11;
    }
    // slacks s = b - A_:S x_S (every row), objective row d = A_R:^T y_R - c
    k_rec_rows_dot<<<grid_for(32LL * m, 256, 8192), 256, 0, s>>>(m, n, h->A, r.S, k, h->b, -1, r.xS, r.s);
    k_rec_cols_dot<<<grid_for(n, 256, 8192), 256, 0, s>>>(n, h->A, r.Rr, k, r.yR, -1, h->c, r.d);
    k_rec_check<256><<<1, 256, 0, s>>>(m, n, r.S, r.Rr, k, r.xS, r.s, r.d, r.yR, r.isbasic, r.inR, h->b, h->c,
                                       r.rp, r.rd, r.chk);
    launches += 3;
    CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    CUDA_TRY(cudaMemcpyAsync(&chk, r.chk, sizeof(RecCheck), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaMemcpyAsync(&singular, r.singular, sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    int rstatus = kRunning;
    CUDA_TRY(cudaMemcpyAsync(&rstatus, &r.rst->status, sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    if (k > 0 && rstatus == kTimeout) {
        set_error("lp_solve: a grid barrier wait of the FP64 refactorisation exceeded its limit");
        return LP_ERR_TIMEOUT;
    }
    if (k > 0 && singular) {
        set_error("lp_solve: the final basis is singular in FP64 (k = %d)", k);
        return LP_ERR_NUMERIC;
    }
    return LP_OPTIMAL;
}

// FP64 recovery of the float phase's final basis: refactorise, check, and
// clean up with revised-form pivots until the checks pass.  Writes the read-out
// into h->sol and the final basic set into h->final_basis.
static lp_status recover(lp_handle* h, const lp_options& o, cudaStream_t s, long long& launches) {
    const int m = h->m, n = h->n;
    std::vector<int> basis(m);
    CUDA_TRY(cudaMemcpyAsync(basis.data(), h->basis, (size_t)m * 4, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    std::vector<int> S, R;
    std::vector<char> slack_basic(m, 0);
    for (int v : basis) {
        if (v < n)
            S.push_back(v);
        else
            slack_basic[v - n] = 1;
    }
    std::sort(S.begin(), S.end());
    for (int i = 0; i < m; ++i)
        if (!slack_basic[i]) R.push_back(i);
    if (S.size() != R.size()) {
        set_error("lp_solve: the float phase left an inconsistent basis");
        return LP_ERR_NUMERIC;
    }
    const double tol = o.recover_tol;
    RecBufs& r = h->rec;
    int cleanup = 0;
    RecCheck chk{};
    lp_status st = LP_OPTIMAL;
    for (;;) {
        st = recover_factor(h, o, s, S, R, chk, launches);
        if (st != LP_OPTIMAL) return st;
        const double pmin = std::min(chk.min_x, chk.min_s);
        const double dmin = std::min(chk.min_d, chk.min_y);
        if (pmin >= -tol && dmin >= -tol) break;                       // optimal in FP64
        if (cleanup >= o.cleanup_max) {
            set_error("lp_solve: FP64 cleanup did not converge in %d pivots", cleanup);
            st = LP_ERR_NUMERIC;
            break;
        }
        const int k = (int)S.size();
        int e_kind, e_at, l_kind, l_at;
        RecChoice ch{};
        if (pmin < -tol) {
            // dual step: the most negative basic value leaves
            const bool structural = chk.min_x <= chk.min_s;
            l_kind = structural ? 0 : 1;
            l_at = structural ? chk.min_x_at : chk.min_s_at;
            k_rec_rho<<<grid_for(k, 256, 1024), 256, 0, s>>>(n, h->A, r.S, k, r.inv, l_kind, l_at, r.rho);
            k_rec_cols_dot<<<grid_for(n, 256, 8192), 256, 0, s>>>(n, h->A, r.Rr, k, r.rho, l_kind == 1 ? l_at : -1,
                                                                  nullptr, r.arow);
            k_rec_dual_ratio<256><<<1, 256, 0, s>>>(n, r.Rr, k, r.arow, r.d, r.isbasic, r.rho, r.yR, 1e-9, r.choice);
            launches += 3;
            CUDA_TRY(cudaMemcpyAsync(&ch, r.choice, sizeof ch, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
            CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
            if (ch.kind < 0) {
                set_error("lp_solve: FP64 dual cleanup found no entering column");
                st = LP_ERR_NUMERIC;
                break;
            }
            e_kind = ch.kind;
            e_at = ch.at;
        } else {
            // primal step: the most negative objective-row entry enters
            const bool structural = chk.min_d <= chk.min_y;
            e_kind = structural ? 0 : 1;
            e_at = structural ? chk.min_d_at : chk.min_y_at;
            k_rec_enter_col<<<grid_for(k, 256, 1024), 256, 0, s>>>(n, h->A, r.Rr, k, e_kind, e_at, r.venter);
            k_rec_matvec<<<grid_for(32LL * k, 256, 4096), 256, 0, s>>>(r.inv, k, r.venter, 0, nullptr, r.aS);
            k_rec_rows_dot<<<grid_for(32LL * m, 256, 8192), 256, 0, s>>>(m, n, h->A, r.S, k, nullptr,
                                                                         e_kind == 0 ? e_at : -1, r.aS, r.aZ);
            k_rec_primal_ratio<256><<<1, 256, 0, s>>>(m, n, r.S, k, r.xS, r.aS, r.s, r.aZ, r.inR, 1e-9, r.choice);
            launches += 4;
            CUDA_TRY(cudaMemcpyAsync(&ch, r.choice, sizeof ch, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
            CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
            if (ch.kind < 0) {
                st = LP_UNBOUNDED;
                break;
            }
            l_kind = ch.kind;
            l_at = ch.at;
        }
        // basis exchange in the (S, R) form
        if (e_kind == 0 && l_kind == 0) {
            S[l_at] = e_at;
        } else if (e_kind == 0 && l_kind == 1) {
            S.push_back(e_at);
            R.push_back(l_at);
        } else if (e_kind == 1 && l_kind == 0) {
            S.erase(S.begin() + l_at);
            R.erase(R.begin() + e_at);
        } else {
            R[e_at] = l_at;
        }
        ++cleanup;
    }
    h->stats.cleanup_pivots = cleanup;
    h->stats.k = (int)S.size();
    h->stats.primal_violation = std::max(0.0, -std::min(chk.min_x, chk.min_s));
    h->stats.dual_violation = std::max(0.0, -std::min(chk.min_d, chk.min_y));
    h->stats.gap = std::fabs(chk.cx - chk.by);
    // read-out: x, y, objective in FP64
    const int k = (int)S.size();
    CUDA_TRY(cudaMemsetAsync(h->sol, 0, (size_t)(n + m + 1) * sizeof(double), s), LP_ERR_CUDA);
    k_rec_output<<<grid_for(std::max(k, 1), 256, 1024), 256, 0, s>>>(m, n, r.S, r.Rr, k, r.xS, r.yR, r.chk, h->sol);
    ++launches;
    std::vector<char> slack_nb(m, 0);
    for (int i : R) slack_nb[i] = 1;
    h->final_basis = S;
    for (int i = 0; i < m; ++i)
        if (!slack_nb[i]) h->final_basis.push_back(n + i);
    std::sort(h->final_basis.begin(), h->final_basis.end());
    return st;
}

template <int NT>
static lp_status solve_nt(lp_handle* h, const lp_options& o, cudaStream_t s) {
    if (!ensure_events(h)) return LP_ERR_CUDA;
    if (!h->checked) {   // created without the input check: run it now
        if (!validate_inputs(h)) {
            h->solved = true;
            h->last_status = LP_ERR_INVALID;
            return LP_ERR_INVALID;
        }
        h->checked = true;
    }
    const int m = h->m;
    // pivot log buffers
    if (o.log_capacity > 0 && o.log_capacity != h->log_cap) {
        dev_free(h, h->logs);
        h->log_cap = 0;
        if (!dev_alloc_block(h, h->logs, (size_t)o.log_capacity * 2 * sizeof(int))) {
            set_error("lp_solve: allocation of the pivot log failed");
            return LP_ERR_NOMEM;
        }
        h->log_cap = o.log_capacity;
    }
    const bool fp32 = o.precision == LP_PREC_FP32;
    lp_status st = ensure_work(h, fp32 ? 4 : 8, o.layout == LP_LAYOUT_CONDENSED ? 1 : 0);
    if (st != LP_OPTIMAL) return st;

    h->stats = lp_stats{};
    h->sol_ready = false;
    h->final_basis.clear();
    DevState hs{};
    long long launches = 0;
    int path = 0, grid = 0;
    if (fp32)
        st = pivot_phase<NT, float>(h, o, s, o.eps_d_fp32, o.eps_p_fp32, hs, launches, path, grid);
    else
        st = pivot_phase<NT, double>(h, o, s, o.eps_d, o.eps_p, hs, launches, path, grid);
    if (st == LP_ERR_CUDA) return st;

    float ms_build = 0.f, ms_pivot = 0.f;
    cudaEventElapsedTime(&ms_build, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&ms_pivot, h->ev[1], h->ev[2]);
    const int ld = h->work.ld, elem = h->work.elem, E = 32 / elem;
    h->stats.iters = hs.iters;
    h->stats.build_ms = ms_build;
    h->stats.pivot_ms = ms_pivot;
    h->stats.dense_update_bytes = 2.0 * (double)(m + 1) * (double)h->W * elem * (double)hs.iters;
    // bytes Step 3 moves: read + write of every listed 32-B group in rows
    // 1..m except p, read + write of the objective row and write of row p over
    // all groups; plus the side traffic of Steps 1-2 and the staging: column q
    // and right-hand-side sectors (m + 1 rows), pivot row read, R write + read.
    {
        const double nsec = (double)(ld / E);
        const double upd = 64.0 * (double)(m - 1) * (double)hs.active_sectors + 96.0 * nsec * (double)hs.iters;
        const double side = (64.0 * (double)(m + 1) + 3.0 * elem * (double)ld) * (double)hs.iters;
        h->stats.update_bytes = upd + side;
    }
    h->stats.path = path;
    h->stats.grid = grid;
    h->stats.block = NT;
    h->stats.ld = ld;
    h->stats.layout = h->work.cond ? LP_LAYOUT_CONDENSED : LP_LAYOUT_FULL;
    h->stats.precision = o.precision;
    h->stats.pivot_status = (int)st;
    for (int k = 0; k < 6; ++k) h->stats.phase_ms[k] = 1e-6 * (double)hs.phase_ns[k];
    h->iters = hs.iters;

    if (fp32 && (st == LP_OPTIMAL || st == LP_ITER_LIMIT || st == LP_UNBOUNDED)) {
        cudaEventRecord(h->ev[3], s);
        long long rl = 0;
        lp_status rs = recover(h, o, s, rl);
        if (rs == LP_ERR_CUDA) return rs;
        cudaEventRecord(h->ev[2], s);
        CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
        float ms_rec = 0.f;
        cudaEventElapsedTime(&ms_rec, h->ev[3], h->ev[2]);
        h->stats.recover_ms = ms_rec;
        launches += rl;
        // a float phase stopped by the iteration cap is finished by the cleanup
        st = rs;
        h->sol_ready = rs == LP_OPTIMAL;
    }
    h->stats.kernel_launches = launches;
    cudaEventRecord(h->ready, s);
    h->solved = true;
    h->last_status = st;
    return st;
}

static bool options_valid(const lp_options& o) {
    return o.eps_d >= 0.0 && o.eps_p >= 0.0 && o.rule >= 0 && o.rule <= 1 && o.path >= 0 && o.path <= 5 &&
           o.path != LP_PATH_TEAM && o.gpu_share >= 0.0 && o.gpu_share <= 1.0 && o.cpu_threads >= 0 &&
           o.log_capacity >= 0 && o.precision >= 0 && o.precision <= 1 && o.eps_d_fp32 >= 0.0 &&
           o.eps_p_fp32 >= 0.0 && o.recover_tol >= 0.0 && o.cleanup_max >= 0 &&
           (o.layout == LP_LAYOUT_CONDENSED || o.layout == LP_LAYOUT_FULL);
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
    if (!options_valid(o)) {
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

// ------------------------------------------------------- many LPs, by teams
// lp_solve_many: one cooperative launch of k_team_solve over the LPs (largest
// first), each LP solved by a team of blocks on its condensed tableau; then
// the per-LP bookkeeping of solve_nt (statistics, and for FP32 the FP64
// recovery) for each handle.

// The dynamic shared-memory limit of a team kernel is raised once to the
// device's maximum (process-wide state, never lowered).
template <int NT, typename V>
static cudaError_t team_allow_smem(size_t& limit) {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    static size_t lim = 0;
    std::call_once(once, [] {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, k_team_solve<NT, V>);
        lim = (size_t)std::max(0, optin - (int)fa.sharedSizeBytes);
        err = cudaFuncSetAttribute(k_team_solve<NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
    });
    limit = lim;
    return err;
}

// Bookkeeping of one LP after the team launch (as solve_nt): statistics and,
// for FP32, the FP64 recovery; *status receives the LP's outcome.
template <typename V>
static lp_status finish_team_lp(lp_handle* h, const lp_options& o, cudaStream_t s, float ms, int C, int NT,
                                lp_status* status) {
    constexpr int elem = (int)sizeof(V);
    const bool fp32 = elem == 4;
    DevState ds{};
    CUDA_TRY(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    lp_status st = ds.status == kRunning ? LP_ERR_TIMEOUT : (lp_status)ds.status;
    if (st == LP_ERR_TIMEOUT) set_error("lp_solve_many: a team barrier wait exceeded its limit");
    if (st == LP_ERR_INVALID) {
        set_error("lp_solve_many: inputs must be finite with b >= 0");
        h->solved = true;
        h->last_status = st;
        *status = st;
        cudaEventRecord(h->ready, s);
        return LP_OPTIMAL;
    }
    h->checked = true;
    const int m = h->m, ld = h->work.ld, E = 32 / elem;
    const double nsec = (double)(ld / E);
    h->stats.iters = ds.iters;
    // ms < 0: a continuous launch, where the LP's team stamped its own start and end
    h->stats.pivot_ms = ms >= 0.f ? (double)ms : 1e-6 * (double)(ds.phase_ns[1] - ds.phase_ns[0]);
    h->stats.dense_update_bytes = 2.0 * (double)(m + 1) * (double)h->W * elem * (double)ds.iters;
    h->stats.update_bytes = ((64.0 * (double)(m - 1) + 96.0) * nsec + 64.0 * (double)(m + 1) +
                             3.0 * elem * (double)ld) * (double)ds.iters;
    h->stats.path = LP_PATH_TEAM;
    h->stats.grid = C;
    h->stats.block = NT;
    h->stats.ld = ld;
    h->stats.layout = LP_LAYOUT_CONDENSED;
    h->stats.precision = o.precision;
    h->stats.pivot_status = (int)st;
    h->stats.kernel_launches = 1;
    h->iters = ds.iters;
    if (fp32 && (st == LP_OPTIMAL || st == LP_ITER_LIMIT || st == LP_UNBOUNDED)) {
        // timed on the host: recovery ends with a synchronisation anyway, and
        // creating events on many threads at once contends in the driver
        const auto t0 = std::chrono::steady_clock::now();
        long long rl = 0;
        lp_status rs = recover(h, o, s, rl);
        if (rs == LP_ERR_CUDA) return rs;
        CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
        h->stats.recover_ms = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        h->stats.kernel_launches += rl;
        st = rs;
        h->sol_ready = rs == LP_OPTIMAL;
    }
    cudaEventRecord(h->ready, s);
    h->solved = true;
    h->last_status = st;
    *status = st;
    return LP_OPTIMAL;
}

#ifndef TSX_TEAM_WIDE
#define TSX_TEAM_WIDE 1   // wide teams for the LPs heavier than a team's share
#endif

template <typename V>
static lp_status solve_many_t(std::vector<lp_handle*>& hs, const lp_options& o, cudaStream_t s,
                              lp_status* status, int reserve_blocks, const std::function<void()>& after_kernel) {
    constexpr int NT = 256;
    constexpr int elem = (int)sizeof(V);
    const bool fp32 = elem == 4;
    const int count = (int)hs.size();
    int device = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&device), LP_ERR_CUDA);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    size_t smem_limit = 0;
    const cudaError_t se = team_allow_smem<NT, V>(smem_limit);
    CUDA_TRY(se, LP_ERR_CUDA);
    int C = o.blocks > 0 ? std::min(o.blocks, kTeamMax) : 16;

    // work buffers and state of every LP (condensed layout)
    for (lp_handle* h : hs) {
        CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ready, 0), LP_ERR_CUDA);
        lp_status st = ensure_work(h, elem, 1);
        if (st != LP_OPTIMAL) return st;
        h->stats = lp_stats{};
        h->sol_ready = false;
        h->final_basis.clear();
        k_reset_state<<<1, 32, 0, h->stream>>>(h->st);
        if (h->stream != s) {   // the launch on s waits for the handle's stream
            if (!ensure_events(h)) return LP_ERR_CUDA;
            CUDA_TRY(cudaEventRecord(h->ev[0], h->stream), LP_ERR_CUDA);
            CUDA_TRY(cudaStreamWaitEvent(s, h->ev[0], 0), LP_ERR_CUDA);
        }
    }
    // the list, largest first; LPs whose pivot row and multipliers exceed the
    // shared memory of one block are solved one at a time afterwards
    std::vector<TeamJob<V>> jobs;
    std::vector<int> who, alone;
    std::vector<double> work;
    int ld_max = 0, rows_max = 0;
    for (int k = 0; k < count; ++k) {
        lp_handle* h = hs[k];
        const int rows = (h->m + 1 + C - 1) / C;
        if ((size_t)(h->work.ld + rows) * elem > smem_limit) {
            alone.push_back(k);
            continue;
        }
        TeamJob<V> J{};
        J.A = h->A;
        J.b = h->b;
        J.c = h->c;
        J.T = (V*)h->work.T;
        J.basis = h->basis;
        J.var = h->work.var;
        J.st = h->st;
        J.m = h->m;
        J.n = h->n;
        J.ld = h->work.ld;
        jobs.push_back(J);
        who.push_back(k);
        work.push_back((double)(h->m + 1) * h->work.ld * (double)(h->m + h->n));
        ld_max = std::max(ld_max, h->work.ld);
        rows_max = std::max(rows_max, rows);
    }
    const int njobs = (int)jobs.size();
    std::vector<int> order(njobs);
    for (int k = 0; k < njobs; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });

    float ms = 0.f;
    if (njobs > 0) {
        const size_t smem = (size_t)(ld_max + ((rows_max + 31) / 32) * 32) * elem;
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_team_solve<NT, V>, NT, smem);
        const int cap = per * nsm - std::max(0, reserve_blocks);
        if (cap <= 0) {
            set_error("lp_solve_many: the team kernel cannot be resident (%zu bytes of shared memory)", smem);
            return LP_ERR_CUDA;
        }
        C = std::min(C, cap);
        // Teams: the LPs heavier than a team's fair share of the whole list
        // would outlast it on C blocks, so up to half the grid forms wide teams
        // (4 C blocks) that take those first; the narrow teams take the rest.
        // Each team drains its own list, then helps with the other.
        double total = 0.0;
        for (double w : work) total += w;
        const int narrow_all = std::max(1, cap / C);
        const double share = total / narrow_all;
        std::vector<int> heavy, light;
        for (int k : order) (work[k] > share ? heavy : light).push_back(k);
        const int CB = std::min(std::min(4 * C, kTeamMax), std::max(C, cap / 2));
        int nwide = heavy.empty() || CB <= C || !TSX_TEAM_WIDE ? 0
                                                               : std::min((int)heavy.size(), std::max(1, (cap / 2) / CB));
        if (nwide == 0) {   // one list
            light.insert(light.begin(), heavy.begin(), heavy.end());
            heavy.clear();
        }
        std::vector<int> first, size, list, team_of;
        for (int t = 0; t < nwide; ++t) {
            first.push_back((int)team_of.size());
            size.push_back(CB);
            list.push_back(1);
            team_of.insert(team_of.end(), CB, (int)first.size() - 1);
        }
        const int nnarrow = std::max(1, std::min((cap - nwide * CB) / C, njobs));
        for (int t = 0; t < nnarrow && (int)team_of.size() + C <= cap; ++t) {
            first.push_back((int)team_of.size());
            size.push_back(C);
            list.push_back(0);
            team_of.insert(team_of.end(), C, (int)first.size() - 1);
        }
        const int nteams = (int)first.size();
        const int grid = (int)team_of.size();
        // scratch: jobs | lists | counters | team tables | team states
        Carve cv;
        const size_t o_jobs = cv.take(sizeof(TeamJob<V>) * (size_t)njobs);
        const size_t o_l0 = cv.take(sizeof(int) * (size_t)std::max<size_t>(1, light.size()));
        const size_t o_l1 = cv.take(sizeof(int) * (size_t)std::max<size_t>(1, heavy.size()));
        const size_t o_tab = cv.take(sizeof(int) * (size_t)(grid + 3 * nteams));
        const size_t o_next = cv.take(2 * sizeof(unsigned));
        const size_t o_teams = cv.take(sizeof(TeamState) * (size_t)nteams);
        const size_t bytes = align_up(cv.off, 256);
        lp_handle* h0 = hs[who[0]];
        void* scratch = h0->alloc ? h0->alloc(bytes, (void*)s, h0->alloc_ctx) : nullptr;
        if (!h0->alloc && pool_alloc(&scratch, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            scratch = nullptr;
        }
        if (!scratch) {
            set_error("lp_solve_many: allocation of %zu bytes of scratch failed", bytes);
            return LP_ERR_NOMEM;
        }
        char* base = (char*)scratch;
        std::vector<int> tab(team_of);
        tab.insert(tab.end(), first.begin(), first.end());
        tab.insert(tab.end(), size.begin(), size.end());
        tab.insert(tab.end(), list.begin(), list.end());
        TeamParams<V> P{};
        P.jobs = (const TeamJob<V>*)(base + o_jobs);
        P.order[0] = (const int*)(base + o_l0);
        P.order[1] = (const int*)(base + o_l1);
        P.count[0] = (int)light.size();
        P.count[1] = (int)heavy.size();
        P.next = (unsigned*)(base + o_next);
        P.teams = (TeamState*)(base + o_teams);
        P.team_of = (const int*)(base + o_tab);
        P.first = P.team_of + grid;
        P.size = P.first + nteams;
        P.list = P.size + nteams;
        P.eps_d = fp32 ? o.eps_d_fp32 : o.eps_d;
        P.eps_p = fp32 ? o.eps_p_fp32 : o.eps_p;
        P.max_iters = o.max_iters;
        P.k_cyc = o.k_cyc;
        P.rule = o.rule;
        P.timeout_ns = std::max(0LL, o.barrier_timeout_ns);
        cudaError_t e = cudaMemcpyAsync(base + o_jobs, jobs.data(), sizeof(TeamJob<V>) * (size_t)njobs,
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !light.empty())
            e = cudaMemcpyAsync(base + o_l0, light.data(), sizeof(int) * light.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !heavy.empty())
            e = cudaMemcpyAsync(base + o_l1, heavy.data(), sizeof(int) * heavy.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + o_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(base + o_next, 0, bytes - o_next, s);
        if (!ensure_events(h0)) return LP_ERR_CUDA;
        cudaEvent_t e0 = h0->ev[1], e1 = h0->ev[2];
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        int ldm = ld_max;
        void* args[] = {(void*)&P, (void*)&ldm};
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel((const void*)k_team_solve<NT, V>, grid, NT, args, smem, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (h0->dealloc)
            h0->dealloc(scratch, bytes, (void*)s, h0->alloc_ctx);
        else
            cudaFreeAsync(scratch, s);
        if (e != cudaSuccess) {
            set_error("lp_solve_many: team launch failed: %s", cudaGetErrorString(e));
            return LP_ERR_CUDA;
        }
    }
    if (after_kernel) after_kernel();
    // the recovery's cooperative refactorisation fits in the reserved blocks
    lp_options of = o;
    of.blocks = std::max(0, reserve_blocks);
    // per-LP bookkeeping (as solve_nt) and the FP64 recovery of FP32 results,
    // spread over host threads with a stream each (the recovery is a chain of
    // small kernels and host decisions per LP)
    const int nthreads = fp32 ? std::max(1, std::min(njobs, 8)) : 1;
    std::vector<lp_status> fail(nthreads, LP_OPTIMAL);
    auto finish = [&](int tid, cudaStream_t ss) -> lp_status {
        for (int t = tid; t < njobs; t += nthreads) {
            const lp_status st = finish_team_lp<V>(hs[who[t]], of, ss, ms, C, NT, status + who[t]);
            if (st == LP_ERR_CUDA) return st;
        }
        return LP_OPTIMAL;
    };
    if (nthreads == 1) {
        fail[0] = finish(0, s);
    } else {
        std::vector<std::thread> th;
        for (int k = 0; k < nthreads; ++k)
            th.emplace_back([&, k] {
                cudaSetDevice(device);
                cudaStream_t ss = stream_get();
                if (!ss) {
                    fail[k] = LP_ERR_CUDA;
                    return;
                }
                fail[k] = finish(k, ss);
                cudaStreamSynchronize(ss);
                stream_put(ss);
            });
        for (auto& t : th) t.join();
    }
    for (lp_status f : fail)
        if (f != LP_OPTIMAL) return f;
    // the rest, one at a time
    for (int k : alone) {
        lp_options oa = o;
        oa.blocks = 0;
        status[k] = solve_nt<NT>(hs[k], oa, s);
    }
    return LP_OPTIMAL;
}

// ------------------------------------------------ continuous team launch
// The request server's lane for large LPs (k_team_serve in tsx_team.cuh):
// one cooperative launch of teams that take jobs from rings in mapped host
// memory while it runs.  The host publishes a job per admitted LP, polls the
// per-job done words, and starts a new launch whenever jobs wait and the last
// one has ended (teams exit after idle_ns without work).
namespace {
constexpr unsigned kLaneCap = 4096;               // ring entries per list
constexpr long long kLaneIdleNs = 2'000'000;      // the teams exit 2 ms after the last one's work
constexpr long long kLaneIdleCapNs = 10'000'000'000LL;   // bound on one team's wait for work
constexpr double kLaneHeavyWork = 1.5e10;         // (m+1) (n+1) (m+n) above this: the wide teams' list
}

struct tsx::TeamLane {
    std::mutex mu;
    lp_options o{};
    int device = 0, nsm = 0;
    bool fp32 = false;
    int reserve = 0;
    int C = 16, CB = 64, grid = 0, nteams = 0;
    size_t smem = 0;
    int ld_cap = 0, rows_cap = 0;
    // mapped host memory: rings, tails, done words, stop word
    char* hmem = nullptr;
    char* hmem_d = nullptr;
    void* ring_h = nullptr;
    unsigned *tail_h = nullptr, *done_h = nullptr, *stop_h = nullptr;
    void* ring_d = nullptr;
    unsigned *tail_d = nullptr, *done_d = nullptr, *stop_d = nullptr;
    // device memory: heads, team states, team tables, job copies
    void* dmem = nullptr;
    size_t dmem_bytes = 0, o_teams = 0, o_tab = 0, o_jc = 0;
    unsigned* head_d = nullptr;
    cudaStream_t ks = nullptr;
    cudaEvent_t kev = nullptr;
    bool running = false;
    long long launches = 0;
    unsigned pub[2] = {0, 0};
    struct Out {
        lp_handle* h;
        unsigned list, seq;
    };
    std::vector<Out> out;
};

template <typename V>
static lp_status lane_launch(TeamLane* L) {
    constexpr int NT = 256;
    const int ntab = L->grid + 3 * L->nteams;
    std::vector<int> tab;
    tab.reserve(ntab);
    std::vector<int> first, size, list;
    int nw = 0;
    {
        int cap = L->grid;
        const int nwide = std::max(0, std::min((cap / 2) / L->CB, 8));
        for (int t = 0; t < nwide; ++t) {
            first.push_back((int)tab.size());
            size.push_back(L->CB);
            list.push_back(1);
            tab.insert(tab.end(), L->CB, (int)first.size() - 1);
        }
        nw = nwide;
        while ((int)tab.size() + L->C <= cap) {
            first.push_back((int)tab.size());
            size.push_back(L->C);
            list.push_back(0);
            tab.insert(tab.end(), L->C, (int)first.size() - 1);
        }
    }
    (void)nw;
    const int grid = (int)tab.size(), nteams = (int)first.size();
    tab.insert(tab.end(), first.begin(), first.end());
    tab.insert(tab.end(), size.begin(), size.end());
    tab.insert(tab.end(), list.begin(), list.end());
    char* base = (char*)L->dmem;
    CUDA_TRY(cudaMemcpyAsync(base + L->o_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, L->ks),
             LP_ERR_CUDA);
    CUDA_TRY(cudaMemsetAsync(base + L->o_teams, 0, sizeof(TeamState) * (size_t)nteams, L->ks), LP_ERR_CUDA);
    CUDA_TRY(cudaMemsetAsync(L->head_d + 2, 0, sizeof(unsigned), L->ks), LP_ERR_CUDA);   // busy teams
    TeamServeParams<V> P{};
    P.tp.teams = (TeamState*)(base + L->o_teams);
    P.tp.team_of = (const int*)(base + L->o_tab);
    P.tp.first = P.tp.team_of + grid;
    P.tp.size = P.tp.first + nteams;
    P.tp.list = P.tp.size + nteams;
    P.tp.eps_d = L->fp32 ? L->o.eps_d_fp32 : L->o.eps_d;
    P.tp.eps_p = L->fp32 ? L->o.eps_p_fp32 : L->o.eps_p;
    P.tp.max_iters = L->o.max_iters;
    P.tp.k_cyc = L->o.k_cyc;
    P.tp.rule = L->o.rule;
    P.tp.timeout_ns = std::max(0LL, L->o.barrier_timeout_ns);
    P.ring.jobs = (TeamJob<V>*)L->ring_d;
    P.ring.tail = L->tail_d;
    P.ring.done = L->done_d;
    P.ring.stop = L->stop_d;
    P.cap = kLaneCap;
    P.head = L->head_d;
    P.busy = L->head_d + 2;
    P.jcopy = (TeamJob<V>*)(base + L->o_jc);
    P.idle_ns = kLaneIdleNs;
    P.idle_cap_ns = kLaneIdleCapNs;
    int ldm = L->ld_cap;
    void* args[] = {(void*)&P, (void*)&ldm};
    CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_team_serve<NT, V>, grid, NT, args, L->smem, L->ks),
             LP_ERR_CUDA);
    CUDA_TRY(cudaEventRecord(L->kev, L->ks), LP_ERR_CUDA);
    L->running = true;
    ++L->launches;
    return LP_OPTIMAL;
}

template <typename V>
static lp_status lane_setup(TeamLane* L) {
    constexpr int NT = 256;
    constexpr int elem = (int)sizeof(V);
    CUDA_TRY(cudaGetDevice(&L->device), LP_ERR_CUDA);
    cudaDeviceGetAttribute(&L->nsm, cudaDevAttrMultiProcessorCount, L->device);
    // shared memory for two blocks per SM: R (ld_cap entries) and the
    // multipliers of a block's rows (rows_cap entries)
    int per_sm = 0, reserved = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, L->device);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, L->device);
    cudaFuncAttributes fa{};
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_team_serve<NT, V>), LP_ERR_CUDA);
    const size_t per_block = (size_t)per_sm / 2 - (size_t)reserved - fa.sharedSizeBytes - 1024;
    const size_t entries = per_block / elem / 32 * 32;
    L->ld_cap = (int)(entries * 3 / 4 / 32 * 32);
    L->rows_cap = (int)entries - L->ld_cap;
    L->smem = entries * elem;
    CUDA_TRY(cudaFuncSetAttribute((const void*)k_team_serve<NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L->smem),
             LP_ERR_CUDA);
    int per = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_team_serve<NT, V>, NT, L->smem), LP_ERR_CUDA);
    L->grid = per * L->nsm - L->reserve;
    L->C = L->o.blocks > 0 ? std::min(L->o.blocks, kTeamMax) : 16;
    if (L->grid < L->C) {
        set_error("lane: the team kernel cannot be resident (%d blocks)", L->grid);
        return LP_ERR_CUDA;
    }
    L->CB = std::min(std::min(4 * L->C, kTeamMax), std::max(L->C, L->grid / 2));
    L->nteams = L->grid;   // upper bound for the tables
    // mapped host memory
    const size_t ring_bytes = sizeof(TeamJob<V>) * 2 * kLaneCap;
    const size_t hbytes = ring_bytes + 64 + sizeof(unsigned) * 2 * kLaneCap + 64;
    CUDA_TRY(cudaHostAlloc((void**)&L->hmem, hbytes, cudaHostAllocMapped), LP_ERR_NOMEM);
    memset(L->hmem, 0, hbytes);
    CUDA_TRY(cudaHostGetDevicePointer((void**)&L->hmem_d, L->hmem, 0), LP_ERR_CUDA);
    L->ring_h = L->hmem;
    L->tail_h = (unsigned*)(L->hmem + ring_bytes);
    L->stop_h = L->tail_h + 4;
    L->done_h = (unsigned*)(L->hmem + ring_bytes + 64);
    L->ring_d = L->hmem_d;
    L->tail_d = (unsigned*)(L->hmem_d + ring_bytes);
    L->stop_d = L->tail_d + 4;
    L->done_d = (unsigned*)(L->hmem_d + ring_bytes + 64);
    // device memory
    Carve cv;
    const size_t o_head = cv.take(4 * sizeof(unsigned));   // heads [2], busy teams
    L->o_teams = cv.take(sizeof(TeamState) * (size_t)L->nteams);
    L->o_tab = cv.take(sizeof(int) * (size_t)(4 * L->grid + 8));
    L->o_jc = cv.take(sizeof(TeamJob<V>) * (size_t)L->nteams);
    L->dmem_bytes = align_up(cv.off, 256);
    CUDA_TRY(cudaMalloc(&L->dmem, L->dmem_bytes), LP_ERR_NOMEM);
    L->head_d = (unsigned*)((char*)L->dmem + o_head);
    CUDA_TRY(cudaMemset(L->dmem, 0, L->dmem_bytes), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamCreateWithFlags(&L->ks, cudaStreamNonBlocking), LP_ERR_CUDA);
    CUDA_TRY(cudaEventCreateWithFlags(&L->kev, cudaEventDisableTiming), LP_ERR_CUDA);
    return LP_OPTIMAL;
}

TeamLane* tsx::lane_open(const lp_options* opt, int reserve_blocks) {
    TeamLane* L = new TeamLane();
    if (opt)
        L->o = *opt;
    else
        lp_options_init(&L->o);
    L->fp32 = L->o.precision == LP_PREC_FP32;
    L->reserve = std::max(0, reserve_blocks);
    const lp_status st = L->fp32 ? lane_setup<float>(L) : lane_setup<double>(L);
    if (st != LP_OPTIMAL) {
        lane_close(L);
        return nullptr;
    }
    return L;
}

long long tsx::lane_submit(TeamLane* L, lp_t h) {
    if (!L || !h) return -1;
    const int elem = L->fp32 ? 4 : 8;
    CUDA_TRY(cudaSetDevice(h->device), -1);
    CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ready, 0), -1);
    if (ensure_work(h, elem, 1) != LP_OPTIMAL) return -1;
    const int rows = (h->m + 1 + L->C - 1) / L->C;
    if (h->work.ld > L->ld_cap || rows > L->rows_cap) return -2;   // solve it another way
    h->stats = lp_stats{};
    h->sol_ready = false;
    h->final_basis.clear();
    // the team resets the LP's state words when it takes the job; the
    // buffers' stream-ordered allocation is complete before it is published
    CUDA_TRY(cudaStreamSynchronize(h->stream), -1);
    TeamJob<double> J{};   // same layout for both element types (pointers and ints)
    J.A = h->A;
    J.b = h->b;
    J.c = h->c;
    J.T = (double*)h->work.T;
    J.basis = h->basis;
    J.var = h->work.var;
    J.st = h->st;
    J.m = h->m;
    J.n = h->n;
    J.ld = h->work.ld;
    const double work = (double)(h->m + 1) * (double)(h->n + 1) * (double)(h->m + h->n);
    const unsigned l = work > kLaneHeavyWork ? 1u : 0u;
    std::lock_guard<std::mutex> lk(L->mu);
    if (L->out.size() >= (size_t)kLaneCap) {
        set_error("lane: %u jobs outstanding", kLaneCap);
        return -1;
    }
    const unsigned seq = L->pub[l];
    const unsigned slot = l * kLaneCap + (seq & (kLaneCap - 1u));
    memcpy((char*)L->ring_h + sizeof(TeamJob<double>) * slot, &J, sizeof J);
    __atomic_store_n(L->done_h + slot, 0u, __ATOMIC_RELAXED);
    L->pub[l] = seq + 1u;
    __atomic_store_n(L->tail_h + l, seq + 1u, __ATOMIC_RELEASE);
    L->out.push_back(TeamLane::Out{h, l, seq});
    if (!L->running) {
        const lp_status st = L->fp32 ? lane_launch<float>(L) : lane_launch<double>(L);
        if (st != LP_OPTIMAL) return -1;
    }
    return (long long)l * kLaneCap + seq;
}

int tsx::lane_poll(TeamLane* L, std::vector<lp_t>& done) {
    std::lock_guard<std::mutex> lk(L->mu);
    for (size_t k = 0; k < L->out.size();) {
        const TeamLane::Out& o = L->out[k];
        const unsigned slot = o.list * kLaneCap + (o.seq & (kLaneCap - 1u));
        if (__atomic_load_n(L->done_h + slot, __ATOMIC_ACQUIRE) == o.seq + 1u) {
            done.push_back(o.h);
            L->out[k] = L->out.back();
            L->out.pop_back();
        } else {
            ++k;
        }
    }
    if (L->running && cudaEventQuery(L->kev) == cudaSuccess) {
        L->running = false;
        unsigned head[2] = {0, 0};
        if (cudaMemcpyAsync(head, L->head_d, sizeof head, cudaMemcpyDeviceToHost, L->ks) == cudaSuccess &&
            cudaStreamSynchronize(L->ks) == cudaSuccess) {
            // jobs a team claimed but did not finish (a team barrier ran out):
            // their state still says running, which the finish reports
            for (size_t k = 0; k < L->out.size();) {
                const TeamLane::Out& o = L->out[k];
                const unsigned slot = o.list * kLaneCap + (o.seq & (kLaneCap - 1u));
                if ((int)(head[o.list] - o.seq) > 0 &&
                    __atomic_load_n(L->done_h + slot, __ATOMIC_ACQUIRE) != o.seq + 1u) {
                    done.push_back(o.h);
                    L->out[k] = L->out.back();
                    L->out.pop_back();
                } else {
                    ++k;
                }
            }
            if (head[0] != L->pub[0] || head[1] != L->pub[1]) {
                if ((L->fp32 ? lane_launch<float>(L) : lane_launch<double>(L)) != LP_OPTIMAL) cudaGetLastError();
            }
        } else {
            cudaGetLastError();
        }
    }
    return (int)L->out.size();
}

lp_status tsx::lane_finish(TeamLane* L, lp_t h, cudaStream_t s, lp_status* status) {
    lp_options of = L->o;
    of.blocks = L->reserve;
    CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
    return L->fp32 ? finish_team_lp<float>(h, of, s, -1.f, L->C, 256, status)
                   : finish_team_lp<double>(h, of, s, -1.f, L->C, 256, status);
}

long long tsx::lane_launches(TeamLane* L) {
    std::lock_guard<std::mutex> lk(L->mu);
    return L->launches;
}

void tsx::lane_close(TeamLane* L) {
    if (!L) return;
    if (L->stop_h) __atomic_store_n(L->stop_h, 1u, __ATOMIC_RELEASE);
    if (L->ks) cudaStreamSynchronize(L->ks);
    if (L->kev) cudaEventDestroy(L->kev);
    if (L->ks) cudaStreamDestroy(L->ks);
    if (L->dmem) cudaFree(L->dmem);
    if (L->hmem) cudaFreeHost(L->hmem);
    delete L;
}

lp_status lp_solve_many(lp_t* handles, int count, const lp_options* opt, lp_status* status) {
    return tsx::solve_many_hooked(handles, count, opt, status, 0, std::function<void()>());
}

lp_status tsx::solve_many_hooked(lp_t* handles, int count, const lp_options* opt, lp_status* status,
                                 int reserve_blocks, const std::function<void()>& after_kernel) {
    if (!handles || !status || count < 0) {
        set_error("lp_solve_many: NULL argument or count < 0");
        return LP_ERR_INVALID;
    }
    lp_options o;
    if (opt)
        o = *opt;
    else
        lp_options_init(&o);
    if (!options_valid(o) || o.layout != LP_LAYOUT_CONDENSED || o.log_capacity != 0 ||
        (o.threads != 0 && o.threads != 256) || o.blocks < 0) {
        set_error("lp_solve_many: invalid options (condensed layout, no pivot log, threads 0 or 256)");
        return LP_ERR_INVALID;
    }
    if (count == 0) return LP_OPTIMAL;
    std::vector<lp_handle*> hs(handles, handles + count);
    for (int k = 0; k < count; ++k) {
        status[k] = LP_ERR_STATE;
        if (!hs[k]) {
            set_error("lp_solve_many: handle %d is NULL", k);
            return LP_ERR_INVALID;
        }
        if (hs[k]->device != hs[0]->device) {
            set_error("lp_solve_many: handle %d lives on another device", k);
            return LP_ERR_INVALID;
        }
    }
    {
        std::vector<lp_handle*> sorted(hs);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
            set_error("lp_solve_many: a handle appears twice");
            return LP_ERR_INVALID;
        }
    }
    CUDA_TRY(cudaSetDevice(hs[0]->device), LP_ERR_CUDA);
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : hs[0]->stream;
    return o.precision == LP_PREC_FP32 ? solve_many_t<float>(hs, o, s, status, reserve_blocks, after_kernel)
                                       : solve_many_t<double>(hs, o, s, status, reserve_blocks, after_kernel);
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
    if ((x || y || obj) && !h->sol_ready) {
        const int ld = h->work.ld, Ws = h->work.Ws, cond = h->work.cond;
        int g = std::min((n + m + 1 + 255) / 256, 1024);
        int gx = std::min((m + 255) / 256, 1024);
        int gy = std::min((n + 255) / 256, 1024);
        if (h->work.elem == 8) {
            const double* T = (const double*)h->work.T;
            k_extract_dense<double><<<g, 256, 0, s>>>(m, n, Ws, ld, T, cond, h->sol);
            if (cond) k_extract_y_cond<double><<<gy, 256, 0, s>>>(m, n, T, h->work.var, h->sol);
            k_extract_x<double><<<gx, 256, 0, s>>>(m, n, Ws, ld, T, h->basis, h->sol);
        } else {
            const float* T = (const float*)h->work.T;
            k_extract_dense<float><<<g, 256, 0, s>>>(m, n, Ws, ld, T, cond, h->sol);
            if (cond) k_extract_y_cond<float><<<gy, 256, 0, s>>>(m, n, T, h->work.var, h->sol);
            k_extract_x<float><<<gx, 256, 0, s>>>(m, n, Ws, ld, T, h->basis, h->sol);
        }
        CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    }
    if (x) CUDA_TRY(cudaMemcpyAsync(x, h->sol, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    if (y) CUDA_TRY(cudaMemcpyAsync(y, h->sol + n, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    if (obj) CUDA_TRY(cudaMemcpyAsync(obj, h->sol + n + m, sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    if (basis) {
        if (!h->final_basis.empty())
            memcpy(basis, h->final_basis.data(), (size_t)m * sizeof(int));
        else
            CUDA_TRY(cudaMemcpyAsync(basis, h->basis, (size_t)m * sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    }
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
    cudaStream_t s = h->stream;
    CUDA_TRY(cudaStreamWaitEvent(s, h->ready, 0), LP_ERR_CUDA);
    const size_t rows = (size_t)h->m + 1, W = (size_t)h->W;
    if (h->work.cond) {
        // condensed: the full Table I tableau is rebuilt on the device
        Block tmp;
        const size_t o_slot = align_up(rows * W * sizeof(double), 256);
        if (!dev_alloc_block(h, tmp, o_slot + (size_t)(h->n + h->m) * sizeof(int))) {
            set_error("lp_get_tableau: allocation of the expanded copy failed");
            return LP_ERR_NOMEM;
        }
        double* out = (double*)tmp.ptr;
        int* slot_of = (int*)((char*)tmp.ptr + o_slot);
        const int m = h->m, n = h->n;
        k_slot_of<<<grid_for(n + m, 256, 1024), 256, 0, s>>>(m, n, h->work.var, slot_of);
        k_slot_of_set<<<grid_for(n, 256, 1024), 256, 0, s>>>(n, h->work.var, slot_of);
        const int ge = grid_for((long long)(rows * W), 256, 152 * 16);
        if (h->work.elem == 8)
            k_expand_cond<double><<<ge, 256, 0, s>>>(m, n, h->work.ld, (const double*)h->work.T, h->work.var,
                                                     slot_of, out);
        else
            k_expand_cond<float><<<ge, 256, 0, s>>>(m, n, h->work.ld, (const float*)h->work.T, h->work.var,
                                                    slot_of, out);
        k_expand_units<<<grid_for(m, 256, 1024), 256, 0, s>>>(m, n, h->basis, out);
        CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
        CUDA_TRY(cudaMemcpyAsync(T, out, rows * W * sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
        CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
        dev_free(h, tmp);
        return LP_OPTIMAL;
    }
    if (h->work.elem == 8) {
        CUDA_TRY(cudaMemcpy2DAsync(T, W * sizeof(double), h->work.T, (size_t)h->work.ld * sizeof(double),
                                   W * sizeof(double), rows, cudaMemcpyDeviceToHost, s),
                 LP_ERR_CUDA);
    } else {
        // float tableau: widened to double on the device, then copied
        Block tmp;
        if (!dev_alloc_block(h, tmp, rows * W * sizeof(double))) {
            set_error("lp_get_tableau: allocation of the widened copy failed");
            return LP_ERR_NOMEM;
        }
        k_widen<float><<<grid_for((long long)(rows * W), 256, 152 * 16), 256, 0, s>>>(
            (int)rows, (int)W, h->work.ld, (const float*)h->work.T, (double*)tmp.ptr);
        CUDA_TRY(cudaMemcpyAsync(T, tmp.ptr, rows * W * sizeof(double), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
        CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
        dev_free(h, tmp);
    }
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
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
    stats->create_copy_ms = h->create_ms[0];
    stats->create_check_ms = h->create_ms[1];
    stats->create_wall_ms = h->create_ms[2];
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
    DevState* st = (DevState*)(base + off_st);
    Params<double> P = make_params<double>(m, n, ld, dT, (double*)base, (double*)(base + off_R),
                                           (int*)(base + off_act), (ArgPart*)(base + off_cp),
                                           (RatPart*)(base + off_rp), st, dbasis, o, o.eps_d, o.eps_p);

    // validate the inputs: the state word starts from zero on every call
    k_reset_state<<<1, 32, 0, s>>>(st);
    {
        const size_t total = (size_t)m * n + m + n;
        int g = (int)std::min<size_t>((total + 255) / 256, 4096);
        k_validate<<<g, 256, 0, s>>>(m, n, dA, db, dc, st);
    }
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, &st->bad, sizeof(int), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    if (bad) {
        set_error("lp_solve_noalloc: inputs must be finite with b >= 0");
        return LP_ERR_INVALID;
    }

    int coresident = 0;
    const int grid = pivot_grid<NT, double>(device, m, ld, kNoAllocMaxGrid, o.blocks, coresident);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    int path = o.path;
    if (path == LP_PATH_AUTO) path = (coop && coresident > 0) ? LP_PATH_PERSISTENT : LP_PATH_MULTILAUNCH;
    if (path == LP_PATH_PERSISTENT && (!coop || coresident <= 0)) {
        set_error("lp_solve_noalloc: persistent path requested but cooperative launch is unavailable");
        return LP_ERR_CUDA;
    }

    k_reset_state<<<1, 32, 0, s>>>(st);
    {
        const size_t groups = (size_t)(m + 1) * (size_t)(ld / 4);
        int g = (int)std::min<size_t>((groups + 255) / 256, 152 * 16);
        k_build<double><<<g, 256, 0, s>>>(m, n, n + m + 1, ld, dA, db, dc, dT, dbasis, nullptr);
    }
    CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    if (path == LP_PATH_PERSISTENT) {
        cudaError_t e = launch_persistent<NT, double>(P, grid, s);
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
        long long launches = 0;
        const int g = multilaunch_grid<NT, double>(device, m, ld, kNoAllocMaxGrid, o.blocks);
        if (run_multilaunch<NT, double>(P, g, s, launches) == LP_ERR_CUDA) return LP_ERR_CUDA;
    }
    DevState hs{};
    CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
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
        o.log_capacity != 0 || o.blocks < 0 || o.blocks > kNoAllocMaxGrid || o.precision != LP_PREC_FP64) {
        set_error("lp_solve_noalloc: invalid options (FP64 only, log_capacity must be 0, blocks <= %d)",
                  kNoAllocMaxGrid);
        return LP_ERR_INVALID;
    }
    {   // the call reads results back and waits for the device: no stream capture
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(static_cast<cudaStream_t>(o.stream), &cs) != cudaSuccess) {
            cudaGetLastError();
            set_error("lp_solve_noalloc: cannot query the stream's capture state");
            return LP_ERR_CUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) {
            set_error("lp_solve_noalloc: the stream is being captured; this call blocks and cannot be captured");
            return LP_ERR_STATE;
        }
    }
    // layout of the array: F | R | act | cpart | rpart | state
    const size_t nstrips = ((size_t)ld + 127) / 128;
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
