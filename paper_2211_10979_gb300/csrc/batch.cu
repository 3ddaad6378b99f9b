// Host side of the batched solve (lp_batch_* in include/tabsimplex.h): many
// small LPs, one thread block per LP with its condensed tableau in shared
// memory (kernel in tsx_batch.cuh).  LPs are grouped in shared-memory size
// classes; each class runs as one persistent launch fed by a work counter, the
// classes run concurrently on their own streams, and the whole solve is
// captured once in a CUDA graph and replayed.  Threads per LP are picked per
// class by timing the candidates on the first solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "tabsimplex.h"
#include "tsx_batch.cuh"
#include "tsx_host.h"

using namespace tsx;

namespace {

constexpr int kClasses = 5;
// shared-memory size classes; the last one holds the LPs that keep their
// tableau in a global workspace slice
constexpr int kGlobal = kClasses - 1;
// The shared-memory classes hold LPs of which 8, 3, 2 and 1 fit one SM at a
// time (bounds from the device's shared memory per SM, see class_bounds).
constexpr int kPerSm[kClasses - 1] = {8, 3, 2, 1};
constexpr int kCandidates[5] = {32, 64, 128, 256, 512};

struct DBlock {
    void* ptr = nullptr;
    size_t bytes = 0;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Threads per LP picked by timing, per device and size class; later batches on
// the same device reuse the choice.
constexpr int kMaxDevices = 64;
std::mutex g_tune_mu;
int g_tuned[kMaxDevices][kClasses] = {};

}  // namespace

struct lp_batch {
    int count = 0;
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side[kClasses] = {};
    cudaStream_t cap = nullptr;      // graphs are captured on and replayed from here
    cudaEvent_t fork = nullptr, join[kClasses] = {}, ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t e_in = nullptr, e_out = nullptr;
    lp_alloc_fn alloc = nullptr;
    lp_free_fn dealloc = nullptr;
    void* actx = nullptr;
    std::vector<BatchLP> lps;
    long long sum_mn = 0, sum_m = 0, sum_n = 0, sum_t = 0;
    DBlock inputs;
    const double *A = nullptr, *b = nullptr, *c = nullptr;
    DBlock work;
    BatchLP* lps_dev = nullptr;
    int* lists[kClasses] = {};
    int class_count[kClasses] = {};
    size_t class_smem[kClasses] = {};
    unsigned* queues = nullptr;
    int* status = nullptr;
    long long* iters = nullptr;
    double* obj = nullptr;
    double* x = nullptr;
    double* y = nullptr;
    unsigned long long* total = nullptr;
    DBlock keep;
    DBlock gwork;                    // global workspace of the kGlobal class
    int tuned[kClasses] = {};
    cudaGraphExec_t graph = nullptr;
    BatchParams graph_params{};
    int graph_nt[kClasses] = {};
    bool graph_valid = false;
    long long solves = 0;            // completed solves (the graph is captured from the second on)
    lp_batch_stats stats{};
    bool solved = false;
    bool kept = false;
};

static void* bdev_alloc(lp_batch* h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (h->alloc) return h->alloc(bytes, (void*)h->stream, h->actx);
    void* p = nullptr;
    if (pool_alloc(&p, bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void bdev_free(lp_batch* h, DBlock& blk) {
    if (!blk.ptr) return;
    if (h->dealloc)
        h->dealloc(blk.ptr, blk.bytes, (void*)h->stream, h->actx);
    else
        cudaFreeAsync(blk.ptr, h->stream);
    blk = DBlock{};
}

static bool bdev_alloc_block(lp_batch* h, DBlock& blk, size_t bytes) {
    blk.ptr = bdev_alloc(h, bytes);
    blk.bytes = blk.ptr ? bytes : 0;
    return blk.ptr != nullptr;
}

void lp_batch_options_init(lp_batch_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->threads = 0;
    o->rule = LP_RULE_DANTZIG;
    o->eps_d = 1e-9;
    o->eps_p = 1e-9;
    o->max_iters = -1;
    o->k_cyc = 50;
    o->use_graph = 1;
    o->keep_tableaux = 0;
    o->stream = nullptr;
}

void lp_batch_destroy(lp_batch_t h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    bdev_free(h, h->keep);
    bdev_free(h, h->gwork);
    bdev_free(h, h->work);
    bdev_free(h, h->inputs);
    if (h->stream) cudaStreamSynchronize(h->stream);
    // the side streams' work was joined into h->stream: all of it is done
    for (int k = 0; k < kClasses; ++k) {
        stream_put(h->side[k]);
        event_put(h->join[k], false);
    }
    event_put(h->fork, false);
    event_put(h->e_in, false);
    event_put(h->e_out, false);
    stream_put(h->cap);
    event_put(h->ev0, true);
    event_put(h->ev1, true);
    if (h->own_stream) stream_put(h->stream);
    delete h;
}

template <int NT>
static size_t kernel_static_smem() {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k_batch_solve<NT>);
    return fa.sharedSizeBytes;
}

static int condensed_ld(int n) { return (n + 1) % 2 == 1 ? n + 1 : n + 2; }

size_t tsx::batch_smem_limit() {
    int device = 0, optin = 0;
    cudaGetDevice(&device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    size_t stat = 0;
    for (size_t v : {kernel_static_smem<32>(), kernel_static_smem<64>(), kernel_static_smem<128>(),
                     kernel_static_smem<256>(), kernel_static_smem<512>()})
        stat = std::max(stat, v);
    return optin > 0 ? (size_t)optin - stat - 256 : 0;
}

// Dynamic shared-memory bound of each shared-memory class: the largest LP
// block of which kPerSm[q] fit on one SM next to each other (each block also
// holds the kernel's static scratch and the per-block reservation).
static void class_bounds(size_t* bound) {
    int device = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&device);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
    size_t stat = 0;
    for (size_t v : {kernel_static_smem<32>(), kernel_static_smem<64>(), kernel_static_smem<128>(),
                     kernel_static_smem<256>(), kernel_static_smem<512>()})
        stat = std::max(stat, v);
    const size_t limit = tsx::batch_smem_limit();
    for (int q = 0; q < kClasses - 1; ++q) {
        const size_t share = (size_t)std::max(per_sm, 0) / (size_t)kPerSm[q];
        const size_t over = stat + (size_t)std::max(reserved, 0);
        bound[q] = share > over ? std::min(limit, (share - over) / 16 * 16) : 0;
    }
    bound[kClasses - 2] = limit;
}

bool tsx::batch_fits(int m, int n, size_t limit) {
    return m > 0 && n > 0 && batch_smem_bytes(m, n, condensed_ld(n)) <= limit;
}

static lp_batch* batch_common(int count, const int* m, const int* n, cudaStream_t stream, bool own_stream) {
    if (count <= 0 || !m || !n) {
        set_error("lp_batch_create: need count > 0 and the m, n arrays");
        return nullptr;
    }
    lp_batch* h = new lp_batch();
    h->count = count;
    cudaGetDevice(&h->device);
    current_allocator(&h->alloc, &h->dealloc, &h->actx);
    cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
    const size_t limit = batch_smem_limit();
    size_t bound[kClasses - 1];
    class_bounds(bound);
    size_t gbytes = 0;
    h->lps.resize(count);
    for (int k = 0; k < count; ++k) {
        if (m[k] <= 0 || n[k] <= 0) {
            set_error("lp_batch_create: LP %d needs m > 0 and n > 0 (got %d, %d)", k, m[k], n[k]);
            delete h;
            return nullptr;
        }
        BatchLP& L = h->lps[k];
        L.m = m[k];
        L.n = n[k];
        L.ldc = condensed_ld(n[k]);
        const size_t smem = batch_smem_bytes(L.m, L.n, L.ldc);
        int cls = kGlobal;
        if (smem <= limit) {
            cls = kGlobal - 1;
            for (int q = 0; q < kGlobal - 1; ++q)
                if (smem <= bound[q]) { cls = q; break; }
            h->class_smem[cls] = std::max(h->class_smem[cls], smem);
            L.w_off = -1;
        } else {
            L.w_off = (long long)gbytes;
            gbytes += align_up(smem, 256);
        }
        L.bucket = cls;
        ++h->class_count[cls];
        L.a_off = h->sum_mn;
        L.b_off = h->sum_m;
        L.c_off = h->sum_n;
        L.t_off = h->sum_t;
        h->sum_mn += (long long)m[k] * n[k];
        h->sum_m += m[k];
        h->sum_n += n[k];
        h->sum_t += (long long)(m[k] + 1) * L.ldc;
    }
    if (own_stream) {
        if (!(h->stream = stream_get())) {
            set_error("lp_batch_create: cudaStreamCreate failed");
            delete h;
            return nullptr;
        }
        h->own_stream = true;
    } else {
        h->stream = stream;
    }
    if (!(h->ev0 = event_get(true)) || !(h->ev1 = event_get(true))) {
        set_error("lp_batch_create: event creation failed");
        lp_batch_destroy(h);
        return nullptr;
    }
    if (gbytes && !bdev_alloc_block(h, h->gwork, gbytes)) {
        set_error("lp_batch_create: device allocation of %zu workspace bytes failed", gbytes);
        lp_batch_destroy(h);
        return nullptr;
    }
    // work block: lps | class lists | queues | status | iters | obj | x | y | total
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = align_up(off, 256);
        off = at + bytes;
        return at;
    };
    const size_t o_lps = take(sizeof(BatchLP) * count);
    size_t o_list[kClasses];
    for (int q = 0; q < kClasses; ++q) o_list[q] = take(sizeof(int) * std::max(1, h->class_count[q]));
    const size_t o_q = take(sizeof(unsigned) * kClasses);
    const size_t o_st = take(sizeof(int) * count);
    const size_t o_it = take(sizeof(long long) * count);
    const size_t o_ob = take(sizeof(double) * count);
    const size_t o_x = take(sizeof(double) * h->sum_n);
    const size_t o_y = take(sizeof(double) * h->sum_m);
    const size_t o_tot = take(sizeof(unsigned long long));
    if (!bdev_alloc_block(h, h->work, align_up(off, 256))) {
        set_error("lp_batch_create: device allocation of %zu bytes failed", off);
        lp_batch_destroy(h);
        return nullptr;
    }
    char* base = (char*)h->work.ptr;
    h->lps_dev = (BatchLP*)(base + o_lps);
    for (int q = 0; q < kClasses; ++q) h->lists[q] = (int*)(base + o_list[q]);
    h->queues = (unsigned*)(base + o_q);
    h->status = (int*)(base + o_st);
    h->iters = (long long*)(base + o_it);
    h->obj = (double*)(base + o_ob);
    h->x = (double*)(base + o_x);
    h->y = (double*)(base + o_y);
    h->total = (unsigned long long*)(base + o_tot);
    // class lists, largest LPs first inside each class (long solves start early)
    std::vector<int> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b2) {
        const long long wa = (long long)h->lps[a].m * h->lps[a].n, wb = (long long)h->lps[b2].m * h->lps[b2].n;
        return wa > wb;
    });
    std::vector<int> lists[kClasses];
    for (int k : order) lists[h->lps[k].bucket].push_back(k);
    bool cp = cudaMemcpyAsync(h->lps_dev, h->lps.data(), sizeof(BatchLP) * count, cudaMemcpyHostToDevice,
                              h->stream) == cudaSuccess;
    for (int q = 0; q < kClasses; ++q)
        if (!lists[q].empty())
            cp = cp && cudaMemcpyAsync(h->lists[q], lists[q].data(), sizeof(int) * lists[q].size(),
                                       cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
    cp = cp && cudaStreamSynchronize(h->stream) == cudaSuccess;
    if (!cp) {
        set_error("lp_batch_create: copy of the batch layout failed");
        lp_batch_destroy(h);
        return nullptr;
    }
    return h;
}

lp_batch_t lp_batch_create(int count, const int* m, const int* n, const double* A, const double* b,
                           const double* c) {
    if (!A || !b || !c) {
        set_error("lp_batch_create: NULL input array");
        return nullptr;
    }
    lp_batch* h = batch_common(count, m, n, nullptr, true);
    if (!h) return nullptr;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = align_up(off, 256);
        off = at + bytes;
        return at;
    };
    const size_t o_A = take(sizeof(double) * h->sum_mn);
    const size_t o_b = take(sizeof(double) * h->sum_m);
    const size_t o_c = take(sizeof(double) * h->sum_n);
    if (!bdev_alloc_block(h, h->inputs, align_up(off, 256))) {
        set_error("lp_batch_create: device allocation of %zu input bytes failed", off);
        lp_batch_destroy(h);
        return nullptr;
    }
    char* base = (char*)h->inputs.ptr;
    h->A = (const double*)(base + o_A);
    h->b = (const double*)(base + o_b);
    h->c = (const double*)(base + o_c);
    const double* gA = host_alias(A, h->sum_mn);
    const double* gb = gA ? host_alias(b, h->sum_m) : nullptr;
    const double* gc = gb ? host_alias(c, h->sum_n) : nullptr;
    if (gc) {   // page-locked inputs: read by one kernel over the host link
        if (launch_ingest(gA, (double*)h->A, (size_t)h->sum_mn, gb, (double*)h->b, (size_t)h->sum_m, gc, (double*)h->c,
                          (size_t)h->sum_n, nullptr, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {   // the caller may reuse its arrays on return
            set_error("lp_batch_create: upload of the inputs failed: %s", cudaGetErrorString(cudaGetLastError()));
            lp_batch_destroy(h);
            return nullptr;
        }
        return h;
    }
    if (cudaMemcpyAsync((void*)h->A, A, sizeof(double) * h->sum_mn, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync((void*)h->b, b, sizeof(double) * h->sum_m, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync((void*)h->c, c, sizeof(double) * h->sum_n, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
        set_error("lp_batch_create: host-to-device copy failed");
        lp_batch_destroy(h);
        return nullptr;
    }
    // a page-locked array among the inputs is copied asynchronously: wait, so
    // that the caller may reuse its arrays on return
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        set_error("lp_batch_create: host-to-device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
        lp_batch_destroy(h);
        return nullptr;
    }
    return h;
}

lp_batch_t lp_batch_create_device(int count, const int* m, const int* n, const double* dA, const double* db,
                                  const double* dc, void* stream) {
    if (!dA || !db || !dc) {
        set_error("lp_batch_create_device: NULL input pointer");
        return nullptr;
    }
    lp_batch* h = batch_common(count, m, n, (cudaStream_t)stream, false);
    if (!h) return nullptr;
    h->A = dA;
    h->b = db;
    h->c = dc;
    return h;
}

// The dynamic shared-memory limit of a kernel is process-wide state: it is
// raised once per kernel instance to the device's maximum (never lowered, so
// concurrent batches on other threads cannot race on it).
template <int NT>
static cudaError_t allow_max_smem() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, k_batch_solve<NT>);
        err = cudaFuncSetAttribute(k_batch_solve<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   optin - (int)fa.sharedSizeBytes);
    });
    return err;
}

template <int NT>
static cudaError_t launch_class(lp_batch* h, const BatchParams& P, int q, cudaStream_t s) {
    if (q == kGlobal) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_solve_global<NT>, NT, 0);
        const int grid = std::max(1, std::min(h->class_count[q], std::max(per, 1) * h->nsm));
        k_batch_solve_global<NT><<<grid, NT, 0, s>>>(P, h->lists[q], h->class_count[q], h->queues + q,
                                                     (unsigned char*)h->gwork.ptr);
        return cudaGetLastError();
    }
    const size_t smem = h->class_smem[q];
    cudaError_t e = allow_max_smem<NT>();
    if (e != cudaSuccess) return e;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_solve<NT>, NT, smem);
    const int grid = std::max(1, std::min(h->class_count[q], std::max(per, 1) * h->nsm));
    k_batch_solve<NT><<<grid, NT, smem, s>>>(P, h->lists[q], h->class_count[q], h->queues + q);
    return cudaGetLastError();
}

static cudaError_t launch_class_nt(lp_batch* h, const BatchParams& P, int q, int nt, cudaStream_t s) {
    switch (nt) {
        case 32: return launch_class<32>(h, P, q, s);
        case 64: return launch_class<64>(h, P, q, s);
        case 128: return launch_class<128>(h, P, q, s);
        case 256: return launch_class<256>(h, P, q, s);
        default: return launch_class<512>(h, P, q, s);
    }
}

// Streams and events of the graph path, created on its first use.
static bool ensure_graph_streams(lp_batch* h) {
    if (h->cap) return true;
    bool ok = (h->fork = event_get(false)) && (h->e_in = event_get(false)) && (h->e_out = event_get(false));
    for (int q = 0; q < kClasses; ++q) ok = ok && (h->side[q] = stream_get()) && (h->join[q] = event_get(false));
    ok = ok && (h->cap = stream_get());
    return ok;
}

// Every class: with `fork`, concurrently on one stream per class joined back
// into s (captured in a graph or launched directly); without, one after the
// other on s.
static cudaError_t enqueue_solve(lp_batch* h, const BatchParams& P, const int* nt, cudaStream_t s, bool fork) {
    cudaError_t e = cudaMemsetAsync(h->queues, 0, sizeof(unsigned) * kClasses, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->total, 0, sizeof(unsigned long long), s);
    if (fork && e == cudaSuccess) e = cudaEventRecord(h->fork, s);
    for (int q = 0; q < kClasses && e == cudaSuccess; ++q) {
        if (!h->class_count[q]) continue;
        if (!fork) {
            e = launch_class_nt(h, P, q, nt[q], s);
            continue;
        }
        e = cudaStreamWaitEvent(h->side[q], h->fork, 0);
        if (e == cudaSuccess) e = launch_class_nt(h, P, q, nt[q], h->side[q]);
        if (e == cudaSuccess) e = cudaEventRecord(h->join[q], h->side[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->join[q], 0);
    }
    return e;
}

lp_status lp_batch_solve(lp_batch_t h, const lp_batch_options* opt) {
    if (!h) {
        set_error("lp_batch_solve: NULL handle");
        return LP_ERR_INVALID;
    }
    lp_batch_options o;
    if (opt)
        o = *opt;
    else
        lp_batch_options_init(&o);
    if (!(o.eps_d >= 0.0) || !(o.eps_p >= 0.0) || o.rule < 0 || o.rule > 1 ||
        (o.threads != 0 && o.threads != 32 && o.threads != 64 && o.threads != 128 && o.threads != 256 &&
         o.threads != 512)) {
        set_error("lp_batch_solve: invalid options (threads must be 0, 32, 64, 128, 256 or 512)");
        return LP_ERR_INVALID;
    }
    TSX_CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : h->stream;
    if (o.keep_tableaux && !h->keep.ptr) {
        const size_t bytes = align_up(sizeof(double) * h->sum_t, 256) + align_up(sizeof(int) * h->sum_n, 256) +
                             sizeof(int) * h->sum_m;
        if (!bdev_alloc_block(h, h->keep, bytes)) {
            set_error("lp_batch_solve: allocation of the kept tableaux failed");
            return LP_ERR_NOMEM;
        }
    }
    BatchParams P{};
    P.lps = h->lps_dev;
    P.A = h->A;
    P.b = h->b;
    P.c = h->c;
    P.status = h->status;
    P.iters = h->iters;
    P.obj = h->obj;
    P.x = h->x;
    P.y = h->y;
    P.total_pivots = h->total;
    if (o.keep_tableaux) {
        char* kb = (char*)h->keep.ptr;
        P.keepT = (double*)kb;
        P.keepvar = (int*)(kb + align_up(sizeof(double) * h->sum_t, 256));
        P.keepbasis = (int*)(kb + align_up(sizeof(double) * h->sum_t, 256) + align_up(sizeof(int) * h->sum_n, 256));
    }
    P.eps_d = o.eps_d;
    P.eps_p = o.eps_p;
    P.max_iters = o.max_iters;
    P.k_cyc = o.k_cyc;
    P.rule = o.rule;

    // threads per LP: given, or timed per class on the first solve
    int nt[kClasses];
    h->stats.tune_ms = 0.0;
    if (o.threads == 0) {
        if (h->device >= 0 && h->device < kMaxDevices) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            for (int q = 0; q < kClasses; ++q)
                if (!h->tuned[q]) h->tuned[q] = g_tuned[h->device][q];
        }
        bool need = false;
        for (int q = 0; q < kClasses; ++q) need |= h->class_count[q] && !h->tuned[q];
        if (need) {
            float total_ms = 0.f;
            for (int q = 0; q < kClasses; ++q) {
                if (!h->class_count[q] || h->tuned[q]) continue;
                float best = 1e30f;
                int best_nt = 128;
                for (int cand : kCandidates) {
                    float ms = 0.f;
                    for (int rep = 0; rep < 2; ++rep) {   // first run warms up
                        TSX_CUDA_TRY(cudaMemsetAsync(h->queues, 0, sizeof(unsigned) * kClasses, s), LP_ERR_CUDA);
                        TSX_CUDA_TRY(cudaEventRecord(h->ev0, s), LP_ERR_CUDA);
                        TSX_CUDA_TRY(launch_class_nt(h, P, q, cand, s), LP_ERR_CUDA);
                        TSX_CUDA_TRY(cudaEventRecord(h->ev1, s), LP_ERR_CUDA);
                        TSX_CUDA_TRY(cudaEventSynchronize(h->ev1), LP_ERR_CUDA);
                        TSX_CUDA_TRY(cudaEventElapsedTime(&ms, h->ev0, h->ev1), LP_ERR_CUDA);
                        total_ms += ms;
                    }
                    if (ms < best) {
                        best = ms;
                        best_nt = cand;
                    }
                }
                h->tuned[q] = best_nt;
                if (h->device >= 0 && h->device < kMaxDevices) {
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    g_tuned[h->device][q] = best_nt;
                }
            }
            h->stats.tune_ms = total_ms;
        }
        for (int q = 0; q < kClasses; ++q) nt[q] = h->tuned[q] ? h->tuned[q] : 128;
    } else {
        for (int q = 0; q < kClasses; ++q) nt[q] = o.threads;
    }

    long long launches = 0;
    for (int q = 0; q < kClasses; ++q) launches += h->class_count[q] ? 1 : 0;
    bool used_graph = false;
    // a batch solved once runs its class launches directly (concurrently, on
    // the side streams); from its second solve on they are captured in a CUDA
    // graph once and replayed -- a capture pays off only when replayed
    if (o.use_graph && h->solves > 0) {
        const bool same = h->graph_valid && memcmp(&h->graph_params, &P, sizeof P) == 0 &&
                          memcmp(h->graph_nt, nt, sizeof nt) == 0;
        if (!same) {
            if (h->graph) cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
            h->graph_valid = false;
            // the attributes are set outside the capture
            for (int q = 0; q < kGlobal; ++q) {
                if (!h->class_count[q]) continue;
                cudaError_t e = cudaSuccess;
                switch (nt[q]) {
                    case 32: e = allow_max_smem<32>(); break;
                    case 64: e = allow_max_smem<64>(); break;
                    case 128: e = allow_max_smem<128>(); break;
                    case 256: e = allow_max_smem<256>(); break;
                    default: e = allow_max_smem<512>(); break;
                }
                TSX_CUDA_TRY(e, LP_ERR_CUDA);
            }
            if (!ensure_graph_streams(h)) {
                set_error("lp_batch_solve: stream/event creation failed");
                return LP_ERR_CUDA;
            }
            cudaGraph_t g = nullptr;
            TSX_CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), LP_ERR_CUDA);
            cudaError_t e = enqueue_solve(h, P, nt, h->cap, true);
            cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
            if (e != cudaSuccess || e2 != cudaSuccess || !g) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                set_error("lp_batch_solve: graph capture failed: %s",
                          cudaGetErrorString(e != cudaSuccess ? e : e2));
                return LP_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            TSX_CUDA_TRY(e, LP_ERR_CUDA);
            h->graph_params = P;
            memcpy(h->graph_nt, nt, sizeof nt);
            h->graph_valid = true;
        }
        TSX_CUDA_TRY(cudaEventRecord(h->e_in, s), LP_ERR_CUDA);
        TSX_CUDA_TRY(cudaStreamWaitEvent(h->cap, h->e_in, 0), LP_ERR_CUDA);
        TSX_CUDA_TRY(cudaEventRecord(h->ev0, h->cap), LP_ERR_CUDA);
        TSX_CUDA_TRY(cudaGraphLaunch(h->graph, h->cap), LP_ERR_CUDA);
        TSX_CUDA_TRY(cudaEventRecord(h->ev1, h->cap), LP_ERR_CUDA);
        TSX_CUDA_TRY(cudaEventRecord(h->e_out, h->cap), LP_ERR_CUDA);
        TSX_CUDA_TRY(cudaStreamWaitEvent(s, h->e_out, 0), LP_ERR_CUDA);
        used_graph = true;
    } else {
        if (!ensure_graph_streams(h)) {
            set_error("lp_batch_solve: stream/event creation failed");
            return LP_ERR_CUDA;
        }
        TSX_CUDA_TRY(cudaEventRecord(h->ev0, s), LP_ERR_CUDA);
        TSX_CUDA_TRY(enqueue_solve(h, P, nt, s, true), LP_ERR_CUDA);
        TSX_CUDA_TRY(cudaEventRecord(h->ev1, s), LP_ERR_CUDA);
    }
    ++h->solves;
    unsigned long long total = 0;
    TSX_CUDA_TRY(cudaMemcpyAsync(&total, h->total, sizeof total, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    TSX_CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    h->stats.solve_ms = ms;
    h->stats.total_pivots = (long long)total;
    h->stats.kernel_launches = launches;
    h->stats.graph = used_graph ? 1 : 0;
    int nb = 0;
    for (int q = 0; q < kClasses; ++q) {
        h->stats.threads[q] = h->class_count[q] ? nt[q] : 0;
        h->stats.lps_per_class[q] = h->class_count[q];
        nb += h->class_count[q] ? 1 : 0;
    }
    h->stats.buckets = nb;
    h->solved = true;
    h->kept = o.keep_tableaux != 0;
    return LP_OPTIMAL;
}

lp_status lp_batch_get(lp_batch_t h, int* status, long long* iters, double* obj, double* x, double* y) {
    if (!h) {
        set_error("lp_batch_get: NULL handle");
        return LP_ERR_INVALID;
    }
    if (!h->solved) {
        set_error("lp_batch_get: no solve has run on this batch");
        return LP_ERR_STATE;
    }
    TSX_CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
    cudaStream_t s = h->stream;
    if (status) TSX_CUDA_TRY(cudaMemcpyAsync(status, h->status, sizeof(int) * h->count, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    if (iters) TSX_CUDA_TRY(cudaMemcpyAsync(iters, h->iters, sizeof(long long) * h->count, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    if (obj) TSX_CUDA_TRY(cudaMemcpyAsync(obj, h->obj, sizeof(double) * h->count, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    if (x) TSX_CUDA_TRY(cudaMemcpyAsync(x, h->x, sizeof(double) * h->sum_n, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    if (y) TSX_CUDA_TRY(cudaMemcpyAsync(y, h->y, sizeof(double) * h->sum_m, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    TSX_CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    return LP_OPTIMAL;
}

lp_status lp_batch_get_tableau(lp_batch_t h, int index, double* T) {
    if (!h || !T || index < 0 || index >= (h ? h->count : 0)) {
        set_error("lp_batch_get_tableau: bad argument");
        return LP_ERR_INVALID;
    }
    if (!h->solved || !h->kept) {
        set_error("lp_batch_get_tableau: needs a solve with keep_tableaux = 1");
        return LP_ERR_STATE;
    }
    TSX_CUDA_TRY(cudaSetDevice(h->device), LP_ERR_CUDA);
    cudaStream_t s = h->stream;
    const BatchLP& L = h->lps[index];
    const size_t bytes = sizeof(double) * (size_t)(L.m + 1) * (L.n + L.m + 1);
    DBlock tmp;
    if (!bdev_alloc_block(h, tmp, bytes)) {
        set_error("lp_batch_get_tableau: allocation failed");
        return LP_ERR_NOMEM;
    }
    char* kb = (char*)h->keep.ptr;
    k_batch_expand<<<1, 256, 0, s>>>(h->lps_dev, index, (const double*)kb,
                                    (const int*)(kb + align_up(sizeof(double) * h->sum_t, 256)),
                                    (const int*)(kb + align_up(sizeof(double) * h->sum_t, 256) +
                                                 align_up(sizeof(int) * h->sum_n, 256)),
                                    (double*)tmp.ptr);
    TSX_CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    TSX_CUDA_TRY(cudaMemcpyAsync(T, tmp.ptr, bytes, cudaMemcpyDeviceToHost, s), LP_ERR_CUDA);
    TSX_CUDA_TRY(cudaStreamSynchronize(s), LP_ERR_CUDA);
    bdev_free(h, tmp);
    return LP_OPTIMAL;
}

lp_status lp_batch_get_stats(lp_batch_t h, lp_batch_stats* stats) {
    if (!h || !stats) {
        set_error("lp_batch_get_stats: NULL argument");
        return LP_ERR_INVALID;
    }
    if (!h->solved) {
        set_error("lp_batch_get_stats: no solve has run on this batch");
        return LP_ERR_STATE;
    }
    *stats = h->stats;
    return LP_OPTIMAL;
}
