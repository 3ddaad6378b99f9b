// Request server for LP solves with continuous batching (lps_* in
// include/tabsimplex.h), and the device-side seeded input generator.
//
// Requests enter a FIFO queue.  A pool of worker threads (each with its own
// CUDA stream) takes work as soon as a worker is free and the device-memory
// budget allows: LPs small enough for the batched solver are taken together --
// every small request waiting at that moment, up to batch_max -- and solved as
// one micro-batch (lp_batch_*); the others are solved one per worker through
// the single-LP path (lp_create / lp_solve, FP32 + FP64 recovery by default).
// Requests that arrive while others are on the GPU join the next micro-batch
// or the next free worker, so their work overlaps on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tabsimplex.h"
#include "tsx_host.h"

using namespace tsx;

// ------------------------------------------------------------- generator
// The seeded dense LP of the benchmarks (the same definition as the Python
// generator lpgen.dense_lp): draw k of seed s is SplitMix64's output function
// applied to s + (k + 1) * 0x9E3779B97F4A7C15; u = (x >> 11) * 2^-53; draws in
// the order A (row-major), b, c; A_ij = 1 + 9u, b_i = 100 + 900u, c_j = 1 + 9u
// (product rounded, then the sum: no fused multiply-add).
__device__ __forceinline__ double gen_u01(unsigned long long seed, unsigned long long k) {
    unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

__global__ void k_generate_dense(int m, int n, unsigned long long seed, double* __restrict__ A,
                                 double* __restrict__ b, double* __restrict__ c) {
    const unsigned long long mn = (unsigned long long)m * n;
    const unsigned long long total = mn + m + n;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const double u = gen_u01(seed, k);
        if (k < mn)
            A[k] = __dadd_rn(1.0, __dmul_rn(9.0, u));
        else if (k < mn + m)
            b[k - mn] = __dadd_rn(100.0, __dmul_rn(900.0, u));
        else
            c[k - mn - m] = __dadd_rn(1.0, __dmul_rn(9.0, u));
    }
}

lp_status lp_generate_dense(int m, int n, unsigned long long seed, double* dA, double* db, double* dc,
                            void* stream) {
    if (m <= 0 || n <= 0 || !dA || !db || !dc) {
        set_error("lp_generate_dense: need m, n > 0 and three device arrays");
        return LP_ERR_INVALID;
    }
    const unsigned long long total = (unsigned long long)m * n + m + n;
    const int grid = (int)std::min<unsigned long long>((total + 255) / 256, 152ull * 32);
    k_generate_dense<<<grid, 256, 0, (cudaStream_t)stream>>>(m, n, seed, dA, db, dc);
    TSX_CUDA_TRY(cudaGetLastError(), LP_ERR_CUDA);
    return LP_OPTIMAL;
}

// ---------------------------------------------------------------- server
namespace {

using Clock = std::chrono::steady_clock;

double seconds(Clock::time_point t) {
    return std::chrono::duration<double>(t.time_since_epoch()).count();
}

struct Request {
    long long id = 0;
    int m = 0, n = 0;
    std::vector<double> hA, hb, hc;       // host inputs (lps_submit)
    const double *dA = nullptr, *db = nullptr, *dc = nullptr;   // device inputs
    bool on_device = false;
    size_t bytes = 0;                     // device memory held while admitted
    bool small = false;
    int status = 100;                     // running until done
    long long iters = 0;
    double obj = 0.0;
    std::vector<double> x, y;
    Clock::time_point t_submit, t_admit, t_done;
    Clock::time_point t_launch, t_kernel;  // its solve's launch began / its kernel completed
    lp_t h = nullptr;                     // its handle while in the continuous lane
    bool done = false;
};

// Device bytes a request holds while it is solved: inputs, the condensed
// tableau and work vectors, and for FP32 the FP64 recovery's k x 2k and k x k
// matrices at their largest (k = min(m, n)).
size_t request_bytes(int m, int n, bool small, int precision) {
    const size_t in = 8ull * ((size_t)m * n + m + n);
    if (small) return 2 * in + 8ull * (size_t)(m + 2) * (n + 3) + 64ull * (m + n) + 4096;
    const size_t elem = precision == LP_PREC_FP32 ? 4 : 8;
    const size_t ld = ((size_t)n + 1 + 31) / 32 * 32;
    const size_t tab = (size_t)(m + 1) * ld * elem + (size_t)(m + 1 + 2 * ld) * elem;
    const size_t k = (size_t)std::min(m, n);
    const size_t rec = precision == LP_PREC_FP32 ? 24ull * k * k + 128ull * (m + n) : 0;
    return in + tab + rec + 64ull * (m + n) + (1ull << 20);
}

}  // namespace

struct lp_server {
    lps_options opt{};
    int device = 0;
    size_t smem_limit = 0;               // batched solver's shared memory per LP
    int blocks = 0;                      // grid cap of a single-lane solve
    std::mutex mu;
    std::condition_variable cv_work;      // workers wait for requests
    std::condition_variable cv_done;      // clients wait for results
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<long long, std::shared_ptr<Request>> all;
    std::vector<std::thread> workers;
    std::vector<double> lat_ms, queue_ms, wait_ms, run_ms, post_ms;
    long long next_id = 0;
    long long used = 0, peak = 0;
    long long submitted = 0, completed = 0, batches = 0, batched_lps = 0, waves = 0, wave_lps = 0;
    double wave_ms = 0.0, wave_kernel_ms = 0.0, wave_create_ms = 0.0, wave_wait_ms = 0.0, wave_launch_ms = 0.0;
    bool wave_running = false;           // a wave's team launch holds the GPU
    bool wave_pending = false;           // a wave is being prepared or waits to launch
    int team_blocks = 0;                 // blocks per team of a wave, < 0: no waves
    std::string last_error;              // message of the latest failed solve
    bool stopping = false;
    bool started = false;
    Clock::time_point t_first, t_last;
    // continuous lane (lps_options.continuous): the team launch, its poller,
    // the requests in it, and those whose team is done (to be finished)
    TeamLane* lane = nullptr;
    std::thread poller;
    std::unordered_map<lp_t, std::shared_ptr<Request>> in_lane;
    std::deque<std::shared_ptr<Request>> finished;
    std::condition_variable cv_fin;       // finishers wait for lane results
    std::vector<std::thread> finishers;
    bool lane_drained = false;            // the poller has ended: no more lane results
    bool workers_done = false;            // every worker has left (no more admissions)
    int lane_admitting = 0;               // workers between taking lane requests and submitting them
    long long lane_lps = 0;
};

void lps_options_init(lps_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->budget_bytes = 64ll << 30;
    o->workers = 8;
    o->precision = LP_PREC_FP32;
    o->batch_small = 1;
    o->batch_max = 1024;
    o->small_max_dim = 0;
    o->blocks_per_lp = 0;
    o->batch_max_bytes = 0;
    o->path = LP_PATH_MULTILAUNCH;
    o->team_blocks = 0;
    o->continuous = 1;
}

// Keeps the calling worker's last library error for lps_last_error.
static void note_error(lp_server* sv, const char* where) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->last_error = std::string(where) + ": " + lp_last_error();
}

// Solves one single-path request on the calling worker thread.
static void solve_single(lp_server* sv, Request& r, cudaStream_t s) {
    lp_t h = r.on_device ? lp_create_device(r.m, r.n, r.dA, r.db, r.dc, (void*)s)
                         : lp_create(r.m, r.n, r.hA.data(), r.hb.data(), r.hc.data());
    if (!h) {
        note_error(sv, "create");
        r.status = LP_ERR_INVALID;
        return;
    }
    lp_options o;
    lp_options_init(&o);
    o.precision = sv->opt.precision;
    o.blocks = sv->blocks;
    o.path = sv->opt.path;
    o.stream = r.on_device ? (void*)s : nullptr;
    r.t_launch = Clock::now();
    r.status = lp_solve(h, &o);
    r.t_kernel = Clock::now();
    if (r.status < 0) note_error(sv, "solve");
    r.x.assign(r.n, 0.0);
    r.y.assign(r.m, 0.0);
    long long it = 0;
    if (r.status >= 0) lp_get_solution(h, r.x.data(), r.y.data(), &r.obj, nullptr, &it);
    r.iters = it;
    lp_destroy(h);
}

// Solves a micro-batch of small requests on the calling worker thread.
static void solve_batch(lp_server* sv, std::vector<std::shared_ptr<Request>>& rs, cudaStream_t s) {
    const int count = (int)rs.size();
    std::vector<int> m(count), n(count);
    size_t smn = 0, sm = 0, sn = 0;
    for (int k = 0; k < count; ++k) {
        m[k] = rs[k]->m;
        n[k] = rs[k]->n;
        smn += (size_t)m[k] * n[k];
        sm += m[k];
        sn += n[k];
    }
    // pack the inputs on the device (host requests: H2D, device requests: D2D)
    double* pack = nullptr;
    const size_t bytes = 8 * (smn + sm + sn);
    auto fail = [&](int st) {
        for (auto& r : rs) r->status = st;
    };
    if (pool_alloc((void**)&pack, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        fail(LP_ERR_NOMEM);
        return;
    }
    double *pA = pack, *pb = pack + smn, *pc = pb + sm;
    size_t oa = 0, ob = 0, oc = 0;
    bool ok = true;
    for (auto& rp : rs) {
        Request& r = *rp;
        const size_t a = (size_t)r.m * r.n;
        const cudaMemcpyKind kind = r.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        ok = ok && cudaMemcpyAsync(pA + oa, r.on_device ? (const void*)r.dA : r.hA.data(), 8 * a, kind, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(pb + ob, r.on_device ? (const void*)r.db : r.hb.data(), 8ull * r.m, kind, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(pc + oc, r.on_device ? (const void*)r.dc : r.hc.data(), 8ull * r.n, kind, s) == cudaSuccess;
        oa += a;
        ob += r.m;
        oc += r.n;
    }
    lp_batch_t h = ok ? lp_batch_create_device(count, m.data(), n.data(), pA, pb, pc, (void*)s) : nullptr;
    if (!h) {
        note_error(sv, "micro-batch create");
        fail(LP_ERR_INVALID);
        cudaFreeAsync(pack, s);
        cudaStreamSynchronize(s);
        return;
    }
    lp_batch_options bo;
    lp_batch_options_init(&bo);
    bo.stream = (void*)s;
    bo.use_graph = 0;   // solved once: a graph would not be replayed
    std::vector<int> st(count);
    std::vector<long long> it(count);
    std::vector<double> obj(count), x(sn), y(sm);
    const auto tl = Clock::now();
    const lp_status bs = lp_batch_solve(h, &bo);
    const auto tk = Clock::now();
    for (auto& r : rs) {
        r->t_launch = tl;
        r->t_kernel = tk;
    }
    if (bs == LP_OPTIMAL &&
        lp_batch_get(h, st.data(), it.data(), obj.data(), x.data(), y.data()) == LP_OPTIMAL) {
        size_t xo = 0, yo = 0;
        for (int k = 0; k < count; ++k) {
            Request& r = *rs[k];
            r.status = st[k];
            r.iters = it[k];
            r.obj = obj[k];
            r.x.assign(x.begin() + xo, x.begin() + xo + r.n);
            r.y.assign(y.begin() + yo, y.begin() + yo + r.m);
            xo += r.n;
            yo += r.m;
        }
    } else {
        note_error(sv, "micro-batch solve");
        fail(LP_ERR_CUDA);
    }
    lp_batch_destroy(h);
    cudaFreeAsync(pack, s);
    cudaStreamSynchronize(s);
    std::lock_guard<std::mutex> lk(sv->mu);
    ++sv->batches;
    sv->batched_lps += count;
}

// Blocks a wave's team launch leaves free (8 SMs' worth on GB300) for the
// previous wave's recovery and the micro-batches.
constexpr int kWaveReserve = 16;
// Blocks the continuous team launch leaves free (16 SMs' worth on GB300): it
// stays resident while requests keep coming, so the micro-batches and the
// FP64 recoveries run beside it all the time.
constexpr int kLaneReserve = 32;

// Solves the requests too large for the micro-batches together: one
// lp_solve_many call (a team of blocks per LP) on the calling worker thread.
static void solve_wave(lp_server* sv, std::vector<std::shared_ptr<Request>>& rs, cudaStream_t s) {
    const auto t0 = Clock::now();
    std::vector<lp_t> hs;
    std::vector<Request*> who;
    for (auto& rp : rs) {
        Request& r = *rp;
        // device inputs: the team kernel checks them while building the tableau
        lp_t h = r.on_device ? create_device_unchecked(r.m, r.n, r.dA, r.db, r.dc, s)
                             : lp_create(r.m, r.n, r.hA.data(), r.hb.data(), r.hc.data());
        if (!h) {
            note_error(sv, "create");
            r.status = LP_ERR_INVALID;
            continue;
        }
        hs.push_back(h);
        who.push_back(&r);
    }
    lp_options o;
    lp_options_init(&o);
    o.precision = sv->opt.precision;
    o.blocks = sv->team_blocks;
    o.stream = (void*)s;
    std::vector<lp_status> st(hs.size(), LP_ERR_STATE);
    // the team launch runs when the previous wave's launch has completed; the
    // previous wave's recovery and read-out overlap this launch on the blocks
    // it leaves free, and the next wave is prepared meanwhile
    const auto t1 = Clock::now();
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->cv_work.wait(lk, [&] { return !sv->wave_running; });
        sv->wave_running = true;
        sv->wave_pending = false;
    }
    sv->cv_work.notify_all();
    const auto t2 = Clock::now();
    auto t3 = t2;
    bool released = false;
    auto release = [&] {
        t3 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->wave_running = false;
        }
        released = true;
        sv->cv_work.notify_all();
    };
    const lp_status rc = hs.empty() ? LP_OPTIMAL
                                    : solve_many_hooked(hs.data(), (int)hs.size(), &o, st.data(), kWaveReserve, release);
    if (!released) release();
    if (rc != LP_OPTIMAL) note_error(sv, "wave");
    for (Request* r : who) {
        r->t_launch = t2;
        r->t_kernel = t3;
    }
    auto ms_of = [](Clock::time_point a, Clock::time_point b) {
        return 1e3 * std::chrono::duration<double>(b - a).count();
    };
    double kernel_ms = 0.0;
    for (size_t k = 0; k < hs.size() && rc == LP_OPTIMAL; ++k) {
        lp_stats ls;
        if (lp_get_stats(hs[k], &ls) == LP_OPTIMAL && ls.path == LP_PATH_TEAM) {
            kernel_ms = ls.pivot_ms;
            break;
        }
    }
    for (size_t k = 0; k < hs.size(); ++k) {
        Request& r = *who[k];
        r.status = rc != LP_OPTIMAL ? rc : st[k];
        if (r.status < 0 && rc == LP_OPTIMAL) note_error(sv, "wave solve");
        r.x.assign(r.n, 0.0);
        r.y.assign(r.m, 0.0);
        long long it = 0;
        if (r.status >= 0) lp_get_solution(hs[k], r.x.data(), r.y.data(), &r.obj, nullptr, &it);
        r.iters = it;
        lp_destroy(hs[k]);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    ++sv->waves;
    sv->wave_lps += (long long)rs.size();
    sv->wave_ms += ms_of(t0, Clock::now());
    sv->wave_kernel_ms += kernel_ms;
    sv->wave_create_ms += ms_of(t0, t1);
    sv->wave_wait_ms += ms_of(t1, t2);
    sv->wave_launch_ms += ms_of(t2, t3);
}

// Continuous lane: creates the handles of admitted large requests and hands
// them to the running team launch; a request that does not fit a team is
// solved here by lp_solve.  Returns the requests completed on this thread.
static std::vector<std::shared_ptr<Request>> lane_admit(lp_server* sv, std::vector<std::shared_ptr<Request>>& rs,
                                                        cudaStream_t s) {
    std::vector<std::shared_ptr<Request>> now;
    for (auto& rp : rs) {
        Request& r = *rp;
        lp_t h = r.on_device ? create_device_unchecked(r.m, r.n, r.dA, r.db, r.dc, s)
                             : lp_create(r.m, r.n, r.hA.data(), r.hb.data(), r.hc.data());
        if (!h) {
            note_error(sv, "create");
            r.status = LP_ERR_INVALID;
            now.push_back(rp);
            continue;
        }
        r.h = h;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->in_lane[h] = rp;
        }
        r.t_launch = Clock::now();
        const long long tok = lane_submit(sv->lane, h);
        if (tok >= 0) continue;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->in_lane.erase(h);
        }
        r.h = nullptr;
        if (tok == -2) {   // larger than a team's shared memory: the single-LP path
            lp_destroy(h);
            solve_single(sv, r, s);
        } else {
            note_error(sv, "lane");
            r.status = LP_ERR_CUDA;
            lp_destroy(h);
        }
        now.push_back(rp);
    }
    return now;
}

// A request whose team is done: statistics, FP64 recovery, read-out.
static void lane_complete(lp_server* sv, Request& r, cudaStream_t s) {
    lp_status st = LP_ERR_STATE;
    if (lane_finish(sv->lane, r.h, s, &st) != LP_OPTIMAL) {
        note_error(sv, "lane finish");
        st = LP_ERR_CUDA;
    }
    r.status = st;
    if (r.status < 0) note_error(sv, "lane solve");
    r.x.assign(r.n, 0.0);
    r.y.assign(r.m, 0.0);
    long long it = 0;
    if (r.status >= 0) lp_get_solution(r.h, r.x.data(), r.y.data(), &r.obj, nullptr, &it);
    r.iters = it;
    lp_destroy(r.h);
    r.h = nullptr;
}

// Polls the lane for requests whose team is done and hands them to the
// workers; relaunches the team kernel when jobs wait (lane_poll).
static void poller_main(lp_server* sv) {
    cudaSetDevice(sv->device);
    std::vector<lp_t> done;
    for (;;) {
        done.clear();
        const int left = lane_poll(sv->lane, done);
        if (!done.empty()) {
            const auto now = Clock::now();
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                for (lp_t h : done) {
                    auto it = sv->in_lane.find(h);
                    if (it == sv->in_lane.end()) continue;
                    it->second->t_kernel = now;
                    sv->finished.push_back(it->second);
                    sv->in_lane.erase(it);
                }
            }
            sv->cv_fin.notify_all();
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (sv->stopping && sv->queue.empty() && sv->in_lane.empty() && sv->lane_admitting == 0 && left == 0 &&
                sv->workers_done)
                break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->lane_drained = true;
    }
    sv->cv_fin.notify_all();
}

// Finishes lane requests whose team is done (FP64 recovery, read-out), on
// threads of their own so that admission and micro-batches never wait for them.
static void finisher_main(lp_server* sv) {
    cudaSetDevice(sv->device);
    use_default_allocator(true);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_fin.wait(lk, [&] { return !sv->finished.empty() || sv->lane_drained; });
            if (sv->finished.empty()) break;
            r = sv->finished.front();
            sv->finished.pop_front();
        }
        lane_complete(sv, *r, s);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            const auto now = Clock::now();
            r->t_done = now;
            r->done = true;
            sv->used -= (long long)r->bytes;
            ++sv->completed;
            ++sv->lane_lps;
            sv->lat_ms.push_back(1e3 * std::chrono::duration<double>(r->t_done - r->t_submit).count());
            sv->queue_ms.push_back(1e3 * std::chrono::duration<double>(r->t_admit - r->t_submit).count());
            sv->wait_ms.push_back(1e3 * std::chrono::duration<double>(r->t_launch - r->t_admit).count());
            sv->run_ms.push_back(1e3 * std::chrono::duration<double>(r->t_kernel - r->t_launch).count());
            sv->post_ms.push_back(1e3 * std::chrono::duration<double>(r->t_done - r->t_kernel).count());
            r->hA.clear();
            r->hA.shrink_to_fit();
            r->hb.clear();
            r->hc.clear();
            sv->t_last = now;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();   // budget freed
    }
    cudaStreamDestroy(s);
}

static void worker_main(lp_server* sv) {
    cudaSetDevice(sv->device);
    use_default_allocator(true);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        std::vector<std::shared_ptr<Request>> take;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // arrival order: the head is admitted first once the budget allows;
            // small requests queued behind it join its micro-batch, and with
            // waves, every large request waiting joins the wave.  While a wave
            // is being prepared or waits for the previous one's launch, large
            // requests wait for the wave after it and the other workers serve
            // the small ones.
            const bool lane = sv->lane != nullptr;
            const bool waves = sv->team_blocks >= 0 && !lane;
            auto pick = [&]() -> std::deque<std::shared_ptr<Request>>::iterator {
                for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
                    const bool large = !((*it)->small && sv->opt.batch_small);
                    if (waves && large && sv->wave_pending) continue;
                    if (sv->used + (long long)(*it)->bytes > sv->opt.budget_bytes) return sv->queue.end();
                    return it;
                }
                return sv->queue.end();
            };
            sv->cv_work.wait(lk, [&] { return sv->stopping || pick() != sv->queue.end(); });
            auto first = pick();
            if (first == sv->queue.end()) {
                if (sv->stopping && sv->queue.empty()) break;
                if (sv->stopping) {
                    sv->cv_work.wait(lk, [&] { return sv->queue.empty() || pick() != sv->queue.end(); });
                    continue;
                }
                continue;
            }
            auto head = *first;
            sv->queue.erase(first);
            sv->used += (long long)head->bytes;
            take.push_back(head);
            const bool head_large = !(head->small && sv->opt.batch_small);
            if ((waves || lane) && head_large) {
                if (waves) sv->wave_pending = true;
                for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)take.size() < sv->opt.batch_max;) {
                    const bool large = !((*it)->small && sv->opt.batch_small);
                    if (large && sv->used + (long long)(*it)->bytes <= sv->opt.budget_bytes) {
                        sv->used += (long long)(*it)->bytes;
                        take.push_back(*it);
                        it = sv->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            } else if (!head_large) {
                for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)take.size() < sv->opt.batch_max;) {
                    if ((*it)->small && sv->used + (long long)(*it)->bytes <= sv->opt.budget_bytes) {
                        sv->used += (long long)(*it)->bytes;
                        take.push_back(*it);
                        it = sv->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
            sv->peak = std::max(sv->peak, sv->used);
            const auto now = Clock::now();
            for (auto& r : take) r->t_admit = now;
            if (lane && head_large) ++sv->lane_admitting;
        }
        const bool large = !(take[0]->small && sv->opt.batch_small);
        if (large && sv->lane) {
            // handed to the running team launch: finished later by a worker,
            // except requests that failed or were solved here
            take = lane_admit(sv, take, s);
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                --sv->lane_admitting;
            }
            sv->cv_work.notify_all();
            if (take.empty()) continue;
        } else if (large && sv->team_blocks >= 0)
            solve_wave(sv, take, s);
        else if (large)
            solve_single(sv, *take[0], s);
        else
            solve_batch(sv, take, s);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            const auto now = Clock::now();
            for (auto& r : take) {
                r->t_done = now;
                r->done = true;
                sv->used -= (long long)r->bytes;
                ++sv->completed;
                sv->lat_ms.push_back(1e3 * std::chrono::duration<double>(r->t_done - r->t_submit).count());
                sv->queue_ms.push_back(1e3 * std::chrono::duration<double>(r->t_admit - r->t_submit).count());
                if (r->t_launch.time_since_epoch().count() && r->t_kernel.time_since_epoch().count()) {
                    sv->wait_ms.push_back(1e3 * std::chrono::duration<double>(r->t_launch - r->t_admit).count());
                    sv->run_ms.push_back(1e3 * std::chrono::duration<double>(r->t_kernel - r->t_launch).count());
                    sv->post_ms.push_back(1e3 * std::chrono::duration<double>(r->t_done - r->t_kernel).count());
                }
                r->hA.clear();
                r->hA.shrink_to_fit();
                r->hb.clear();
                r->hc.clear();
            }
            sv->t_last = now;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    cudaStreamDestroy(s);
}

lps_t lps_open(const lps_options* opt) {
    lp_server* sv = new lp_server();
    if (opt)
        sv->opt = *opt;
    else
        lps_options_init(&sv->opt);
    if (sv->opt.workers <= 0 || sv->opt.budget_bytes <= 0 || sv->opt.batch_max <= 0 || sv->opt.precision < 0 ||
        sv->opt.precision > 1 || sv->opt.path < LP_PATH_AUTO || sv->opt.path > LP_PATH_MULTILAUNCH) {
        set_error("lps_open: invalid options");
        delete sv;
        return nullptr;
    }
    cudaGetDevice(&sv->device);
    sv->smem_limit = batch_smem_limit();
    // each single-lane solve gets a share of the GPU's blocks (a quarter with
    // the default 8 workers), so that solves of several workers run side by side
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, sv->device);
    sv->team_blocks = sv->opt.team_blocks < 0 ? -1 : sv->opt.team_blocks;
    sv->blocks = sv->opt.blocks_per_lp > 0 ? sv->opt.blocks_per_lp
                                           : std::max(16, 4 * nsm / std::max(1, sv->opt.workers));
    if (sv->opt.continuous && sv->team_blocks >= 0) {
        lp_options lo;
        lp_options_init(&lo);
        lo.precision = sv->opt.precision;
        lo.blocks = sv->team_blocks;
        sv->lane = lane_open(&lo, kLaneReserve);
        if (!sv->lane) {
            delete sv;
            return nullptr;
        }
        sv->poller = std::thread(poller_main, sv);
        for (int w = 0; w < sv->opt.workers; ++w) sv->finishers.emplace_back(finisher_main, sv);
    }
    for (int w = 0; w < sv->opt.workers; ++w) sv->workers.emplace_back(worker_main, sv);
    return sv;
}

static long long enqueue(lp_server* sv, std::shared_ptr<Request> r) {
    // the batch lane: LPs whose condensed tableau fits shared memory, or is at
    // most batch_max_bytes (solved from global memory, one block per LP)
    const size_t cbytes = 8ull * (size_t)(r->m + 1) * (size_t)(r->n + 2);
    r->small = sv->opt.batch_small &&
               (batch_fits(r->m, r->n, sv->smem_limit) || cbytes <= (size_t)sv->opt.batch_max_bytes) &&
               (sv->opt.small_max_dim <= 0 || (r->m <= sv->opt.small_max_dim && r->n <= sv->opt.small_max_dim));
    r->bytes = request_bytes(r->m, r->n, r->small, sv->opt.precision);
    if ((long long)r->bytes > sv->opt.budget_bytes) {
        set_error("lps_submit: request needs %zu bytes, more than the budget", r->bytes);
        return -1;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) {
            set_error("lps_submit: server is closing");
            return -1;
        }
        r->id = sv->next_id++;
        r->t_submit = Clock::now();
        if (!sv->started) {
            sv->started = true;
            sv->t_first = r->t_submit;
        }
        sv->all[r->id] = r;
        sv->queue.push_back(r);
        ++sv->submitted;
    }
    sv->cv_work.notify_one();
    return r->id;
}

long long lps_submit(lps_t sv, int m, int n, const double* A, const double* b, const double* c) {
    if (!sv || m <= 0 || n <= 0 || !A || !b || !c) {
        set_error("lps_submit: bad argument");
        return -1;
    }
    auto r = std::make_shared<Request>();
    r->m = m;
    r->n = n;
    r->hA.assign(A, A + (size_t)m * n);
    r->hb.assign(b, b + m);
    r->hc.assign(c, c + n);
    return enqueue(sv, r);
}

long long lps_submit_device(lps_t sv, int m, int n, const double* dA, const double* db, const double* dc) {
    if (!sv || m <= 0 || n <= 0 || !dA || !db || !dc) {
        set_error("lps_submit_device: bad argument");
        return -1;
    }
    auto r = std::make_shared<Request>();
    r->m = m;
    r->n = n;
    r->dA = dA;
    r->db = db;
    r->dc = dc;
    r->on_device = true;
    return enqueue(sv, r);
}

int lps_wait(lps_t sv, long long ticket, double timeout_s) {
    if (!sv) return LP_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) {
        set_error("lps_wait: unknown ticket %lld", ticket);
        return LP_ERR_INVALID;
    }
    auto r = it->second;
    const auto pred = [&] { return r->done; };
    if (timeout_s < 0)
        sv->cv_done.wait(lk, pred);
    else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
        return 100;
    return r->status;
}

lp_status lps_result(lps_t sv, long long ticket, double* x, double* y, double* obj, long long* iters,
                     double* times) {
    if (!sv) return LP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) {
        set_error("lps_result: unknown ticket %lld", ticket);
        return LP_ERR_INVALID;
    }
    Request& r = *it->second;
    if (!r.done) {
        set_error("lps_result: request %lld is not finished", ticket);
        return LP_ERR_STATE;
    }
    if (x && !r.x.empty()) memcpy(x, r.x.data(), sizeof(double) * r.n);
    if (y && !r.y.empty()) memcpy(y, r.y.data(), sizeof(double) * r.m);
    if (obj) *obj = r.obj;
    if (iters) *iters = r.iters;
    if (times) {
        times[0] = seconds(r.t_submit);
        times[1] = seconds(r.t_admit);
        times[2] = seconds(r.t_done);
    }
    return (lp_status)r.status;
}

lp_status lps_release(lps_t sv, long long ticket) {
    if (!sv) return LP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end() || !it->second->done) {
        set_error("lps_release: unknown or unfinished ticket %lld", ticket);
        return LP_ERR_STATE;
    }
    sv->all.erase(it);
    return LP_OPTIMAL;
}

static double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

lp_status lps_get_stats(lps_t sv, lps_stats* st) {
    if (!sv || !st) return LP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(st, 0, sizeof *st);
    st->submitted = sv->submitted;
    st->completed = sv->completed;
    st->wall_s = sv->completed ? std::chrono::duration<double>(sv->t_last - sv->t_first).count() : 0.0;
    st->lat_p50_ms = percentile(sv->lat_ms, 0.50);
    st->lat_p99_ms = percentile(sv->lat_ms, 0.99);
    st->lat_max_ms = sv->lat_ms.empty() ? 0.0 : *std::max_element(sv->lat_ms.begin(), sv->lat_ms.end());
    double sum = 0.0;
    for (double v : sv->lat_ms) sum += v;
    st->lat_mean_ms = sv->lat_ms.empty() ? 0.0 : sum / (double)sv->lat_ms.size();
    st->queue_p50_ms = percentile(sv->queue_ms, 0.50);
    st->queue_p99_ms = percentile(sv->queue_ms, 0.99);
    st->wait_p50_ms = percentile(sv->wait_ms, 0.50);
    st->wait_p99_ms = percentile(sv->wait_ms, 0.99);
    st->run_p50_ms = percentile(sv->run_ms, 0.50);
    st->run_p99_ms = percentile(sv->run_ms, 0.99);
    st->post_p50_ms = percentile(sv->post_ms, 0.50);
    st->post_p99_ms = percentile(sv->post_ms, 0.99);
    st->batches = sv->batches;
    st->batched_lps = sv->batched_lps;
    st->waves = sv->waves;
    st->wave_lps = sv->wave_lps;
    st->wave_ms = sv->wave_ms;
    st->wave_kernel_ms = sv->wave_kernel_ms;
    st->wave_create_ms = sv->wave_create_ms;
    st->wave_wait_ms = sv->wave_wait_ms;
    st->wave_launch_ms = sv->wave_launch_ms;
    st->peak_bytes = sv->peak;
    st->lane_lps = sv->lane_lps;
    st->lane_launches = sv->lane ? lane_launches(sv->lane) : 0;
    return LP_OPTIMAL;
}

const char* lps_last_error(lps_t sv) {
    if (!sv) return "";
    thread_local std::string copy;
    std::lock_guard<std::mutex> lk(sv->mu);
    copy = sv->last_error;
    return copy.c_str();
}

void lps_close(lps_t sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->workers_done = true;
    }
    if (sv->poller.joinable()) sv->poller.join();
    for (auto& t : sv->finishers) t.join();
    if (sv->lane) lane_close(sv->lane);
    delete sv;
}
