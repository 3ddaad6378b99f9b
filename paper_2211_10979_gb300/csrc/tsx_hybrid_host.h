// Host share of the CPU+GPU split (arXiv 2211.10979, Section IV: the OpenMP
// threads' part, here a team of std::threads on the Grace cores).  The host
// holds nC column slots of the condensed tableau plus a copy of the
// right-hand side and of the basis, and runs Steps 1-3 on them in lockstep
// with the GPU kernel k_pivot_hybrid (tsx_hybrid.cuh), exchanging the Step 1
// candidates, the owner's Step 2 result and column q through the mailbox.
// Arithmetic as on the GPU: IEEE division for the pivot row and the ratios,
// std::fma for the update (built with -ffp-contract=off), the same candidate
// tests and tie rules, so every value equals the GPU-only solve's.
#pragma once

#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <thread>
#include <vector>

#include "tsx_hybrid.cuh"

namespace tsx {

struct HybHost {
    int m = 0, nC = 0, ldC = 0;
    double* T = nullptr;          // (m+1) x ldC: nC slots, right-hand side at column nC
    int* var = nullptr;           // nC: variable of each slot
    int* basis = nullptr;         // m: the host's copy of the basis
    double* F = nullptr;          // m+1: column q
    double* R = nullptr;          // ldC: scaled pivot row
    HybMailbox* mb = nullptr;     // host view of the mailbox
    const double* gF = nullptr;   // 2 x (m+1): column q from the GPU
    double* cF = nullptr;         // 2 x (m+1): column q for the GPU
    double eps_d = 1e-9, eps_p = 1e-9;
    long long max_iters = 0;
    int k_cyc = 50, rule = 0;
    long long wait_ns = 2'000'000'000LL;
    int nthreads = 1;
    int status = kRunning;        // outcome as seen by the host
    long long iters = 0;
};

class HybTeam {
public:
    explicit HybTeam(HybHost& h) : H(h), args(h.nthreads), rats(h.nthreads) {}

    // Runs the host share to the end on H.nthreads threads (the caller's
    // thread is one of them).
    void run() {
        std::vector<std::thread> th;
        for (int t = 1; t < H.nthreads; ++t) th.emplace_back([this, t] { work(t); });
        work(0);
        for (auto& t : th) t.join();
    }

private:
    struct alignas(64) Arg {
        double v;
        int key, slot, fkey, fslot;
    };
    struct alignas(64) Rat {
        double r;
        int key, i;
        double a;
    };
    HybHost& H;
    std::vector<Arg> args;
    std::vector<Rat> rats;
    std::atomic<unsigned> bar_count{0}, bar_gen{0};
    std::atomic<int> failed{0};
    // decisions of the current pivot (thread 0 writes them between barriers)
    int owner = 0, qC = -1, qv = INT_MAX, p = -1, leaving = -1, done = kRunning;
    double piv = 0.0, ratio = 0.0;

    static long long now_ns() {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(
                   std::chrono::steady_clock::now().time_since_epoch())
            .count();
    }

    // Spin barrier of the team, bounded like the device barriers.
    bool barrier() {
        const unsigned gen = bar_gen.load(std::memory_order_acquire);
        if (bar_count.fetch_add(1, std::memory_order_acq_rel) == (unsigned)H.nthreads - 1) {
            bar_count.store(0, std::memory_order_relaxed);
            bar_gen.store(gen + 1, std::memory_order_release);
            return failed.load(std::memory_order_acquire) == 0;
        }
        const long long t0 = now_ns();
        for (unsigned long long spins = 0; bar_gen.load(std::memory_order_acquire) == gen; ++spins) {
            if ((spins & 1023ull) == 0 && (failed.load(std::memory_order_acquire) || now_ns() - t0 > H.wait_ns)) {
                failed.store(1, std::memory_order_release);
                return false;
            }
        }
        return failed.load(std::memory_order_acquire) == 0;
    }

    // Bounded wait (thread 0) for the GPU's post of iteration want - 1.
    bool wait_seq(const unsigned* seq, unsigned want) {
        const long long t0 = now_ns();
        for (unsigned long long spins = 0;; ++spins) {
            if (__atomic_load_n(seq, __ATOMIC_ACQUIRE) == want) return true;
            if ((spins & 255ull) == 0) {
                if (__atomic_load_n(&H.mb->fail, __ATOMIC_ACQUIRE) != 0u || now_ns() - t0 > H.wait_ns) {
                    __atomic_store_n(&H.mb->fail, 1u, __ATOMIC_RELEASE);
                    return false;
                }
            }
        }
    }

    void fail_all() {
        failed.store(1, std::memory_order_release);
        __atomic_store_n(&H.mb->fail, 1u, __ATOMIC_RELEASE);
    }

    void work(int tid) {
        const int m = H.m, nC = H.nC, ld = H.ldC, T1 = H.nthreads;
        // the thread's slots, rows and pivot-row entries
        const int s0 = (int)((long long)nC * tid / T1), s1 = (int)((long long)nC * (tid + 1) / T1);
        const int r0 = (int)((long long)(m + 1) * tid / T1), r1 = (int)((long long)(m + 1) * (tid + 1) / T1);
        const int c0 = (int)((long long)(nC + 1) * tid / T1), c1 = (int)((long long)(nC + 1) * (tid + 1) / T1);
        const size_t mF = (size_t)m + 1;
        double* T = H.T;
        long long it = 0;
        int bland = H.rule == 1 ? 1 : 0, degen = 0;
        int end = kRunning;   // this thread's view of the outcome (the same on every thread)
        for (;;) {
            const int par = (int)(it & 1);
            const unsigned want = (unsigned)(it + 1);
            // Step 1 on the host's slots
            Arg a{INFINITY, INT_MAX, -1, INT_MAX, -1};
            for (int j = s0; j < s1; ++j) {
                const double v = T[j];
                if (v < -H.eps_d) {
                    const int vj = H.var[j];
                    if (v < a.v || (v == a.v && vj < a.key)) {
                        a.v = v;
                        a.key = vj;
                        a.slot = j;
                    }
                    if (vj < a.fkey) {
                        a.fkey = vj;
                        a.fslot = j;
                    }
                }
            }
            args[tid] = a;
            if (!barrier()) break;
            if (tid == 0) {
                Arg c = args[0];
                for (int t = 1; t < T1; ++t) {
                    const Arg& b = args[t];
                    if (b.key != INT_MAX && (c.key == INT_MAX || b.v < c.v || (b.v == c.v && b.key < c.key))) {
                        c.v = b.v;
                        c.key = b.key;
                        c.slot = b.slot;
                    }
                    if (b.fkey < c.fkey) {
                        c.fkey = b.fkey;
                        c.fslot = b.fslot;
                    }
                }
                HybPost* post = &H.mb->c1[par];
                post->v = c.v;
                post->key = c.key;
                post->slot = c.slot;
                post->fkey = c.fkey;
                post->fslot = c.fslot;
                __atomic_store_n(&post->seq, want, __ATOMIC_RELEASE);
                if (!wait_seq(&H.mb->g1[par].seq, want)) {
                    fail_all();
                } else {
                    const HybPost* g = &H.mb->g1[par];
                    const double gv = g->v;
                    const int gk = g->key, gf = g->fkey;
                    bool host_best;
                    if (bland) {
                        host_best = c.fkey < gf;
                        qv = host_best ? c.fkey : gf;
                        qC = host_best ? c.fslot : -1;
                    } else {
                        host_best = c.key != INT_MAX && (gk == INT_MAX || c.v < gv || (c.v == gv && c.key < gk));
                        qv = host_best ? c.key : gk;
                        qC = host_best ? c.slot : -1;
                    }
                    owner = host_best ? 1 : 0;
                    done = qv == INT_MAX ? kOptimal : (it >= H.max_iters ? kIterLimit : kRunning);
                }
            }
            if (!barrier()) break;
            if (done != kRunning) {
                end = done;
                break;
            }
            // Step 2: on the host's column, or the GPU's result
            if (owner == 1) {
                Rat best{INFINITY, INT_MAX, INT_MAX, 0.0};
                double* out = H.cF + (size_t)par * mF;
                for (int i = r0; i < r1; ++i) {
                    const double av = T[(size_t)i * ld + qC];
                    H.F[i] = av;
                    out[i] = av;
                    if (i >= 1 && av > H.eps_p) {
                        const double r = T[(size_t)i * ld + nC] / av;
                        if (!std::isnan(r)) {
                            const int key = bland ? H.basis[i - 1] : i;
                            if (best.i == INT_MAX || r < best.r || (r == best.r && key < best.key)) {
                                best.r = r;
                                best.key = key;
                                best.i = i;
                                best.a = av;
                            }
                        }
                    }
                }
                rats[tid] = best;
                if (!barrier()) break;
                if (tid == 0) {
                    Rat b = rats[0];
                    for (int t = 1; t < T1; ++t) {
                        const Rat& x = rats[t];
                        if (x.i != INT_MAX && (b.i == INT_MAX || x.r < b.r || (x.r == b.r && x.key < b.key))) b = x;
                    }
                    p = b.i == INT_MAX ? -1 : b.i;
                    piv = b.a;
                    ratio = b.r;
                    leaving = p > 0 ? H.basis[p - 1] : -1;
                    HybPost* post = &H.mb->c2[par];
                    post->p = p;
                    post->piv = piv;
                    post->ratio = ratio;
                    post->leaving = leaving;
                    post->entering = qv;
                    __atomic_store_n(&post->seq, want, __ATOMIC_RELEASE);
                }
            } else if (tid == 0) {
                if (!wait_seq(&H.mb->g2[par].seq, want)) {
                    fail_all();
                } else {
                    const HybPost* g = &H.mb->g2[par];
                    p = g->p;
                    piv = g->piv;
                    ratio = g->ratio;
                    leaving = g->leaving;
                }
            }
            if (!barrier()) break;
            if (p < 0) {
                end = kUnbounded;
                break;
            }
            if (!std::isfinite(piv) || !std::isfinite(ratio)) {
                end = kNumeric;
                break;
            }
            if (owner == 0) {
                const double* src = H.gF + (size_t)par * mF;
                for (int i = r0; i < r1; ++i) H.F[i] = src[i];
            }
            // Step 3: the host's part of the pivot row; the leaving variable
            // takes slot qC when the host holds it
            const double* rowp = T + (size_t)p * ld;
            for (int j = c0; j < c1; ++j) H.R[j] = (j == qC ? 1.0 : rowp[j]) / piv;
            if (!barrier()) break;
            if (tid == 0) {
                H.basis[p - 1] = qv;
                if (owner == 1) H.var[qC] = leaving;
            }
            for (int i = r0; i < r1; ++i) {
                double* row = T + (size_t)i * ld;
                if (i == p) {
                    for (int j = 0; j <= nC; ++j) row[j] = H.R[j];
                    continue;
                }
                const double f = H.F[i];
                for (int j = 0; j <= nC; ++j) row[j] = std::fma(-f, H.R[j], j == qC ? 0.0 : row[j]);
            }
            ++it;
            if (H.rule == 0) {
                if (ratio <= 0.0) {
                    ++degen;
                    if (H.k_cyc > 0 && degen >= H.k_cyc) bland = 1;
                } else {
                    degen = 0;
                    bland = 0;
                }
            }
            if (!barrier()) break;
        }
        if (tid == 0) {
            H.status = failed.load() ? kTimeout : end;
            H.iters = it;
        }
    }
};

}  // namespace tsx
