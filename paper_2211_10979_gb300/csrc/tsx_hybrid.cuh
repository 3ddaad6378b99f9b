// The paper's CPU+GPU split of the tableau (arXiv 2211.10979, Section IV:
// Setup, Initialization and Steps 1-4), on one GB300 and its Grace host.
//
// The condensed tableau's nonbasic column slots are split: the GPU keeps the
// first nG slots (a fraction theta of them), host threads the other nC; both
// keep a copy of the right-hand side and of the basis.  Per pivot:
//   Step 1  each side finds its own most negative objective-row entry; the
//           two posts are exchanged and both take the same minimum (value,
//           then variable) -- the owner of the entering slot is known to both;
//   Step 2  the owner runs the minimum-ratio test on its column q and posts the
//           leaving row, the pivot element, the minimum ratio, the leaving and
//           entering variables, and column q itself (the paper's "data of the
//           winning column are sent");
//   Step 3  both sides scale their part of the pivot row and update their
//           columns and their copy of the right-hand side.
// The GPU side is the persistent kernel's phases on its (m+1) x (nG+1)
// condensed tableau, with the two exchanges added; the host side does the
// same arithmetic (IEEE division, one fused multiply-add per entry, the same
// tie rules), so every pivot and value equals the GPU-only solve's.
// Posts go through a mailbox in mapped host memory: a writer fills a post and
// then stores its sequence number (iteration + 1) with release semantics; a
// reader waits (bounded) until it sees that number with acquire semantics.
// Posts are double-buffered by iteration parity: a side can only overwrite
// the post of iteration i after reading the other side's Step 1 post of
// iteration i + 1, which the other side makes only after finishing iteration i.
#pragma once

#include "tsx_kernels.cuh"

namespace tsx {

struct HybPost {
    unsigned seq;              // iteration + 1 once the post is complete
    int owner;                 // Step 1: 0 (this post is a candidate); Step 2: unused
    double v;                  // Step 1: most negative entry (+inf if none)
    int key, slot;             // Step 1: its variable (INT_MAX if none) and local slot
    int fkey, fslot;           // Step 1: lowest candidate variable (Bland) and its slot
    int p;                     // Step 2: leaving row (-1: no eligible row, unbounded)
    int leaving, entering;     // Step 2: the variables that leave and enter
    int pad;
    double piv, ratio;         // Step 2: pivot element and minimum ratio
};

struct HybMailbox {            // mapped host memory
    HybPost g1[2], c1[2];      // Step 1 posts of the GPU and of the host, by parity
    HybPost g2[2], c2[2];      // Step 2 posts of the owner, by parity
    unsigned fail;             // a side gave up waiting: the other leaves too
    unsigned pad[15];
};

struct HybParams {
    HybMailbox* mb;            // device pointer of the mailbox
    double* gF;                // column q from the GPU, 2 x (m+1) (mapped host memory)
    const double* cF;          // column q from the host, 2 x (m+1) (mapped host memory)
    long long wait_ns;         // bound on one wait for the other side
};

__device__ __forceinline__ unsigned hyb_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void hyb_st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait (one thread) until *seq == want; false if the time ran out or
// the other side gave up.
__device__ inline bool hyb_wait(HybMailbox* mb, const unsigned* seq, unsigned want, long long wait_ns) {
    const long long t0 = global_ns();
    const unsigned long long max_spins = (unsigned long long)(wait_ns > 0 ? wait_ns : 0) / 64ull + 4096ull;
    for (unsigned long long spins = 0;; ++spins) {
        if (hyb_ld_acquire(seq) == want) return true;
        if ((spins & 15ull) == 0) {
            if (*(volatile unsigned*)&mb->fail != 0u) return false;
            if (global_ns() - t0 >= wait_ns || spins > max_spins) {
                hyb_st_release(&mb->fail, 1u);
                return false;
            }
        }
        __nanosleep(64);
    }
}

// Step 2 of the persistent kernel (phase_ratio) that also writes column q to
// the mailbox for the host.
__device__ void hyb_phase_ratio(const Params<double>& P, int q, int bland, BlockScratch& s, double* F_host) {
    RatPart best = rat_none();
    const long long nth = (long long)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.st->nact = 0;
        P.st->next_slot = 0;
    }
    for (long long i = (long long)threadIdx.x * gridDim.x + blockIdx.x; i <= P.m; i += nth) {
        const double* row = P.T + (size_t)i * (size_t)P.ld;
        const double a = __ldcg(row + q);
        __stcg(P.F + i, a);
        F_host[i] = a;
        if (i >= 1 && a > P.eps_p) {
            RatPart c;
            c.r = div_rn(__ldcg(row + (P.W - 1)), a);
            c.i = (int)i;
            c.key = bland ? __ldcg(P.basis + (i - 1)) : (int)i;
            c.a = a;
            if (!dbits_nan(c.r)) rat_merge(best, c);
        }
    }
    __threadfence_system();   // column q reaches the host before the post
    best = block_rat(best, s);
    if (threadIdx.x == 0) store_rat(P.rpart + blockIdx.x, best);
}

struct HybShared {             // a block's copy of the exchanged decisions
    int owner;                 // 0: the GPU holds the entering slot, 1: the host
    int q;                     // the GPU's local slot (owner 0), else -1
    int qv;                    // entering variable, INT_MAX: optimal
    int p, leaving;
    double piv, ratio;
    int ok;
};

template <int NT>
__global__ void __launch_bounds__(NT, persistent_sm_threads(NT) / NT) k_pivot_hybrid(Params<double> P, HybParams H) {
    __shared__ BlockScratch s;
    __shared__ HybShared hs;
    __shared__ PhaseClock clk;
    if (threadIdx.x == 0) s.passed = 0;
    clk.start();
    phase_init_argmin(P);
    if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
    long long it = 0;
    int bland = P.rule == 1 ? 1 : 0;
    int degen = 0;
    HybMailbox* mb = H.mb;
    const size_t mF = (size_t)P.m + 1;
    for (;;) {
        const int par = (int)(it & 1);
        const unsigned want = (unsigned)(it + 1);
        // Step 1: this side's candidate, exchanged with the host's
        const ArgPart e = phase_entering(P, s);
        if (threadIdx.x == 0) {
            if (blockIdx.x == 0) {
                HybPost* g = &mb->g1[par];
                g->v = e.v;
                g->key = e.key;
                g->slot = e.slot;
                g->fkey = e.fkey;
                g->fslot = e.fslot;
                __threadfence_system();
                hyb_st_release(&g->seq, want);
            }
            hs.ok = hyb_wait(mb, &mb->c1[par].seq, want, H.wait_ns) ? 1 : 0;
            if (hs.ok) {
                const HybPost* c = &mb->c1[par];
                const double cv = *(volatile const double*)&c->v;
                const int ck = *(volatile const int*)&c->key, cf = *(volatile const int*)&c->fkey;
                // the same minimum on both sides: value, then variable
                bool host_best;
                if (bland) {
                    host_best = cf < e.fkey;
                    hs.qv = host_best ? cf : e.fkey;
                    hs.q = host_best ? -1 : e.fslot;
                } else {
                    const long long ek = dkey(e.v), hk = dkey(cv);
                    host_best = ck != INT_MAX && (e.key == INT_MAX || hk < ek || (hk == ek && ck < e.key));
                    hs.qv = host_best ? ck : e.key;
                    hs.q = host_best ? -1 : e.slot;
                }
                hs.owner = host_best ? 1 : 0;
            }
        }
        __syncthreads();
        const int ok1 = hs.ok, owner = hs.owner, q = hs.q, qv = hs.qv;
        __syncthreads();   // hs is written again below
        if (!ok1) { finish(P, kTimeout, it, bland, degen, clk.acc); return; }
        if (qv == INT_MAX) { finish(P, kOptimal, it, bland, degen, clk.acc); return; }
        if (it >= P.max_iters) { finish(P, kIterLimit, it, bland, degen, clk.acc); return; }
        clk.lap(0);
        int p;
        double piv, ratio;
        int leaving;
        if (owner == 0) {
            // Step 2 on the GPU's column; column q goes to the host as well
            hyb_phase_ratio(P, q, bland, s, H.gF + (size_t)par * mF);
            if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
            const RatPart l = phase_leaving(P, s);
            p = l.i == INT_MAX ? -1 : l.i;
            piv = l.a;
            ratio = l.r;
            leaving = -1;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                // block 0 alone reads the leaving variable: it updates the basis below
                leaving = p > 0 ? P.basis[p - 1] : -1;
                HybPost* g = &mb->g2[par];
                g->p = p;
                g->piv = piv;
                g->ratio = ratio;
                g->leaving = leaving;
                g->entering = qv;
                __threadfence_system();
                hyb_st_release(&g->seq, want);
            }
        } else {
            // Step 2 on the host: its result and column q.  The update's work
            // counters start from zero each pivot (phase_ratio resets them
            // when the GPU runs Step 2).
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                P.st->nact = 0;
                P.st->next_slot = 0;
            }
            if (threadIdx.x == 0) {
                hs.ok = hyb_wait(mb, &mb->c2[par].seq, want, H.wait_ns) ? 1 : 0;
                if (hs.ok) {
                    const volatile HybPost* c = &mb->c2[par];
                    hs.p = c->p;
                    hs.piv = c->piv;
                    hs.ratio = c->ratio;
                    hs.leaving = c->leaving;
                }
            }
            __syncthreads();
            const int ok2 = hs.ok;
            p = hs.p;
            piv = hs.piv;
            ratio = hs.ratio;
            leaving = hs.leaving;
            __syncthreads();   // hs is written again in the next iteration
            if (!ok2) { finish(P, kTimeout, it, bland, degen, clk.acc); return; }
            if (p > 0) {
                const volatile double* src = H.cF + (size_t)par * mF;
                for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= P.m;
                     i += (long long)gridDim.x * blockDim.x)
                    __stcg(P.F + i, src[i]);
            }
        }
        if (p < 0) { finish(P, kUnbounded, it, bland, degen, clk.acc); return; }
        if (!isfinite(piv) || !isfinite(ratio)) { finish(P, kNumeric, it, bland, degen, clk.acc); return; }
        // Step 3: the GPU's part of the pivot row; the leaving variable takes
        // slot q when the GPU holds it
        phase_stage_row(P, p, q, piv);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.basis[p - 1] = qv;
            if (owner == 0) P.var[q] = leaving;
            if (it < P.log_cap) {
                P.qlog[it] = qv;
                P.plog[it] = p;
            }
        }
        clk.lap(1);
        if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(4);
        phase_update<double, persistent_rows(NT)>(P, p, q, it);
        ++it;
        degeneracy_step(P, ratio, bland, degen);
        clk.lap(2);
        if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(5);
    }
}

}  // namespace tsx
