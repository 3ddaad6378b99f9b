// Team solve: many LPs at once, each by a team of C thread blocks (the
// full-tableau simplex of arXiv 2211.10979, Section III, Steps 1-3), for LPs
// too large for one block's shared memory and too small to fill the GPU.
//
// One cooperative launch holds every team; a team takes the next LP from a
// list (largest first) and solves it on its condensed tableau in global
// memory.  Block b of the team owns a contiguous range of rows: it runs the
// ratio test on its rows (keeping their column-q entries, the multipliers, in
// shared memory), stages the whole scaled pivot row R in its own shared memory
// (each block divides row p by the pivot itself), and updates its rows.  Block
// 0 owns row 0 and finds the next entering column while it updates it.  Two
// team barriers per pivot: after the ratio test (every block learns p) and
// after the update (every block learns the next entering column, and every
// block has read row p, so its owner may now overwrite it with R).  The
// arithmetic and the tie rules are those of the single-LP kernels, so every
// pivot and value equals lp_solve's.
#pragma once

#include "tsx_device.cuh"

namespace tsx {

constexpr int kTeamMax = 160;  // blocks per team, upper bound
#ifndef TSX_TEAM_SM_THREADS
#define TSX_TEAM_SM_THREADS 512   // threads per SM the team kernel is compiled for
#endif
#ifndef TSX_TEAM_SLICE_LD
#define TSX_TEAM_SLICE_LD 1024   // FP64 rows this long or longer: row p scaled a slice per block
#endif
// Threads per SM of the team kernel with blocks of nt threads, and the rows a
// warp of its update keeps in flight (16 where a thread may hold 255 registers).
__host__ __device__ constexpr int team_sm_threads(int nt) { return nt > TSX_TEAM_SM_THREADS ? nt : TSX_TEAM_SM_THREADS; }
__host__ __device__ constexpr int team_rows_in_flight(int nt) { return team_sm_threads(nt) <= 256 ? 16 : kRowsInFlight; }

template <typename V>
struct TeamJob {
    const double* A;           // inputs (device), m x n row-major, m, n
    const double* b;
    const double* c;
    V* T;                      // condensed tableau (m+1) x ld
    int* basis;                // m
    int* var;                  // n
    DevState* st;              // the LP's state words: status, iters, bland, degen_run
    int m, n, ld;
    int pad;
};

struct __align__(256) TeamState {   // one per team
    unsigned bar_count;
    unsigned bar_gen;
    int job;
    int fail;                  // set when a team barrier wait ran out
    int bad;                   // the current LP's inputs are not finite or b < 0
    unsigned seq;              // continuous launch: sequence number of the job
    ArgPart ent;               // next entering candidate (block 0)
    RatPart rat[kTeamMax];     // ratio-test partial of each block
};

template <typename V>
struct TeamParams {
    const TeamJob<V>* jobs;
    const int* order[2];       // job indices of the two lists, largest first
    int count[2];              // their lengths
    unsigned* next;            // list position counters (2)
    TeamState* teams;
    const int* team_of;        // grid: the team of each block
    const int* first;          // teams: first block, size, own list (0 or 1)
    const int* size;
    const int* list;
    double eps_d, eps_p;
    long long max_iters;       // < 0: 50 (m + n)
    int k_cyc, rule;
    long long timeout_ns;
};

// Barrier of the C blocks of one team; bounded like grid_barrier.  Returns
// false (in every thread) if the wait ran out or another block of the team
// gave up.
// With TSX_BARRIER_COUNT the arrival counter only grows within a launch (the
// team states are zeroed before it): a block adds 1 (release, no returned
// value) and waits for (barriers passed + 1) x C, `passed` counting its own
// barriers; otherwise the last arrival resets the counter and bumps a
// generation word.
__device__ inline bool team_barrier(TeamState* ts, unsigned C, long long timeout_ns, int& sok, unsigned& passed) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        bool done = false;
        unsigned gen = 0, target = 0;
        if (TSX_BARRIER_COUNT) {
            target = (passed + 1u) * C;
            red_add_release(&ts->bar_count, 1u);
        } else {
            gen = ld_acquire(&ts->bar_gen);
            const unsigned arrived = atom_add_acq_rel(&ts->bar_count, 1u);
            if (arrived == C - 1) {
                ts->bar_count = 0;
                st_release(&ts->bar_gen, gen + 1);
                done = true;
            }
        }
        if (!done) {
            const long long t0 = global_ns();
            const unsigned long long max_spins = (unsigned long long)(timeout_ns > 0 ? timeout_ns : 0) + 4096ull;
            unsigned long long spins = 0;
            while (TSX_BARRIER_COUNT ? (int)(ld_acquire(&ts->bar_count) - target) < 0
                                     : ld_acquire(&ts->bar_gen) == gen) {
                ++spins;
                if ((spins & 31ull) == 1) {
                    if (ld_relaxed(&ts->fail) != 0) { ok = 0; break; }
                    if (global_ns() - t0 >= timeout_ns || spins > max_spins) {
                        atomicExch(&ts->fail, 1);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        passed += 1u;
        __threadfence();
        sok = ok;
    }
    __syncthreads();
    return sok != 0;
}

// Rows of block bt among C: [r0, r1) of 0..m.
__device__ __forceinline__ void team_rows(int m, int C, int bt, int& r0, int& r1) {
    const int per = (m + 1 + C - 1) / C;
    r0 = min(m + 1, bt * per);
    r1 = min(m + 1, r0 + per);
}

// Condensed Table I rows [r0, r1) (slack basis): row 0 = [-c | 0], row i =
// [A_i | b_i], padding zero; the LP's basis words of those rows; var[] by block
// 0.  Inputs that are not finite, or b_i < 0, mark the LP bad in the team state
// (the input check of lp_create, done while the data pass by).
template <typename V>
__device__ void team_build(const TeamJob<V>& J, int r0, int r1, int bt, TeamState* ts) {
    constexpr int E = Lanes<V>::E;
    const int n = J.n, ld = J.ld;
    const long long per_row = ld / E;
    const long long total = (long long)(r1 - r0) * per_row;
    int bad = 0;
    for (long long g = threadIdx.x; g < total; g += blockDim.x) {
        const int i = r0 + (int)(g / per_row);
        const int j0 = (int)(g - (long long)(i - r0) * per_row) * E;
        Sector<V> out;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = j0 + e;
            double v = 0.0;
            if (i == 0) {
                if (j < n) v = -J.c[j];
            } else if (j < n) {
                v = J.A[(size_t)(i - 1) * (size_t)n + j];
            } else if (j == n) {
                v = J.b[i - 1];
                bad |= !(v >= 0.0);
            }
            bad |= !isfinite(v);
            out.v[e] = (V)v;
        }
        st_sector(J.T + (size_t)i * (size_t)ld + j0, out);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ts->bad, 1);
    for (int i = max(r0, 1) + threadIdx.x; i < r1; i += blockDim.x) J.basis[i - 1] = n + i - 1;
    if (bt == 0)
        for (int j = threadIdx.x; j < n; j += blockDim.x) J.var[j] = j;
}

// Objective row (block 0): T[0][j] = fma(-f0, R[j], T[0][j]) (q: from the
// leaving variable's unit column, 0 off row p) when R != null, then the
// entering candidate of the new row over all slots, posted to the team.
template <typename V>
__device__ void team_row0(const TeamJob<V>& J, const V* R, V f0, int q, const TeamParams<V>& P, TeamState* ts,
                          BlockScratch& s) {
    constexpr int E = Lanes<V>::E;
    const int nsec = J.ld / E;
    ArgPart a = arg_none();
    for (int g = threadIdx.x; g < nsec; g += blockDim.x) {
        const int j = g * E;
        Sector<V> o = ld_sector_cg(J.T + j);
        if (R) {
            const Sector<V> r = *reinterpret_cast<const Sector<V>*>(R + j);
#pragma unroll
            for (int e = 0; e < E; ++e) o.v[e] = fma_rn(-f0, r.v[e], j + e == q ? V(0) : o.v[e]);
            st_sector(J.T + j, o);
        }
        arg_consider_sector(a, o, j, J.n, P.eps_d, J.var);
    }
    a = block_arg(a, s);
    if (threadIdx.x == 0) store_arg(&ts->ent, a);
}

// Rank-1 update of the block's rows [lo, r1) except p, R and the multipliers
// (Floc, indexed from r0) in shared memory; slots of RF rows x 32 column
// groups, one group per lane.
template <typename V, int RF>
__device__ void team_update(const TeamJob<V>& J, const V* R, const V* Floc, int r0, int lo, int r1, int p, int q) {
    constexpr int E = Lanes<V>::E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nsec = J.ld / E;
    const int nchunks = (nsec + 31) / 32;
    const int nrg = (r1 - lo + RF - 1) / RF;
    const long long total = (long long)nrg * nchunks;
    for (long long u = warp; u < total; u += nw) {
        const int rg = (int)(u / nchunks), ch = (int)(u - (long long)rg * nchunks);
        const int i0 = lo + rg * RF;
        const int nrows = min(RF, r1 - i0);
        const int gidx = ch * 32 + lane;
        if (gidx >= nsec) continue;
        const size_t col = (size_t)E * (size_t)gidx;
        const Sector<V> r = *reinterpret_cast<const Sector<V>*>(R + col);
        const int eq = q - (int)col;
        Sector<V> v[RF];
#pragma unroll
        for (int k = 0; k < RF; ++k) {
            const int i = i0 + k;
            if (k < nrows && i != p) v[k] = ld_sector_stream(J.T + (size_t)i * (size_t)J.ld + col);
        }
#pragma unroll
        for (int k = 0; k < RF; ++k) {
            const int i = i0 + k;
            if (k < nrows && i != p) {
                const V f = Floc[i - r0];
#pragma unroll
                for (int e2 = 0; e2 < E; ++e2) v[k].v[e2] = fma_rn(-f, r.v[e2], e2 == eq ? V(0) : v[k].v[e2]);
                st_sector(J.T + (size_t)i * (size_t)J.ld + col, v[k]);
            }
        }
    }
}

// Solves one LP with the team of C blocks; false if a team barrier failed.
template <int RF, typename V>
__device__ bool team_solve_one(const TeamParams<V>& P, const TeamJob<V>& J, TeamState* ts, int bt, unsigned C,
                               V* R, V* Floc, BlockScratch& s, int& sok, unsigned& tpass) {
    const int m = J.m, n = J.n, ld = J.ld;
    int r0, r1;
    team_rows(m, (int)C, bt, r0, r1);
    team_build(J, r0, r1, bt, ts);
    __syncthreads();
    if (bt == 0) team_row0(J, (const V*)nullptr, V(0), -1, P, ts, s);   // Step 1 of the first pivot
    if (!team_barrier(ts, C, P.timeout_ns, sok, tpass)) return false;
    const long long cap = P.max_iters < 0 ? 50LL * ((long long)m + n) : P.max_iters;
    long long it = 0;
    int bland = P.rule == 1, degen = 0;
    int status = ld_relaxed(&ts->bad) ? kInvalid : kRunning;
    const int lo = max(r0, 1);
    const int i_first = lo + (int)threadIdx.x;   // the thread's first row in Step 2
    while (status == kRunning) {
        // its right-hand side, in flight while Step 1's candidate is read
        const V rhs0 = i_first < r1 ? __ldcg(J.T + (size_t)i_first * (size_t)ld + n) : V(0);
        const ArgPart e = load_arg(&ts->ent);                // Step 1
        const int q = bland ? e.fslot : e.slot;
        const int qv = bland ? e.fkey : e.key;
        if (qv == INT_MAX) { status = kOptimal; break; }
        if (it >= cap) { status = kIterLimit; break; }
        // Step 2 on the block's rows; their column-q entries become the multipliers
        RatPart best = rat_none();
        if (bt == 0 && threadIdx.x == 0) Floc[0] = __ldcg(J.T + q);
        for (int i = i_first; i < r1; i += blockDim.x) {
            const V* row = J.T + (size_t)i * (size_t)ld;
            const V a = __ldcg(row + q);
            Floc[i - r0] = a;
            if ((double)a > P.eps_p) {
                RatPart c;
                c.r = (double)div_rn(i == i_first ? rhs0 : __ldcg(row + n), a);
                c.i = i;
                c.key = bland ? __ldcg(J.basis + (i - 1)) : i;
                c.a = (double)a;
                c.pad = 0.0;
                if (!dbits_nan(c.r)) rat_merge(best, c);
            }
        }
        best = block_rat(best, s);
        if (threadIdx.x == 0) store_rat(&ts->rat[bt], best);
        if (!team_barrier(ts, C, P.timeout_ns, sok, tpass)) return false;
        RatPart l = rat_none();
        if (threadIdx.x < (int)C) l = load_rat(&ts->rat[threadIdx.x]);
        l = block_rat(l, s);
        if (l.i == INT_MAX) { status = kUnbounded; break; }
        const int p = l.i;
        const V piv = (V)l.a;
        if (!isfinite((double)piv) || !isfinite(l.r)) { status = kNumeric; break; }
        // Step 3, pivot row; the leaving variable takes slot q.  FP64 rows of
        // TSX_TEAM_SLICE_LD entries or more: each block scales its slice of
        // row p in place (the new row p), a team barrier, then every block
        // reads the whole row (GB300's FP64 pipe charges ~9 fused
        // multiply-adds per division, ld of them a block otherwise).  Shorter
        // or FP32 rows: every block scales the whole row itself.
        V* rowp = J.T + (size_t)p * (size_t)ld;
        const bool slice = sizeof(V) == 8 && ld >= TSX_TEAM_SLICE_LD;
        if (slice) {
            const int sl = (ld + (int)C - 1) / (int)C;
            const int j0 = min(ld, bt * sl), j1 = min(ld, j0 + sl);
            for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x)
                rowp[j] = div_rn(j == q ? V(1) : __ldcg(rowp + j), piv);
        } else {
            for (int j = threadIdx.x; j < ld; j += blockDim.x) R[j] = div_rn(j == q ? V(1) : __ldcg(rowp + j), piv);
        }
        if (bt == 0 && threadIdx.x == 0) {
            const int leaving = J.basis[p - 1];
            J.basis[p - 1] = qv;
            J.var[q] = leaving;
        }
        if (P.rule == 0) {
            if (l.r <= 0.0) {
                ++degen;
                if (P.k_cyc > 0 && degen >= P.k_cyc) bland = 1;
            } else {
                degen = 0;
                bland = 0;
            }
        }
        if (slice) {
            if (!team_barrier(ts, C, P.timeout_ns, sok, tpass)) return false;
            for (int j = threadIdx.x; j < ld; j += blockDim.x) R[j] = __ldcg(rowp + j);
        }
        __syncthreads();
        if (bt == 0) team_row0(J, R, Floc[0], q, P, ts, s);   // the next Step 1 on the new row 0
        team_update<V, RF>(J, R, Floc, r0, lo, r1, p, q);
        ++it;
        if (!team_barrier(ts, C, P.timeout_ns, sok, tpass)) return false;
        if (!slice && p >= r0 && p < r1) {   // every block has read row p: its owner stores R there
            for (int j = threadIdx.x; j < ld; j += blockDim.x) J.T[(size_t)p * (size_t)ld + j] = R[j];
            __syncthreads();
        }
    }
    // commit: the status is written only once every block of the team has
    // finished its part (a block that gave up at a barrier never gets here,
    // and the LP stays unfinished)
    if (!team_barrier(ts, C, P.timeout_ns, sok, tpass)) return false;
    if (bt == 0 && threadIdx.x == 0) {
        J.st->status = status;
        J.st->iters = it;
        J.st->bland = bland;
        J.st->degen_run = degen;
    }
    return true;
}

// One cooperative launch: team t (blocks first[t] .. first[t] + size[t] - 1)
// takes entries of its own list, then of the other one, until both are empty.
// Dynamic shared memory per block: R (ld_max entries) then the multipliers
// (rows per block, max over the lists for the smallest team).
template <int NT, typename V>
__global__ void __launch_bounds__(NT, team_sm_threads(NT) / NT) k_team_solve(TeamParams<V> P, int ld_max) {
    extern __shared__ __align__(32) unsigned char team_smem[];
    __shared__ BlockScratch s;
    __shared__ int sok;
    __shared__ unsigned tpass;   // counted team barriers passed (thread 0)
    if (threadIdx.x == 0) tpass = 0;
    const int t = P.team_of[blockIdx.x];
    const int bt = blockIdx.x - P.first[t];
    const unsigned C = (unsigned)P.size[t];
    TeamState* ts = P.teams + t;
    V* R = reinterpret_cast<V*>(team_smem);
    V* Floc = R + ld_max;
    int li = P.list[t];
    for (;;) {
        if (bt == 0 && threadIdx.x == 0) {
            ts->bad = 0;   // read after the next barrier; set during the build
            int k = -1;
            for (int pass = 0; pass < 2 && k < 0; ++pass) {
                const int l = pass == 0 ? li : 1 - li;
                const int pos = (int)atomicAdd(P.next + l, 1u);
                if (pos < P.count[l]) k = P.order[l][pos];
            }
            ts->job = k;
        }
        if (!team_barrier(ts, C, P.timeout_ns, sok, tpass)) return;
        const int k = *(volatile const int*)&ts->job;
        if (k < 0) return;
        const TeamJob<V> J = P.jobs[k];
        if (!team_solve_one<team_rows_in_flight(NT)>(P, J, ts, bt, C, R, Floc, s, sok, tpass)) return;
    }
}

// ---------------------------------------------------------------------------
// Continuous team launch (the request server's lane for large LPs): the same
// teams and the same team_solve_one, but the jobs come from rings that the
// host appends to while the launch runs, so an LP admitted at any moment is
// taken by the next team that finishes one, and each LP reports its end on
// its own instead of at the end of a launch.
//   - rings in mapped host memory, one per list (light / heavy LPs): the host
//     writes a job entry, then publishes it by a release store of the list's
//     tail; a team's leader claims the next entry with a compare-and-swap on
//     the list's head (device memory) after an acquire load of the tail, and
//     copies the entry into device memory for the team;
//   - when an LP is solved (after the team's commit barrier) the leader
//     stores the job's sequence number + 1 into its done word (release,
//     system scope), which the host polls;
//   - a team that finds nothing to claim keeps polling while another team
//     still works (a job published meanwhile is taken at once); once no team
//     has had work for idle_ns (or the stop word is set) every team exits, and
//     the host starts a new launch when jobs are waiting and none runs.  Every
//     wait is bounded: the claim loop by idle_cap_ns and a spin cap, the team
//     barriers as in k_team_solve (a team that gives up clears its busy mark).
// ---------------------------------------------------------------------------
template <typename V>
struct ServeRing {
    TeamJob<V>* jobs;          // host memory: 2 lists x cap entries
    unsigned* tail;            // host memory: jobs published per list [2]
    unsigned* done;            // host memory: per entry, its sequence number + 1 once solved
    unsigned* stop;            // host memory: nonzero: teams with nothing to claim exit now
};

template <typename V>
struct TeamServeParams {
    TeamParams<V> tp;          // tolerances, rules and team tables (jobs, order, count, next unused)
    ServeRing<V> ring;
    unsigned cap;              // entries per list, a power of two
    unsigned* head;            // device memory: jobs claimed per list [2]
    unsigned* busy;            // device memory: teams solving a job (zero at launch)
    TeamJob<V>* jcopy;         // device memory: per team, the job it solves
    long long idle_ns;         // every team leaves once none has had work for this long
    long long idle_cap_ns;     // bound on a team's wait while others still work
};

__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned* p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int NT, typename V>
__global__ void __launch_bounds__(NT, team_sm_threads(NT) / NT) k_team_serve(TeamServeParams<V> P, int ld_max) {
    extern __shared__ __align__(32) unsigned char team_smem[];
    __shared__ BlockScratch s;
    __shared__ int sok;
    __shared__ unsigned tpass;
    if (threadIdx.x == 0) tpass = 0;
    const int t = P.tp.team_of[blockIdx.x];
    const int bt = blockIdx.x - P.tp.first[t];
    const unsigned C = (unsigned)P.tp.size[t];
    TeamState* ts = P.tp.teams + t;
    V* R = reinterpret_cast<V*>(team_smem);
    V* Floc = R + ld_max;
    const int li = P.tp.list[t];
    TeamJob<V>* jc = P.jcopy + t;
    for (;;) {
        if (bt == 0 && threadIdx.x == 0) {
            ts->bad = 0;   // read after the next barrier; set during the build
            int got = -1;
            unsigned gseq = 0;
            const long long t0 = global_ns();
            const unsigned long long max_spins =
                (unsigned long long)(P.idle_cap_ns > 0 ? P.idle_cap_ns : 0) / 500ull + 64ull;
            long long t_idle = t0;   // since when no team has been seen working
            for (unsigned long long spins = 0;; ++spins) {
                for (int pass = 0; pass < 2 && got < 0; ++pass) {
                    const int l = pass == 0 ? li : 1 - li;
                    const unsigned tl = ld_acquire_sys(P.ring.tail + l);
                    unsigned h = *(volatile unsigned*)(P.head + l);
                    while ((int)(tl - h) > 0) {
                        const unsigned prev = atomicCAS(P.head + l, h, h + 1u);
                        if (prev == h) {
                            got = l;
                            gseq = h;
                            break;
                        }
                        h = prev;
                    }
                }
                if (got >= 0) {
                    atomicAdd(P.busy, 1u);
                    break;
                }
                const long long now = global_ns();
                if (*(volatile unsigned*)P.busy != 0u) t_idle = now;
                if (ld_acquire_sys(P.ring.stop) != 0u || now - t_idle >= P.idle_ns || now - t0 >= P.idle_cap_ns ||
                    spins >= max_spins)
                    break;
                __nanosleep(500);
            }
            if (got >= 0) {
                const unsigned slot = (unsigned)got * P.cap + (gseq & (P.cap - 1u));
                const volatile unsigned long long* src =
                    reinterpret_cast<const volatile unsigned long long*>(P.ring.jobs + slot);
                unsigned long long* dst = reinterpret_cast<unsigned long long*>(jc);
                for (int w = 0; w < (int)(sizeof(TeamJob<V>) / 8); ++w) dst[w] = src[w];
                ts->job = (int)slot;
                ts->seq = gseq;
            } else {
                ts->job = -1;
            }
        }
        if (!team_barrier(ts, C, P.tp.timeout_ns, sok, tpass)) return;
        const int slot = *(volatile const int*)&ts->job;
        if (slot < 0) return;
        TeamJob<V> J;
        {
            const unsigned long long* src = reinterpret_cast<const unsigned long long*>(jc);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(&J);
            for (int w = 0; w < (int)(sizeof(TeamJob<V>) / 8); ++w) dst[w] = __ldcg(src + w);
        }
        if (bt == 0 && threadIdx.x == 0) {
            // the LP's state words start from zero here (no reset launch per job)
            DevState* st = J.st;
            st->status = kRunning;
            st->q = -1;
            st->p = -1;
            st->bland = 0;
            st->degen_run = 0;
            st->bad = 0;
            st->iters = 0;
            st->active_sectors = 0;
            st->theta = 0.0;
            st->bar_count = 0;
            st->bar_gen = 0;
            st->nact = 0;
            st->next_slot = 0;
            for (int q = 2; q < 6; ++q) st->phase_ns[q] = 0;
            st->phase_ns[1] = 0;
            st->phase_ns[0] = global_ns();
        }
        if (!team_solve_one<team_rows_in_flight(NT)>(P.tp, J, ts, bt, C, R, Floc, s, sok, tpass)) {
            if (bt == 0 && threadIdx.x == 0) atomicSub(P.busy, 1u);
            return;
        }
        if (bt == 0 && threadIdx.x == 0) {
            J.st->phase_ns[1] = global_ns();
            __threadfence_system();
            st_release_sys(P.ring.done + slot, *(volatile unsigned*)&ts->seq + 1u);
            atomicSub(P.busy, 1u);
        }
    }
}

}  // namespace tsx
