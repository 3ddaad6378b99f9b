// Device side of the dense full-tableau simplex pivot (arXiv 2211.10979,
// Section III Steps 1-3; Section IV Steps 1-4 for one GPU).
//
// One pivot is four phases over the row-major tableau T ((m+1) x ld entries of
// type V = double or float; the last logical column W-1 is the right-hand
// side).  The full layout holds Table I itself (W = n + m + 1 columns); the
// condensed layout holds the n nonbasic columns and the right-hand side
// (W = n + 1) with var[j] = the variable of column slot j -- the basic columns
// are exact unit vectors, and the leaving variable takes the entering slot:
//   P1  entering column q: reduce the per-strip (value, variable, slot)
//       partials of the objective row left by the previous P4 (Section III
//       Step 1, Dantzig's most negative coefficient, lowest variable on ties;
//       Section IV Step 1's local-then-global reduction, here warp -> strip ->
//       block).
//   P2  minimum-ratio test on column q (Section III Step 2, Section IV Step 2):
//       every block scans a share of the rows, copies column q into F and keeps
//       its best (ratio, key, row, pivot element) -> one partial per block.
//   P3  leaving row p = reduce of the P2 partials; pivot-row staging
//       R[j] = T[p][j] / T[p][q] (Section III Step 3's pivot row; condensed:
//       R[q] = 1 / T[p][q], the leaving variable's new column) and, in the
//       full layout, the list of 32-byte column groups of row p holding a
//       nonzero entry.
//   P4  rank-1 update T[i][j] = fma(-F[i], R[j], T[i][j]) for i != p (condensed:
//       slot q starts from 0) and T[p][j] = R[j] (Section III Step 3, Section
//       IV Step 4), streamed with 256-bit accesses; the objective row is
//       updated first, one warp per strip, each emitting that strip's argmin
//       partial of the new objective row (the next P1's input).
// Between phases every block of the grid passes a device-wide barrier whose
// wait is bounded in time (the paper's per-iteration synchronisation,
// Section IV Iterate/Finalization).
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

namespace tsx {

constexpr int kRunning = 100;      // status while the iteration is in progress
#ifndef TSX_ROWS_IN_FLIGHT
#define TSX_ROWS_IN_FLIGHT 0   // rows in flight of the persistent update; 0: by registers per thread
#endif
#ifndef TSX_GRAB
#define TSX_GRAB 0     // work slots per grab of the update; 0: 1 for double, 2 for float
#endif
#ifndef TSX_SM_THREADS
#define TSX_SM_THREADS 256   // threads per SM the persistent kernel is compiled for
#endif
#ifndef TSX_TMA
#define TSX_TMA 0          // 1: condensed persistent update through bulk copies into shared memory
#endif
#ifndef TSX_TMA_ROWS
#define TSX_TMA_ROWS 4
#endif
#ifndef TSX_TMA_STAGES
#define TSX_TMA_STAGES 3
#endif
#ifndef TSX_TMA_BATCH
#define TSX_TMA_BATCH 4    // rows of a stage read from shared memory before their FMAs
#endif
#ifndef TSX_ALTERNATE
#define TSX_ALTERNATE 1   // alternate the update's sweep direction per pivot
#endif
#ifndef TSX_SLOT_PIPE
#define TSX_SLOT_PIPE 1      // the update's next grab read after the current slot, not before it
#endif
#ifndef TSX_STATIC_FIRST
#define TSX_STATIC_FIRST 1   // each warp's first update slot given by its index, not the counter
#endif
#ifndef TSX_RHS_PREFETCH
#define TSX_RHS_PREFETCH 1   // persistent kernel: P2's first right-hand side loaded before P1
#endif
constexpr int kRowsInFlight = 8;   // rows a warp loads before its first store (128 registers a thread)

// Threads per SM of the persistent kernel with blocks of nt threads, and the
// rows a warp of its update keeps in flight: 16 where a thread may hold 255
// registers (at most 256 threads per SM), else 8.  A warp's bytes in flight
// set the update's bandwidth once the tableau outgrows L2.
__host__ __device__ constexpr int persistent_sm_threads(int nt) { return nt > TSX_SM_THREADS ? nt : TSX_SM_THREADS; }
__host__ __device__ constexpr int persistent_rows(int nt) {
    return TSX_ROWS_IN_FLIGHT > 0 ? TSX_ROWS_IN_FLIGHT : persistent_sm_threads(nt) <= 256 ? 16 : kRowsInFlight;
}
constexpr int kMaxWarps = 32;      // warps per block upper bound (1024 threads)

// status codes (same values as lp_status in tabsimplex.h)
constexpr int kOptimal = 0, kUnbounded = 1, kIterLimit = 2, kNumeric = 3, kInvalid = -1, kTimeout = -4;

struct __align__(16) ArgPart {   // best entering candidate of a column range
    double v;         // most negative objective-row entry (< -eps_d), +inf if none
    int key;          // its variable (lowest on ties), INT_MAX if none
    int slot;         // its column in the stored tableau
    int fkey;         // lowest variable with entry < -eps_d (Bland), INT_MAX if none
    int fslot;        // its column
    int pad[2];
};

struct __align__(16) RatPart {   // best leaving candidate of a row range
    double r;         // minimum ratio rhs_i / T[i][q], +inf if none
    int key;          // tie-break key: row index (Dantzig) or basic variable (Bland)
    int i;            // its row (1..m), INT_MAX if none
    double a;         // its pivot element T[i][q] (exact in double for both tableau types)
    double pad;
};

struct DevState {
    int status;                        // kRunning or the final lp_status
    int q;                             // entering column (one-launch-per-phase path)
    int p;                             // leaving row
    int bland;                         // 1 while Bland's rule is in force
    int degen_run;                     // consecutive pivots with minimum ratio <= 0
    int bad;                           // input validation flag (create)
    long long iters;                   // pivots completed
    unsigned long long active_sectors; // sum over pivots of updated 32-B column groups
    double theta;                      // minimum ratio of the current pivot
    unsigned bar_count;                // grid barrier: blocks arrived
    unsigned bar_gen;                  // grid barrier: generation
    int qvar;                          // entering variable (one-launch-per-phase path)
    unsigned nact;                     // active 32-B column groups of this pivot
    unsigned next_slot;                // P4 work counter (slots handed out)
    long long phase_ns[6];             // block 0's time per phase: work of
                                       // {select+ratio, stage, update}, then the
                                       // barrier wait after each of them
};

// Entries of type V per 32-byte sector (one lane's share of a warp access).
template <typename V> struct Lanes;
template <> struct Lanes<double> { static constexpr int E = 4; };
template <> struct Lanes<float> { static constexpr int E = 8; };

template <typename V>
struct Params {
    V* T;                // tableau, (m+1) x ld
    int ld, m, n, W;
    int* basis;          // m: variable basic in row i+1
    V* F;                // m+1: column q of the tableau before the update
    V* R;                // ld: scaled pivot row
    int* act;            // ld/E: indices of the 32-B column groups Step 3 updates
    ArgPart* cpart;      // nstrips: objective-row argmin partial per strip
    RatPart* rpart;      // grid blocks: ratio-test partial per block
    DevState* st;
    int* qlog;           // log_cap entries (may be null)
    int* plog;
    long long log_cap;
    double eps_d, eps_p;
    long long max_iters;
    int k_cyc, rule;
    long long timeout_ns;
    int nstrips;         // ceil(ld / (32 E)): warp strips of the objective row
    int skip_zero;       // leave column groups whose R entries are all zero
    int cond;            // 1: condensed tableau (nonbasic columns + RHS), 0: full
    int* var;            // condensed: n, the variable held by each column slot
};

// ------------------------------------------------------------------ helpers
// One 32-byte sector of the tableau: E consecutive entries.
template <typename V>
struct __align__(32) Sector {
    V v[Lanes<V>::E];
};

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// 256-bit accesses of one 32-byte sector; addresses 32-byte aligned.
// "stream": the bulk update's loads (no L1 allocation); "cg": L2 loads of data
// another block wrote before the last barrier.
__device__ __forceinline__ Sector<double> ld_sector_stream(const double* p) {
    Sector<double> s;
    asm volatile("ld.global.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(s.v[0]), "=d"(s.v[1]), "=d"(s.v[2]), "=d"(s.v[3]) : "l"(p));
    return s;
}
__device__ __forceinline__ Sector<double> ld_sector_cg(const double* p) {
    Sector<double> s;
    asm volatile("ld.global.cg.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(s.v[0]), "=d"(s.v[1]), "=d"(s.v[2]), "=d"(s.v[3]) : "l"(p));
    return s;
}
__device__ __forceinline__ void st_sector(double* p, const Sector<double>& s) {
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};"
                 ::"l"(p), "d"(s.v[0]), "d"(s.v[1]), "d"(s.v[2]), "d"(s.v[3]) : "memory");
}
__device__ __forceinline__ Sector<float> ld_sector_stream(const float* p) {
    Sector<float> s;
    asm volatile("ld.global.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(s.v[0]), "=f"(s.v[1]), "=f"(s.v[2]), "=f"(s.v[3]),
                   "=f"(s.v[4]), "=f"(s.v[5]), "=f"(s.v[6]), "=f"(s.v[7]) : "l"(p));
    return s;
}
__device__ __forceinline__ Sector<float> ld_sector_cg(const float* p) {
    Sector<float> s;
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(s.v[0]), "=f"(s.v[1]), "=f"(s.v[2]), "=f"(s.v[3]),
                   "=f"(s.v[4]), "=f"(s.v[5]), "=f"(s.v[6]), "=f"(s.v[7]) : "l"(p));
    return s;
}
__device__ __forceinline__ void st_sector(float* p, const Sector<float>& s) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"l"(p), "f"(s.v[0]), "f"(s.v[1]), "f"(s.v[2]), "f"(s.v[3]),
                   "f"(s.v[4]), "f"(s.v[5]), "f"(s.v[6]), "f"(s.v[7]) : "memory");
}

// One rounding per operation, in the tableau's own precision.
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }

template <typename V>
__device__ __forceinline__ bool sector_nonzero(const Sector<V>& s) {
    bool nz = false;
#pragma unroll
    for (int e = 0; e < Lanes<V>::E; ++e) nz |= s.v[e] != V(0);
    return nz;
}

// The reductions of Steps 1-2 compare 64-bit integer keys with the order of
// the doubles they stand for: on GB300 every FP64 comparison occupies the
// SM's FP64 pipe (16 cycles a warp instruction), the pipe that also runs the
// update's DFMAs, while integer compares run on the ALU pipes.  For doubles
// that are not NaN, x < y iff dkey(x) < dkey(y), and x == y iff
// dkey(x) == dkey(y) (-0 and +0 share the key of +0), so every decision and
// tie is the one the floating-point comparisons take.  NaN values never win
// a floating-point `<` or `==` comparison; the kernel keeps them out of the
// candidates instead.  The map is its own inverse up to the sign of zero.
__device__ __forceinline__ long long dkey(double x) {
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ULL) b = 0;
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dkey_value(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ bool dbits_nan(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool dbits_finite(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
constexpr long long kKeyInf = 0x7ff0000000000000LL;   // dkey(+inf)

__device__ __forceinline__ ArgPart arg_none() {
    return ArgPart{__longlong_as_double(0x7ff0000000000000LL), INT_MAX, INT_MAX, INT_MAX, INT_MAX, {0, 0}};
}
__device__ __forceinline__ RatPart rat_none() { return RatPart{__longlong_as_double(0x7ff0000000000000LL), INT_MAX, INT_MAX, 0.0, 0.0}; }

// (v, key) lexicographic minimum: the most negative entry, lowest variable on
// ties; and the lowest candidate variable (Bland).  The key of a column is its
// variable: the column index itself in the full tableau, var[] in the
// condensed one.
// Merges of Step 1-2 partials (shuffle trees, block and grid reductions)
// compare keys: measured 5888 vs 5817 pivots/s at 8192^2 (the ratio and
// staging phases 2 us shorter per pivot).  Keys in the per-entry candidate
// scans as well cost more ALU work in the objective-row pass than the FP64
// comparisons they replace (5709).
#ifndef TSX_KEYS
#define TSX_KEYS 1   // 0: FP64 comparisons; 1: merges of partials on keys; 2: the candidate scans too
#endif
// Values of partials are +inf (none) or candidates (never NaN).
__device__ __forceinline__ void arg_merge(ArgPart& a, const ArgPart& b) {
#if TSX_KEYS >= 1
    const long long bk = dkey(b.v), ak = dkey(a.v);
    if (bk < ak || (bk == ak && b.key < a.key)) { a.v = b.v; a.key = b.key; a.slot = b.slot; }
#else
    if (b.v < a.v || (b.v == a.v && b.key < a.key)) { a.v = b.v; a.key = b.key; a.slot = b.slot; }
#endif
    if (b.fkey < a.fkey) { a.fkey = b.fkey; a.fslot = b.fslot; }
}

__device__ __forceinline__ void arg_consider(ArgPart& a, double v, int j, int key, int jend, double eps_d) {
#if TSX_KEYS >= 2
    const long long vk = dkey(v);
    if (j < jend && !dbits_nan(v) && vk < dkey(-eps_d)) {
        const long long ak = dkey(a.v);
        if (vk < ak || (vk == ak && key < a.key)) { a.v = v; a.key = key; a.slot = j; }
        if (key < a.fkey) { a.fkey = key; a.fslot = j; }
    }
#else
    if (j < jend && v < -eps_d) {
        if (v < a.v || (v == a.v && key < a.key)) { a.v = v; a.key = key; a.slot = j; }
        if (key < a.fkey) { a.fkey = key; a.fslot = j; }
    }
#endif
}

// Columns j .. j+E-1 of the objective row; var == null: full tableau (key = j).
template <typename V>
__device__ __forceinline__ void arg_consider_sector(ArgPart& a, const Sector<V>& s, int j, int jend, double eps_d,
                                                    const int* var) {
#pragma unroll
    for (int e = 0; e < Lanes<V>::E; ++e) {
        const int jj = j + e;
        const int key = (var && jj < jend) ? __ldcg(var + jj) : jj;
        arg_consider(a, (double)s.v[e], jj, key, jend, eps_d);
    }
}

// (r, key) lexicographic minimum: smallest ratio, lowest key on ties.
// Ratios are +inf (none) or candidates; a NaN ratio is never made a
// candidate (it would lose every comparison).
__device__ __forceinline__ void rat_merge(RatPart& a, const RatPart& b) {
#if TSX_KEYS >= 1
    const long long bk = dkey(b.r), ak = dkey(a.r);
    if (bk < ak || (bk == ak && b.key < a.key)) a = b;
#else
    if (b.r < a.r || (b.r == a.r && b.key < a.key)) a = b;
#endif
}

__device__ __forceinline__ ArgPart warp_arg(ArgPart a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ArgPart b;
        b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
        b.key = __shfl_xor_sync(0xffffffffu, a.key, o);
        b.slot = __shfl_xor_sync(0xffffffffu, a.slot, o);
        b.fkey = __shfl_xor_sync(0xffffffffu, a.fkey, o);
        b.fslot = __shfl_xor_sync(0xffffffffu, a.fslot, o);
        arg_merge(a, b);
    }
    return a;
}

__device__ __forceinline__ RatPart warp_rat(RatPart a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        RatPart b;
        b.r = __shfl_xor_sync(0xffffffffu, a.r, o);
        b.key = __shfl_xor_sync(0xffffffffu, a.key, o);
        b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
        b.a = __shfl_xor_sync(0xffffffffu, a.a, o);
        rat_merge(a, b);
    }
    return a;
}

// Partials are read by other blocks after a barrier: 128-bit L2 accesses.
__device__ __forceinline__ void store_arg(ArgPart* dst, const ArgPart& a) {
    long long bits = __double_as_longlong(a.v);
    __stcg(reinterpret_cast<int4*>(dst), make_int4((int)(bits & 0xffffffff), (int)(bits >> 32), a.key, a.slot));
    __stcg(reinterpret_cast<int4*>(dst) + 1, make_int4(a.fkey, a.fslot, 0, 0));
}
__device__ __forceinline__ ArgPart load_arg(const ArgPart* src) {
    int4 w = __ldcg(reinterpret_cast<const int4*>(src));
    int4 u = __ldcg(reinterpret_cast<const int4*>(src) + 1);
    long long bits = ((long long)(unsigned)w.y << 32) | (unsigned)w.x;
    return ArgPart{__longlong_as_double(bits), w.z, w.w, u.x, u.y, {0, 0}};
}
__device__ __forceinline__ void store_rat(RatPart* dst, const RatPart& a) {
    long long bits = __double_as_longlong(a.r);
    __stcg(reinterpret_cast<int4*>(dst), make_int4((int)(bits & 0xffffffff), (int)(bits >> 32), a.key, a.i));
    __stcg(reinterpret_cast<double2*>(dst) + 1, make_double2(a.a, 0.0));
}
__device__ __forceinline__ RatPart load_rat(const RatPart* src) {
    int4 w = __ldcg(reinterpret_cast<const int4*>(src));
    double2 x = __ldcg(reinterpret_cast<const double2*>(src) + 1);
    long long bits = ((long long)(unsigned)w.y << 32) | (unsigned)w.x;
    return RatPart{__longlong_as_double(bits), w.z, w.w, x.x, 0.0};
}

struct BlockScratch {
    ArgPart arg[kMaxWarps];
    RatPart rat[kMaxWarps];
    ArgPart arg_out;
    RatPart rat_out;
    int ok;
    unsigned passed;   // counted grid barriers this block has passed (thread 0)
};

// Block-wide reductions; every thread returns the block result.
__device__ inline ArgPart block_arg(ArgPart a, BlockScratch& s) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_arg(a);
    __syncthreads();
    if (lane == 0) s.arg[w] = a;
    __syncthreads();
    if (w == 0) {
        ArgPart b = lane < nw ? s.arg[lane] : arg_none();
        b = warp_arg(b);
        if (lane == 0) s.arg_out = b;
    }
    __syncthreads();
    return s.arg_out;
}

__device__ inline RatPart block_rat(RatPart a, BlockScratch& s) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_rat(a);
    __syncthreads();
    if (lane == 0) s.rat[w] = a;
    __syncthreads();
    if (w == 0) {
        RatPart b = lane < nw ? s.rat[lane] : rat_none();
        b = warp_rat(b);
        if (lane == 0) s.rat_out = b;
    }
    __syncthreads();
    return s.rat_out;
}

// ------------------------------------------------------------- grid barrier
// All blocks of the (co-resident) grid meet here.  Thread 0 of each block
// arrives on a counter; the last arrival resets it and bumps the generation
// word with release semantics; the others spin on the generation with acquire
// loads.  Each wait is bounded: after timeout_ns (globaltimer) or a spin-count
// limit, the block marks the solve LP_ERR_TIMEOUT and returns false; a block
// that sees a negative status while waiting returns false as well, so every
// block of a failed solve exits without waiting for the others.
__device__ inline bool grid_barrier(DevState* st, long long timeout_ns, BlockScratch& s) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned nblocks = gridDim.x;
        const unsigned gen = ld_acquire(&st->bar_gen);
        const unsigned arrived = atom_add_acq_rel(&st->bar_count, 1u);
        if (arrived == nblocks - 1) {
            st->bar_count = 0;
            st_release(&st->bar_gen, gen + 1);
        } else {
            const long long t0 = global_ns();
            // spin-count bound on top of the clock bound: >= 1 ns per spin
            const unsigned long long max_spins = (unsigned long long)(timeout_ns > 0 ? timeout_ns : 0) + 4096ull;
            unsigned long long spins = 0;
            while (ld_acquire(&st->bar_gen) == gen) {
                ++spins;
                if ((spins & 31ull) == 1) {   // first spin, then every 32
                    if (ld_relaxed(&st->status) < 0) { ok = 0; break; }
                    if (global_ns() - t0 >= timeout_ns || spins > max_spins) {
                        atomicCAS(&st->status, kRunning, kTimeout);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        s.ok = ok;
    }
    __syncthreads();
    return s.ok != 0;
}

#ifndef TSX_BARRIER_COUNT
#define TSX_BARRIER_COUNT 1   // counted barriers in the pivot and team kernels
#endif

// Counted grid barrier (the pivot kernel): the arrival counter only grows
// within a launch (it starts at 0: the state block is reset before every
// launch); thread 0 of each block adds 1 with release semantics and no
// returned value, then waits until the counter reaches (barriers passed + 1)
// x G.  One L2 round trip less than the generation barrier above (no read
// of the generation, no returning atomic before the release).  The 32-bit
// counter may wrap: blocks are at most one barrier apart, so the signed
// difference decides.  Bounded and failing exactly like grid_barrier.
__device__ inline bool grid_barrier_counted(DevState* st, long long timeout_ns, BlockScratch& s) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (s.passed + 1u) * gridDim.x;
        red_add_release(&st->bar_count, 1u);
        const long long t0 = global_ns();
        const unsigned long long max_spins = (unsigned long long)(timeout_ns > 0 ? timeout_ns : 0) + 4096ull;
        unsigned long long spins = 0;
        while ((int)(ld_acquire(&st->bar_count) - target) < 0) {
            ++spins;
            if ((spins & 31ull) == 1) {
                if (ld_relaxed(&st->status) < 0) { ok = 0; break; }
                if (global_ns() - t0 >= timeout_ns || spins > max_spins) {
                    atomicCAS(&st->status, kRunning, kTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        s.passed += 1u;
        __threadfence();
        s.ok = ok;
    }
    __syncthreads();
    return s.ok != 0;
}

__device__ __forceinline__ bool pivot_barrier(DevState* st, long long timeout_ns, BlockScratch& s) {
    return TSX_BARRIER_COUNT ? grid_barrier_counted(st, timeout_ns, s) : grid_barrier(st, timeout_ns, s);
}

// ------------------------------------------------------------------ phases
// Initial objective-row argmin (before the first pivot): one warp per strip.
template <typename V>
__device__ void phase_init_argmin(const Params<V>& P) {
    constexpr int E = Lanes<V>::E;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long s = gw; s < P.nstrips; s += nw) {
        const int j = (int)s * 32 * E + lane * E;
        ArgPart a = arg_none();
        if (j < P.ld) arg_consider_sector(a, ld_sector_cg(P.T + j), j, P.W - 1, P.eps_d, P.cond ? P.var : nullptr);
        a = warp_arg(a);
        if (lane == 0) store_arg(P.cpart + s, a);
    }
}

// P1: global entering candidate from the strip partials (every block).
template <typename V>
__device__ ArgPart phase_entering(const Params<V>& P, BlockScratch& s) {
    ArgPart a = arg_none();
    for (int k = threadIdx.x; k < P.nstrips; k += blockDim.x) arg_merge(a, load_arg(P.cpart + k));
    return block_arg(a, s);
}

// The right-hand side of the first row a thread scans in P2 (the row depends
// only on the thread's index), loaded before P1 has found the entering column
// so that P2 waits on one load instead of two in a row.
template <typename V>
__device__ __forceinline__ V ratio_rhs_first(const Params<V>& P) {
    const long long i = (long long)threadIdx.x * gridDim.x + blockIdx.x;
    return i <= P.m ? __ldcg(P.T + (size_t)i * (size_t)P.ld + (P.W - 1)) : V(0);
}

// P2: ratio test on column q and copy of column q into F; one partial per block.
// Row i goes to block i mod G, so the divisions spread over every SM.
// rhs0: the first row's right-hand side from ratio_rhs_first, or null.
template <typename V>
__device__ void phase_ratio(const Params<V>& P, int q, int bland, BlockScratch& s, const V* rhs0 = nullptr) {
    RatPart best = rat_none();
    const long long nth = (long long)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // counted again in P3 / P4
        P.st->nact = 0;
        P.st->next_slot = 0;
    }
    const long long i0 = (long long)threadIdx.x * gridDim.x + blockIdx.x;
    for (long long i = i0; i <= P.m; i += nth) {
        const V* row = P.T + (size_t)i * (size_t)P.ld;
        const V a = __ldcg(row + q);
        __stcg(P.F + i, a);
        if (i >= 1 && (double)a > P.eps_p) {
            RatPart c;
            c.r = (double)div_rn(i == i0 && rhs0 ? *rhs0 : __ldcg(row + (P.W - 1)), a);
            c.i = (int)i;
            c.key = bland ? __ldcg(P.basis + (i - 1)) : (int)i;
            c.a = (double)a;
            if (!dbits_nan(c.r)) rat_merge(best, c);
        }
    }
    best = block_rat(best, s);
    if (threadIdx.x == 0) store_rat(P.rpart + blockIdx.x, best);
}

// P3a: global leaving candidate from the block partials (every block).
template <typename V>
__device__ RatPart phase_leaving(const Params<V>& P, BlockScratch& s) {
    RatPart a = rat_none();
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) rat_merge(a, load_rat(P.rpart + k));
    return block_rat(a, s);
}

// P3b: pivot-row staging.  (1) R[j] = T[p][j] / piv over the padded row,
// element j on block j mod G so the divisions spread over all SMs.  (2) The
// 32-B column groups of row p holding a nonzero entry -- exactly the groups
// whose R entries can be nonzero -- compacted into P.act (warp ballot, one
// atomic per warp; the order of the list does not matter, every group is
// updated independently).  With skip_zero == 0 every group is listed.  The
// first element and the first sector of each thread are loaded together, so
// both parts wait on one round trip.
template <typename V>
__device__ void phase_stage_row(const Params<V>& P, int p, int q, V piv) {
    constexpr int E = Lanes<V>::E;
    const V* row = P.T + (size_t)p * (size_t)P.ld;
    if (P.cond) {   // condensed: every column is updated; slot q takes the leaving variable's column
        const long long nth = (long long)gridDim.x * blockDim.x;
        for (long long e = (long long)threadIdx.x * gridDim.x + blockIdx.x; e < P.ld; e += nth)
            __stcg(P.R + e, div_rn(e == q ? V(1) : __ldcg(row + e), piv));
        return;
    }
    const int lane = threadIdx.x & 31;
    const long long nsec = P.ld / E;
    const long long nth = (long long)gridDim.x * blockDim.x;
    const long long e0 = (long long)threadIdx.x * gridDim.x + blockIdx.x;
    const long long wi = (long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const long long nwi = (long long)(blockDim.x >> 5) * gridDim.x;
    const long long k0 = wi * 32 + lane;
    V x = V(0);
    Sector<V> t;
    if (e0 < P.ld) x = __ldcg(row + e0);
    if (k0 < nsec) t = ld_sector_cg(row + E * k0);
    if (e0 < P.ld) __stcg(P.R + e0, div_rn(x, piv));
    for (long long e = e0 + nth; e < P.ld; e += nth) __stcg(P.R + e, div_rn(__ldcg(row + e), piv));
    for (long long base = wi * 32; base < nsec; base += nwi * 32) {
        const long long k = base + lane;
        bool nz = false;
        if (k < nsec) {
            if (base != wi * 32) t = ld_sector_cg(row + E * k);
            nz = P.skip_zero ? sector_nonzero(t) : true;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, nz);
        if (mask) {
            unsigned off = 0;
            if (lane == 0) off = atomicAdd(&P.st->nact, (unsigned)__popc(mask));
            off = __shfl_sync(0xffffffffu, off, 0);
            if (nz) P.act[off + __popc(mask & ((1u << lane) - 1u))] = (int)k;
        }
    }
}

// P4a: the objective row and the pivot row, every column group.  One warp per
// strip: T[0][j] = fma(-F[0], R[j], T[0][j]) with the strip's argmin partial of
// the new objective row (the next Step 1's input), and T[p][j] = R[j].
template <typename V>
__device__ void phase_update_edge_rows(const Params<V>& P, int p, int q) {
    constexpr int E = Lanes<V>::E;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const V f0 = __ldcg(P.F);
    const int jend = P.W - 1;
    const int zq = P.cond ? q : -1;   // condensed: slot q starts from the unit column e_p
    for (long long s = gw; s < P.nstrips; s += nw) {
        const int j = (int)s * 32 * E + lane * E;
        ArgPart a = arg_none();
        if (j < P.ld) {
            const Sector<V> r = ld_sector_cg(P.R + j);
            Sector<V> o = ld_sector_stream(P.T + j);
#pragma unroll
            for (int e = 0; e < E; ++e) o.v[e] = fma_rn(-f0, r.v[e], j + e == zq ? V(0) : o.v[e]);
            st_sector(P.T + j, o);
            st_sector(P.T + (size_t)p * (size_t)P.ld + j, r);
            arg_consider_sector(a, o, j, jend, P.eps_d, P.cond ? P.var : nullptr);
        }
        a = warp_arg(a);
        if (lane == 0) store_arg(P.cpart + s, a);
    }
}

// One work slot: rows i0 .. i0+nrows-1 (row p excluded) of the column group
// listed at entry c*32 + lane.
template <typename V, int R>
__device__ __forceinline__ void update_slot(const Params<V>& P, int p, int zq, unsigned nact, long long c, int i0,
                                            int nrows, const V* f) {
    constexpr int E = Lanes<V>::E;
    const long long e = c * 32 + (threadIdx.x & 31);
    if (e >= (long long)nact) return;
    const size_t col = (size_t)E * (size_t)(P.cond ? (int)e : __ldcg(P.act + e));
    const Sector<V> r = ld_sector_cg(P.R + col);
    // condensed: the entry of slot q starts from the leaving variable's unit column (0 off row p)
    const int eq = zq - (int)col;
    Sector<V> v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = i0 + k;
        if (k < nrows && i != p) v[k] = ld_sector_stream(P.T + (size_t)i * (size_t)P.ld + col);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = i0 + k;
        if (k < nrows && i != p) {
#pragma unroll
            for (int e2 = 0; e2 < E; ++e2) v[k].v[e2] = fma_rn(-f[k], r.v[e2], e2 == eq ? V(0) : v[k].v[e2]);
            st_sector(P.T + (size_t)i * (size_t)P.ld + col, v[k]);
        }
    }
}

// P4b: the rank-1 update of rows 1..m except p on the listed column groups:
// T[i][j] = fma(-F[i], R[j], T[i][j]).  Work slots are (group of kRowsInFlight
// rows, chunk of 32 listed column groups), numbered row-group-major, so that
// consecutive slots stream along the same rows and the rows' F values stay in
// registers while the row group is unchanged.  One listed column group per
// lane.  Groups not listed have R == 0: their update is the identity.
template <typename V, int R>
__device__ void phase_update_bulk(const Params<V>& P, int p, int zq, unsigned nact, int rev) {
    const int lane = threadIdx.x & 31;
    const long long nchunks = ((long long)nact + 31) / 32;
    const long long ngroups = ((long long)P.m + R - 1) / R;
    const long long total = nchunks * ngroups;
    long long gcur = -1;
    V f[R];
    int i0 = 1, nrows = 0;
    // Slots are handed out `grab` at a time from a counter (a static split
    // leaves the slowest blocks ~15% behind the mean); the next grab is
    // requested before the current one is processed.
    // (measured: single slots shorten the tail of the double update; the
    // float update has twice the slots per pivot, and pairs keep the counter's
    // atomics off its critical path)
    constexpr unsigned grab = TSX_GRAB > 0 ? (unsigned)TSX_GRAB : (sizeof(V) == 8 ? 1u : 2u);
    // TSX_STATIC_FIRST: warp w of the grid takes slots w*grab .. first, without
    // the counter, and the counter hands out the slots after the first
    // (warps x grab).  TSX_SLOT_PIPE: the grab for a warp's next slot is
    // requested before the current slot and read after it, so its round trip
    // never holds the warp (reading it at once would).
    const long long base = TSX_STATIC_FIRST ? (((long long)gridDim.x * blockDim.x) >> 5) * grab : 0;
    unsigned mine = 0;   // lane 0: a requested grab
    if (lane == 0) mine = atomicAdd(&P.st->next_slot, grab);
    long long cur;
    if (TSX_STATIC_FIRST) {
        cur = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * grab;
    } else {
        cur = (long long)__shfl_sync(0xffffffffu, mine, 0);
        if (lane == 0 && cur < total) mine = atomicAdd(&P.st->next_slot, grab);
    }
    while (cur < total) {
        const long long u0 = cur;
        const long long u1 = min(total, u0 + (long long)grab);
        if (!TSX_SLOT_PIPE) {
            cur = base + (long long)__shfl_sync(0xffffffffu, mine, 0);
            if (lane == 0 && cur < total) mine = atomicAdd(&P.st->next_slot, grab);
        }
        for (long long u = u0; u < u1; ++u) {
            // odd pivots sweep backwards: they start on the rows the previous
            // sweep wrote last, which are still in L2
            const long long ur = rev ? total - 1 - u : u;
            const long long g = ur / nchunks;
            const long long c = ur - g * nchunks;
            if (g != gcur) {
                gcur = g;
                i0 = 1 + (int)g * R;
                nrows = min(R, P.m + 1 - i0);
#pragma unroll
                for (int k = 0; k < R; ++k) f[k] = k < nrows ? __ldcg(P.F + i0 + k) : V(0);
            }
            update_slot<V, R>(P, p, zq, nact, c, i0, nrows, f);
        }
        if (TSX_SLOT_PIPE) {
            cur = base + (long long)__shfl_sync(0xffffffffu, mine, 0);
            if (lane == 0 && cur < total) mine = atomicAdd(&P.st->next_slot, grab);
        }
    }
}

// ------------------------------------------- P4b with bulk copies (TMA)
// Condensed layout: a slot's rows are contiguous 1 KB pieces of the tableau
// (32 sectors of one chunk), so each warp streams its slots into a ring of
// shared-memory stages with cp.async.bulk and an mbarrier per stage.  The
// loads of the next stages are in flight while the warp runs the FMAs and
// stores of the current one, without holding registers for them.
constexpr int kTmaRows = TSX_TMA_ROWS;       // rows per slot
constexpr int kTmaBatch = TSX_TMA_BATCH;
constexpr int kChunkBytes = 32 * 32;          // one chunk of one row: 32 sectors
constexpr int kTmaSmPerSm = 200 * 1024;       // ring bytes per SM (of 228 KB)

// Stages per warp for blocks of nt threads: TSX_TMA_STAGES, fewer where the
// rings of all resident warps would not fit the budget; 0 (no ring: the
// register path) where fewer than two fit.
__host__ __device__ constexpr int tma_fit(int nt) {
    return kTmaSmPerSm / (((nt > TSX_SM_THREADS ? nt : TSX_SM_THREADS) / 32) * (kTmaRows * kChunkBytes + 8));
}
__host__ __device__ constexpr int tma_stages(int nt) {
    return !TSX_TMA ? 0 : tma_fit(nt) >= TSX_TMA_STAGES ? TSX_TMA_STAGES : tma_fit(nt) >= 2 ? tma_fit(nt) : 0;
}
__host__ __device__ constexpr size_t tma_smem_bytes(int nt) {
    return (size_t)(nt / 32) * tma_stages(nt) * ((size_t)kTmaRows * kChunkBytes + 8);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity to complete; bounded by the
// solve's barrier timeout (globaltimer) and a spin count.
__device__ inline bool mbar_wait(unsigned bar, unsigned parity, long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    const unsigned long long max_spins = (unsigned long long)(timeout_ns > 0 ? timeout_ns : 0) + 4096ull;
    for (unsigned long long spins = 1;; ++spins) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spins & 15ull) == 0 && (global_ns() - t0 >= timeout_ns || spins > max_spins)) return false;
    }
}
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// Orders this thread's view of global memory (generic proxy: the stores of
// the previous pivot, published by the grid barrier) before its bulk copies.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// 16-byte pieces: a lane takes bytes [16 lane, 16 lane + 16) and
// [512 + 16 lane, 528 + 16 lane) of a chunk, so its shared-memory reads are
// conflict-free and its stores coalesce per warp instruction.
template <typename V>
struct Piece {
    static constexpr int N = 16 / (int)sizeof(V);
    V v[N];
};
__device__ __forceinline__ Piece<double> ld_piece_cg(const double* p) {
    Piece<double> x;
    asm volatile("ld.global.cg.v2.f64 {%0,%1}, [%2];" : "=d"(x.v[0]), "=d"(x.v[1]) : "l"(p));
    return x;
}
__device__ __forceinline__ Piece<float> ld_piece_cg(const float* p) {
    Piece<float> x;
    asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(x.v[0]), "=f"(x.v[1]), "=f"(x.v[2]), "=f"(x.v[3]) : "l"(p));
    return x;
}
template <typename V>
__device__ Piece<V> ld_piece_smem(unsigned a);
template <>
__device__ __forceinline__ Piece<double> ld_piece_smem<double>(unsigned a) {
    Piece<double> x;
    asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];" : "=d"(x.v[0]), "=d"(x.v[1]) : "r"(a) : "memory");
    return x;
}
template <>
__device__ __forceinline__ Piece<float> ld_piece_smem<float>(unsigned a) {
    Piece<float> x;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(x.v[0]), "=f"(x.v[1]), "=f"(x.v[2]), "=f"(x.v[3]) : "r"(a) : "memory");
    return x;
}
__device__ __forceinline__ void st_piece(double* p, const Piece<double>& x) {
    asm volatile("st.global.v2.f64 [%0], {%1,%2};" ::"l"(p), "d"(x.v[0]), "d"(x.v[1]) : "memory");
}
__device__ __forceinline__ void st_piece(float* p, const Piece<float>& x) {
    asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(x.v[0]), "f"(x.v[1]), "f"(x.v[2]),
                 "f"(x.v[3]) : "memory");
}

// A warp's ring: kTmaStages stages of kTmaRows x 1 KB and one mbarrier each.
// `phase` bit s is the parity of stage s's next completion; it persists
// across pivots (every issued stage is consumed before the phase ends).
template <int S>
struct TmaRing {
    static_assert(S >= 2, "a ring needs two stages");
    unsigned data;    // shared address of stage 0
    unsigned bar;     // shared address of stage 0's mbarrier
    unsigned phase;
};

template <int NT>
__device__ inline TmaRing<tma_stages(NT)> tma_ring_init(unsigned char* dyn) {
    constexpr int S = tma_stages(NT), nw = NT / 32;
    const int w = threadIdx.x >> 5;
    TmaRing<S> r;
    r.data = smem_u32(dyn) + (unsigned)(w * S * kTmaRows * kChunkBytes);
    r.bar = smem_u32(dyn) + (unsigned)(nw * S * kTmaRows * kChunkBytes + w * S * 8);
    r.phase = 0;
    if ((threadIdx.x & 31) == 0) {
        for (int s = 0; s < S; ++s) mbar_init(r.bar + 8 * s);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    return r;
}

// Slot u of a pivot's update (same numbering as phase_update_bulk with
// kTmaRows rows per group): rows i0 .. i0+nrows-1, chunk c.  Slot numbers
// fit 32 bits: the slot counter is 32 bits wide and a slot covers 4 KB or
// more of the tableau.
struct TmaSlot {
    unsigned c;
    int i0, nrows;
    unsigned bytes;   // bytes of each row's piece of the chunk (32 per sector)
};

__device__ __forceinline__ TmaSlot tma_slot(unsigned u, unsigned total, unsigned nchunks, unsigned nact, int m,
                                            int rev) {
    const unsigned ur = rev ? total - 1 - u : u;
    const unsigned g = ur / nchunks;
    TmaSlot t;
    t.c = ur - g * nchunks;
    t.i0 = 1 + (int)g * kTmaRows;
    t.nrows = min(kTmaRows, m + 1 - t.i0);
    t.bytes = 32u * min(32u, nact - t.c * 32u);
    return t;
}

// Lane 0: the stage's expected bytes, then one bulk copy per row (row p is
// skipped: the edge-row phase rewrites it meanwhile).
template <typename V>
__device__ __forceinline__ void tma_issue(const Params<V>& P, int p, const TmaSlot& t, unsigned dst, unsigned bar) {
    constexpr int E = Lanes<V>::E;
    const int skip = (p >= t.i0 && p < t.i0 + t.nrows) ? 1 : 0;
    mbar_arrive_expect_tx(bar, t.bytes * (unsigned)(t.nrows - skip));
    for (int k = 0; k < t.nrows; ++k) {
        const int i = t.i0 + k;
        if (i != p) bulk_load(dst + k * kChunkBytes, P.T + (size_t)i * (size_t)P.ld + (size_t)t.c * 32 * E, t.bytes, bar);
    }
}

template <typename V>
struct TmaOperands {   // a lane's R pieces and the slot's F values
    Piece<V> r0, r1;
    V f[kTmaRows];
};

template <typename V>
__device__ __forceinline__ TmaOperands<V> tma_operands(const Params<V>& P, const TmaSlot& t) {
    constexpr int E = Lanes<V>::E, N = Piece<V>::N;
    const int lane = threadIdx.x & 31;
    TmaOperands<V> o;
    const size_t col = (size_t)t.c * 32 * E + (size_t)lane * N;
    if ((unsigned)(16 * lane) < t.bytes) o.r0 = ld_piece_cg(P.R + col);
    if ((unsigned)(512 + 16 * lane) < t.bytes) o.r1 = ld_piece_cg(P.R + col + 32 * N);
#pragma unroll
    for (int k = 0; k < kTmaRows; ++k) o.f[k] = k < t.nrows ? __ldcg(P.F + t.i0 + k) : V(0);
    return o;
}

// All lanes: the FMAs and stores of one staged slot.
template <typename V>
__device__ __forceinline__ void tma_compute(const Params<V>& P, int p, int zq, const TmaSlot& t,
                                            const TmaOperands<V>& o, unsigned src) {
    constexpr int E = Lanes<V>::E, N = Piece<V>::N;
    const int lane = threadIdx.x & 31;
    const int col0 = (int)t.c * 32 * E + lane * N;
    const bool h0 = (unsigned)(16 * lane) < t.bytes, h1 = (unsigned)(512 + 16 * lane) < t.bytes;
    const int eq0 = zq - col0, eq1 = zq - (col0 + 32 * N);
    // the reads of kTmaBatch rows first, then their FMAs and stores
    constexpr int B = kTmaBatch < kTmaRows ? kTmaBatch : kTmaRows;
#pragma unroll
    for (int k0 = 0; k0 < kTmaRows; k0 += B) {
    Piece<V> x0[B], x1[B];
#pragma unroll
    for (int kk = 0; kk < B; ++kk) {
        const int k = k0 + kk;
        if (k < t.nrows && h0) x0[kk] = ld_piece_smem<V>(src + k * kChunkBytes + 16 * lane);
        if (k < t.nrows && h1) x1[kk] = ld_piece_smem<V>(src + k * kChunkBytes + 512 + 16 * lane);
    }
#pragma unroll
    for (int kk = 0; kk < B; ++kk) {
        const int k = k0 + kk;
        const int i = t.i0 + k;
        if (k < t.nrows && i != p) {
            V* row = P.T + (size_t)i * (size_t)P.ld + col0;
            const V f = -o.f[k];
            if (h0) {
#pragma unroll
                for (int e = 0; e < N; ++e) x0[kk].v[e] = fma_rn(f, o.r0.v[e], e == eq0 ? V(0) : x0[kk].v[e]);
                st_piece(row, x0[kk]);
            }
            if (h1) {
#pragma unroll
                for (int e = 0; e < N; ++e) x1[kk].v[e] = fma_rn(f, o.r1.v[e], e == eq1 ? V(0) : x1[kk].v[e]);
                st_piece(row + 32 * N, x1[kk]);
            }
        }
    }
    }
}

// P4b through the ring.  Slots come from the same counter as in
// phase_update_bulk: the prologue takes kTmaStages consecutive slots, each
// consumed stage is refilled with a slot requested one stage earlier.  Slot
// numbers grow in the order the stages are consumed, so the first stage with
// no slot ends the phase with nothing left in flight.
template <typename V, int kTmaStages>
__device__ void phase_update_bulk_tma(const Params<V>& P, int p, int zq, unsigned nact, int rev,
                                      TmaRing<kTmaStages>& ring) {
    const int lane = threadIdx.x & 31;
    const unsigned nchunks = (nact + 31) / 32;
    const unsigned ngroups = (unsigned)((P.m + kTmaRows - 1) / kTmaRows);
    const unsigned total = nchunks * ngroups;
    constexpr unsigned kStageBytes = kTmaRows * kChunkBytes;
    unsigned u[kTmaStages];
    unsigned base = 0;
    if (lane == 0) {
        fence_proxy_async_global();
        base = atomicAdd(&P.st->next_slot, (unsigned)kTmaStages);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
    for (int s = 0; s < kTmaStages; ++s) {
        u[s] = base + s;
        if (lane == 0 && u[s] < total)
            tma_issue(P, p, tma_slot(u[s], total, nchunks, nact, P.m, rev), ring.data + s * kStageBytes, ring.bar + 8 * s);
    }
    if (u[0] >= total) return;
    TmaSlot t = tma_slot(u[0], total, nchunks, nact, P.m, rev);
    TmaOperands<V> o = tma_operands(P, t);
    for (;;) {
#pragma unroll
        for (int s = 0; s < kTmaStages; ++s) {
            const int sn = (s + 1) % kTmaStages;
            unsigned req = 0;
            if (lane == 0) req = atomicAdd(&P.st->next_slot, 1u);   // the refill of stage s
            const bool more = u[sn] < total;
            TmaSlot tn = t;
            TmaOperands<V> on = o;
            if (more) {   // the next stage's operands, loaded ahead
                tn = tma_slot(u[sn], total, nchunks, nact, P.m, rev);
                on = tma_operands(P, tn);
            }
            const bool ok = mbar_wait(ring.bar + 8 * s, (ring.phase >> s) & 1u, P.timeout_ns);
            if (!__all_sync(0xffffffffu, ok)) goto drain;
            ring.phase ^= 1u << s;
            tma_compute(P, p, zq, t, o, ring.data + s * kStageBytes);
            __syncwarp();
            u[s] = __shfl_sync(0xffffffffu, req, 0);
            if (lane == 0 && u[s] < total)
                tma_issue(P, p, tma_slot(u[s], total, nchunks, nact, P.m, rev), ring.data + s * kStageBytes,
                          ring.bar + 8 * s);
            if (!more) return;
            t = tn;
            o = on;
        }
    }
drain:
    // a wait ran out: mark the solve, wait (bounded) for the stages' copies
    // so that none lands after the block exits
    if (lane == 0) atomicCAS(&P.st->status, kRunning, kTimeout);
#pragma unroll
    for (int s = 0; s < kTmaStages; ++s) {
        if (u[s] < total) {
            mbar_wait(ring.bar + 8 * s, (ring.phase >> s) & 1u, 1000000);
            ring.phase ^= 1u << s;
        }
    }
}

template <typename V, int R = kRowsInFlight, int S = 2>
__device__ void phase_update(const Params<V>& P, int p, int q, long long it, TmaRing<S>* ring = nullptr) {
    constexpr int E = Lanes<V>::E;
    const unsigned nact = P.cond ? (unsigned)(P.ld / E) : *(volatile const unsigned*)&P.st->nact;
    if (blockIdx.x == 0 && threadIdx.x == 0) P.st->active_sectors += nact;
    phase_update_edge_rows(P, p, q);
    const int rev = TSX_ALTERNATE ? (int)(it & 1) : 0;
    if (ring && P.cond)
        phase_update_bulk_tma(P, p, q, nact, rev, *ring);
    else
        phase_update_bulk<V, R>(P, p, P.cond ? q : -1, nact, rev);
}

}  // namespace tsx
