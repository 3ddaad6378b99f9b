// Device side of the dense full-tableau simplex pivot (arXiv 2211.10979,
// Section III Steps 1-3; Section IV Steps 1-4 for one GPU).
//
// One pivot is four phases over the row-major tableau T ((m+1) x ld doubles,
// W = n + m + 1 logical columns, the last one the right-hand side):
//   P1  entering column q: reduce the per-strip (value, index) partials of the
//       objective row left by the previous P4 (Section III Step 1, Dantzig's
//       most negative coefficient; Section IV Step 1's local-then-global
//       reduction, here warp -> strip -> block).
//   P2  minimum-ratio test on column q (Section III Step 2, Section IV Step 2):
//       every block scans a share of the rows, copies column q into F and keeps
//       its best (ratio, key, row) -> one partial per block.
//   P3  leaving row p = reduce of the P2 partials; pivot-row staging
//       R[j] = T[p][j] / T[p][q] (Section III Step 3's pivot row).
//   P4  rank-1 update T[i][j] = fma(-F[i], R[j], T[i][j]) for i != p and
//       T[p][j] = R[j] (Section III Step 3, Section IV Step 4), streamed with
//       256-bit accesses, one warp per strip of 128 columns; the warp holding the
//       objective row of a strip also emits that strip's argmin partial of the
//       new objective row (the next P1's input).
// Between phases every block of the grid passes a device-wide barrier whose
// wait is bounded in time (the paper's per-iteration synchronisation,
// Section IV Iterate/Finalization).
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

namespace tsx {

constexpr int kRunning = 100;      // status while the iteration is in progress
constexpr int kStripCols = 128;    // columns of one warp strip (32 lanes x 4)
constexpr int kUnitRows = 32;      // rows of one work unit (one strip)
constexpr int kRowsInFlight = 8;   // rows loaded before the first store
constexpr int kMaxWarps = 32;      // warps per block upper bound (1024 threads)

// status codes (same values as lp_status in tabsimplex.h)
constexpr int kOptimal = 0, kUnbounded = 1, kIterLimit = 2, kNumeric = 3, kTimeout = -4;

struct ArgPart {      // best entering candidate of a column range
    double v;         // most negative objective-row entry (< -eps_d), +inf if none
    int j;            // its column (lowest on ties), INT_MAX if none
    int jfirst;       // lowest column with entry < -eps_d (Bland), INT_MAX if none
};

struct RatPart {      // best leaving candidate of a row range
    double r;         // minimum ratio rhs_i / T[i][q], +inf if none
    int key;          // tie-break key: row index (Dantzig) or basic variable (Bland)
    int i;            // its row (1..m), INT_MAX if none
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
};

struct Params {
    double* T;           // tableau, (m+1) x ld
    int ld, m, n, W;
    int* basis;          // m: variable basic in row i+1
    double* F;           // m+1: column q of the tableau before the update
    double* R;           // ld: scaled pivot row
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
    int nstrips;         // ceil(ld / kStripCols)
    int nrc;             // ceil((m+1) / kUnitRows)
    long long nunits;    // nstrips * nrc
    int skip_zero;       // leave column groups whose R entries are all zero
};

// ------------------------------------------------------------------ helpers
// One 32-byte sector of the tableau: four consecutive doubles.
struct __align__(32) sec4 {
    double x, y, z, w;
};

__device__ __forceinline__ sec4 make_sec4(double x, double y, double z, double w) {
    sec4 v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = w;
    return v;
}

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

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// 256-bit accesses of one 32-byte sector (4 doubles); addresses 32-B aligned.
__device__ __forceinline__ sec4 ld_sector_stream(const double* p) {
    sec4 v;
    asm volatile("ld.global.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v.x), "=d"(v.y), "=d"(v.z), "=d"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ sec4 ld_sector_cg(const double* p) {
    sec4 v;
    asm volatile("ld.global.cg.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v.x), "=d"(v.y), "=d"(v.z), "=d"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_sector(double* p, sec4 v) {
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};"
                 ::"l"(p), "d"(v.x), "d"(v.y), "d"(v.z), "d"(v.w) : "memory");
}

__device__ __forceinline__ ArgPart arg_none() { return ArgPart{__longlong_as_double(0x7ff0000000000000LL), INT_MAX, INT_MAX}; }
__device__ __forceinline__ RatPart rat_none() { return RatPart{__longlong_as_double(0x7ff0000000000000LL), INT_MAX, INT_MAX}; }

// (v, j) lexicographic minimum: the most negative entry, lowest column on ties.
__device__ __forceinline__ void arg_merge(ArgPart& a, const ArgPart& b) {
    if (b.v < a.v || (b.v == a.v && b.j < a.j)) { a.v = b.v; a.j = b.j; }
    a.jfirst = min(a.jfirst, b.jfirst);
}

__device__ __forceinline__ void arg_consider(ArgPart& a, double v, int j, int jend, double eps_d) {
    if (j < jend && v < -eps_d) {
        if (v < a.v || (v == a.v && j < a.j)) { a.v = v; a.j = j; }
        a.jfirst = min(a.jfirst, j);
    }
}

// (r, key) lexicographic minimum: smallest ratio, lowest key on ties.
__device__ __forceinline__ void rat_merge(RatPart& a, const RatPart& b) {
    if (b.r < a.r || (b.r == a.r && b.key < a.key)) a = b;
}

__device__ __forceinline__ ArgPart warp_arg(ArgPart a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ArgPart b;
        b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
        b.j = __shfl_xor_sync(0xffffffffu, a.j, o);
        b.jfirst = __shfl_xor_sync(0xffffffffu, a.jfirst, o);
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
        rat_merge(a, b);
    }
    return a;
}

// Partials are read by other blocks after a barrier: 128-bit L2 accesses.
__device__ __forceinline__ void store_arg(ArgPart* dst, const ArgPart& a) {
    long long bits = __double_as_longlong(a.v);
    __stcg(reinterpret_cast<int4*>(dst), make_int4((int)(bits & 0xffffffff), (int)(bits >> 32), a.j, a.jfirst));
}
__device__ __forceinline__ ArgPart load_arg(const ArgPart* src) {
    int4 w = __ldcg(reinterpret_cast<const int4*>(src));
    long long bits = ((long long)(unsigned)w.y << 32) | (unsigned)w.x;
    return ArgPart{__longlong_as_double(bits), w.z, w.w};
}
__device__ __forceinline__ void store_rat(RatPart* dst, const RatPart& a) {
    long long bits = __double_as_longlong(a.r);
    __stcg(reinterpret_cast<int4*>(dst), make_int4((int)(bits & 0xffffffff), (int)(bits >> 32), a.key, a.i));
}
__device__ __forceinline__ RatPart load_rat(const RatPart* src) {
    int4 w = __ldcg(reinterpret_cast<const int4*>(src));
    long long bits = ((long long)(unsigned)w.y << 32) | (unsigned)w.x;
    return RatPart{__longlong_as_double(bits), w.z, w.w};
}

struct BlockScratch {
    ArgPart arg[kMaxWarps];
    RatPart rat[kMaxWarps];
    unsigned long long cnt[kMaxWarps];
    ArgPart arg_out;
    RatPart rat_out;
    unsigned long long cnt_out;
    int ok;
};

// Block-wide reductions; every thread returns the block result.
__device__ ArgPart block_arg(ArgPart a, BlockScratch& s) {
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

__device__ RatPart block_rat(RatPart a, BlockScratch& s) {
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

__device__ unsigned long long block_sum(unsigned long long v, BlockScratch& s) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) s.cnt[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned long long b = lane < nw ? s.cnt[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (lane == 0) s.cnt_out = b;
    }
    __syncthreads();
    return s.cnt_out;
}

// ------------------------------------------------------------- grid barrier
// All blocks of the (co-resident) grid meet here.  Thread 0 of each block
// arrives on a counter; the last arrival resets it and bumps the generation
// word with release semantics; the others spin on the generation with acquire
// loads.  Each wait is bounded: after timeout_ns (globaltimer) or a spin-count
// limit, the block marks the solve LP_ERR_TIMEOUT and returns false; a block
// that sees a negative status while waiting returns false as well, so every
// block of a failed solve exits without waiting for the others.
__device__ bool grid_barrier(DevState* st, long long timeout_ns, BlockScratch& s) {
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

// ------------------------------------------------------------------ phases
// Initial objective-row argmin (before the first pivot): one warp per strip.
__device__ void phase_init_argmin(const Params& P) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long s = gw; s < P.nstrips; s += nw) {
        const int j = (int)s * kStripCols + lane * 4;
        ArgPart a = arg_none();
        if (j < P.ld) {
            sec4 v = ld_sector_cg(P.T + j);
            arg_consider(a, v.x, j, P.W - 1, P.eps_d);
            arg_consider(a, v.y, j + 1, P.W - 1, P.eps_d);
            arg_consider(a, v.z, j + 2, P.W - 1, P.eps_d);
            arg_consider(a, v.w, j + 3, P.W - 1, P.eps_d);
        }
        a = warp_arg(a);
        if (lane == 0) store_arg(P.cpart + s, a);
    }
}

// P1: global entering candidate from the strip partials (every block).
__device__ ArgPart phase_entering(const Params& P, BlockScratch& s) {
    ArgPart a = arg_none();
    for (int k = threadIdx.x; k < P.nstrips; k += blockDim.x) arg_merge(a, load_arg(P.cpart + k));
    return block_arg(a, s);
}

// P2: ratio test on column q and copy of column q into F; one partial per block.
__device__ void phase_ratio(const Params& P, int q, int bland, BlockScratch& s) {
    RatPart best = rat_none();
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= P.m; i += nth) {
        const double* row = P.T + (size_t)i * (size_t)P.ld;
        const double a = __ldcg(row + q);
        __stcg(P.F + i, a);
        if (i >= 1 && a > P.eps_p) {
            RatPart c;
            c.r = __ldcg(row + (P.W - 1)) / a;
            c.i = (int)i;
            c.key = bland ? __ldcg(P.basis + (i - 1)) : (int)i;
            rat_merge(best, c);
        }
    }
    best = block_rat(best, s);
    if (threadIdx.x == 0) store_rat(P.rpart + blockIdx.x, best);
}

// P3a: global leaving candidate from the block partials (every block).
__device__ RatPart phase_leaving(const Params& P, BlockScratch& s) {
    RatPart a = rat_none();
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) rat_merge(a, load_rat(P.rpart + k));
    return block_rat(a, s);
}

// P3b: R[j] = T[p][j] / piv over the padded row; counts the 32-B column groups
// with a nonzero entry (the groups P4 has to update when skipping).
__device__ void phase_stage_row(const Params& P, int p, double piv, BlockScratch& s) {
    const double* row = P.T + (size_t)p * (size_t)P.ld;
    const long long nsec = P.ld / 4;
    const long long nth = (long long)gridDim.x * blockDim.x;
    unsigned long long nz = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nsec; k += nth) {
        sec4 v = ld_sector_cg(row + 4 * k);
        sec4 r;
        r.x = v.x / piv;
        r.y = v.y / piv;
        r.z = v.z / piv;
        r.w = v.w / piv;
        st_sector(P.R + 4 * k, r);
        nz += (r.x != 0.0 || r.y != 0.0 || r.z != 0.0 || r.w != 0.0) ? 1ull : 0ull;
    }
    nz = block_sum(nz, s);
    if (threadIdx.x == 0 && nz) atomicAdd(&P.st->active_sectors, nz);
}

// P4: the rank-1 update, one warp per (strip, 32-row unit), contiguous unit
// ranges per warp in strip-major order (the scaled pivot row of a strip stays
// in registers across the warp's units).  Rows i != p: T = fma(-F[i], R, T);
// row p: T = R.  With skip_zero, a lane whose four R entries are all zero
// touches only the objective row and row p.  The warp that updates the
// objective row of a strip writes that strip's argmin partial.
__device__ void phase_update(const Params& P, int p) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long u0 = gw * P.nunits / nw;
    const long long u1 = (gw + 1) * P.nunits / nw;
    const int rows = P.m + 1;
    const int jend = P.W - 1;
    int strip = -1, j = 0;
    bool act = false, live = false;
    sec4 r = make_sec4(0.0, 0.0, 0.0, 0.0);
    for (long long u = u0; u < u1; ++u) {
        const int s = (int)(u / P.nrc);
        const int rc = (int)(u - (long long)s * P.nrc);
        if (s != strip) {
            strip = s;
            j = s * kStripCols + lane * 4;
            act = j < P.ld;
            r = act ? ld_sector_cg(P.R + j) : make_sec4(0.0, 0.0, 0.0, 0.0);
            live = act && (!P.skip_zero || r.x != 0.0 || r.y != 0.0 || r.z != 0.0 || r.w != 0.0);
        }
        const int i0 = rc * kUnitRows;
        const int i1 = min(i0 + kUnitRows, rows);
        const double fl = (i0 + lane < i1) ? __ldcg(P.F + i0 + lane) : 0.0;
        ArgPart a = arg_none();
        for (int ib = i0; ib < i1; ib += kRowsInFlight) {
            sec4 v[kRowsInFlight];
#pragma unroll
            for (int k = 0; k < kRowsInFlight; ++k) {
                const int i = ib + k;
                const bool go = act && i < i1 && (live || i == 0) && i != p;
                if (go) v[k] = ld_sector_stream(P.T + (size_t)i * (size_t)P.ld + j);
            }
#pragma unroll
            for (int k = 0; k < kRowsInFlight; ++k) {
                const int i = ib + k;
                const double f = __shfl_sync(0xffffffffu, fl, (i - i0) & 31);
                if (act && i < i1 && (live || i == 0 || i == p)) {
                    sec4 o;
                    if (i == p) {
                        o = r;
                    } else {
                        o.x = __fma_rn(-f, r.x, v[k].x);
                        o.y = __fma_rn(-f, r.y, v[k].y);
                        o.z = __fma_rn(-f, r.z, v[k].z);
                        o.w = __fma_rn(-f, r.w, v[k].w);
                    }
                    st_sector(P.T + (size_t)i * (size_t)P.ld + j, o);
                    if (i == 0) {
                        arg_consider(a, o.x, j, jend, P.eps_d);
                        arg_consider(a, o.y, j + 1, jend, P.eps_d);
                        arg_consider(a, o.z, j + 2, jend, P.eps_d);
                        arg_consider(a, o.w, j + 3, jend, P.eps_d);
                    }
                }
            }
        }
        if (i0 == 0) {
            a = warp_arg(a);
            if (lane == 0) store_arg(P.cpart + s, a);
        }
    }
}

}  // namespace tsx
