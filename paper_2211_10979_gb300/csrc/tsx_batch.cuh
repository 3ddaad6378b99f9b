// Batched solve of many small LPs (the full-tableau simplex of arXiv 2211.10979,
// Section III, one LP per block, the whole LP in shared memory).
//
// Each block keeps the CONDENSED tableau of its LP: the objective row and the m
// constraint rows over the n nonbasic columns plus the right-hand side, with
// var[j] = the variable held by column slot j.  The full tableau's basic
// columns are exact unit vectors (the pivot column becomes e_p exactly, and a
// basic column's pivot-row entry is zero so later pivots leave it unchanged),
// so dropping them changes no stored value: at a pivot on (p, slot q) the
// leaving variable takes slot q, whose new entries are what the full tableau
// computes for the leaving variable's unit column e_p:
//     row p:  1 / piv;     row i != p:  fma(-T[i][q], 1 / piv, 0),
// and every other slot follows Step 3 unchanged.  Ties are broken by the
// original variable index, so pivots and values equal the full-tableau run.
// The largest LP of m = n = 128 needs (m+1) x (n+1) doubles = 133 KB.  An LP
// whose condensed tableau does not fit in shared memory keeps it in a global
// workspace slice instead (k_batch_solve_global; L2-resident for medium LPs).
#pragma once

#include "tsx_select.cuh"

namespace tsx {

struct BatchLP {              // one LP of the batch
    int m, n;
    int ldc;                  // padded row length of the condensed tableau (odd)
    int bucket;
    long long a_off;          // offset of A (m x n row-major) in the packed A
    long long b_off;          // offset of b (and of y) in the packed b / y
    long long c_off;          // offset of c (and of x) in the packed c / x
    long long t_off;          // offset of the kept condensed tableau ((m+1) x ldc)
    long long w_off;          // byte offset of its global workspace slice, -1 if in shared memory
};

struct BatchParams {
    const BatchLP* lps;
    const double* A;
    const double* b;
    const double* c;
    int* status;              // per LP
    long long* iters;         // per LP
    double* obj;              // per LP
    double* x;                // packed like c
    double* y;                // packed like b
    double* keepT;            // kept condensed tableaux (null: not kept)
    int* keepvar;             // kept var maps (packed like c) (null: not kept)
    int* keepbasis;           // kept basis (packed like b)
    unsigned long long* total_pivots;
    double eps_d, eps_p;
    long long max_iters;      // < 0: 50 (m + n)
    int k_cyc, rule;
};

#ifndef TSX_BATCH_FLAT
#define TSX_BATCH_FLAT 1      // 1: flattened update + screened ratio test (batch_solve_one_flat)
#endif

// Shared-memory bytes of one LP's block.
__host__ __device__ inline size_t batch_smem_bytes(int m, int n, int ldc) {
    size_t bytes = (size_t)(m + 1) * ldc * 8      // tableau
                 + (size_t)(m + 1) * 8             // F (pivot column)
                 + (size_t)ldc * 8                 // R (scaled pivot row)
                 + (size_t)n * 4 + (size_t)m * 4;  // var, basis
#if TSX_BATCH_FLAT
    bytes += (size_t)m * 4;                        // ratio-test candidate rows
#endif
    return (bytes + 15) / 16 * 16;
}

constexpr int kRc = 4;        // scaled-pivot-row entries per lane kept in registers

struct BatchScratch {
    BArg arg[kMaxWarps];
    BRat rat[kMaxWarps];
    BArg arg_out;
    BRat rat_out;
    int lp;
    int ncand;                // flat solver: rows on the candidate list
};

// Block-wide ratio-test minimum with one barrier: each warp reduces, lane 0
// posts the warp's partial, every thread merges the posted partials.  The
// partials' slots are next written after at least one more barrier.
template <int NT>
__device__ BRat batch_block_rat(BRat a, BatchScratch& s) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_brat(a);
    if (NT == 32) return a;
    if (lane == 0) s.rat[w] = a;
    __syncthreads();
    BRat r = s.rat[0];
#pragma unroll
    for (int k = 1; k < NT / 32; ++k) brat_merge(r, s.rat[k]);
    return r;
}

// Solves LP `k` of the batch (NT threads) with its tableau at `smem` (shared
// memory, or the LP's global workspace slice).
template <int NT>
__device__ void batch_solve_one(const BatchParams& P, int k, unsigned char* smem, BatchScratch& sc) {
    const BatchLP L = P.lps[k];
    const int m = L.m, n = L.n, ldc = L.ldc;
    double* T = reinterpret_cast<double*>(smem);
    double* F = T + (size_t)(m + 1) * ldc;
    double* R = F + (m + 1);
    int* var = reinterpret_cast<int*>(R + ldc);
    int* basis = var + n;
    const double* A = P.A + L.a_off;
    const double* b = P.b + L.b_off;
    const double* c = P.c + L.c_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;

    // Initialization Step: condensed Table I (slack basis), plus input checks
    int bad = 0;
    for (long long t = tid; t < (long long)(m + 1) * ldc; t += NT) {
        const int i = (int)(t / ldc), j = (int)(t - (long long)i * ldc);
        double v = 0.0;
        if (j < n)
            v = i == 0 ? -c[j] : A[(size_t)(i - 1) * n + j];
        else if (j == n && i > 0)
            v = b[i - 1];
        if (j <= n) bad |= !dbits_finite(v) || (j == n && i > 0 && !(v >= 0.0));
        T[t] = v;
    }
    for (int j = tid; j < n; j += NT) var[j] = j;
    for (int i = tid; i < m; i += NT) basis[i] = n + i;
    bad = __syncthreads_or(bad);
    const long long cap = P.max_iters < 0 ? 50LL * (m + n) : P.max_iters;
    int status = kRunning;
    if (bad) status = -1;   // LP_ERR_INVALID
    long long it = 0;
    int bland = P.rule == 1, degen = 0;
    // Step 1 of the first pivot: warp 0 scans the objective row
    if (warp == 0) {
        BArg a0 = barg_none();
        for (int j = lane; j < n; j += 32) barg_consider(a0, T[j], var[j], j, P.eps_d);
        a0 = warp_barg(a0);
        if (lane == 0) sc.arg_out = a0;
    }
    __syncthreads();
    while (status == kRunning) {
        // Step 1: entering slot (most negative objective-row entry; ties and
        // Bland's rule by variable index), left by the previous update
        const BArg a = sc.arg_out;
        const int qs = bland ? a.fslot : a.slot;
        if (qs < 0) { status = kOptimal; break; }
        if (it >= cap) { status = kIterLimit; break; }
        // Step 2: minimum ratio on slot qs (ties: row, or basic variable in
        // Bland mode); column qs is copied to F on the way
        BRat best = brat_none();
        if (tid == 0) F[0] = T[qs];
        for (int i = 1 + tid; i <= m; i += NT) {
            const double av = T[(size_t)i * ldc + qs];
            F[i] = av;
            if (av > P.eps_p) {
                const double r = __ddiv_rn(T[(size_t)i * ldc + n], av);
                if (!dbits_nan(r)) {   // a NaN ratio never wins the comparison
                    BRat cnd;
                    cnd.rk = dkey(r);
                    cnd.i = i;
                    cnd.key = bland ? basis[i - 1] : i;
                    cnd.a = av;
                    brat_merge(best, cnd);
                }
            }
        }
        best = batch_block_rat<NT>(best, sc);
        if (best.i == INT_MAX) { status = kUnbounded; break; }
        const int p = best.i;
        const double piv = best.a;
        const double ratio = dkey_value(best.rk);
        if (!dbits_finite(piv) || !dbits_finite(ratio)) { status = kNumeric; break; }
        // Step 3: scaled pivot row; the leaving variable takes slot qs
        for (int j = tid; j <= n; j += NT) R[j] = __ddiv_rn(j == qs ? 1.0 : T[(size_t)p * ldc + j], piv);
        if (tid == 0) {
            const int leaving = basis[p - 1];
            basis[p - 1] = var[qs];
            var[qs] = leaving;
        }
        ++it;
        if (P.rule == 0) {
            if (best.rk <= 0) {   // ratio <= 0
                ++degen;
                if (P.k_cyc > 0 && degen >= P.k_cyc) bland = 1;
            } else {
                degen = 0;
                bland = 0;
            }
        }
        __syncthreads();
        // rank-1 update; the warp of row 0 also finds the next entering slot.
        // The first kRc entries of R per lane stay in registers for all rows.
        double rr[kRc];
#pragma unroll
        for (int t = 0; t < kRc; ++t) {
            const int j = lane + 32 * t;
            rr[t] = j <= n ? R[j] : 0.0;
        }
        for (int i = warp; i <= m; i += NW) {
            double* row = T + (size_t)i * ldc;
            if (i == p) {
                for (int j = lane; j <= n; j += 32) row[j] = R[j];
            } else if (i == 0) {
                const double f = F[0];
                BArg an = barg_none();
                for (int j = lane; j <= n; j += 32) {
                    const double v = __fma_rn(-f, R[j], j == qs ? 0.0 : row[j]);
                    row[j] = v;
                    if (j < n) barg_consider(an, v, var[j], j, P.eps_d);
                }
                an = warp_barg(an);
                if (lane == 0) sc.arg_out = an;
            } else {
                const double f = F[i];
#pragma unroll
                for (int t = 0; t < kRc; ++t) {
                    const int j = lane + 32 * t;
                    if (j <= n) row[j] = __fma_rn(-f, rr[t], j == qs ? 0.0 : row[j]);
                }
                for (int j = lane + 32 * kRc; j <= n; j += 32) row[j] = __fma_rn(-f, R[j], j == qs ? 0.0 : row[j]);
            }
        }
        __syncthreads();
    }
    // read-out (Table I layout): x from the basis, y from the objective row
    double* x = P.x + L.c_off;
    double* y = P.y + L.b_off;
    for (int j = tid; j < n; j += NT) x[j] = 0.0;
    for (int i = tid; i < m; i += NT) y[i] = 0.0;
    __syncthreads();
    if (status != -1) {
        for (int i = tid; i < m; i += NT)
            if (basis[i] < n) x[basis[i]] = T[(size_t)(i + 1) * ldc + n];
        for (int j = tid; j < n; j += NT)
            if (var[j] >= n) y[var[j] - n] = T[j];
    }
    if (tid == 0) {
        P.status[k] = status;
        P.iters[k] = it;
        P.obj[k] = status == -1 ? 0.0 : T[n];
        if (it) atomicAdd(P.total_pivots, (unsigned long long)it);
    }
    if (P.keepT) {
        double* kt = P.keepT + L.t_off;
        for (long long t = tid; t < (long long)(m + 1) * ldc; t += NT) kt[t] = T[t];
        for (int j = tid; j < n; j += NT) P.keepvar[L.c_off + j] = var[j];
        for (int i = tid; i < m; i += NT) P.keepbasis[L.b_off + i] = basis[i];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// The same solve with every FP64 instruction of a pivot as full as it can be.
// GB300 issues an FP64 warp instruction to its one FP64 pipe per SM for the
// same 16 cycles whether 1 or 32 lanes are active, and an IEEE division costs
// about nine of them, so the pipe time of a pivot is counted in warp
// instructions:
//   - Step 3 runs over the (m+1) x (n+1) entries as one flat index space (each
//     warp instruction updates 32 consecutive entries, across row ends), not
//     row by row (a row of n+1 entries fills ceil((n+1)/32) instructions);
//   - Step 2 screens the rows in single precision first: a row whose FP32
//     ratio estimate is more than a factor 1 + 2^-18 above its warp's
//     smallest estimate cannot hold the minimum ratio (the estimate's relative
//     error is below 2^-21), so only the remaining rows -- usually one per
//     warp, plus any row the estimate cannot represent -- get the exact IEEE
//     division, all of them in one warp;
//   - the candidate tests of Steps 1-2 compare integer keys, not doubles.
// Every decision is taken on the same correctly rounded values as before, so
// pivots and results are unchanged.  Four block barriers per pivot: after the
// screen, after the exact minimum, after the pivot-row staging, after Step 3.
// ---------------------------------------------------------------------------

template <int NT>
__device__ void batch_solve_one_flat(const BatchParams& P, int k, unsigned char* smem, BatchScratch& sc) {
    const BatchLP L = P.lps[k];
    const int m = L.m, n = L.n, ldc = L.ldc;
    double* T = reinterpret_cast<double*>(smem);
    double* F = T + (size_t)(m + 1) * ldc;
    double* R = F + (m + 1);
    int* var = reinterpret_cast<int*>(R + ldc);
    int* basis = var + n;
    int* cand = basis + m;
    const double* A = P.A + L.a_off;
    const double* b = P.b + L.b_off;
    const double* c = P.c + L.c_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    const long long epsk = dkey(-P.eps_d);
    // bit pattern of eps_p >= 0, with -0 taken as +0
    const long long eps_bits = max(0LL, (long long)__double_as_longlong(P.eps_p));

    // Initialization Step: condensed Table I (slack basis), plus input checks
    int bad = 0;
    for (long long t = tid; t < (long long)(m + 1) * ldc; t += NT) {
        const int i = (int)(t / ldc), j = (int)(t - (long long)i * ldc);
        double v = 0.0;
        if (j < n)
            v = i == 0 ? -c[j] : A[(size_t)(i - 1) * n + j];
        else if (j == n && i > 0)
            v = b[i - 1];
        if (j <= n) bad |= !dbits_finite(v) || (j == n && i > 0 && !(v >= 0.0));
        T[t] = v;
    }
    for (int j = tid; j < n; j += NT) var[j] = j;
    for (int i = tid; i < m; i += NT) basis[i] = n + i;
    // Step 1 of the first pivot: warp 0 scans the objective row
    {
        BArg a0 = barg_none();
        if (warp == 0) {
            for (int j = lane; j < n; j += 32) barg_consider_key(a0, -c[j], j, j, epsk);
            a0 = warp_barg(a0);
        }
        if (lane == 0) sc.arg[warp] = a0;
        if (tid == 0) sc.ncand = 0;
    }
    bad = __syncthreads_or(bad);
    const long long cap = P.max_iters < 0 ? 50LL * (m + n) : P.max_iters;
    int status = kRunning;
    if (bad) status = -1;   // LP_ERR_INVALID
    long long it = 0;
    int bland = P.rule == 1, degen = 0;
    // this thread's first entry of the flat (m+1) x (n+1) index space, and
    // the step between its entries
    const int W1 = n + 1;
    const int i_first = tid / W1, j_first = tid - (tid / W1) * W1;
    const int di = NT / W1, dj = NT - (NT / W1) * W1;
    const bool row0_warp = warp * 32 < W1;   // warps whose entries include row 0
    const int NW0 = min(NW, (W1 + 31) / 32);   // ... are the first NW0 (the others post none)
    while (status == kRunning) {
        // Step 1: merge the objective-row partials of the previous update
        BArg a = sc.arg[0];
#pragma unroll 1
        for (int w = 1; w < NW0; ++w) barg_merge(a, sc.arg[w]);
        const int qs = bland ? a.fslot : a.slot;
        if (qs < 0) { status = kOptimal; break; }
        if (it >= cap) { status = kIterLimit; break; }
        // Step 2, screen: F = column qs; each warp keeps the rows whose FP32
        // ratio estimate is within 1 + 2^-18 of its smallest estimate, and
        // every eligible row without a usable estimate, on the candidate list
        if (tid == 0) F[0] = T[qs];
        float emin = __int_as_float(0x7f800000);   // +inf
        // the thread's first row (its only one when m <= NT) keeps its screen
        // result in a register for the second pass: -1 not eligible, NaN
        // eligible without a usable estimate, else the estimate (> 0)
        float scr0 = -1.f;
        for (int i = 1 + tid; i <= m; i += NT) {
            const double av = T[(size_t)i * ldc + qs];
            F[i] = av;
            float scr = -1.f;
            if (eligible_bits(av, eps_bits)) {
                float est;
                if (ratio_estimate(T[(size_t)i * ldc + n], av, est)) {
                    scr = est;
                    emin = fminf(emin, est);
                } else {
                    scr = __int_as_float(0x7fc00000);
                }
            }
            if (i == 1 + tid) scr0 = scr;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emin = fminf(emin, __shfl_xor_sync(0xffffffffu, emin, o));
        const float band = __fmul_ru(emin, 1.0f + 0x1p-18f);
        for (int base = 1 + warp * 32; base <= m; base += NT) {
            const int i = base + lane;   // base == 1 + warp * 32: the row 1 + tid of the first pass
            bool keep = false;
            if (i <= m) {
                if (base == 1 + warp * 32) {
                    keep = isnan(scr0) || (scr0 >= 0.f && scr0 <= band);
                } else {
                    const double av = F[i];
                    if (eligible_bits(av, eps_bits)) {
                        float est;
                        keep = !ratio_estimate(T[(size_t)i * ldc + n], av, est) || est <= band;
                    }
                }
            }
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            if (ball) {
                int at = 0;
                if (lane == 0) at = atomicAdd(&sc.ncand, __popc(ball));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (keep) cand[at + __popc(ball & ((1u << lane) - 1u))] = i;
            }
        }
        __syncthreads();
        // Step 2, exact: warp 0 divides the candidates (IEEE division) and
        // takes the minimum (ties: row, or basic variable in Bland mode).  One
        // warp only: GB300's FP64 pipe charges a division by warp
        // instruction, however few lanes are active.
        if (warp == 0) {
            BRat best = brat_none();
            const int nc = sc.ncand;
            for (int t = lane; t < nc; t += 32) {
                const int i = cand[t];
                const double av = F[i];
                const double r = __ddiv_rn(T[(size_t)i * ldc + n], av);
                if (!dbits_nan(r)) {   // a NaN ratio never wins the comparison
                    BRat cnd;
                    cnd.rk = dkey(r);
                    cnd.i = i;
                    cnd.key = bland ? basis[i - 1] : i;
                    cnd.a = av;
                    brat_merge(best, cnd);
                }
            }
            // lanes nc.. hold none while nc < 32: fold only the lanes with
            // candidates into lane 0 (nothing to fold for a single candidate)
            if (nc >= 32) {
                best = warp_brat(best);
            } else {
                for (int o = 1; o < nc; o <<= 1) {
                    BRat b;
                    b.rk = __shfl_down_sync(0xffffffffu, best.rk, o);
                    b.key = __shfl_down_sync(0xffffffffu, best.key, o);
                    b.i = __shfl_down_sync(0xffffffffu, best.i, o);
                    b.a = __shfl_down_sync(0xffffffffu, best.a, o);
                    brat_merge(best, b);
                }
            }
            if (lane == 0) sc.rat_out = best;
        }
        __syncthreads();
        const BRat best = sc.rat_out;
        if (best.i == INT_MAX) { status = kUnbounded; break; }
        const int p = best.i;
        const double piv = best.a;
        const double ratio = dkey_value(best.rk);
        if (!dbits_finite(piv) || !dbits_finite(ratio)) { status = kNumeric; break; }
        // Step 3: scaled pivot row; the leaving variable takes slot qs (the
        // swap is written after the barrier below, when no warp reads them)
        const int leaving = basis[p - 1];
        const int entering = var[qs];
        for (int j = tid; j <= n; j += NT) R[j] = __ddiv_rn(j == qs ? 1.0 : T[(size_t)p * ldc + j], piv);
        ++it;
        if (P.rule == 0) {
            if (best.rk <= 0) {   // ratio <= 0
                ++degen;
                if (P.k_cyc > 0 && degen >= P.k_cyc) bland = 1;
            } else {
                degen = 0;
                bland = 0;
            }
        }
        __syncthreads();
        if (tid == 0) {
            sc.ncand = 0;   // every warp has read these before the barrier above
            basis[p - 1] = entering;
            var[qs] = leaving;
        }
        // rank-1 update over the flat index space; row p becomes R; the
        // objective row's new entries feed the next Step 1
        BArg an = flat_update(T, ldc, m, W1, n, F, R, qs, p, var, epsk, i_first, j_first, di, dj, leaving);
        if (row0_warp) an = warp_barg_rule(an, bland);   // the next Step 1 reads these fields only
        if (lane == 0) sc.arg[warp] = an;
        __syncthreads();
    }
    // read-out (Table I layout): x from the basis, y from the objective row
    double* x = P.x + L.c_off;
    double* y = P.y + L.b_off;
    for (int j = tid; j < n; j += NT) x[j] = 0.0;
    for (int i = tid; i < m; i += NT) y[i] = 0.0;
    __syncthreads();
    if (status != -1) {
        for (int i = tid; i < m; i += NT)
            if (basis[i] < n) x[basis[i]] = T[(size_t)(i + 1) * ldc + n];
        for (int j = tid; j < n; j += NT)
            if (var[j] >= n) y[var[j] - n] = T[j];
    }
    if (tid == 0) {
        P.status[k] = status;
        P.iters[k] = it;
        P.obj[k] = status == -1 ? 0.0 : T[n];
        if (it) atomicAdd(P.total_pivots, (unsigned long long)it);
    }
    if (P.keepT) {
        double* kt = P.keepT + L.t_off;
        for (long long t = tid; t < (long long)(m + 1) * ldc; t += NT) kt[t] = T[t];
        for (int j = tid; j < n; j += NT) P.keepvar[L.c_off + j] = var[j];
        for (int i = tid; i < m; i += NT) P.keepbasis[L.b_off + i] = basis[i];
    }
    __syncthreads();
}

template <int NT>
__device__ __forceinline__ void batch_solve_lp(const BatchParams& P, int k, unsigned char* smem, BatchScratch& sc) {
#if TSX_BATCH_FLAT
    batch_solve_one_flat<NT>(P, k, smem, sc);
#else
    batch_solve_one<NT>(P, k, smem, sc);
#endif
}

// One bucket: persistent blocks take LPs of `list` from a counter until none is left.
template <int NT>
__global__ void __launch_bounds__(NT, TSX_BATCH_MINB ? (1024 / NT > 0 ? 1024 / NT : 1) : 1) k_batch_solve(BatchParams P, const int* __restrict__ list, int count,
                                                   unsigned* __restrict__ queue) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BatchScratch sc;
    for (;;) {
        if (threadIdx.x == 0) sc.lp = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int t = sc.lp;
        __syncthreads();
        if (t >= count) return;
        batch_solve_lp<NT>(P, list[t], smem, sc);
    }
}

// LPs too large for shared memory: the same solve on a global workspace slice.
template <int NT>
__global__ void __launch_bounds__(NT, TSX_BATCH_MINB ? (1024 / NT > 0 ? 1024 / NT : 1) : 1) k_batch_solve_global(BatchParams P, const int* __restrict__ list, int count,
                                                          unsigned* __restrict__ queue, unsigned char* work) {
    __shared__ BatchScratch sc;
    for (;;) {
        if (threadIdx.x == 0) sc.lp = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int t = sc.lp;
        __syncthreads();
        if (t >= count) return;
        const int k = list[t];
        batch_solve_lp<NT>(P, k, work + P.lps[k].w_off, sc);
    }
}

// Full (m+1) x (n+m+1) tableau of one LP from its kept condensed tableau: the
// nonbasic columns where var[] puts them, unit columns for the basic variables,
// the right-hand side last.
__global__ void k_batch_expand(const BatchLP* lps, int k, const double* keepT, const int* keepvar,
                               const int* keepbasis, double* out) {
    const BatchLP L = lps[k];
    const int m = L.m, n = L.n, W = n + m + 1;
    const double* T = keepT + L.t_off;
    const int* var = keepvar + L.c_off;
    const int* basis = keepbasis + L.b_off;
    const size_t total = (size_t)(m + 1) * W;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
        out[t] = 0.0;
    __syncthreads();
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < (size_t)(m + 1) * (n + 1);
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / (n + 1)), j = (int)(t - (size_t)i * (n + 1));
        const int col = j < n ? var[j] : W - 1;
        out[(size_t)i * W + col] = T[(size_t)i * L.ldc + j];
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        out[(size_t)(i + 1) * W + basis[i]] = 1.0;
}

}  // namespace tsx
