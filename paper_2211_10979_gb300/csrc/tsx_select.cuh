// Selection helpers shared by the block-per-LP (tsx_batch.cuh) and
// cluster-per-LP (tsx_cluster.cuh) solvers: Step 1 and Step 2 candidates of
// the full-tableau simplex (arXiv 2211.10979, Section III) with the
// reductions on integer keys, and the single-precision screen of the ratio
// test.
#pragma once

#include "tsx_device.cuh"

#ifndef TSX_FLAT_UNROLL
#define TSX_FLAT_UNROLL 2   // entries of the flat update in flight per thread
#endif
#ifndef TSX_BATCH_MINB
#define TSX_BATCH_MINB 1    // 1: the batch kernel is compiled for 1024 threads per SM (64 registers)
#endif

namespace tsx {

// The reductions of Steps 1-2 compare the integer keys of tsx_device.cuh
// (dkey), not the doubles: no FP64-pipe instruction in the argmin trees.
struct BArg {                 // entering candidate
    long long vk;             // dkey of its objective-row entry
    int var;                  // its variable (tie-break), INT_MAX if none
    int slot;
    int fvar;                 // Bland: lowest candidate variable
    int fslot;
};

__device__ __forceinline__ void barg_merge(BArg& a, const BArg& b) {
    if (b.vk < a.vk || (b.vk == a.vk && b.var < a.var)) { a.vk = b.vk; a.var = b.var; a.slot = b.slot; }
    if (b.fvar < a.fvar) { a.fvar = b.fvar; a.fslot = b.fslot; }
}

struct BRat {                 // leaving candidate
    long long rk;             // dkey of the ratio rhs_i / T[i][q]; dkey(+inf) if none
    int key;                  // tie-break key: row (Dantzig) or basic variable (Bland)
    int i;                    // its row, INT_MAX if none
    double a;                 // its pivot element
};

__device__ __forceinline__ BRat brat_none() { return BRat{kKeyInf, INT_MAX, INT_MAX, 0.0}; }

__device__ __forceinline__ void brat_merge(BRat& a, const BRat& b) {
    if (b.rk < a.rk || (b.rk == a.rk && b.key < a.key)) a = b;
}

__device__ __forceinline__ BRat warp_brat(BRat a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        BRat b;
        b.rk = __shfl_xor_sync(0xffffffffu, a.rk, o);
        b.key = __shfl_xor_sync(0xffffffffu, a.key, o);
        b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
        b.a = __shfl_xor_sync(0xffffffffu, a.a, o);
        brat_merge(a, b);
    }
    return a;
}

// Warp-wide entering candidate (every lane returns the warp's result).
__device__ __forceinline__ BArg warp_barg(BArg a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        BArg b;
        b.vk = __shfl_xor_sync(0xffffffffu, a.vk, o);
        b.var = __shfl_xor_sync(0xffffffffu, a.var, o);
        b.slot = __shfl_xor_sync(0xffffffffu, a.slot, o);
        b.fvar = __shfl_xor_sync(0xffffffffu, a.fvar, o);
        b.fslot = __shfl_xor_sync(0xffffffffu, a.fslot, o);
        barg_merge(a, b);
    }
    return a;
}

// The same for the fields the next Step 1 reads under the rule in force
// (Dantzig: value, variable, slot; Bland: lowest variable and its slot); the
// other fields keep the lane's own values.
__device__ __forceinline__ BArg warp_barg_rule(BArg a, int bland) {
    if (bland) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int fv = __shfl_xor_sync(0xffffffffu, a.fvar, o);
            const int fs = __shfl_xor_sync(0xffffffffu, a.fslot, o);
            if (fv < a.fvar) { a.fvar = fv; a.fslot = fs; }
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long vk = __shfl_xor_sync(0xffffffffu, a.vk, o);
            const int v = __shfl_xor_sync(0xffffffffu, a.var, o);
            const int sl = __shfl_xor_sync(0xffffffffu, a.slot, o);
            if (vk < a.vk || (vk == a.vk && v < a.var)) { a.vk = vk; a.var = v; a.slot = sl; }
        }
    }
    return a;
}

__device__ __forceinline__ BArg barg_none() {
    return BArg{kKeyInf, INT_MAX, -1, INT_MAX, -1};
}

// Step 1 candidate of objective-row slot j (value v, variable var); a NaN
// entry fails the test v < -eps_d and is no candidate.
__device__ __forceinline__ void barg_consider(BArg& a, double v, int vj, int j, double eps_d) {
    if (v < -eps_d) {
        const long long vk = dkey(v);
        if (vk < a.vk || (vk == a.vk && vj < a.var)) { a.vk = vk; a.var = vj; a.slot = j; }
        if (vj < a.fvar) { a.fvar = vj; a.fslot = j; }
    }
}

// FP32 value of a positive double whose exponent lies in float's normal range,
// its mantissa truncated to 23 bits (relative error below 2^-23); false for
// zero, negative, subnormal, out-of-range, infinite or NaN input.
__device__ __forceinline__ bool f32_trunc(double x, float& f) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    if (hi < (897u << 20) || hi >= (1151u << 20)) return false;   // sign 0, exponent 897..1150
    f = __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
    return true;
}

__device__ __forceinline__ float f32_rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Screen of one eligible row: its FP32 ratio estimate, or false when the
// estimate is unusable (non-positive right-hand side, out-of-range values, an
// estimate outside [2^-100, 2^100]); such a row always takes the exact path.
__device__ __forceinline__ bool ratio_estimate(double rhs, double a, float& est) {
    float rf, af;
    if (!f32_trunc(rhs, rf) || !f32_trunc(a, af)) return false;
    est = __fmul_rn(rf, f32_rcp_approx(af));
    return est >= 0x1p-100f && est <= 0x1p100f;
}

// Row i is eligible for Step 2 iff T[i][q] > eps_p (eps_p >= 0), decided on the
// bit patterns: for a non-NaN double the signed 64-bit pattern orders like the
// value above zero, and every negative value or -0 has a negative pattern.
__device__ __forceinline__ bool eligible_bits(double a, long long eps_bits) {
    return !dbits_nan(a) && __double_as_longlong(a) > eps_bits;
}

// Step 1 candidate test on integer keys (epsk = dkey(-eps_d)).
__device__ __forceinline__ void barg_consider_key(BArg& a, double v, int vj, int j, long long epsk) {
    const long long vk = dkey(v);
    if (!dbits_nan(v) && vk < epsk) {
        if (vk < a.vk || (vk == a.vk && vj < a.var)) { a.vk = vk; a.var = vj; a.slot = j; }
        if (vj < a.fvar) { a.fvar = vj; a.fslot = j; }
    }
}


// Step 3 over a flat index space: local rows 0..last of a row-major tableau
// (stride ld, n + 1 = W1 stored columns each), 32 consecutive entries per warp
// instruction across row ends.  T[l][j] = fma(-F[l], R[j], T[l][j]) with slot
// qs starting from 0 (the leaving variable's unit column), and row lp (< 0:
// none) becomes R.  Local row 0 is the objective row: its new entries j < n
// are the next Step 1's candidates (integer keys, var[] as tie-break), which
// the returned partial holds.  (i, j) is the calling thread's first entry and
// (di, dj) the step between its entries (NT threads).  Four entries are in
// flight per thread.
// var_qs >= 0: the variable slot qs holds after this pivot, for the
// objective-row candidates (var[qs] may still be changing meanwhile).
__device__ __forceinline__ BArg flat_update(double* T, int ld, int last, int W1, int n, const double* F,
                                           const double* R, int qs, int lp, const int* var, long long epsk,
                                           int i, int j, int di, int dj, int var_qs = -1) {
    BArg an = barg_none();
    // the objective row's entries (candidate test on each)
    for (; i == 0 && i <= last;) {
        double* tp = T + j;
        const double r = R[j];
        double v = __fma_rn(-F[0], r, j == qs ? 0.0 : *tp);
        if (lp == 0) v = r;
        *tp = v;
        if (j < n) barg_consider_key(an, v, j == qs && var_qs >= 0 ? var_qs : var[j], j, epsk);
        i += di;
        j += dj;
        if (j >= W1) { j -= W1; ++i; }
    }
    // the constraint rows, U entries per thread at a time
    constexpr int U = TSX_FLAT_UNROLL;
    while (i <= last) {
        int ii[U], jj[U];
#pragma unroll
        for (int e = 0; e < U; ++e) {
            ii[e] = i;
            jj[e] = j;
            i += di;
            j += dj;
            if (j >= W1) { j -= W1; ++i; }
        }
        double old[U], r[U], f[U];
#pragma unroll
        for (int e = 0; e < U; ++e) {
            if (ii[e] <= last) {
                old[e] = jj[e] == qs ? 0.0 : T[(size_t)ii[e] * ld + jj[e]];
                r[e] = R[jj[e]];
                f[e] = F[ii[e]];
            }
        }
#pragma unroll
        for (int e = 0; e < U; ++e) {
            if (ii[e] <= last) {
                double v = __fma_rn(-f[e], r[e], old[e]);
                if (ii[e] == lp) v = r[e];
                T[(size_t)ii[e] * ld + jj[e]] = v;
            }
        }
    }
    return an;
}

}  // namespace tsx
