// Kernels of the full-tableau simplex (arXiv 2211.10979, Section III), for a
// tableau of doubles or floats (V):
//   k_reset_state         zero the per-solve state word block
//   k_validate            inputs finite, b >= 0 (create)
//   k_ingest              create from page-locked host inputs: read over the
//                         host link, copied and checked in one pass
//   k_build<V>            Initialization Step: Table I tableau (full or
//                         condensed), slack basis
//   k_pivot_persistent    Steps 1-3 iterated inside one cooperative launch
//   k_ml_*                the same phases, one launch each (fallback, profiling)
//   k_extract_*<V>        read-out of x, y, objective from the tableau
//   k_expand_cond<V> etc. Table I rebuilt from a condensed tableau
#pragma once

#include "tsx_device.cuh"

namespace tsx {

__global__ void k_reset_state(DevState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
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
        for (int k = 0; k < 6; ++k) st->phase_ns[k] = 0;
    }
}

// Input check: every entry finite, b >= 0.
__global__ void k_validate(int m, int n, const double* __restrict__ A, const double* __restrict__ b,
                           const double* __restrict__ c, DevState* st) {
    const size_t mn = (size_t)m * (size_t)n;
    const size_t total = mn + (size_t)m + (size_t)n;
    int bad = 0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        double v;
        if (k < mn) {
            v = A[k];
            bad |= !isfinite(v);
        } else if (k < mn + m) {
            v = b[k - mn];
            bad |= !isfinite(v) || !(v >= 0.0);
        } else {
            v = c[k - mn - m];
            bad |= !isfinite(v);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->bad, 1);
}

// lp_create from page-locked host inputs: the GPU reads A, b, c over the host
// link itself (src = the arrays' device aliases) and checks them in the same
// pass -- entries finite, b >= 0 (-0 allowed) -- so the inputs are read once
// and no check kernel follows (st == null: copy only, the batched solver's
// upload, whose solve reports invalid inputs per LP).  Checks on the bits (integer pipes).  16-byte
// accesses for A where both addresses allow them; four in flight per thread.
__device__ __forceinline__ int ingest_bad(unsigned long long u, int nonneg) {
    const int nonfinite = ((u >> 52) & 0x7ffull) == 0x7ffull;
    const int negative = nonneg && (u >> 63) && (u & 0x7fffffffffffffffull) != 0ull;
    return nonfinite | negative;
}

__global__ void k_ingest(const double* __restrict__ sA, double* __restrict__ dA, size_t mn,
                         const double* __restrict__ sb, double* __restrict__ db, size_t m,
                         const double* __restrict__ sc, double* __restrict__ dc, size_t n, DevState* st) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    int bad = 0;
    if ((((unsigned long long)sA | (unsigned long long)dA) & 15ull) == 0ull) {
        const size_t np = mn / 2;
        const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sA);
        ulonglong2* d2 = reinterpret_cast<ulonglong2*>(dA);
        constexpr int U = 4;
        size_t k = tid;
        for (; k + (U - 1) * nth < np; k += U * nth) {
            ulonglong2 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = s2[k + u * nth];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                d2[k + u * nth] = v[u];
                bad |= ingest_bad(v[u].x, 0) | ingest_bad(v[u].y, 0);
            }
        }
        for (; k < np; k += nth) {
            const ulonglong2 v = s2[k];
            d2[k] = v;
            bad |= ingest_bad(v.x, 0) | ingest_bad(v.y, 0);
        }
        if ((mn & 1) && tid == 0) {
            const unsigned long long u = __double_as_longlong(sA[mn - 1]);
            dA[mn - 1] = __longlong_as_double(u);
            bad |= ingest_bad(u, 0);
        }
    } else {
        for (size_t k = tid; k < mn; k += nth) {
            const unsigned long long u = __double_as_longlong(sA[k]);
            dA[k] = __longlong_as_double(u);
            bad |= ingest_bad(u, 0);
        }
    }
    for (size_t k = tid; k < m; k += nth) {
        const unsigned long long u = __double_as_longlong(sb[k]);
        db[k] = __longlong_as_double(u);
        bad |= ingest_bad(u, 1);
    }
    for (size_t k = tid; k < n; k += nth) {
        const unsigned long long u = __double_as_longlong(sc[k]);
        dc[k] = __longlong_as_double(u);
        bad |= ingest_bad(u, 0);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && st) atomicOr(&st->bad, 1);
}

// Initialization Step (Section III, Table I): row 0 = [-c, 0 | 0],
// row i = [A_i, e_i | b_i]; padding columns [W, ld) are zero.  One thread per
// 32-byte sector; the float tableau takes the inputs rounded to nearest.
// Also seeds the slack basis.
// W is the stored width: n + m + 1 (full) or n + 1 (condensed, var != null:
// the slack columns are basic unit vectors and are not stored; var[j] = j).
template <typename V>
__global__ void k_build(int m, int n, int W, int ld, const double* __restrict__ A,
                        const double* __restrict__ b, const double* __restrict__ c,
                        V* __restrict__ T, int* __restrict__ basis, int* __restrict__ var) {
    constexpr int E = Lanes<V>::E;
    const size_t per_row = (size_t)ld / E;
    const size_t total = (size_t)(m + 1) * per_row;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / per_row);
        const int j0 = (int)(g - (size_t)i * per_row) * E;
        Sector<V> out;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = j0 + e;
            double v = 0.0;
            if (i == 0) {
                if (j < n) v = -c[j];
            } else {
                if (j < n)
                    v = A[(size_t)(i - 1) * (size_t)n + j];
                else if (j == W - 1)
                    v = b[i - 1];
                else if (!var && j == n + i - 1)
                    v = 1.0;
            }
            out.v[e] = (V)v;
        }
        st_sector(T + (size_t)i * (size_t)ld + j0, out);
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)m;
         i += (size_t)gridDim.x * blockDim.x)
        basis[i] = n + (int)i;
    if (var)
        for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < (size_t)n;
             j += (size_t)gridDim.x * blockDim.x)
            var[j] = (int)j;
}

// Pivot bookkeeping shared by both paths (one thread): basis update, pivot
// log (entering variable qv, leaving row p); condensed: the leaving variable
// takes column slot q.
template <typename V>
__device__ __forceinline__ void record_pivot(const Params<V>& P, long long it, int q, int qv, int p) {
    const int leaving = P.basis[p - 1];
    P.basis[p - 1] = qv;
    if (P.cond) P.var[q] = leaving;
    if (it < P.log_cap) {
        P.qlog[it] = qv;
        P.plog[it] = p;
    }
}

// Cycling guard: a pivot with minimum ratio <= 0 does not move the objective;
// k_cyc of them in a row switch to Bland's rule until a positive-ratio pivot.
template <typename V>
__device__ __forceinline__ void degeneracy_step(const Params<V>& P, double theta, int& bland, int& degen) {
    if (P.rule != 0) return;
    if (theta <= 0.0) {
        ++degen;
        if (P.k_cyc > 0 && degen >= P.k_cyc) bland = 1;
    } else {
        degen = 0;
        bland = 0;
    }
}

template <typename V>
__device__ __forceinline__ void finish(const Params<V>& P, int status, long long it, int bland, int degen,
                                       const long long* ph) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicCAS(&P.st->status, kRunning, status);
        P.st->iters = it;
        P.st->bland = bland;
        P.st->degen_run = degen;
        for (int k = 0; k < 6; ++k) P.st->phase_ns[k] = ph[k];
    }
}

// Phase timer of block 0, thread 0, kept in shared memory so that no
// registers are held across the pivot loop.
struct PhaseClock {
    long long acc[6];
    long long t;
    __device__ void start() {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            for (int k = 0; k < 6; ++k) acc[k] = 0;
            t = global_ns();
        }
    }
    __device__ void lap(int k) {   // closes interval k, opens the next one
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const long long now = global_ns();
            acc[k] += now - t;
            t = now;
        }
    }
};

// Steps 1-3 iterated inside one cooperative launch; three grid barriers per
// pivot (after P2, after P3, after P4).  Every block takes the same decisions
// from the same reduced values, so all leave the loop together.
// RS: rows of an update slot (fewer for LPs whose slots would be too few to
// spread evenly over the grid's warps).
template <int NT, typename V, int RS = persistent_rows(NT)>
__global__ void __launch_bounds__(NT, persistent_sm_threads(NT) / NT) k_pivot_persistent(Params<V> P) {
    __shared__ BlockScratch s;
    __shared__ PhaseClock clk;
    extern __shared__ __align__(128) unsigned char tsx_dyn[];
    TmaRing<(tma_stages(NT) >= 2 ? tma_stages(NT) : 2)> ring;
    auto* ringp = tma_stages(NT) >= 2 ? &ring : nullptr;
    if constexpr (tma_stages(NT) >= 2) ring = tma_ring_init<NT>(tsx_dyn);
    if (threadIdx.x == 0) s.passed = 0;
    clk.start();
    phase_init_argmin(P);
    if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
    long long it = 0;
    int bland = P.rule == 1 ? 1 : 0;
    int degen = 0;
    clk.start();
    for (;;) {
        V rhs0 = V(0);
        if (TSX_RHS_PREFETCH) rhs0 = ratio_rhs_first(P);   // in flight during Step 1
        const ArgPart e = phase_entering(P, s);           // Step 1
        const int q = bland ? e.fslot : e.slot;
        const int qv = bland ? e.fkey : e.key;
        if (qv == INT_MAX) { finish(P, kOptimal, it, bland, degen, clk.acc); return; }
        if (it >= P.max_iters) { finish(P, kIterLimit, it, bland, degen, clk.acc); return; }
        phase_ratio(P, q, bland, s, TSX_RHS_PREFETCH ? &rhs0 : nullptr);   // Step 2 (block partials)
        clk.lap(0);
        if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(3);
        const RatPart l = phase_leaving(P, s);            // Step 2 (global)
        if (l.i == INT_MAX) { finish(P, kUnbounded, it, bland, degen, clk.acc); return; }
        const V piv = (V)l.a;   // the pivot element, carried by the partial
        if (!isfinite((double)piv) || !isfinite(l.r)) { finish(P, kNumeric, it, bland, degen, clk.acc); return; }
        phase_stage_row(P, l.i, q, piv);                  // Step 3 (pivot row)
        if (blockIdx.x == 0 && threadIdx.x == 0) record_pivot(P, it, q, qv, l.i);
        clk.lap(1);
        if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(4);
        phase_update<V, RS>(P, l.i, q, it, ringp);   // Step 3 (rank-1 update)
        ++it;
        degeneracy_step(P, l.r, bland, degen);
        clk.lap(2);
        if (!pivot_barrier(P.st, P.timeout_ns, s)) return;
        clk.lap(5);
    }
}

// ---- one launch per phase (same device functions; state in DevState)
template <typename V>
__global__ void k_ml_init(Params<V> P) {
    if (blockIdx.x == 0 && threadIdx.x == 0) P.st->bland = P.rule == 1 ? 1 : 0;
    phase_init_argmin(P);
}

template <int NT, typename V>
__global__ void __launch_bounds__(NT) k_ml_select(Params<V> P) {
    __shared__ BlockScratch s;
    if (P.st->status != kRunning) return;
    const int bland = P.st->bland;
    const long long it = P.st->iters;
    const ArgPart e = phase_entering(P, s);
    const int q = bland ? e.fslot : e.slot;
    const int qv = bland ? e.fkey : e.key;
    if (qv == INT_MAX || it >= P.max_iters) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicCAS(&P.st->status, kRunning, qv == INT_MAX ? kOptimal : kIterLimit);
        return;
    }
    phase_ratio(P, q, bland, s);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.st->q = q;
        P.st->qvar = qv;
    }
}

template <int NT, typename V>
__global__ void __launch_bounds__(NT) k_ml_stage(Params<V> P) {
    __shared__ BlockScratch s;
    if (P.st->status != kRunning) return;
    const RatPart l = phase_leaving(P, s);
    if (l.i == INT_MAX) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&P.st->status, kRunning, kUnbounded);
        return;
    }
    const V piv = (V)l.a;   // the pivot element, carried by the partial
    if (!isfinite((double)piv) || !isfinite(l.r)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&P.st->status, kRunning, kNumeric);
        return;
    }
    phase_stage_row(P, l.i, P.st->q, piv);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        record_pivot(P, P.st->iters, P.st->q, P.st->qvar, l.i);
        P.st->p = l.i;
        P.st->theta = l.r;
    }
}

template <int NT, typename V>
__global__ void __launch_bounds__(NT, 512 / NT) k_ml_update(Params<V> P) {
    if (P.st->status != kRunning) return;
    const int p = P.st->p;
    phase_update(P, p, P.st->q, P.st->iters);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int bland = P.st->bland, degen = P.st->degen_run;
        degeneracy_step(P, P.st->theta, bland, degen);
        P.st->bland = bland;
        P.st->degen_run = degen;
        P.st->iters += 1;
    }
}

// Solution read-out (Table I layout), widened to double: y_i = T[0][n+i],
// obj = T[0][W-1], x zeroed, then x[basis[i]] = T[i+1][W-1] for structural
// basics.
// Condensed tableau: y_i = 0 for basic slacks; the nonbasic slacks' entries
// are scattered by k_extract_y_cond afterwards.
template <typename V>
__global__ void k_extract_dense(int m, int n, int W, int ld, const V* __restrict__ T, int cond,
                                double* __restrict__ sol) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n + m + 1; k += gridDim.x * blockDim.x) {
        if (k < n)
            sol[k] = 0.0;
        else if (k < n + m)
            sol[k] = cond ? 0.0 : (double)T[n + (k - n)];
        else
            sol[k] = (double)T[W - 1];
    }
}

// Condensed tableau: y_i = T[0][j] for the slot j holding slack n + i.
template <typename V>
__global__ void k_extract_y_cond(int m, int n, const V* __restrict__ T, const int* __restrict__ var,
                                 double* __restrict__ sol) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int v = var[j];
        if (v >= n) sol[v] = (double)T[j];   // sol + n + (v - n)
    }
}

// Full (m+1) x (n+m+1) tableau widened to double from the condensed one:
// column var[j] <- slot j, column n+m <- the RHS, unit columns for the basic
// variables, zero elsewhere.  Two passes: zero-and-scatter of the stored
// columns (every output entry written once by its own thread), then the units.
template <typename V>
__global__ void k_expand_cond(int m, int n, int ld, const V* __restrict__ T, const int* __restrict__ var,
                              const int* __restrict__ slot_of, double* __restrict__ out) {
    const size_t W = (size_t)n + m + 1;
    const size_t total = (size_t)(m + 1) * W;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = t / W, col = t - i * W;
        double v = 0.0;
        if (col == W - 1)
            v = (double)T[i * (size_t)ld + n];
        else if (slot_of[col] >= 0)
            v = (double)T[i * (size_t)ld + slot_of[col]];
        out[t] = v;
    }
}

// slot_of[v] = the slot holding variable v, -1 if v is basic; then the basic
// variables' unit entries.
__global__ void k_slot_of(int m, int n, const int* __restrict__ var, int* __restrict__ slot_of) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n + m; v += gridDim.x * blockDim.x) slot_of[v] = -1;
}
__global__ void k_slot_of_set(int n, const int* __restrict__ var, int* __restrict__ slot_of) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) slot_of[var[j]] = j;
}
__global__ void k_expand_units(int m, int n, const int* __restrict__ basis, double* __restrict__ out) {
    const size_t W = (size_t)n + m + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        out[(size_t)(i + 1) * W + basis[i]] = 1.0;
}

template <typename V>
__global__ void k_extract_x(int m, int n, int W, int ld, const V* __restrict__ T, const int* __restrict__ basis,
                            double* __restrict__ sol) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int v = basis[i];
        if (v < n) sol[v] = (double)T[(size_t)(i + 1) * (size_t)ld + (W - 1)];
    }
}

// Tableau copy-out widened to double (row-major, W columns).
template <typename V>
__global__ void k_widen(int rows, int W, int ld, const V* __restrict__ T, double* __restrict__ out) {
    const size_t total = (size_t)rows * (size_t)W;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const size_t i = k / (size_t)W, j = k - i * (size_t)W;
        out[k] = (double)T[i * (size_t)ld + j];
    }
}

}  // namespace tsx
