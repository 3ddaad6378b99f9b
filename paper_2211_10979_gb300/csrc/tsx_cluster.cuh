// One LP solved by one thread-block cluster, its condensed tableau held in the
// cluster's distributed shared memory (the full-tableau simplex of arXiv
// 2211.10979, Section III, Steps 1-3; Section IV's split of the tableau over
// processors, here over the C <= 16 SMs of one cluster).
//
// For LPs whose pivots are too small to fill the GPU, the cost of a pivot on
// the grid-wide kernel is its fixed part: three device-wide barriers through
// L2 and the reductions' round trips (~20 us at m = n = 256, where the update
// itself moves 1 MB).  Here a cluster of C blocks keeps the tableau on chip
// and synchronises with the hardware cluster barrier:
//   - block r owns constraint rows [g0, g1) of the condensed tableau (the n
//     nonbasic columns plus the right-hand side, var[] giving each slot's
//     variable) in its shared memory, and every block keeps its own copy of
//     the objective row and of var[], updated identically, so every block
//     finds the same entering slot without an exchange (Step 1);
//   - Step 2: each block screens its rows in single precision and divides
//     the few rows that can hold the minimum (the screen of the batched
//     solver), and posts its best (ratio key, tie key, row, pivot element,
//     basic variable) in its shared memory;
//   - cluster barrier; every block reads the C posts through distributed
//     shared memory and takes the same minimum (row p, pivot element);
//   - Step 3, pivot row: block r divides its slice of row p (read from the
//     owner's shared memory) by the pivot element and stores that slice of R
//     into every block's shared memory;
//   - cluster barrier; every block updates its rows and its copy of row 0
//     over one flat index space (full warp instructions), and the new row 0
//     gives the next entering slot.
// Two cluster barriers per pivot.  Every value is computed by the same
// operations as in the other kernels (one IEEE division per R entry and per
// ratio, one fused multiply-add per updated entry, decisions on the correctly
// rounded values), so pivots and results are lp_solve's on every path.
// The cluster's blocks are co-scheduled by the hardware; they pass every
// barrier the same number of times (all decisions are taken on identical
// data), so no wait can be left without its partners.
#pragma once

#include <cstddef>

#include "tsx_select.cuh"

namespace tsx {

constexpr int kClusterMax = 16;

struct ClusterParams {
    double* T;                 // the handle's condensed tableau (built), (m+1) x ldg
    int ldg;
    int m, n;
    int* basis;                // m: variable basic in row i+1
    int* var;                  // n: variable held by each column slot
    DevState* st;
    int* qlog;                 // pivot log (may be null)
    int* plog;
    long long log_cap;
    double eps_d, eps_p;
    long long max_iters;       // < 0: 50 (m + n)
    int k_cyc, rule;
};

struct CRat {                  // a block's Step 2 result, read by the cluster
    long long rk;              // dkey of the minimum ratio, kKeyInf if none
    int key;                   // tie-break key (row, or basic variable in Bland mode)
    int i;                     // its row, INT_MAX if none
    double a;                  // its pivot element
    int bvar;                  // the variable basic in row i (the leaving variable)
    int pad;
};

__device__ __forceinline__ void crat_merge(CRat& a, const CRat& b) {
    if (b.rk < a.rk || (b.rk == a.rk && b.key < a.key)) a = b;
}

__device__ __forceinline__ CRat warp_crat(CRat a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CRat b;
        b.rk = __shfl_xor_sync(0xffffffffu, a.rk, o);
        b.key = __shfl_xor_sync(0xffffffffu, a.key, o);
        b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
        b.a = __shfl_xor_sync(0xffffffffu, a.a, o);
        b.bvar = __shfl_xor_sync(0xffffffffu, a.bvar, o);
        crat_merge(a, b);
    }
    return a;
}

// ---- distributed shared memory (sm_90+ cluster PTX) -----------------------
__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Barrier of every thread of every block of the cluster; the arrive releases
// this thread's shared-memory writes (local and remote), the wait acquires the
// others'.
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// Address of the same shared-memory location in block `rank` of the cluster.
__device__ __forceinline__ unsigned cl_map(unsigned addr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ double cl_ld_f64(unsigned a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ long long cl_ld_s64(unsigned a) {
    long long v;
    asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int cl_ld_s32(unsigned a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void cl_st_f64(unsigned a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// Rows of block r among C: constraint rows [g0, g1) of 1..m.
__host__ __device__ __forceinline__ int cluster_rows_per(int m, int C) { return (m + C - 1) / C; }

__host__ __device__ inline int cluster_ldc(int n) { return (n + 1) | 1; }

// Dynamic shared memory of one block: [row 0 | own rows] (stride ldc), R,
// F (row 0 + own rows), var, own basis, candidate list.
__host__ __device__ inline size_t cluster_smem_bytes(int m, int n, int C) {
    const int ldc = cluster_ldc(n), per = cluster_rows_per(m, C);
    size_t bytes = (size_t)(per + 1) * ldc * 8 + (size_t)ldc * 8 + (size_t)(per + 1) * 8;
    bytes += (size_t)n * 4 + (size_t)per * 4 + (size_t)per * 4;
    return (bytes + 15) / 16 * 16;
}

struct ClusterScratch {
    BArg arg[kMaxWarps];
    CRat part;                 // this block's Step 2 result (read remotely)
    CRat merged;               // the cluster's minimum
    int ncand;
};

template <int NT>
__global__ void __launch_bounds__(NT) k_cluster_solve(ClusterParams P) {
    static_assert(NT >= 64, "warp 0 takes the objective row, the others the constraint rows");
    extern __shared__ __align__(16) unsigned char cl_smem[];
    __shared__ ClusterScratch sc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned me = cl_rank(), C = cl_size();
    const int m = P.m, n = P.n, ldc = cluster_ldc(n), W1 = n + 1;
    const int per = cluster_rows_per(m, (int)C);
    const int g0 = min(m + 1, 1 + (int)me * per), g1 = min(m + 1, g0 + per);
    const int nr = g1 - g0;   // own constraint rows: local rows 1..nr
    double* Tl = reinterpret_cast<double*>(cl_smem);          // local row 0 = objective row
    double* R = Tl + (size_t)(per + 1) * ldc;
    double* F = R + ldc;                                       // F[l], local rows
    int* var = reinterpret_cast<int*>(F + (per + 1));
    int* bas = var + n;                                        // own rows' basic variables
    int* cand = bas + per;
    const long long epsk = dkey(-P.eps_d);
    const long long eps_bits = max(0LL, (long long)__double_as_longlong(P.eps_p));

    // load the built tableau: row 0 and the own rows, var[], own basis
    for (long long t = tid; t < (long long)(nr + 1) * W1; t += NT) {
        const int l = (int)(t / W1), j = (int)(t - (long long)l * W1);
        const int g = l == 0 ? 0 : g0 + l - 1;
        Tl[(size_t)l * ldc + j] = P.T[(size_t)g * P.ldg + j];
    }
    for (int j = tid; j < n; j += NT) var[j] = P.var[j];
    for (int l = tid; l < nr; l += NT) bas[l] = P.basis[g0 + l - 1];
    if (tid == 0) sc.ncand = 0;
    __syncthreads();
    // Step 1 of the first pivot on the local copy of row 0 (warp 0)
    if (warp == 0) {
        BArg a0 = barg_none();
        for (int j = lane; j < n; j += 32) barg_consider_key(a0, Tl[j], var[j], j, epsk);
        a0 = warp_barg(a0);
        if (lane == 0) sc.arg[0] = a0;
    }
    // every block has started before any distributed shared-memory access
    cl_sync();

    const long long cap = P.max_iters < 0 ? 50LL * (m + n) : P.max_iters;
    int status = kRunning;
    long long it = 0;
    int bland = P.rule == 1, degen = 0;
    // the update's flat index space over the own rows 1..nr, warps 1..NW-1
    constexpr int NU = NT - 32;
    const int tu = tid - 32;
    const int i_first = 1 + (tu >= 0 ? tu / W1 : 0), j_first = tu >= 0 ? tu - (tu / W1) * W1 : 0;
    const int di = NU / W1, dj = NU - (NU / W1) * W1;
    // block 0's time per phase (thread 0): Step 2, wait at barrier 1, the
    // cluster minimum and R slices, wait at barrier 2, Step 3, and Step 1
    long long ph[6] = {0, 0, 0, 0, 0, 0};
    long long tph = (me == 0 && tid == 0) ? global_ns() : 0;
    auto mark = [&](int k) {
        if (me == 0 && tid == 0) {
            const long long t = global_ns();
            ph[k] += t - tph;
            tph = t;
        }
    };
    const int sl = (W1 + (int)C - 1) / (int)C;                 // R slice per block
    const int j0 = min(W1, (int)me * sl), j1 = min(W1, j0 + sl);
    while (status == kRunning) {
        // Step 1 (identical in every block): warp 0's result on row 0
        const BArg a = sc.arg[0];
        const int qs = bland ? a.fslot : a.slot;
        mark(5);
        if (qs < 0) { status = kOptimal; break; }
        if (it >= cap) { status = kIterLimit; break; }
        // Step 2 on the own rows.  Up to 32 rows: warp 0 divides every
        // eligible row itself.  More: single-precision screen, then exact
        // divisions of the candidates by warp 0.
        if (nr <= 32) {
            if (warp == 0) {
                if (lane == 0) F[0] = Tl[qs];
                CRat best{kKeyInf, INT_MAX, INT_MAX, 0.0, 0, 0};
                const int l = 1 + lane;
                if (l <= nr) {
                    const double av = Tl[(size_t)l * ldc + qs];
                    F[l] = av;
                    if (eligible_bits(av, eps_bits)) {
                        const double r = __ddiv_rn(Tl[(size_t)l * ldc + n], av);
                        if (!dbits_nan(r)) {
                            const int g = g0 + l - 1;
                            best = CRat{dkey(r), bland ? bas[l - 1] : g, g, av, bas[l - 1], 0};
                        }
                    }
                }
                best = warp_crat(best);
                if (lane == 0) sc.part = best;
            }
        } else {
        if (tid == 0) F[0] = Tl[qs];
        float emin = __int_as_float(0x7f800000);
        for (int l = 1 + tid; l <= nr; l += NT) {
            const double av = Tl[(size_t)l * ldc + qs];
            F[l] = av;
            float est;
            if (eligible_bits(av, eps_bits) && ratio_estimate(Tl[(size_t)l * ldc + n], av, est))
                emin = fminf(emin, est);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emin = fminf(emin, __shfl_xor_sync(0xffffffffu, emin, o));
        const float band = __fmul_ru(emin, 1.0f + 0x1p-18f);
        for (int base = 1 + warp * 32; base <= nr; base += NT) {
            const int l = base + lane;
            bool keep = false;
            if (l <= nr) {
                const double av = F[l];
                if (eligible_bits(av, eps_bits)) {
                    float est;
                    keep = !ratio_estimate(Tl[(size_t)l * ldc + n], av, est) || est <= band;
                }
            }
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            if (ball) {
                int at = 0;
                if (lane == 0) at = atomicAdd(&sc.ncand, __popc(ball));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (keep) cand[at + __popc(ball & ((1u << lane) - 1u))] = l;
            }
        }
        __syncthreads();
        if (warp == 0) {
            CRat best{kKeyInf, INT_MAX, INT_MAX, 0.0, 0, 0};
            const int nc = sc.ncand;
            for (int t = lane; t < nc; t += 32) {
                const int l = cand[t];
                const double av = F[l];
                const double r = __ddiv_rn(Tl[(size_t)l * ldc + n], av);
                if (!dbits_nan(r)) {
                    const int g = g0 + l - 1;
                    CRat cnd{dkey(r), bland ? bas[l - 1] : g, g, av, bas[l - 1], 0};
                    crat_merge(best, cnd);
                }
            }
            best = warp_crat(best);
            if (lane == 0) {
                sc.part = best;
                sc.ncand = 0;
            }
        }
        }
        mark(0);
        cl_sync();   // #1: every block's Step 2 result is posted
        mark(1);
        // the cluster's minimum: lane r of warp 0 reads block r's post
        if (warp == 0) {
            CRat b{kKeyInf, INT_MAX, INT_MAX, 0.0, 0, 0};
            if (lane < (int)C) {
                const unsigned base = cl_map(smem_addr(&sc.part), (unsigned)lane);
                b.rk = cl_ld_s64(base + offsetof(CRat, rk));
                b.key = cl_ld_s32(base + offsetof(CRat, key));
                b.i = cl_ld_s32(base + offsetof(CRat, i));
                b.a = cl_ld_f64(base + offsetof(CRat, a));
                b.bvar = cl_ld_s32(base + offsetof(CRat, bvar));
            }
            b = warp_crat(b);
            if (lane == 0) sc.merged = b;
        }
        __syncthreads();
        const CRat best = sc.merged;
        if (best.i == INT_MAX) { status = kUnbounded; break; }
        const int p = best.i;
        const double piv = best.a;
        const double ratio = dkey_value(best.rk);
        if (!dbits_finite(piv) || !dbits_finite(ratio)) { status = kNumeric; break; }
        const unsigned owner = (unsigned)((p - 1) / per);
        const int pl = p - (1 + (int)owner * per) + 1;             // local row of p at its owner
        // Step 3, pivot row: this block's slice of R from row p at the owner
        for (int j = j0 + tid; j < j1; j += NT) {
            const double v = cl_ld_f64(cl_map(smem_addr(Tl + (size_t)pl * ldc + j), owner));
            R[j] = __ddiv_rn(j == qs ? 1.0 : v, piv);   // one division, whichever operand
        }
        __syncthreads();
        for (int t = tid; t < (j1 - j0) * (int)C; t += NT) {
            const int j = j0 + t / (int)C;
            const unsigned rr = (unsigned)(t - (j - j0) * (int)C);
            if (rr != me) cl_st_f64(cl_map(smem_addr(R + j), rr), R[j]);
        }
        const int entering = var[qs];
        if (tid == 0) {
            if (me == 0 && P.qlog && it < P.log_cap) {
                P.qlog[it] = entering;
                P.plog[it] = p;
            }
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
        mark(2);
        cl_sync();   // #2: R is complete in every block; row p and the posts have been read
        mark(3);
        if (tid == 0) {
            var[qs] = best.bvar;                                   // the leaving variable takes slot qs
            if (owner == me) bas[pl - 1] = entering;
        }
        // Step 3, update of row 0 and the own rows over one flat index space;
        // the owner's row p becomes R
        const int plocal = owner == me ? pl : -1;
        __syncthreads();   // var[qs] is read by the objective-row candidates
        if (warp == 0) {
            // row 0 and the next Step 1
            BArg an = barg_none();
            const double f0 = F[0];
            for (int j = lane; j < W1; j += 32) {
                const double v = __fma_rn(-f0, R[j], j == qs ? 0.0 : Tl[j]);
                Tl[j] = v;
                if (j < n) barg_consider_key(an, v, var[j], j, epsk);
            }
            an = warp_barg_rule(an, bland);   // the next Step 1 reads these fields only
            if (lane == 0) sc.arg[0] = an;
        } else {
            // the own constraint rows, flat over warps 1..NW-1
            flat_update(Tl, ldc, nr, W1, n, F, R, qs, plocal, var, epsk, i_first, j_first, di, dj);
        }
        __syncthreads();
        mark(4);
    }
    // write back: own rows (block 0 also row 0 and var), own basis, state
    for (long long t = tid; t < (long long)(nr + 1) * W1; t += NT) {
        const int l = (int)(t / W1), j = (int)(t - (long long)l * W1);
        if (l == 0 && me != 0) continue;
        const int g = l == 0 ? 0 : g0 + l - 1;
        P.T[(size_t)g * P.ldg + j] = Tl[(size_t)l * ldc + j];
    }
    if (me == 0)
        for (int j = tid; j < n; j += NT) P.var[j] = var[j];
    for (int l = tid; l < nr; l += NT) P.basis[g0 + l - 1] = bas[l];
    if (me == 0 && tid == 0) {
        P.st->status = status;
        P.st->iters = it;
        P.st->bland = bland;
        P.st->degen_run = degen;
        P.st->active_sectors = (unsigned long long)it * (unsigned long long)(P.ldg / 4);
        for (int k = 0; k < 6; ++k) P.st->phase_ns[k] = ph[k];
    }
    // no block leaves while another may still read its shared memory
    cl_sync();
}

}  // namespace tsx
