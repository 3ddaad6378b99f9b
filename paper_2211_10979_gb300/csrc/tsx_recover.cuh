// FP64 recovery of an LP solved on a float tableau.
//
// The float pivots (Section III Steps 1-3 on a float tableau) end at a basis;
// its exact meaning is recomputed here in double precision from the original
// data, and checked.  With S = structural basic variables (k of them), Z = the
// constraints whose slack is basic and R = the other k constraints (their slack
// is nonbasic, the constraint is tight), the basis matrix has the block form
//     B = [A_RS 0; A_ZS I]   so   B^-1 = [A_RS^-1 0; -A_ZS A_RS^-1 I],
// and everything needs only the k x k block A_RS:
//     x_S = A_RS^-1 b_R,  s_Z = b_Z - A_ZS x_S,  y_R = A_RS^-T c_S,  y_Z = 0,
//     objective-row entries d_j = (A^T y)_j - c_j (structural), y_r (slacks).
// Optimal iff x_S, s_Z >= -tol and d_j, y_R >= -tol.  Otherwise cleanup pivots
// in this revised form: primal (an entry d < -tol enters; column B^-1 a_q;
// minimum-ratio test) or dual (a basic value < -tol leaves; row of B^-1 [A I];
// dual ratio test).  A_RS^-1 comes from Gauss-Jordan elimination with partial
// pivoting in a cooperative kernel (one grid barrier per column).
#pragma once

#include "tsx_device.cuh"

namespace tsx {

struct RecCheck {
    double min_x;  int min_x_at;     // smallest x_S entry, its position in S
    double min_s;  int min_s_at;     // smallest basic slack s_i (i in Z), its row i
    double min_d;  int min_d_at;     // most negative d_j over nonbasic structural j
    double min_y;  int min_y_at;     // most negative y_r over r in R (position in R)
    double cx, by;                   // c^T x and b^T y
    double res_p, res_d;             // max |b_R - A_RS x_S|, max |c_S - A_RS^T y_R|
};

// M = [A_RS | I_k], k x 2k row-major.
__global__ void k_rec_gather(int n, const double* __restrict__ A, const int* __restrict__ S,
                             const int* __restrict__ Rr, int k, double* __restrict__ M) {
    const size_t total = (size_t)k * 2 * k;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / (2 * (size_t)k)), b = (int)(t - (size_t)a * 2 * k);
        M[t] = b < k ? A[(size_t)Rr[a] * n + S[b]] : (b - k == a ? 1.0 : 0.0);
    }
}

struct PivPart {
    double v;   // |pivot candidate|
    int r;      // its row (lowest on ties), INT_MAX if none
};

__device__ __forceinline__ void piv_merge(PivPart& a, const PivPart& b) {
    if (b.v > a.v || (b.v == a.v && b.r < a.r)) a = b;
}

// Gauss-Jordan elimination of M = [A_RS | I] (k x 2k), cooperative.  Column c:
// every block picks the same pivot row (largest |M[r][c]| among rows not used
// yet, lowest row on ties), then the other rows subtract their multiple of the
// pivot row on columns > c.  Rows are not swapped (pivrow[c] records the row)
// and the pivot rows are scaled at the end (k_rec_finish).  Sets *singular if a
// pivot is zero.  Each block keeps the used rows in its own shared-memory
// bitmap (ceil(k / 32) words of dynamic shared memory), so no block's choice
// can see a later step's mark.
template <int NT>
__global__ void __launch_bounds__(NT) k_rec_gauss_jordan(double* M, int k, int* pivrow, int* singular,
                                                        DevState* st, long long timeout_ns) {
    __shared__ PivPart sp[NT / 32];
    __shared__ PivPart sbest;
    __shared__ BlockScratch s;
    extern __shared__ unsigned used_bits[];
    const size_t w2 = 2 * (size_t)k;
    const int nwords = (k + 31) / 32;
    for (int w = threadIdx.x; w < nwords; w += NT) used_bits[w] = 0u;
    __syncthreads();
    for (int c = 0; c < k; ++c) {
        PivPart best{-1.0, INT_MAX};
        for (int r = threadIdx.x; r < k; r += NT)
            if (!((used_bits[r >> 5] >> (r & 31)) & 1u)) piv_merge(best, PivPart{fabs(__ldcg(M + r * w2 + c)), r});
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            PivPart b{__shfl_xor_sync(0xffffffffu, best.v, o), __shfl_xor_sync(0xffffffffu, best.r, o)};
            piv_merge(best, b);
        }
        if ((threadIdx.x & 31) == 0) sp[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            PivPart b = sp[0];
            for (int w = 1; w < NT / 32; ++w) piv_merge(b, sp[w]);
            sbest = b;
        }
        __syncthreads();
        const int pr = sbest.r;
        if (pr == INT_MAX || !(sbest.v > 0.0)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *singular = 1;
            return;   // every block takes the same branch
        }
        const double ip = 1.0 / __ldcg(M + pr * w2 + c);
        const size_t width = w2 - (size_t)c - 1;
        const size_t total = (size_t)k * width;
        for (size_t t = (size_t)blockIdx.x * NT + threadIdx.x; t < total; t += (size_t)gridDim.x * NT) {
            const size_t r = t / width, j = c + 1 + (t - r * width);
            if ((int)r == pr) continue;
            const double l = __ldcg(M + r * w2 + c) * ip;
            if (l != 0.0) M[r * w2 + j] = __fma_rn(-l, __ldcg(M + pr * w2 + j), __ldcg(M + r * w2 + j));
        }
        if (threadIdx.x == 0) {
            used_bits[pr >> 5] |= 1u << (pr & 31);   // this block's copy; read after the barrier
            if (blockIdx.x == 0) pivrow[c] = pr;
        }
        if (!grid_barrier(st, timeout_ns, s)) return;
    }
}

// The same elimination in place on the k x k block (the default): step c
// frees column c of M, which then holds the right-hand column of the pivot
// row pr_c, i.e. what column k + pr_c of [A_RS | I] would hold (that column is
// the unit vector of row pr_c until step c: M[pr_c][c] becomes 1, and every
// other row r gets fma(-l_r, 1, 0) = -l_r).  Every stored value goes through
// the same operations as in k_rec_gauss_jordan, in k^3 instead of 1.5 k^3
// fused multiply-adds and half the memory.  A warp updates one row at a time
// (its multiplier l_r = M[r][c] / M[pr][c] computed once), the pivot row is
// staged in shared memory, and the next column's pivot search rides on the
// update: each block posts its best (|M[r][c+1]|, r) over its unused rows, so
// a step has one grid barrier.  dpiv[c] = the pivot element of step c.
struct PivVal {
    double v;     // |pivot candidate|, -1 if none
    double val;   // its signed value
    int r;        // its row (lowest on ties), INT_MAX if none
    int pad;
};

__device__ __forceinline__ void pivval_merge(PivVal& a, const PivVal& b) {
    if (b.v > a.v || (b.v == a.v && b.r < a.r)) a = b;
}

__device__ __forceinline__ PivVal warp_pivval(PivVal a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        PivVal b;
        b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
        b.val = __shfl_xor_sync(0xffffffffu, a.val, o);
        b.r = __shfl_xor_sync(0xffffffffu, a.r, o);
        pivval_merge(a, b);
    }
    return a;
}

template <int NT>
__device__ __forceinline__ void block_post_pivval(PivVal a, PivVal* sp, PivVal* dst) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_pivval(a);
    if (lane == 0) sp[w] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        PivVal b = sp[0];
        for (int q = 1; q < NT / 32; ++q) pivval_merge(b, sp[q]);
        *dst = b;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_rec_gj_inplace(double* M, int k, int* pivrow, double* dpiv, PivVal* parts,
                                                      int* singular, DevState* st, long long timeout_ns) {
    __shared__ PivVal sp[NT / 32];
    __shared__ BlockScratch s;
    extern __shared__ double gj_smem[];
    double* P = gj_smem;                                            // pivot row, k entries
    unsigned* used_bits = reinterpret_cast<unsigned*>(P + k);      // rows used as pivots
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (NT / 32) + warp, nwarps = gridDim.x * (NT / 32);
    const size_t kk = (size_t)k;
    const int nwords = (k + 31) / 32;
    for (int w = threadIdx.x; w < nwords; w += NT) used_bits[w] = 0u;
    // pivot search of column 0
    {
        PivVal best{-1.0, 0.0, INT_MAX, 0};
        for (int r = blockIdx.x * NT + threadIdx.x; r < k; r += gridDim.x * NT) {
            const double v = __ldcg(M + r * kk);
            pivval_merge(best, PivVal{fabs(v), v, r, 0});
        }
        block_post_pivval<NT>(best, sp, parts + blockIdx.x);
    }
    if (!grid_barrier(st, timeout_ns, s)) return;
    for (int c = 0; c < k; ++c) {
        const PivVal* cur = parts + (size_t)(c & 1) * gridDim.x;
        PivVal* nxt = parts + (size_t)((c + 1) & 1) * gridDim.x;
        // the pivot of column c: warp 0 of every block merges the same posts
        if (warp == 0) {
            PivVal pv{-1.0, 0.0, INT_MAX, 0};
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const PivVal q{__ldcg(&cur[b].v), __ldcg(&cur[b].val), __ldcg(&cur[b].r), 0};
                pivval_merge(pv, q);
            }
            pv = warp_pivval(pv);
            if (lane == 0) sp[0] = pv;
        }
        __syncthreads();
        const PivVal pv = sp[0];
        __syncthreads();   // sp is written again by this step's post
        const int pr = pv.r;
        if (pr == INT_MAX || !(pv.v > 0.0)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *singular = 1;
            return;   // every block takes the same branch
        }
        const double ip = 1.0 / pv.val;
        for (int j = threadIdx.x; j < k; j += NT) P[j] = j == c ? 1.0 : __ldcg(M + pr * kk + j);
        if (threadIdx.x == 0) used_bits[pr >> 5] |= 1u << (pr & 31);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            pivrow[c] = pr;
            dpiv[c] = pv.val;
        }
        __syncthreads();
        PivVal best{-1.0, 0.0, INT_MAX, 0};
        const int cn = c + 1;
        for (int r = gw; r < k; r += nwarps) {
            double* row = M + r * kk;
            if (r == pr) {
                if (lane == 0) row[c] = 1.0;
                continue;
            }
            const double l = __ldcg(row + c) * ip;
            const bool unused = !((used_bits[r >> 5] >> (r & 31)) & 1u);
            // eight entries per lane in flight: all loads of a chunk before its stores
            for (int j0 = lane; j0 < k; j0 += 32 * 8) {
                double v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = j0 + 32 * u;
                    v[u] = j < k ? __ldcg(row + j) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = j0 + 32 * u;
                    if (j < k) row[j] = __fma_rn(-l, P[j], j == c ? 0.0 : v[u]);
                }
            }
            // the next column's candidate of this row, read back once (no
            // predicated FP64 work inside the loop above)
            __syncwarp();
            if (lane == 0 && unused && cn < k) {
                const double w = row[cn];
                pivval_merge(best, PivVal{fabs(w), w, r, 0});
            }
        }
        if (cn < k) block_post_pivval<NT>(best, sp, nxt + blockIdx.x);
        if (!grid_barrier(st, timeout_ns, s)) return;
    }
}

// inv[c][a] = M[pivrow[c]][pivstep[a]] / dpiv[c] (pivstep = the inverse of
// pivrow): the rows of A_RS^-1 from the in-place elimination.
__global__ void k_rec_finish_inplace(const double* __restrict__ M, int k, const int* __restrict__ pivrow,
                                     const int* __restrict__ pivstep, const double* __restrict__ dpiv,
                                     double* __restrict__ inv) {
    const size_t total = (size_t)k * k;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / k), a = (int)(t - (size_t)c * k);
        inv[t] = M[(size_t)pivrow[c] * k + pivstep[a]] / dpiv[c];
    }
}

__global__ void k_rec_pivstep(const int* __restrict__ pivrow, int k, int* __restrict__ pivstep) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) pivstep[pivrow[c]] = c;
}

// M = A_RS, k x k row-major.
__global__ void k_rec_gather_square(int n, const double* __restrict__ A, const int* __restrict__ S,
                                    const int* __restrict__ Rr, int k, double* __restrict__ M) {
    const size_t total = (size_t)k * k;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / k), b = (int)(t - (size_t)a * k);
        M[t] = A[(size_t)Rr[a] * n + S[b]];
    }
}

// inv[c][a] = M[pivrow[c]][k + a] / M[pivrow[c]][c]: the rows of A_RS^-1.
__global__ void k_rec_finish(const double* __restrict__ M, int k, const int* __restrict__ pivrow,
                             double* __restrict__ inv) {
    const size_t total = (size_t)k * k;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / k), a = (int)(t - (size_t)c * k);
        const size_t pr = (size_t)pivrow[c];
        const double* row = M + pr * 2 * (size_t)k;
        inv[t] = row[k + a] / row[c];
    }
}

// out[c] = sum_a inv[c][a] v[a] (trans = 0) or sum_a inv[a][c] v[a] (trans = 1);
// if acc != null: out = acc + that (refinement).
__global__ void k_rec_matvec(const double* __restrict__ inv, int k, const double* __restrict__ v, int trans,
                             const double* __restrict__ acc, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    if (!trans) {   // one warp per output entry (rows of inv are contiguous)
        const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
        for (long long c = w; c < k; c += nw) {
            double sum = 0.0;
            for (int a = lane; a < k; a += 32) sum = __fma_rn(inv[(size_t)c * k + a], v[a], sum);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) out[c] = acc ? acc[c] + sum : sum;
        }
    } else {        // one thread per output entry (columns: coalesced across threads)
        for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (long long)gridDim.x * blockDim.x) {
            double sum = 0.0;
            for (int a = 0; a < k; ++a) sum = __fma_rn(inv[(size_t)a * k + c], v[a], sum);
            out[c] = acc ? acc[c] + sum : sum;
        }
    }
}

// Right-hand sides: bR[a] = b[R[a]], cS[b] = c[S[b]].
__global__ void k_rec_gather_rhs(const double* __restrict__ b, const double* __restrict__ c, const int* __restrict__ S,
                                 const int* __restrict__ Rr, int k, double* __restrict__ bR, double* __restrict__ cS) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        bR[t] = b[Rr[t]];
        cS[t] = c[S[t]];
    }
}

// Residuals for one refinement step: rp[a] = b_R[a] - sum_b A[R[a]][S[b]] x_S[b],
// rd[b] = c_S[b] - sum_a A[R[a]][S[b]] y_R[a].  One warp per entry.
__global__ void k_rec_residual(int n, const double* __restrict__ A, const int* __restrict__ S, const int* __restrict__ Rr,
                               int k, const double* __restrict__ bR, const double* __restrict__ cS,
                               const double* __restrict__ xS, const double* __restrict__ yR,
                               double* __restrict__ rp, double* __restrict__ rd) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = w; t < 2LL * k; t += nw) {
        double sum = 0.0;
        if (t < k) {
            const double* row = A + (size_t)Rr[t] * n;
            for (int b2 = lane; b2 < k; b2 += 32) sum = __fma_rn(row[S[b2]], xS[b2], sum);
        } else {
            const int col = S[t - k];
            for (int a = lane; a < k; a += 32) sum = __fma_rn(A[(size_t)Rr[a] * n + col], yR[a], sum);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            if (t < k) rp[t] = bR[t] - sum;
            else rd[t - k] = cS[t - k] - sum;
        }
    }
}

// Slacks of every constraint: s_i = b_i - sum_b A[i][S[b]] x_S[b] (one warp per row).
// With col != null, also alpha_Z: out2[i] = colv_i - sum_b A[i][S[b]] w[b]
// where colv_i = A[i][col_j] (structural entering) or 0 (slack entering).
__global__ void k_rec_rows_dot(int m, int n, const double* __restrict__ A, const int* __restrict__ S, int k,
                               const double* __restrict__ base, int base_col, const double* __restrict__ w,
                               double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long wi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = wi; i < m; i += nw) {
        const double* row = A + (size_t)i * n;
        double sum = 0.0;
        for (int b2 = lane; b2 < k; b2 += 32) sum = __fma_rn(row[S[b2]], w[b2], sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            const double b0 = base ? base[i] : (base_col >= 0 ? row[base_col] : 0.0);
            out[i] = b0 - sum;
        }
    }
}

// Columns of the objective row (or of any tableau row given its B^-1 row rho
// restricted to R): out[j] = sum_a rho[a] A[R[a]][j] + extra_row_j - cj, where
// extra_row_j = A[extra_row][j] if extra_row >= 0 and cj = c[j] if c != null.
// One thread per structural column j (coalesced along rows of A).
__global__ void k_rec_cols_dot(int n, const double* __restrict__ A, const int* __restrict__ Rr, int k,
                               const double* __restrict__ rho, int extra_row, const double* __restrict__ c,
                               double* __restrict__ out) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        double sum = extra_row >= 0 ? A[(size_t)extra_row * n + j] : 0.0;
        for (int a = 0; a < k; ++a) sum = __fma_rn(A[(size_t)Rr[a] * n + j], rho[a], sum);
        out[j] = c ? sum - c[j] : sum;
    }
}

// Basic-status flags: isbasic[v] for variables v < n + m; inR[i] for rows.
__global__ void k_rec_flags(int m, int n, const int* __restrict__ S, const int* __restrict__ Rr, int k,
                            int* __restrict__ isbasic, int* __restrict__ inR) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n + m; t += gridDim.x * blockDim.x) {
        isbasic[t] = t < n ? 0 : 1;   // slacks basic unless their row is in R
        if (t < m) inR[t] = 0;
    }
}
__global__ void k_rec_flags2(int m, int n, const int* __restrict__ S, const int* __restrict__ Rr, int k,
                             int* __restrict__ isbasic, int* __restrict__ inR) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        isbasic[S[t]] = 1;
        isbasic[n + Rr[t]] = 0;
        inR[Rr[t]] = 1;
    }
}

// The optimality checks, one block: minima (lowest index on ties) of x_S, of
// the basic slacks, of d over nonbasic structural columns and of y_R, plus
// c^T x, b^T y and the residual maxima.
template <int NT>
__global__ void __launch_bounds__(NT) k_rec_check(int m, int n, const int* __restrict__ S, const int* __restrict__ Rr,
                                                 int k, const double* __restrict__ xS, const double* __restrict__ s,
                                                 const double* __restrict__ d, const double* __restrict__ yR,
                                                 const int* __restrict__ isbasic, const int* __restrict__ inR,
                                                 const double* __restrict__ b, const double* __restrict__ c,
                                                 const double* __restrict__ rp, const double* __restrict__ rd,
                                                 RecCheck* out) {
    __shared__ double sv[4][NT / 32];
    __shared__ int si[4][NT / 32];
    __shared__ double ss[4][NT / 32];
    double v[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
    int ix[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // cx, by, res_p, res_d
    auto take = [&](int q, double val, int at) {
        if (val < v[q] || (val == v[q] && at < ix[q])) { v[q] = val; ix[q] = at; }
    };
    for (int t = threadIdx.x; t < k; t += NT) {
        take(0, xS[t], t);
        take(3, yR[t], t);
        acc[0] = __fma_rn(c[S[t]], xS[t], acc[0]);
        acc[1] = __fma_rn(b[Rr[t]], yR[t], acc[1]);
        acc[2] = fmax(acc[2], fabs(rp[t]));
        acc[3] = fmax(acc[3], fabs(rd[t]));
    }
    for (int i = threadIdx.x; i < m; i += NT)
        if (!inR[i]) take(1, s[i], i);
    for (int j = threadIdx.x; j < n; j += NT)
        if (!isbasic[j]) take(2, d[j], j);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, v[q], o);
            const int oi = __shfl_xor_sync(0xffffffffu, ix[q], o);
            if (ov < v[q] || (ov == v[q] && oi < ix[q])) { v[q] = ov; ix[q] = oi; }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
        acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
        acc[2] = fmax(acc[2], __shfl_xor_sync(0xffffffffu, acc[2], o));
        acc[3] = fmax(acc[3], __shfl_xor_sync(0xffffffffu, acc[3], o));
    }
    if (lane == 0)
        for (int q = 0; q < 4; ++q) {
            sv[q][w] = v[q];
            si[q][w] = ix[q];
            ss[q][w] = acc[q];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        RecCheck r;
        double bv[4];
        int bi[4];
        double ba[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q = 0; q < 4; ++q) {
            bv[q] = INFINITY;
            bi[q] = INT_MAX;
            for (int ww = 0; ww < NT / 32; ++ww) {
                if (sv[q][ww] < bv[q] || (sv[q][ww] == bv[q] && si[q][ww] < bi[q])) { bv[q] = sv[q][ww]; bi[q] = si[q][ww]; }
                if (q < 2) ba[q] += ss[q][ww];
                else ba[q] = fmax(ba[q], ss[q][ww]);
            }
        }
        r.min_x = bv[0]; r.min_x_at = bi[0];
        r.min_s = bv[1]; r.min_s_at = bi[1];
        r.min_d = bv[2]; r.min_d_at = bi[2];
        r.min_y = bv[3]; r.min_y_at = bi[3];
        r.cx = ba[0]; r.by = ba[1]; r.res_p = ba[2]; r.res_d = ba[3];
        *out = r;
    }
}

struct RecChoice {
    double ratio;
    int kind;    // 0: position in S (structural basic / entering), 1: row i (slack), -1: none
    int at;
};

// Primal ratio test over the basic variables: min value/alpha over alpha > eps,
// ties to the lowest variable index (S[b], or n + i for the slack of row i).
template <int NT>
__global__ void __launch_bounds__(NT) k_rec_primal_ratio(int m, int n, const int* __restrict__ S, int k,
                                                        const double* __restrict__ xS, const double* __restrict__ aS,
                                                        const double* __restrict__ s, const double* __restrict__ aZ,
                                                        const int* __restrict__ inR, double eps, RecChoice* out) {
    __shared__ double sr[NT / 32];
    __shared__ int sv[NT / 32], sk[NT / 32], sa[NT / 32];
    double best = INFINITY;
    int bvar = INT_MAX, bkind = -1, bat = -1;
    auto take = [&](double r, int var, int kind, int at) {
        if (r < best || (r == best && var < bvar)) { best = r; bvar = var; bkind = kind; bat = at; }
    };
    for (int t = threadIdx.x; t < k; t += NT)
        if (aS[t] > eps) take(xS[t] / aS[t], S[t], 0, t);
    for (int i = threadIdx.x; i < m; i += NT)
        if (!inR[i] && aZ[i] > eps) take(s[i] / aZ[i], n + i, 1, i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double orr = __shfl_xor_sync(0xffffffffu, best, o);
        const int ov = __shfl_xor_sync(0xffffffffu, bvar, o);
        const int ok2 = __shfl_xor_sync(0xffffffffu, bkind, o);
        const int oa = __shfl_xor_sync(0xffffffffu, bat, o);
        if (orr < best || (orr == best && ov < bvar)) { best = orr; bvar = ov; bkind = ok2; bat = oa; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sr[w] = best; sv[w] = bvar; sk[w] = bkind; sa[w] = bat; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < NT / 32; ++ww)
            if (sr[ww] < sr[0] || (sr[ww] == sr[0] && sv[ww] < sv[0])) { sr[0] = sr[ww]; sv[0] = sv[ww]; sk[0] = sk[ww]; sa[0] = sa[ww]; }
        *out = RecChoice{sr[0], sk[0], sa[0]};
    }
}

// Dual ratio test over the nonbasic variables: among tableau-row entries
// alpha < -eps, min (objective-row entry) / (-alpha), ties to the lowest
// variable index.  Structural j: alpha = arow[j], row-0 entry d[j]; slack of
// the constraint R[a]: alpha = rho[a], row-0 entry y_R[a].
template <int NT>
__global__ void __launch_bounds__(NT) k_rec_dual_ratio(int n, const int* __restrict__ Rr, int k,
                                                      const double* __restrict__ arow, const double* __restrict__ d,
                                                      const int* __restrict__ isbasic, const double* __restrict__ rho,
                                                      const double* __restrict__ yR, double eps, RecChoice* out) {
    __shared__ double sr[NT / 32];
    __shared__ int sv[NT / 32], sk[NT / 32], sa[NT / 32];
    double best = INFINITY;
    int bvar = INT_MAX, bkind = -1, bat = -1;
    auto take = [&](double r, int var, int kind, int at) {
        if (r < best || (r == best && var < bvar)) { best = r; bvar = var; bkind = kind; bat = at; }
    };
    for (int j = threadIdx.x; j < n; j += NT)
        if (!isbasic[j] && arow[j] < -eps) take(fmax(d[j], 0.0) / -arow[j], j, 0, j);
    for (int a = threadIdx.x; a < k; a += NT)
        if (rho[a] < -eps) take(fmax(yR[a], 0.0) / -rho[a], n + Rr[a], 1, a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double orr = __shfl_xor_sync(0xffffffffu, best, o);
        const int ov = __shfl_xor_sync(0xffffffffu, bvar, o);
        const int ok2 = __shfl_xor_sync(0xffffffffu, bkind, o);
        const int oa = __shfl_xor_sync(0xffffffffu, bat, o);
        if (orr < best || (orr == best && ov < bvar)) { best = orr; bvar = ov; bkind = ok2; bat = oa; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sr[w] = best; sv[w] = bvar; sk[w] = bkind; sa[w] = bat; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < NT / 32; ++ww)
            if (sr[ww] < sr[0] || (sr[ww] == sr[0] && sv[ww] < sv[0])) { sr[0] = sr[ww]; sv[0] = sv[ww]; sk[0] = sk[ww]; sa[0] = sa[ww]; }
        *out = RecChoice{sr[0], sk[0], sa[0]};
    }
}

// rho = row b of A_RS^-1 (leaving structural S[b]) or -(A[i][S] A_RS^-1)
// (leaving slack of row i): rho[a] = -sum_b A[i][S[b]] inv[b][a].
__global__ void k_rec_rho(int n, const double* __restrict__ A, const int* __restrict__ S, int k,
                          const double* __restrict__ inv, int leave_kind, int leave_at, double* __restrict__ rho) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
        if (leave_kind == 0) {
            rho[a] = inv[(size_t)leave_at * k + a];
        } else {
            const double* row = A + (size_t)leave_at * n;
            double sum = 0.0;
            for (int b2 = 0; b2 < k; ++b2) sum = __fma_rn(row[S[b2]], inv[(size_t)b2 * k + a], sum);
            rho[a] = -sum;
        }
    }
}

// Entering column restricted to R: v[a] = A[R[a]][j] (structural j) or e_{a0}
// (slack of the constraint R[a0]).
__global__ void k_rec_enter_col(int n, const double* __restrict__ A, const int* __restrict__ Rr, int k, int kind,
                                int at, double* __restrict__ v) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x)
        v[a] = kind == 0 ? A[(size_t)Rr[a] * n + at] : (a == at ? 1.0 : 0.0);
}

// Final x (n), y (m) and objective c^T x in the read-out layout (sol zeroed first).
__global__ void k_rec_output(int m, int n, const int* __restrict__ S, const int* __restrict__ Rr, int k,
                              const double* __restrict__ xS, const double* __restrict__ yR, const RecCheck* chk,
                              double* __restrict__ sol) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        sol[S[t]] = xS[t];
        sol[n + Rr[t]] = yR[t];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sol[n + m] = chk->cx;
}

}  // namespace tsx
