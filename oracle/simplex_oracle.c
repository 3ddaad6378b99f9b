/*
 * Plain single-threaded FP64 full-tableau simplex: the ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or constant with the CUDA
 * path (it re-declares its own status codes below).
 *
 * It follows Section III of arXiv 2211.10979 ("The standard simplex method")
 * step by step, in the paper's order:
 *
 *   Initialization Step (Sec. III, Table I): build the full tableau from
 *     (A, b, c) with the slack variables x_{n+1..n+m} as the starting basis.
 *   Step 1 (Sec. III): entering variable = column of the objective row with the
 *     most negative coefficient (Dantzig's rule).
 *   Step 2 (Sec. III): leaving variable = row with the minimum ratio
 *     rhs_i / T[i][q] over the rows with a positive entry in column q.
 *   Step 3 (Sec. III): pivot on (p, q): the pivot row is divided by the pivot
 *     element and every other row has that multiple of it subtracted.
 *   Iterate/Finalization Step (Sec. III): repeat until no negative objective
 *     coefficient is left (optimal) or column q has no positive entry
 *     (unbounded).
 *
 * Readings where the paper is silent (each stated again where it is used):
 *   - maximize c^T x s.t. A x <= b, x >= 0 with b >= 0 (Table I's -c row and
 *     slack identity); the constant z column of Table I is dropped, so the
 *     tableau has W = n + m + 1 columns, the last one being the right-hand side.
 *   - a column is a candidate to enter iff T[0][j] < -eps_d; a row is eligible
 *     to leave iff T[i][q] > eps_p.
 *   - ties: the lowest column index enters; the lowest row index leaves
 *     (Bland mode: the row whose basic variable has the lowest index leaves).
 *   - arithmetic of Step 3: r_j = T[p][j] / T[p][q] (IEEE division), then
 *     T[i][j] = fma(-T[i][q], r_j, T[i][j]) for i != p (one rounding), row p = r.
 *   - cycling guard (not in the paper): after k_cyc consecutive pivots whose
 *     minimum ratio is <= 0 the rule becomes Bland's (lowest-index entering
 *     column, lowest basic-variable index among tied rows) until the next
 *     pivot with a positive minimum ratio.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math: the
 * one fused multiply-add is the explicit fma() call of Step 3).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* oracle-local status codes (the values of the paper's two outcomes and of the
 * guards added here) */
enum {
    ORC_OPTIMAL = 0,
    ORC_UNBOUNDED = 1,
    ORC_ITER_LIMIT = 2,
    ORC_NUMERIC = 3,
    ORC_INVALID = -1
};

typedef struct {
    int rule;          /* 0 = Dantzig with Bland fallback, 1 = Bland throughout */
    double eps_d;      /* optimality tolerance on objective-row entries        */
    double eps_p;      /* pivot tolerance on column-q entries                  */
    long max_iters;    /* pivot cap; <0 means 50 (m + n)                       */
    int k_cyc;         /* consecutive degenerate pivots before Bland; <=0: off */
} orc_options;

#define TAB(T, W, i, j) ((T)[(size_t)(i) * (size_t)(W) + (size_t)(j)])

/* Initialization Step (Sec. III, Table I).  T is (m+1) x W, W = n + m + 1.
 * Row 0 = [-c_1 .. -c_n, 0 .. 0 | 0]; row i (1..m) = [a_i1 .. a_in, e_i | b_i].
 * basis[i-1] = n + i - 1 (the slack of constraint i, 0-based variable index). */
int orc_build(int m, int n, const double *A, const double *b, const double *c,
              double *T, int *basis)
{
    if (m <= 0 || n <= 0 || !A || !b || !c || !T || !basis)
        return ORC_INVALID;
    const int W = n + m + 1;
    for (int i = 0; i < m; ++i)
        if (!(b[i] >= 0.0) || !isfinite(b[i]))
            return ORC_INVALID;
    memset(T, 0, sizeof(double) * (size_t)(m + 1) * (size_t)W);
    for (int j = 0; j < n; ++j)
        TAB(T, W, 0, j) = -c[j];
    for (int i = 1; i <= m; ++i) {
        for (int j = 0; j < n; ++j)
            TAB(T, W, i, j) = A[(size_t)(i - 1) * (size_t)n + (size_t)j];
        TAB(T, W, i, n + i - 1) = 1.0;
        TAB(T, W, i, W - 1) = b[i - 1];
        basis[i - 1] = n + i - 1;
    }
    return ORC_OPTIMAL;
}

/* Step 1 (Sec. III): the entering column.  Scans j = 0 .. W-2 (every variable
 * column; the right-hand side is not a candidate).  Dantzig: the most negative
 * T[0][j] below -eps_d, lowest j on ties.  Bland: the lowest j below -eps_d.
 * Returns -1 when no column qualifies (the current basis is optimal). */
int orc_entering(int m, int n, const double *T, int bland, double eps_d)
{
    const int W = n + m + 1;
    int q = -1;
    double best = 0.0;
    for (int j = 0; j < W - 1; ++j) {
        double v = TAB(T, W, 0, j);
        if (v < -eps_d) {
            if (bland)
                return j;
            if (q < 0 || v < best) {
                q = j;
                best = v;
            }
        }
    }
    return q;
}

/* Step 2 (Sec. III): the minimum-ratio test on column q.  Rows i = 1..m with
 * T[i][q] > eps_p are eligible; ratio_i = T[i][W-1] / T[i][q].  The smallest
 * ratio wins; ties go to the lowest row index (Dantzig mode) or to the row whose
 * basic variable has the lowest index (Bland mode).  Returns -1 if no row is
 * eligible (the LP is unbounded along column q). */
int orc_leaving(int m, int n, const double *T, const int *basis, int q,
                int bland, double eps_p, double *ratio_out)
{
    const int W = n + m + 1;
    int p = -1;
    double best = 0.0;
    for (int i = 1; i <= m; ++i) {
        double a = TAB(T, W, i, q);
        if (a > eps_p) {
            double r = TAB(T, W, i, W - 1) / a;
            int take;
            if (p < 0)
                take = 1;
            else if (r < best)
                take = 1;
            else if (r == best && bland)
                take = basis[i - 1] < basis[p - 1];
            else
                take = 0;
            if (take) {
                p = i;
                best = r;
            }
        }
    }
    if (ratio_out)
        *ratio_out = best;
    return p;
}

/* Step 3 (Sec. III): pivot on (p, q).  The pivot row and the pivot column are
 * copied before any element changes: r_j = T[p][j] / T[p][q] for every j, and
 * f_i = T[i][q] for every i.  Then T[i][j] = fma(-f_i, r_j, T[i][j]) for every
 * row i != p and row p becomes r.  Since r_q = 1 exactly and
 * fma(-f_i, 1, f_i) = 0 exactly, column q becomes the unit vector e_p. */
void orc_pivot(int m, int n, double *T, int p, int q, double *r, double *f)
{
    const int W = n + m + 1;
    const double piv = TAB(T, W, p, q);
    for (int j = 0; j < W; ++j)
        r[j] = TAB(T, W, p, j) / piv;
    for (int i = 0; i <= m; ++i)
        f[i] = TAB(T, W, i, q);
    for (int i = 0; i <= m; ++i) {
        if (i == p)
            continue;
        for (int j = 0; j < W; ++j)
            TAB(T, W, i, j) = fma(-f[i], r[j], TAB(T, W, i, j));
    }
    for (int j = 0; j < W; ++j)
        TAB(T, W, p, j) = r[j];
}

/* Separation of the decisions of one Dantzig pivot (a check of the instance,
 * not part of the method): with q and p chosen by Steps 1 and 2,
 *   *dgap = (second most negative candidate T[0][j], j != q) - T[0][q],
 *   *rgap = (second smallest eligible ratio, i != p) - ratio of row p,
 * each +INFINITY when there is no second candidate.  A pivot whose gaps are
 * positive would pick the same (q, p) under any order of the comparisons. */
void orc_pivot_gaps(int m, int n, const double *T, int q, int p, double eps_d,
                    double eps_p, double *dgap, double *rgap)
{
    const int W = n + m + 1;
    const double vq = TAB(T, W, 0, q);
    double second = INFINITY;
    for (int j = 0; j < W - 1; ++j) {
        double v = TAB(T, W, 0, j);
        if (j != q && v < -eps_d && v < second)
            second = v;
    }
    *dgap = second - vq;
    const double rp = TAB(T, W, p, W - 1) / TAB(T, W, p, q);
    second = INFINITY;
    for (int i = 1; i <= m; ++i) {
        double a = TAB(T, W, i, q);
        if (i != p && a > eps_p) {
            double r = TAB(T, W, i, W - 1) / a;
            if (r < second)
                second = r;
        }
    }
    *rgap = second - rp;
}

/* Iterate/Finalization Step (Sec. III): Steps 1-3 until optimal or unbounded.
 * Runs on a tableau built by orc_build (or one already pivoted by an earlier
 * call; the degenerate-run state then starts from zero).  The i-th pivot's
 * (q, p) pair is written to qlog[i], plog[i] while i < log_cap; when
 * dgap/rgap/thetalog/dval are not NULL, the pivot's minimum ratio, its
 * objective-row entry T[0][q] and the gaps of orc_pivot_gaps (NAN for a pivot
 * taken under Bland's rule) go there too. */
int orc_solve_traced(int m, int n, double *T, int *basis, const orc_options *opt,
                     long *iters_out, int *qlog, int *plog, long log_cap,
                     double *dgap, double *rgap, double *thetalog, double *dval)
{
    if (m <= 0 || n <= 0 || !T || !basis || !opt)
        return ORC_INVALID;
    const int W = n + m + 1;
    const long cap = opt->max_iters < 0 ? 50L * ((long)m + (long)n) : opt->max_iters;
    double *r = (double *)malloc(sizeof(double) * (size_t)W);
    double *f = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    if (!r || !f) {
        free(r);
        free(f);
        return ORC_INVALID;
    }
    int bland = opt->rule == 1;
    int degen_run = 0;
    long it = 0;
    int status;
    for (;;) {
        int q = orc_entering(m, n, T, bland, opt->eps_d);
        if (q < 0) {
            status = ORC_OPTIMAL;
            break;
        }
        if (it >= cap) {
            status = ORC_ITER_LIMIT;
            break;
        }
        double theta = 0.0;
        int p = orc_leaving(m, n, T, basis, q, bland, opt->eps_p, &theta);
        if (p < 0) {
            status = ORC_UNBOUNDED;
            break;
        }
        if (!isfinite(TAB(T, W, p, q)) || !isfinite(theta)) {
            status = ORC_NUMERIC;
            break;
        }
        if (it < log_cap) {
            if (qlog)
                qlog[it] = q;
            if (plog)
                plog[it] = p;
            if (thetalog)
                thetalog[it] = theta;
            if (dval)
                dval[it] = TAB(T, W, 0, q);
            if (dgap && rgap) {
                if (bland) {
                    dgap[it] = NAN;
                    rgap[it] = NAN;
                } else {
                    orc_pivot_gaps(m, n, T, q, p, opt->eps_d, opt->eps_p, &dgap[it], &rgap[it]);
                }
            }
        }
        orc_pivot(m, n, T, p, q, r, f);
        basis[p - 1] = q;
        ++it;
        /* cycling guard: a pivot with minimum ratio <= 0 leaves the objective
         * unchanged; k_cyc of them in a row switch to Bland's rule, and the
         * first pivot with a positive ratio switches back to Dantzig's. */
        if (opt->rule == 0) {
            if (theta <= 0.0) {
                ++degen_run;
                if (opt->k_cyc > 0 && degen_run >= opt->k_cyc)
                    bland = 1;
            } else {
                degen_run = 0;
                bland = 0;
            }
        }
    }
    free(r);
    free(f);
    if (iters_out)
        *iters_out = it;
    return status;
}

int orc_solve(int m, int n, double *T, int *basis, const orc_options *opt,
              long *iters_out, int *qlog, int *plog, long log_cap)
{
    return orc_solve_traced(m, n, T, basis, opt, iters_out, qlog, plog, log_cap,
                            NULL, NULL, NULL, NULL);
}

/* Read the solution out of a tableau (Sec. III, Table I layout): x_j is the
 * right-hand side of the row where x_j is basic (0 if nonbasic); the dual value
 * of constraint i is the objective-row entry of its slack column n + i - 1; the
 * objective value is the objective row's right-hand side. */
void orc_extract(int m, int n, const double *T, const int *basis, double *x,
                 double *y, double *obj)
{
    const int W = n + m + 1;
    if (x) {
        for (int j = 0; j < n; ++j)
            x[j] = 0.0;
        for (int i = 1; i <= m; ++i)
            if (basis[i - 1] < n)
                x[basis[i - 1]] = TAB(T, W, i, W - 1);
    }
    if (y)
        for (int i = 1; i <= m; ++i)
            y[i - 1] = TAB(T, W, 0, n + i - 1);
    if (obj)
        *obj = TAB(T, W, 0, W - 1);
}

/* ------------------------------------------------------------------------
 * The same steps on a float tableau (the single-precision variant of the
 * method): the tableau entries are the inputs rounded to float, r_j and the
 * ratios are float divisions, the update is one fmaf per entry.  Comparisons
 * against the tolerances are made in double on the float values.  Used to
 * check a float pivot kernel step by step; the result of the method itself is
 * checked against the double oracle above.
 * ------------------------------------------------------------------------ */
int orc32_build(int m, int n, const double *A, const double *b, const double *c,
                float *T, int *basis)
{
    if (m <= 0 || n <= 0 || !A || !b || !c || !T || !basis)
        return ORC_INVALID;
    const int W = n + m + 1;
    for (int i = 0; i < m; ++i)
        if (!(b[i] >= 0.0) || !isfinite(b[i]))
            return ORC_INVALID;
    memset(T, 0, sizeof(float) * (size_t)(m + 1) * (size_t)W);
    for (int j = 0; j < n; ++j)
        TAB(T, W, 0, j) = (float)(-c[j]);
    for (int i = 1; i <= m; ++i) {
        for (int j = 0; j < n; ++j)
            TAB(T, W, i, j) = (float)A[(size_t)(i - 1) * (size_t)n + (size_t)j];
        TAB(T, W, i, n + i - 1) = 1.0f;
        TAB(T, W, i, W - 1) = (float)b[i - 1];
        basis[i - 1] = n + i - 1;
    }
    return ORC_OPTIMAL;
}

int orc32_entering(int m, int n, const float *T, int bland, double eps_d)
{
    const int W = n + m + 1;
    int q = -1;
    float best = 0.0f;
    for (int j = 0; j < W - 1; ++j) {
        float v = TAB(T, W, 0, j);
        if ((double)v < -eps_d) {
            if (bland)
                return j;
            if (q < 0 || v < best) {
                q = j;
                best = v;
            }
        }
    }
    return q;
}

int orc32_leaving(int m, int n, const float *T, const int *basis, int q,
                  int bland, double eps_p, float *ratio_out)
{
    const int W = n + m + 1;
    int p = -1;
    float best = 0.0f;
    for (int i = 1; i <= m; ++i) {
        float a = TAB(T, W, i, q);
        if ((double)a > eps_p) {
            float r = TAB(T, W, i, W - 1) / a;
            int take;
            if (p < 0)
                take = 1;
            else if (r < best)
                take = 1;
            else if (r == best && bland)
                take = basis[i - 1] < basis[p - 1];
            else
                take = 0;
            if (take) {
                p = i;
                best = r;
            }
        }
    }
    if (ratio_out)
        *ratio_out = best;
    return p;
}

void orc32_pivot(int m, int n, float *T, int p, int q, float *r, float *f)
{
    const int W = n + m + 1;
    const float piv = TAB(T, W, p, q);
    for (int j = 0; j < W; ++j)
        r[j] = TAB(T, W, p, j) / piv;
    for (int i = 0; i <= m; ++i)
        f[i] = TAB(T, W, i, q);
    for (int i = 0; i <= m; ++i) {
        if (i == p)
            continue;
        for (int j = 0; j < W; ++j)
            TAB(T, W, i, j) = fmaf(-f[i], r[j], TAB(T, W, i, j));
    }
    for (int j = 0; j < W; ++j)
        TAB(T, W, p, j) = r[j];
}

int orc32_solve(int m, int n, float *T, int *basis, const orc_options *opt,
                long *iters_out, int *qlog, int *plog, long log_cap)
{
    if (m <= 0 || n <= 0 || !T || !basis || !opt)
        return ORC_INVALID;
    const int W = n + m + 1;
    const long cap = opt->max_iters < 0 ? 50L * ((long)m + (long)n) : opt->max_iters;
    float *r = (float *)malloc(sizeof(float) * (size_t)W);
    float *f = (float *)malloc(sizeof(float) * (size_t)(m + 1));
    if (!r || !f) {
        free(r);
        free(f);
        return ORC_INVALID;
    }
    int bland = opt->rule == 1;
    int degen_run = 0;
    long it = 0;
    int status;
    for (;;) {
        int q = orc32_entering(m, n, T, bland, opt->eps_d);
        if (q < 0) {
            status = ORC_OPTIMAL;
            break;
        }
        if (it >= cap) {
            status = ORC_ITER_LIMIT;
            break;
        }
        float theta = 0.0f;
        int p = orc32_leaving(m, n, T, basis, q, bland, opt->eps_p, &theta);
        if (p < 0) {
            status = ORC_UNBOUNDED;
            break;
        }
        if (!isfinite(TAB(T, W, p, q)) || !isfinite(theta)) {
            status = ORC_NUMERIC;
            break;
        }
        if (it < log_cap) {
            if (qlog)
                qlog[it] = q;
            if (plog)
                plog[it] = p;
        }
        orc32_pivot(m, n, T, p, q, r, f);
        basis[p - 1] = q;
        ++it;
        if (opt->rule == 0) {
            if (theta <= 0.0f) {
                ++degen_run;
                if (opt->k_cyc > 0 && degen_run >= opt->k_cyc)
                    bland = 1;
            } else {
                degen_run = 0;
                bland = 0;
            }
        }
    }
    free(r);
    free(f);
    if (iters_out)
        *iters_out = it;
    return status;
}
