/*
 * PANDA message-passing oracle: plain FP64 CPU loops (see panda_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.
 *
 * Every similarity is Eq. 1 evaluated as the three running sums of Eq. 8,
 * summed in index order, with no blocking and no reassociation (the library is
 * built with -ffp-contract=off so a product and a sum are rounded separately
 * on every machine).  Loops over output elements may run on several threads;
 * each element is computed on its own, so the thread count never changes a
 * result.
 *
 * Readings of the paper taken here (each one is listed with its reason in the
 * design notes of the repository):
 *   - Eq. 4 uses the previous state W^(t-1), C^(t-1), as the equation prints
 *     (the sentence above it says (t), which would make Eq. 2 circular).
 *   - Eq. 5: the index printed as p is the row index m; P and C are updated
 *     from the new W^(t) ("the updates of W, then P and C").
 *   - Eq. 6: sigma_i is the population standard deviation of the off-diagonal
 *     entries of row i of the updated network; rule D1 damps the increment by
 *     alpha (see the header for D0 and D2); t is 1-based.
 *   - Eq. 7 ("hamming distance") is the mean absolute change of W.
 *   - The Z-score uses one global mean and population std per network.
 *   - Tan is 0 when its denominator is 0 (both vectors zero).
 *   - P and C are symmetric (Section II-A); the oracle checks this and reads
 *     column j of C as its row j.
 */
#include "panda_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int oracle_get_threads(void) { return g_threads; }

/* ---- Eq. 1 / Eq. 8 ------------------------------------------------------ */

double oracle_tanimoto(const double *x, long incx, const double *y, long incy, long n)
{
    double sxy = 0.0; /* numerator: x . y            */
    double sxx = 0.0; /* |x|^2                        */
    double syy = 0.0; /* |y|^2                        */
    for (long k = 0; k < n; ++k) {
        double a = x[k * incx];
        double b = y[k * incy];
        sxy += a * b;
        sxx += a * a;
        syy += b * b;
    }
    double den = sqrt(sxx + syy - fabs(sxy));
    if (den == 0.0)
        return 0.0;
    return sxy / den;
}

/* ---- input normalisation (NormalizeNetwork) ----------------------------- */

int oracle_zscore(double *a, long n)
{
    if (n <= 0)
        return -1;
    double s = 0.0;
    for (long k = 0; k < n; ++k)
        s += a[k];
    double mean = s / (double)n;
    double ss = 0.0;
    for (long k = 0; k < n; ++k) {
        double d = a[k] - mean;
        ss += d * d;
    }
    double sd = sqrt(ss / (double)n);
    if (!(sd > 0.0))
        return -6;
    for (long k = 0; k < n; ++k)
        a[k] = (a[k] - mean) / sd;
    return 0;
}

int oracle_pearson(int G, int N, const double *X, double *C)
{
    if (G <= 0 || N <= 0 || !X || !C)
        return -1;
    double *mean = (double *)malloc(sizeof(double) * (size_t)G);
    double *ss = (double *)malloc(sizeof(double) * (size_t)G);
    if (!mean || !ss) {
        free(mean);
        free(ss);
        return -1;
    }
    int degenerate = 0;
    for (int g = 0; g < G; ++g) {
        const double *x = X + (long)g * N;
        double m = 0.0;
        for (int k = 0; k < N; ++k)
            m += x[k];
        m /= (double)N;
        double q = 0.0;
        for (int k = 0; k < N; ++k)
            q += (x[k] - m) * (x[k] - m);
        mean[g] = m;
        ss[g] = q;
        if (!(q > 0.0))
            degenerate = 1;
    }
    if (degenerate) {
        free(mean);
        free(ss);
        return -6;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int g = 0; g < G; ++g) {
        const double *x = X + (long)g * N;
        C[(long)g * G + g] = 1.0;
        for (int h = g + 1; h < G; ++h) {
            const double *y = X + (long)h * N;
            double s = 0.0;
            for (int k = 0; k < N; ++k)
                s += (x[k] - mean[g]) * (y[k] - mean[h]);
            const double r = s / sqrt(ss[g] * ss[h]);
            C[(long)g * G + h] = r;
            C[(long)h * G + g] = r;
        }
    }
    free(mean);
    free(ss);
    return 0;
}

int oracle_normalize(int T, int G, double *W, double *P, double *C)
{
    if (T <= 0 || G <= 0 || !W || !P || !C)
        return -1;
    int rc = oracle_zscore(W, (long)T * G);
    if (rc)
        return rc;
    rc = oracle_zscore(P, (long)T * T);
    if (rc)
        return rc;
    return oracle_zscore(C, (long)G * G);
}

/* ---- helpers ------------------------------------------------------------ */

static int is_symmetric(const double *X, int n)
{
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (X[(long)i * n + j] != X[(long)j * n + i])
                return 0;
    return 1;
}

/* Out-of-place transpose of a rows x cols matrix (data movement only). */
static double *transposed(const double *X, int rows, int cols)
{
    double *Y = (double *)malloc(sizeof(double) * (size_t)rows * (size_t)cols);
    if (!Y)
        return NULL;
    for (long r = 0; r < rows; ++r)
        for (long c = 0; c < cols; ++c)
            Y[c * rows + r] = X[r * cols + c];
    return Y;
}

/* ---- Eqs. 3, 4, 2: responsibility, availability, new W ------------------ */

double oracle_responsibility(int T, int G, const double *W, const double *P, int i, int j)
{
    /* R_ij = Tan(P_i., W_.j): row i of P against column j of W (Eq. 3). */
    return oracle_tanimoto(P + (long)i * T, 1, W + j, G, T);
}

double oracle_availability(int T, int G, const double *W, const double *C, int i, int j)
{
    /* A_ij = Tan(W_i., C_.j): row i of W against column j of C (Eq. 4). */
    (void)T;
    return oracle_tanimoto(W + (long)i * G, 1, C + j, G, G);
}

static double w_update(double w, double alpha, double r, double a)
{
    /* Eq. 2 */
    return (1.0 - alpha) * w + alpha / 2.0 * (a + r);
}

double oracle_w_entry(int T, int G, const double *W, const double *P, const double *C,
                      double alpha, int i, int j)
{
    double r = oracle_responsibility(T, G, W, P, i, j);
    double a = oracle_availability(T, G, W, C, i, j);
    return w_update(W[(long)i * G + j], alpha, r, a);
}

/* Rows of W' for the listed TFs.  Column j of W is read from a transposed
 * copy and column j of the symmetric C as its row j, so both vectors of every
 * similarity are contiguous; the sums are the same as in Eq. 3 and Eq. 4. */
static void w_rows_impl(int T, int G, const double *W, const double *Wt, const double *P,
                        const double *C, double alpha, int n, const int *rows, double *out)
{
    for (int q = 0; q < n; ++q) {
        long i = rows[q];
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int j = 0; j < G; ++j) {
            double r = oracle_tanimoto(P + i * T, 1, Wt + (long)j * T, 1, T);
            double a = oracle_tanimoto(W + i * G, 1, C + (long)j * G, 1, G);
            out[(long)q * G + j] = w_update(W[i * G + j], alpha, r, a);
        }
    }
}

int oracle_w_rows(int T, int G, const double *W, const double *P, const double *C,
                  double alpha, int n, const int *rows, double *out)
{
    if (T <= 0 || G <= 0 || n < 0 || !W || !P || !C || (n && (!rows || !out)))
        return -1;
    if (!is_symmetric(C, G) || !is_symmetric(P, T))
        return -5;
    double *Wt = transposed(W, T, G);
    if (!Wt)
        return -2;
    w_rows_impl(T, G, W, Wt, P, C, alpha, n, rows, out);
    free(Wt);
    return 0;
}

void oracle_w_row(int T, int G, const double *W, const double *P, const double *C,
                  double alpha, int i, double *out)
{
    for (int j = 0; j < G; ++j)
        out[j] = oracle_w_entry(T, G, W, P, C, alpha, i, j);
}

void oracle_w_col(int T, int G, const double *W, const double *P, const double *C,
                  double alpha, int j, double *out)
{
    for (int i = 0; i < T; ++i)
        out[i] = oracle_w_entry(T, G, W, P, C, alpha, i, j);
}

/* ---- Eq. 5: off-diagonal P and C from the new W ------------------------- */

double oracle_eq5_entry(double old, double alpha, const double *x, long incx, const double *y,
                        long incy, long n)
{
    double s = oracle_tanimoto(x, incx, y, incy, n);
    return (1.0 - alpha) * old + alpha * s;
}

/* Row i of P' (Eq. 5, first line) for each listed i: entries m != i get
 * (1-a) P_im + a Tan(W'_i., W'_m.); the diagonal entry is copied unchanged
 * (Eq. 6 updates it afterwards).  sim (may be NULL) receives the bare
 * similarities Tan(W'_i., W'_m.) with 0 on the diagonal. */
int oracle_p_rows(int T, int G, const double *Wn, const double *P, double alpha, int n,
                  const int *rows, double *out, double *sim)
{
    if (T <= 0 || G <= 0 || n < 0 || !Wn || !P || (n && (!rows || !out)))
        return -1;
    for (int q = 0; q < n; ++q) {
        long i = rows[q];
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int m = 0; m < T; ++m) {
            double s = 0.0, v = P[i * T + m];
            if (m != i) {
                v = oracle_eq5_entry(P[i * T + m], alpha, Wn + i * G, 1, Wn + (long)m * G, 1, G);
                if (sim)
                    s = oracle_tanimoto(Wn + i * G, 1, Wn + (long)m * G, 1, G);
            }
            out[(long)q * T + m] = v;
            if (sim)
                sim[(long)q * T + m] = s;
        }
    }
    return 0;
}

/* Row k of C' (Eq. 5, second line): entries j != k get
 * (1-a) C_kj + a Tan(W'_.k, W'_.j), columns of W' read from a transposed copy. */
int oracle_c_rows(int T, int G, const double *Wn, const double *C, double alpha, int n,
                  const int *rows, double *out, double *sim)
{
    if (T <= 0 || G <= 0 || n < 0 || !Wn || !C || (n && (!rows || !out)))
        return -1;
    double *Wnt = transposed(Wn, T, G);
    if (!Wnt)
        return -2;
    for (int q = 0; q < n; ++q) {
        long k = rows[q];
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int j = 0; j < G; ++j) {
            double s = 0.0, v = C[k * G + j];
            if (j != k) {
                v = oracle_eq5_entry(C[k * G + j], alpha, Wnt + k * T, 1, Wnt + (long)j * T, 1, T);
                if (sim)
                    s = oracle_tanimoto(Wnt + k * T, 1, Wnt + (long)j * T, 1, T);
            }
            out[(long)q * G + j] = v;
            if (sim)
                sim[(long)q * G + j] = s;
        }
    }
    free(Wnt);
    return 0;
}

/* ---- Eq. 6: diagonals ---------------------------------------------------- */

/* Population standard deviation of the n-1 off-diagonal entries of row i of
 * the n x n matrix X (0 when the row has no off-diagonal entry). */
static double offdiag_row_std(const double *X, int n, int i)
{
    if (n < 2)
        return 0.0;
    double s = 0.0;
    for (int m = 0; m < n; ++m)
        if (m != i)
            s += X[(long)i * n + m];
    double mean = s / (double)(n - 1);
    double ss = 0.0;
    for (int m = 0; m < n; ++m)
        if (m != i) {
            double d = X[(long)i * n + m] - mean;
            ss += d * d;
        }
    return sqrt(ss / (double)(n - 1));
}

double oracle_diag_value(const double *row, int n, int i, double mult, double old, double alpha,
                         int t, int rule)
{
    double growth = exp(2.0 * alpha * (double)t);
    double gain = (rule == ORACLE_DIAG_D0) ? 1.0 : alpha;
    double sigma = offdiag_row_std(row - (long)i * n, n, i);
    return (1.0 - alpha) * old + gain * mult * sigma * growth;
}

/* Xn holds the updated off-diagonal entries; its diagonal is overwritten with
 * Eq. 6.  mult is N_a (= G) for P and N_e (= T) for C. */
static void diag_update(int n, double mult, double *Xn, const double *Xold, const double *sim,
                        double alpha, int t, int rule)
{
    const double *src = (rule == ORACLE_DIAG_D2) ? sim : Xn;
    for (int i = 0; i < n; ++i)
        Xn[(long)i * n + i] = oracle_diag_value(src + (long)i * n, n, i, mult, Xold[(long)i * n + i],
                                                alpha, t, rule);
}

/* ---- one iteration -------------------------------------------------------- */

int oracle_step(int T, int G, const double *W, const double *P, const double *C,
                double alpha, int t, int diag_rule, double *Wn, double *Pn, double *Cn, double *h)
{
    if (T <= 0 || G <= 0 || !W || !P || !C || !Wn || !Pn || !Cn || !h)
        return -1;
    if (diag_rule < 0 || diag_rule > 2 || t < 1)
        return -1;
    if (!is_symmetric(C, G) || !is_symmetric(P, T))
        return -5;

    /* Eqs. 3, 4, 2 for every row of W. */
    int *idx = (int *)malloc(sizeof(int) * (size_t)(T > G ? T : G));
    double *Wt = transposed(W, T, G);
    double *Psim = NULL, *Csim = NULL;
    if (diag_rule == ORACLE_DIAG_D2) {
        Psim = (double *)malloc(sizeof(double) * (size_t)T * T);
        Csim = (double *)malloc(sizeof(double) * (size_t)G * G);
    }
    if (!idx || !Wt || (diag_rule == ORACLE_DIAG_D2 && (!Psim || !Csim))) {
        free(idx); free(Wt); free(Psim); free(Csim);
        return -2;
    }
    for (int q = 0; q < (T > G ? T : G); ++q)
        idx[q] = q;
    w_rows_impl(T, G, W, Wt, P, C, alpha, T, idx, Wn);
    free(Wt);

    /* Eq. 7 */
    double s = 0.0;
    for (long q = 0; q < (long)T * G; ++q)
        s += fabs(Wn[q] - W[q]);
    *h = s / ((double)T * (double)G);

    /* Eq. 5 from the new W */
    oracle_p_rows(T, G, Wn, P, alpha, T, idx, Pn, Psim);
    int rc = oracle_c_rows(T, G, Wn, C, alpha, G, idx, Cn, Csim);
    free(idx);
    if (rc) {
        free(Psim); free(Csim);
        return rc;
    }

    /* Eq. 6: N_a (= G) with P, N_e (= T) with C */
    diag_update(T, (double)G, Pn, P, Psim, alpha, t, diag_rule);
    diag_update(G, (double)T, Cn, C, Csim, alpha, t, diag_rule);
    free(Psim);
    free(Csim);
    return 0;
}

int oracle_run(int T, int G, double *W, double *P, double *C, double alpha, double tol,
               int max_iter, int t0, int diag_rule, int *iters, double *h_hist)
{
    if (T <= 0 || G <= 0 || !W || !P || !C || !iters || max_iter < 0 || t0 < 0 || tol < 0)
        return -1;
    size_t nw = (size_t)T * G, np = (size_t)T * T, nc = (size_t)G * G;
    double *Wn = (double *)malloc(sizeof(double) * nw);
    double *Pn = (double *)malloc(sizeof(double) * np);
    double *Cn = (double *)malloc(sizeof(double) * nc);
    if (!Wn || !Pn || !Cn) {
        free(Wn); free(Pn); free(Cn);
        return -2;
    }
    int rc = 1;
    *iters = 0;
    for (int it = 1; it <= max_iter; ++it) {
        double h = 0.0;
        int e = oracle_step(T, G, W, P, C, alpha, t0 + it, diag_rule, Wn, Pn, Cn, &h);
        if (e) {
            rc = e;
            break;
        }
        memcpy(W, Wn, sizeof(double) * nw);
        memcpy(P, Pn, sizeof(double) * np);
        memcpy(C, Cn, sizeof(double) * nc);
        *iters = it;
        if (h_hist)
            h_hist[it - 1] = h;
        if (h < tol) { /* strict test after the whole iteration */
            rc = 0;
            break;
        }
    }
    free(Wn); free(Pn); free(Cn);
    return rc;
}
