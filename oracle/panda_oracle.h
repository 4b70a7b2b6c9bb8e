/*
 * PANDA message-passing oracle: plain FP64 CPU loops, written straight from the
 * paper's element-wise equations (Glass, Quackenbush, Kepner, "High Performance
 * Computing of Gene Regulatory Networks using a Message-Passing Model").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this code; it exists so the CUDA path can be checked against an obviously
 * correct statement of the method.  It shares no code, header or constant with
 * the CUDA library.
 *
 * Conventions
 *   T  = number of effector nodes (transcription factors, the paper's N_e)
 *   G  = number of affected nodes (genes, the paper's N_a)
 *   W  = T x G regulatory network, row-major, W[i*G + j]
 *   P  = T x T cooperativity network, row-major, full (diagonal included)
 *   C  = G x G co-regulatory network, row-major, full (diagonal included)
 *   t  = 1-based iteration index used in the diagonal factor e^{2 alpha t}
 *
 * Diagonal rules (Eq. 6; the paper prints no alpha on the increment):
 *   ORACLE_DIAG_D1 = 0  damped:  X_ii <- (1-a) X_ii + a * N * sigma_i * e^{2 a t}
 *   ORACLE_DIAG_D0 = 1  literal: X_ii <- (1-a) X_ii +     N * sigma_i * e^{2 a t}
 *   ORACLE_DIAG_D2 = 2  as D1, sigma over row i of the new similarity matrix
 *                       instead of row i of the updated network
 *   with N = G for P (N_a) and N = T for C (N_e), as Eq. 6 pairs them.
 *
 * Parity status: every function here is pinned by the CPU tests (closed forms
 * of the similarity, the matrix form of Eq. 9, alpha = 0 and alpha = 1 cases,
 * identity-prior closed forms, a hand-worked 2 x 3 example, symmetry and
 * permutation equivariance; the Pearson initialisation against a library
 * correlation, a worked 3 x 3 case, affine invariance and sign flips).  Multi-iteration trajectories beyond those pins
 * rest on the same per-step functions; the paper prints no worked trajectory.
 */
#ifndef PANDA_ORACLE_H
#define PANDA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_DIAG_D1 = 0, ORACLE_DIAG_D0 = 1, ORACLE_DIAG_D2 = 2 };

/* The initial co-regulation network (Sec. II-A): Pearson correlation between
 * pairs of genes across all samples.  X is the G x N expression matrix
 * (row-major, gene g's samples in X[g*N .. g*N + N-1]); C (G x G, row-major,
 * full) receives r_gh = s_gh / sqrt(s_gg s_hh), s_gh = sum_k (x_gk - m_g)(x_hk - m_h)
 * with m_g the mean of row g, and r_gg = 1.  Two passes in FP64 (means, then
 * centred sums).  Returns 0; -1 for bad arguments; -6 when a row has zero
 * variance (its correlations are undefined). */
int oracle_pearson(int G, int N, const double *X, double *C);

/* Eq. 1, in the three-sum form of Eq. 8: x.y / sqrt(|x|^2 + |y|^2 - |x.y|).
 * x and y are strided FP64 vectors of length n.  Both-zero vectors give 0. */
double oracle_tanimoto(const double *x, long incx, const double *y, long incy, long n);

/* Z-score one network in place (the paper's NormalizeNetwork): one global mean
 * and population standard deviation over all n entries.  Returns 0, or -6 when
 * the standard deviation is zero (the transform is undefined). */
int oracle_zscore(double *a, long n);

/* Z-score W, P and C, each on its own (Section II-A, input preparation). */
int oracle_normalize(int T, int G, double *W, double *P, double *C);

/* Responsibility R_ij = Tan(P_i., W_.j) (Eq. 3) and availability
 * A_ij = Tan(W_i., C_.j) (Eq. 4) of one edge, from the previous state. */
double oracle_responsibility(int T, int G, const double *W, const double *P, int i, int j);
double oracle_availability(int T, int G, const double *W, const double *C, int i, int j);

/* Updated regulatory edge W'_ij (Eq. 2) and whole rows / columns of W'. */
double oracle_w_entry(int T, int G, const double *W, const double *P, const double *C,
                      double alpha, int i, int j);
void oracle_w_row(int T, int G, const double *W, const double *P, const double *C,
                  double alpha, int i, double *out /* G */);
void oracle_w_col(int T, int G, const double *W, const double *P, const double *C,
                  double alpha, int j, double *out /* T */);

/* The listed rows of W' (n x G), computed with the similarities' vectors made
 * contiguous first.  Returns 0, -1 bad argument, -2 no memory, -5 P or C not
 * exactly symmetric. */
int oracle_w_rows(int T, int G, const double *W, const double *P, const double *C,
                  double alpha, int n, const int *rows, double *out);

/* Eq. 5 for one off-diagonal entry: (1 - alpha) old + alpha Tan(x, y). */
double oracle_eq5_entry(double old, double alpha, const double *x, long incx, const double *y,
                        long incy, long n);

/* Eq. 6 for one diagonal entry: row holds row i of the updated n x n network
 * (or of the new similarity matrix under rule D2; its diagonal entry is not
 * read); mult is N_a (= G) for P and N_e (= T) for C; old is X_ii^(t-1). */
double oracle_diag_value(const double *row, int n, int i, double mult, double old, double alpha,
                         int t, int rule);

/* The listed rows of P' (n x T) and C' (n x G) after the off-diagonal update of
 * Eq. 5 from the new W' (Wn); diagonal entries are copied unchanged.  sim (may
 * be NULL) receives the bare similarities, 0 on the diagonal. */
int oracle_p_rows(int T, int G, const double *Wn, const double *P, double alpha, int n,
                  const int *rows, double *out, double *sim);
int oracle_c_rows(int T, int G, const double *Wn, const double *C, double alpha, int n,
                  const int *rows, double *out, double *sim);

/* One full iteration (Eqs. 2-7): W', then P' and C' from W', then the
 * diagonals.  Inputs are not modified; outputs must not alias inputs.
 * *h receives the mean absolute change of W (Eq. 7).  Returns 0, or -1 on a
 * bad argument. */
int oracle_step(int T, int G, const double *W, const double *P, const double *C,
                double alpha, int t, int diag_rule,
                double *Wn, double *Pn, double *Cn, double *h);

/* Iterate oracle_step in place from iteration t0+1 until h < tol (strictly,
 * tested after the whole iteration) or max_iter iterations.  *iters receives
 * the number of iterations run; h_hist (may be NULL) receives h per iteration
 * and must hold max_iter entries.  Returns 0 when converged, 1 when max_iter
 * was reached first, negative on a bad argument. */
int oracle_run(int T, int G, double *W, double *P, double *C, double alpha, double tol,
               int max_iter, int t0, int diag_rule, int *iters, double *h_hist);

/* Threads used by the loops of oracle_step (each output element is computed
 * on its own, so results do not depend on the thread count). */
void oracle_set_threads(int n);
int oracle_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
