/*
 * fastpfp_oracle.h -- plain FP64 CPU oracle for FastPFP (Lu, Huang & Liu,
 * "A Fast Projected Fixed-Point Algorithm for Large Graph Matching").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this library.
 * It shares no code, header, table or helper with the CUDA library under
 * paper_1207_1114_gb300/csrc, and the product path never calls it.
 *
 * All matrices are dense, row-major, double precision.  Orientation follows
 * the paper's convention (Section 3): the larger graph indexes the rows, so
 * in the step functions below N >= m, X and K are N x m and the slacked
 * matrix Y is N x N (Section 4.3).  orc_solve() takes the caller's
 * orientation and performs the swap itself.
 */
#ifndef FASTPFP_ORACLE_H
#define FASTPFP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double lambda;      /* weight of the node term, Eq. (1) / Eq. (3)           */
    double alpha;       /* step size of the FastPFP update, Eq. (fastPFP)       */
    double tol_outer;   /* eps_1: stop when max|X(t+1)-X(t)| < eps_1 (Sec. 5)   */
    double tol_inner;   /* eps_2: stop when max|Y(u+1)-Y(u)| < eps_2 (Sec. 5)   */
    int max_outer;      /* I_0: at most this many outer iterations (Sec. 5)     */
    int max_inner;      /* I_1: at most this many inner iterations (Sec. 5)     */
    int normalize_max;  /* 1: X <- X / max(X) each outer iteration (Alg. 1)     */
    int slack_policy;   /* 0: slack columns of Y carry over (Alg. 1), 1: reset  */
    int algorithm;      /* 0: FastPFP, Eq. (fastPFP); 1: projected gradient,
                           Eq. (pg): X <- P_d(X + alpha (A X A' + lambda K))  */
} orc_params;

typedef struct {
    int outer_iters;        /* outer iterations run                              */
    int inner_total;        /* sum of inner iterations over all outer iterations */
    int inner_max;          /* largest inner count of one outer iteration        */
    int converged;          /* 1 if max|dX| < eps_1 was reached                  */
    int transposed;         /* 1 if the caller's graphs were swapped (n_a < n_b) */
    double final_delta;     /* last max|X(t+1)-X(t)|                             */
    double objective;       /* Eq. (3) at the discrete result                    */
    double error;           /* Eq. (1) at the discrete result                    */
} orc_stats;

/* Number of OpenMP threads the oracle will use (1 when built without OpenMP). */
int orc_num_threads(void);
void orc_set_num_threads(int n);

/* K = B * B2^T  (N x m), the attribute affinity below Eq. (4). */
void orc_affinity(const double* B, const double* B2, int N, int m, int k, double* K);

/* G = A * X * A2 + lambda * K (N x m), the gradient of f in Section 4.1.
 * The product is formed as T = A*X first, then T*A2.  K may be NULL when
 * lambda == 0. */
void orc_gradient(const double* A, const double* X, const double* A2, const double* K,
                  double lambda, int N, int m, double* G);

/* One P1 step, Eq. (P1), in place on the N x N matrix Y, with the total sum
 * taken over Y (the reading of Algorithm 1). */
void orc_p1(double* Y, int N);

/* One P2 step, Eq. (P2): Y <- (Y + |Y|) / 2. */
void orc_p2(double* Y, int N);

/* Successive projection P_D(Y) = ...P2 P1 P2 P1 (Y) of Section 4.3, in
 * place.  Runs iterations of (P1 then P2) until max|Y_new - Y_old| < tol or
 * max_iter iterations have run.  When fixed_iters > 0 exactly that many
 * iterations run and tol is ignored (replay mode).  Returns the number of
 * iterations run; *last_delta (nullable) receives the last max|dY|. */
int orc_pd(double* Y, int N, double tol, int max_iter, int fixed_iters, double* last_delta);

/* X_new = (1-alpha) X + alpha Y[:, :m]; if normalize, X_new /= max(X_new)
 * (Algorithm 1 and the Remarks after Theorem 1).  X (N x m) is overwritten
 * with X_new; returns max|X_new - X_old|. */
double orc_blend(double* X, const double* Y, int N, int m, double alpha, int normalize);

/* Greedy discretisation of Section 4.5, written as its Steps 1-3 with an
 * explicit index set L.  Ties between equal maxima go to the lowest
 * row-major index i*m+j.  row_of_col[j] receives the row matched to column
 * j (every column is matched since N >= m).  */
void orc_greedy_literal(const double* X, int N, int m, int* row_of_col);

/* The same greedy as a scan over all entries sorted by (value desc, index
 * asc), accepting an entry when its row and its column are both free. */
void orc_greedy_sorted(const double* X, int N, int m, int* row_of_col);

/* Objective of Eq. (3): 1/2 tr(P^T A P A2) + lambda tr(P^T K) for the
 * partial permutation given by row_of_col (N x m, one 1 per column). */
double orc_qap_objective(const double* A, const double* A2, const double* K, double lambda,
                         const int* row_of_col, int N, int m);

/* Objective of Eq. (1): 1/2 ||A - P A2 P^T||_F^2 + lambda ||B - P B2||_F^2
 * for the partial permutation given by row_of_col. */
double orc_error_objective(const double* A, const double* A2, const double* B, const double* B2,
                           int k, double lambda, const int* row_of_col, int N, int m);

/* Relaxed objective f(X) of Section 4.1 for a real N x m matrix X. */
double orc_relaxed_objective(const double* A, const double* A2, const double* K, double lambda,
                             const double* X, int N, int m);

/* Algorithm 1 end to end in the caller's orientation.
 *   A  : n_a x n_a symmetric,  A2 : n_b x n_b symmetric
 *   B  : n_a x k,              B2 : n_b x k        (NULL when k == 0)
 *   X0 : n_a x n_b initial X (NULL: the uniform start 11^T / (n n'))
 *   replay_inner : nullable; when given, outer iteration t runs exactly
 *                  replay_inner[t] inner iterations (tolerance ignored)
 *   replay_outer : > 0 runs exactly that many outer iterations
 *   perm_out     : n_a entries, the node of graph 2 matched to node i of
 *                  graph 1, or -1
 *   X_out        : nullable, n_a x n_b final soft assignment
 *   inner_trace  : nullable, max_outer entries, inner count per outer iter
 *   delta_trace  : nullable, max_outer entries, max|dX| per outer iter
 * Returns 0, or -1 on bad arguments. */
int orc_solve(const double* A, int n_a, const double* A2, int n_b,
              const double* B, const double* B2, int k,
              const orc_params* p, const double* X0,
              const int* replay_inner, int replay_outer,
              int* perm_out, double* X_out, int* inner_trace, double* delta_trace,
              orc_stats* st);

#ifdef __cplusplus
}
#endif
#endif
