/*
 * fastpfp_oracle.c -- plain FP64 CPU oracle for FastPFP.
 *
 * TEST INFRASTRUCTURE ONLY (see fastpfp_oracle.h).  Every function is a
 * direct transcription of the paper's definitions: plain loops, sums taken
 * in ascending index order, no blocking, fusion or algebraic rewriting.
 * OpenMP only splits independent output elements across threads; the
 * arithmetic of each element is the same for any thread count.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -shared -fPIC
 * (-ffp-contract=off keeps a*b+c as two rounded operations on every host, so
 * x86 and Arm builds give identical results).
 *
 * Parity status of each function (what pins it outside itself lives in
 * tests/test_oracle_*.py):
 *   orc_affinity, orc_gradient   pinned (finite differences of f, Sec. 4.1)
 *   orc_p1                       pinned (KKT least-squares solve, Eq. (P1))
 *   orc_p2                       pinned (definition of P2, Eq. (P2))
 *   orc_pd                       pinned (invariants, exact cases, Sec. 4.3)
 *   orc_blend                    pinned (closure, Theorem 1 rate, Sec. 4.1/4.4)
 *   orc_greedy_*                 pinned (each other, Hungarian on separable cases)
 *   orc_*_objective              pinned (brute force, Appendix identity)
 *   orc_solve                    pinned (exact recovery, brute force on N<=7)
 *   orc_solve, algorithm = PG    pinned (a feasible point is fixed at alpha = 0;
 *                                linear objective -> its assignment optimum;
 *                                relabelling equivariance)
 * The inner cap I_1, the slack carry-over and the comparison details are
 * readings of an underspecified paper; those choices are "parity unpinned".
 */
#include "fastpfp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* K = B B2^T, defined below Eq. (4): K_ij = sum_c B_ic B2_jc. */
void orc_affinity(const double* B, const double* B2, int N, int m, int k, double* K) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int c = 0; c < k; ++c) acc += B[(size_t)i * k + c] * B2[(size_t)j * k + c];
            K[(size_t)i * m + j] = acc;
        }
    }
}

/* Gradient of f(X) = 1/2 tr(X^T A X A2) + lambda tr(X^T K), Section 4.1:
 * grad f = A X A2 + lambda K.  T = A X (N x m), then G = T A2 + lambda K.
 * Each entry accumulates its products in ascending order of the summed index. */
void orc_gradient(const double* A, const double* X, const double* A2, const double* K,
                  double lambda, int N, int m, double* G) {
    double* T = (double*)malloc((size_t)N * m * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double* t = T + (size_t)i * m;
        for (int j = 0; j < m; ++j) t[j] = 0.0;
        for (int l = 0; l < N; ++l) {
            const double a = A[(size_t)i * N + l];
            const double* x = X + (size_t)l * m;
            for (int j = 0; j < m; ++j) t[j] += a * x[j];
        }
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double* g = G + (size_t)i * m;
        const double* t = T + (size_t)i * m;
        for (int j = 0; j < m; ++j) g[j] = 0.0;
        for (int l = 0; l < m; ++l) {
            const double a = t[l];
            const double* b = A2 + (size_t)l * m;
            for (int j = 0; j < m; ++j) g[j] += a * b[j];
        }
        if (lambda != 0.0 && K) {
            const double* kk = K + (size_t)i * m;
            for (int j = 0; j < m; ++j) g[j] += lambda * kk[j];
        }
    }
    free(T);
}

/* Row sums r = Y 1, column sums c = Y^T 1 and total s = 1^T Y 1 = sum_i r_i. */
static double row_col_sums(const double* Y, int N, double* r, double* c) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j) acc += Y[(size_t)i * N + j];
        r[i] = acc;
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < N; ++j) {
        double acc = 0.0;
        for (int i = 0; i < N; ++i) acc += Y[(size_t)i * N + j];
        c[j] = acc;
    }
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += r[i];
    return s;
}

/* Eq. (P1): P1(Y) = Y + (I/n + (1^T Y 1) I / n^2 - Y/n) 1 1^T - 1 1^T Y / n.
 * Entry (i,j) of the right-hand side is
 *   Y_ij + 1/n + s/n^2 - r_i/n - c_j/n,   r = Y1, c = Y^T 1, s = 1^T Y 1,
 * since (I/n) 1 1^T has every entry 1/n, (s I/n^2) 1 1^T every entry s/n^2,
 * (Y/n) 1 1^T has entry r_i/n and 1 1^T Y/n has entry c_j/n.  n is the size
 * of the square slacked matrix. */
static void p1_apply(double* Y, int N, const double* r, const double* c, double s) {
    const double n = (double)N;
    const double a = 1.0 / n + s / (n * n);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        const double ri = r[i] / n;
        double* y = Y + (size_t)i * N;
        for (int j = 0; j < N; ++j) y[j] = y[j] + a - ri - c[j] / n;
    }
}

void orc_p1(double* Y, int N) {
    double* r = (double*)malloc((size_t)N * sizeof(double));
    double* c = (double*)malloc((size_t)N * sizeof(double));
    const double s = row_col_sums(Y, N, r, c);
    p1_apply(Y, N, r, c, s);
    free(r);
    free(c);
}

/* Eq. (P2): (Y + |Y|)/2, i.e. the elementwise positive part. */
void orc_p2(double* Y, int N) {
    const size_t total = (size_t)N * N;
#pragma omp parallel for schedule(static)
    for (size_t e = 0; e < total; ++e) Y[e] = (Y[e] + fabs(Y[e])) / 2.0;
}

/* Successive projection of Section 4.3 as written in Algorithm 1: repeat
 * {P1; P2} until Y converges (Section 5: max|Y(u+1) - Y(u)| < eps_2, or the
 * cap I_1). */
int orc_pd(double* Y, int N, double tol, int max_iter, int fixed_iters, double* last_delta) {
    const size_t total = (size_t)N * N;
    double* Yo = (double*)malloc(total * sizeof(double));
    double* r = (double*)malloc((size_t)N * sizeof(double));
    double* c = (double*)malloc((size_t)N * sizeof(double));
    const int cap = fixed_iters > 0 ? fixed_iters : max_iter;
    int it = 0;
    double delta = 0.0;
    while (it < cap) {
        memcpy(Yo, Y, total * sizeof(double));
        const double s = row_col_sums(Y, N, r, c);
        p1_apply(Y, N, r, c, s);
        orc_p2(Y, N);
        ++it;
        delta = 0.0;
#pragma omp parallel for reduction(max : delta) schedule(static)
        for (size_t e = 0; e < total; ++e) {
            const double d = fabs(Y[e] - Yo[e]);
            if (d > delta) delta = d;
        }
        if (fixed_iters <= 0 && delta < tol) break;
    }
    if (last_delta) *last_delta = delta;
    free(Yo);
    free(r);
    free(c);
    return it;
}

/* Algorithm 1, the update and normalisation of X:
 *   X <- (1-alpha) X + alpha Y[:, :m];  X <- X / max(X). */
double orc_blend(double* X, const double* Y, int N, int m, double alpha, int normalize) {
    const size_t total = (size_t)N * m;
    double* Xn = (double*)malloc(total * sizeof(double));
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < m; ++j)
            Xn[(size_t)i * m + j] = (1.0 - alpha) * X[(size_t)i * m + j] + alpha * Y[(size_t)i * N + j];
    if (normalize) {
        double mx = -INFINITY;
        for (size_t e = 0; e < total; ++e)
            if (Xn[e] > mx) mx = Xn[e];
        for (size_t e = 0; e < total; ++e) Xn[e] = Xn[e] / mx;
    }
    double d = 0.0;
    for (size_t e = 0; e < total; ++e) {
        const double v = fabs(Xn[e] - X[e]);
        if (v > d) d = v;
        X[e] = Xn[e];
    }
    free(Xn);
    return d;
}

/* Section 4.5, Steps 1-3: L holds every index (i,j); repeatedly take the
 * maximum of X over L, record it, and drop every index sharing its row or
 * its column.  Scanning L in row-major order with a strict '>' keeps the
 * first (lowest-index) maximum. */
void orc_greedy_literal(const double* X, int N, int m, int* row_of_col) {
    unsigned char* row_live = (unsigned char*)malloc((size_t)N);
    unsigned char* col_live = (unsigned char*)malloc((size_t)m);
    memset(row_live, 1, (size_t)N);
    memset(col_live, 1, (size_t)m);
    for (int j = 0; j < m; ++j) row_of_col[j] = -1;
    const int rounds = N < m ? N : m;
    for (int t = 0; t < rounds; ++t) {
        int bi = -1, bj = -1;
        double bv = 0.0;
        for (int i = 0; i < N; ++i) {
            if (!row_live[i]) continue;
            for (int j = 0; j < m; ++j) {
                if (!col_live[j]) continue;
                const double v = X[(size_t)i * m + j];
                if (bi < 0 || v > bv) { bi = i; bj = j; bv = v; }
            }
        }
        row_of_col[bj] = bi;
        row_live[bi] = 0;
        col_live[bj] = 0;
    }
    free(row_live);
    free(col_live);
}

typedef struct { double v; long long idx; } orc_entry;

static int entry_cmp(const void* pa, const void* pb) {
    const orc_entry* a = (const orc_entry*)pa;
    const orc_entry* b = (const orc_entry*)pb;
    if (a->v > b->v) return -1;
    if (a->v < b->v) return 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

void orc_greedy_sorted(const double* X, int N, int m, int* row_of_col) {
    const size_t total = (size_t)N * m;
    orc_entry* e = (orc_entry*)malloc(total * sizeof(orc_entry));
    for (size_t t = 0; t < total; ++t) { e[t].v = X[t]; e[t].idx = (long long)t; }
    qsort(e, total, sizeof(orc_entry), entry_cmp);
    unsigned char* row_used = (unsigned char*)calloc((size_t)N, 1);
    unsigned char* col_used = (unsigned char*)calloc((size_t)m, 1);
    for (int j = 0; j < m; ++j) row_of_col[j] = -1;
    int left = N < m ? N : m;
    for (size_t t = 0; t < total && left > 0; ++t) {
        const int i = (int)(e[t].idx / m), j = (int)(e[t].idx % m);
        if (row_used[i] || col_used[j]) continue;
        row_used[i] = 1;
        col_used[j] = 1;
        row_of_col[j] = i;
        --left;
    }
    free(e);
    free(row_used);
    free(col_used);
}

/* Eq. (3) at a partial permutation P (P_ij = 1 iff i = row_of_col[j]):
 *   tr(P^T A P A2) = sum_{j,l} A[r(j), r(l)] A2[l, j],  tr(P^T K) = sum_j K[r(j), j]. */
double orc_qap_objective(const double* A, const double* A2, const double* K, double lambda,
                         const int* row_of_col, int N, int m) {
    double quad = 0.0;
    for (int j = 0; j < m; ++j) {
        const int rj = row_of_col[j];
        for (int l = 0; l < m; ++l) quad += A[(size_t)rj * N + row_of_col[l]] * A2[(size_t)l * m + j];
    }
    double lin = 0.0;
    if (K && lambda != 0.0)
        for (int j = 0; j < m; ++j) lin += K[(size_t)row_of_col[j] * m + j];
    return 0.5 * quad + lambda * lin;
}

/* Eq. (1) at a partial permutation: (P A2 P^T)_{ab} = A2[c(a), c(b)] when
 * rows a and b are both matched (c = column matched to a row), else 0;
 * (P B2)_a = B2[c(a)] when row a is matched, else 0. */
double orc_error_objective(const double* A, const double* A2, const double* B, const double* B2,
                           int k, double lambda, const int* row_of_col, int N, int m) {
    int* col_of_row = (int*)malloc((size_t)N * sizeof(int));
    for (int i = 0; i < N; ++i) col_of_row[i] = -1;
    for (int j = 0; j < m; ++j) col_of_row[row_of_col[j]] = j;
    double e1 = 0.0;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            const int ca = col_of_row[a], cb = col_of_row[b];
            const double pap = (ca >= 0 && cb >= 0) ? A2[(size_t)ca * m + cb] : 0.0;
            const double d = A[(size_t)a * N + b] - pap;
            e1 += d * d;
        }
    double e2 = 0.0;
    if (k > 0 && B && B2)
        for (int a = 0; a < N; ++a)
            for (int c = 0; c < k; ++c) {
                const double pb = col_of_row[a] >= 0 ? B2[(size_t)col_of_row[a] * k + c] : 0.0;
                const double d = B[(size_t)a * k + c] - pb;
                e2 += d * d;
            }
    free(col_of_row);
    return 0.5 * e1 + lambda * e2;
}

/* f(X) = 1/2 tr(X^T A X A2) + lambda tr(X^T K), Section 4.1. */
double orc_relaxed_objective(const double* A, const double* A2, const double* K, double lambda,
                             const double* X, int N, int m) {
    double* G = (double*)malloc((size_t)N * m * sizeof(double));
    orc_gradient(A, X, A2, NULL, 0.0, N, m, G); /* G = A X A2 */
    double quad = 0.0, lin = 0.0;
    for (size_t e = 0; e < (size_t)N * m; ++e) quad += X[e] * G[e];
    if (K && lambda != 0.0)
        for (size_t e = 0; e < (size_t)N * m; ++e) lin += X[e] * K[e];
    free(G);
    return 0.5 * quad + lambda * lin;
}

/* Algorithm 1 with the initialisation recommended after it
 * (X = 1 1^T / (n n'), Y = 0) and the stopping rules of Section 5.  With
 * algorithm = 1 the same loop runs the projected gradient method of
 * Eq. (pg) instead: Y_{1:n,1:n'} = X + alpha (A X A' + lambda K), then
 * X = P_d(.) = P_D(Y)_{1:n,1:n'} (the slack columns handled as for
 * FastPFP), optionally normalised by its maximum. */
int orc_solve(const double* A_in, int n_a, const double* A2_in, int n_b,
              const double* B_in, const double* B2_in, int k,
              const orc_params* p, const double* X0,
              const int* replay_inner, int replay_outer,
              int* perm_out, double* X_out, int* inner_trace, double* delta_trace,
              orc_stats* st) {
    if (!A_in || !A2_in || !p || !perm_out || n_a <= 0 || n_b <= 0 || k < 0) return -1;
    if (k > 0 && p->lambda != 0.0 && (!B_in || !B2_in)) return -1;
    /* Section 3 assumes n >= n' without loss of generality: swap otherwise. */
    const int transposed = n_a < n_b;
    const double* A = transposed ? A2_in : A_in;
    const double* A2 = transposed ? A_in : A2_in;
    const double* B = transposed ? B2_in : B_in;
    const double* B2 = transposed ? B_in : B2_in;
    const int N = transposed ? n_b : n_a;
    const int m = transposed ? n_a : n_b;
    const size_t NM = (size_t)N * m, NN = (size_t)N * N;

    double* K = NULL;
    const int use_k = (k > 0 && p->lambda != 0.0);
    if (use_k) {
        K = (double*)malloc(NM * sizeof(double));
        orc_affinity(B, B2, N, m, k, K);
    }
    double* X = (double*)malloc(NM * sizeof(double));
    double* Y = (double*)calloc(NN, sizeof(double));
    double* G = (double*)malloc(NM * sizeof(double));
    if (X0) {
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < m; ++j)
                X[(size_t)i * m + j] = transposed ? X0[(size_t)j * N + i] : X0[(size_t)i * m + j];
    } else {
        const double u = 1.0 / ((double)N * (double)m);
        for (size_t e = 0; e < NM; ++e) X[e] = u;
    }

    const int outer_cap = replay_outer > 0 ? replay_outer : p->max_outer;
    int t = 0, converged = 0, inner_total = 0, inner_max = 0;
    double delta = 0.0;
    while (t < outer_cap) {
        /* Y_{1:n,1:n'} = A X A' + lambda K (FastPFP) or X + alpha (A X A' + lambda K) (PG) */
        orc_gradient(A, X, A2, K, p->lambda, N, m, G);
        const int pg = p->algorithm == 1;
        for (int i = 0; i < N; ++i) {
            for (int j = 0; j < m; ++j)
                Y[(size_t)i * N + j] = pg ? X[(size_t)i * m + j] + p->alpha * G[(size_t)i * m + j]
                                          : G[(size_t)i * m + j];
            if (p->slack_policy == 1)
                for (int j = m; j < N; ++j) Y[(size_t)i * N + j] = 0.0;
        }
        const int fixed = replay_inner ? replay_inner[t] : 0;
        const int inner = orc_pd(Y, N, p->tol_inner, p->max_inner, fixed, NULL);
        /* FastPFP blends; PG takes the projection itself (a blend with weight 1) */
        delta = orc_blend(X, Y, N, m, pg ? 1.0 : p->alpha, p->normalize_max);
        if (inner_trace) inner_trace[t] = inner;
        if (delta_trace) delta_trace[t] = delta;
        inner_total += inner;
        if (inner > inner_max) inner_max = inner;
        ++t;
        if (delta < p->tol_outer) {
            converged = 1;
            if (replay_outer <= 0) break;
        }
    }

    int* row_of_col = (int*)malloc((size_t)m * sizeof(int));
    orc_greedy_literal(X, N, m, row_of_col);

    if (transposed) {
        /* caller's graph 1 is our column side: node j of graph 1 -> row */
        for (int j = 0; j < m; ++j) perm_out[j] = row_of_col[j];
    } else {
        for (int i = 0; i < N; ++i) perm_out[i] = -1;
        for (int j = 0; j < m; ++j) perm_out[row_of_col[j]] = j;
    }
    if (X_out) {
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < m; ++j) {
                if (transposed) X_out[(size_t)j * N + i] = X[(size_t)i * m + j];
                else X_out[(size_t)i * m + j] = X[(size_t)i * m + j];
            }
    }
    if (st) {
        st->outer_iters = t;
        st->inner_total = inner_total;
        st->inner_max = inner_max;
        st->converged = converged;
        st->transposed = transposed;
        st->final_delta = delta;
        st->objective = orc_qap_objective(A, A2, K, p->lambda, row_of_col, N, m);
        st->error = orc_error_objective(A, A2, use_k ? B : NULL, use_k ? B2 : NULL, use_k ? k : 0,
                                        p->lambda, row_of_col, N, m);
    }
    free(row_of_col);
    free(K);
    free(X);
    free(Y);
    free(G);
    return 0;
}
