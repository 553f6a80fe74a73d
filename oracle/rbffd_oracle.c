/* rbffd_oracle.c -- TEST INFRASTRUCTURE: the CPU oracle for the overlapped RBF-FD
 * differentiation matrix.  Plain, slow, single-threaded, FP64, no blocking or fusion.
 * It shares no code with the CUDA library and is loaded only by the tests, the smoke
 * check and the benchmark's CPU-baseline leg.
 *
 * Paper: V. Shankar, "The Overlapped Radial Basis Function-Finite Difference (RBF-FD)
 * Method: A Generalization of RBF-FD".  Sections followed:
 *   §2      augmented local RBF interpolant, degree rule
 *   §4.1    stencils P_k, local block system, stencil width rho_k, retention distance
 *           r_k = (1-delta) rho_k, retention set R_k, multi-RHS system A_k W_k = B_k,
 *           scatter L(R_i, I_j) = W(j, i), "weights are never recomputed" traversal rule
 *   §4.2.1  local L-Lebesgue function Lambda = ||w||_1 and the acceptance test
 *           Lambda(x_i) <= Lambda(x_k)
 * Readings where the paper is silent or ambiguous (traversal = index order, closed ball,
 * reference point of the Lebesgue test = the stencil's own center, scaled local
 * coordinates, graded monomial order, ties in kNN by index) are the ones stated in the
 * header of each function below.
 *
 * Build with -ffp-contract=off: squared distances and radii must be formed without FMA.
 */
#include "rbffd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- small helpers */

/* Squared distance in the fixed order ((dx*dx + dy*dy) + dz*dz), each op rounded. */
static double sqdist(const double* a, const double* b, int d) {
    double t = a[0] - b[0];
    double s = t * t;
    t = a[1] - b[1];
    s = s + t * t;
    if (d == 3) {
        t = a[2] - b[2];
        s = s + t * t;
    }
    return s;
}

/* r^k for odd k >= 1 from r and r2 = r*r, by repeated multiplication: r * r2^((k-1)/2). */
static double odd_power(double r, double r2, int k) {
    double p = r;
    for (int s = 0; s < (k - 1) / 2; ++s) p = p * r2;
    return p;
}

/* x^e for a small non-negative integer e, by repeated multiplication. */
static double ipow(double x, int e) {
    double p = 1.0;
    for (int s = 0; s < e; ++s) p = p * x;
    return p;
}

static int64_t binom(int a, int b) {
    if (b < 0 || b > a) return 0;
    int64_t r = 1;
    for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

/* ---------------------------------------------------------------- §2 degree rule */

int ora_degree_for_n(int n, int d, int* M_out) {
    int s;
    if (n < 2 || (d != 2 && d != 3)) return ORA_EINVAL;
    if (d == 2) {
        /* the positive root of C(s+2,2) = n/2, rounded down */
        s = (int)floor(0.5 * (sqrt(4.0 * n + 1.0) - 3.0));
    } else {
        /* "solve a cubic": the largest s with C(s+3,3) <= n/2 */
        s = 0;
        while (2 * binom(s + 1 + 3, 3) <= n) ++s;
    }
    if (s < 0) s = 0;
    if (M_out) *M_out = (int)binom(s + d, d);
    return s;
}

/* ---------------------------------------------------------------- monomial basis (§2, §4.1) */

int ora_poly_terms(int d, int ell, int* exps) {
    int M = 0;
    for (int g = 0; g <= ell; ++g) {
        if (d == 2) {
            for (int a = g; a >= 0; --a) {
                if (exps) { exps[M * 2 + 0] = a; exps[M * 2 + 1] = g - a; }
                ++M;
            }
        } else {
            for (int a = g; a >= 0; --a)
                for (int b = g - a; b >= 0; --b) {
                    if (exps) {
                        exps[M * 3 + 0] = a; exps[M * 3 + 1] = b; exps[M * 3 + 2] = g - a - b;
                    }
                    ++M;
                }
        }
    }
    return M;
}

/* psi(x) = prod_a x_a^alpha_a */
static double mono(const double* x, const int* alpha, int d) {
    double p = 1.0;
    for (int a = 0; a < d; ++a) p = p * ipow(x[a], alpha[a]);
    return p;
}

/* Laplacian of psi: sum_a alpha_a (alpha_a - 1) x^(alpha - 2 e_a) */
static double lap_mono(const double* x, const int* alpha, int d) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
        if (alpha[a] < 2) continue;
        double p = (double)(alpha[a] * (alpha[a] - 1));
        for (int b = 0; b < d; ++b) p = p * ipow(x[b], b == a ? alpha[b] - 2 : alpha[b]);
        s = s + p;
    }
    return s;
}

/* Directional derivative of psi along nrm: sum_a nrm_a alpha_a x^(alpha - e_a) */
static double dn_mono(const double* x, const int* alpha, const double* nrm, int d) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
        if (alpha[a] < 1) continue;
        double p = (double)alpha[a];
        for (int b = 0; b < d; ++b) p = p * ipow(x[b], b == a ? alpha[b] - 1 : alpha[b]);
        s = s + nrm[a] * p;
    }
    return s;
}

/* ---------------------------------------------------------------- §2/§4.1 kNN */

int ora_knn(const double* X, int64_t N, int d, int n, int32_t* nbr, double* d2) {
    if (N < 1 || n < 1 || n > N || (d != 2 && d != 3)) return ORA_EINVAL;
    for (int64_t k = 0; k < N; ++k) {
        int32_t* bi = nbr + k * n;
        double* bd = d2 + k * n;
        int cnt = 0;
        for (int64_t j = 0; j < N; ++j) {
            double s = sqdist(X + k * d, X + j * d, d);
            /* is (s, j) smaller than the current n-th best (bd[n-1], bi[n-1])? */
            if (cnt == n && !(s < bd[n - 1] || (s == bd[n - 1] && j < bi[n - 1]))) continue;
            int pos = (cnt < n) ? cnt : n - 1;
            while (pos > 0 && (s < bd[pos - 1] || (s == bd[pos - 1] && j < bi[pos - 1]))) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = s;
            bi[pos] = (int32_t)j;
            if (cnt < n) ++cnt;
        }
        if (bi[0] != k) return ORA_EDUPLICATE; /* another node at distance 0 with lower index */
        for (int t = 1; t < n; ++t)
            if (bd[t] == 0.0) return ORA_EDUPLICATE;
    }
    return ORA_OK;
}

/* ---------------------------------------------------------------- §4.1 retention balls */

int ora_ball_len(const double* d2, int64_t N, int n, double delta, int32_t* ball_len) {
    if (!(delta > 0.0 && delta <= 1.0)) return ORA_EINVAL;
    double f = (1.0 - delta) * (1.0 - delta);
    for (int64_t k = 0; k < N; ++k) {
        double r2 = f * d2[k * n + n - 1];
        int len = 0;
        for (int t = 0; t < n; ++t)
            if (d2[k * n + t] <= r2) len = t + 1; /* d2 is sorted: the ball is a prefix */
        ball_len[k] = len;
    }
    return ORA_OK;
}

/* ---------------------------------------------------------------- dense LU (partial pivoting) */

/* In-place LU of the K x K row-major matrix A with partial pivoting: at step p the pivot is
 * the row with the largest |A[i][p]|, i >= p, the lowest such row on ties.  piv[p] is the
 * row swapped with p.  Returns ORA_ESINGULAR on an exactly zero pivot. */
static int lu_factor(double* A, int K, int* piv) {
    for (int p = 0; p < K; ++p) {
        int best = p;
        double bv = fabs(A[p * K + p]);
        for (int i = p + 1; i < K; ++i)
            if (fabs(A[i * K + p]) > bv) { bv = fabs(A[i * K + p]); best = i; }
        if (bv == 0.0) return ORA_ESINGULAR;
        piv[p] = best;
        if (best != p)
            for (int j = 0; j < K; ++j) {
                double t = A[p * K + j]; A[p * K + j] = A[best * K + j]; A[best * K + j] = t;
            }
        for (int i = p + 1; i < K; ++i) {
            double l = A[i * K + p] / A[p * K + p];
            A[i * K + p] = l;
            for (int j = p + 1; j < K; ++j) A[i * K + j] = A[i * K + j] - l * A[p * K + j];
        }
    }
    return ORA_OK;
}

/* Solve (LU) x = P b for one right-hand side b (overwritten by x). */
static void lu_solve(const double* A, int K, const int* piv, double* b) {
    for (int p = 0; p < K; ++p)
        if (piv[p] != p) { double t = b[p]; b[p] = b[piv[p]]; b[piv[p]] = t; }
    for (int i = 1; i < K; ++i) {          /* unit lower triangle */
        double s = b[i];
        for (int j = 0; j < i; ++j) s = s - A[i * K + j] * b[j];
        b[i] = s;
    }
    for (int i = K - 1; i >= 0; --i) {     /* upper triangle */
        double s = b[i];
        for (int j = i + 1; j < K; ++j) s = s - A[i * K + j] * b[j];
        b[i] = s / A[i * K + i];
    }
}

/* ---------------------------------------------------------------- §4.1 local system */

/* The stencil is scaled to local coordinates xi = (x - x_c) / rho_c with rho_c the stencil
 * width (§4.1).  The PHS space is invariant under this map (r^m only gains the factor
 * rho^-m) and so is the polynomial space, so the weights of the scaled problem are those
 * of the original one times rho^2 for the Laplacian (rho^0 for the identity). */
int ora_local_weights(const double* X, int d, const int32_t* idx, int n, int ell, int m, int op,
                      const double* Y, int q, double* W, double* lam) {
    if (op == ORA_OP_NORMAL) return ORA_EINVAL;  /* needs normals: ora_local_weights_dn */
    return ora_local_weights_dn(X, d, idx, n, ell, m, op, Y, NULL, q, W, lam);
}

/* The same with the operator ORA_OP_NORMAL allowed: the derivative along the unit vector
 * Nrm[e] at evaluation point e (§5, the Neumann operator of the boundary condition).  For
 * it the weights of the scaled problem are those of the original one times rho. */
int ora_local_weights_dn(const double* X, int d, const int32_t* idx, int n, int ell, int m,
                         int op, const double* Y, const double* Nrm, int q, double* W,
                         double* lam) {
    if ((d != 2 && d != 3) || n < 1 || q < 0 || m < 3 || (m % 2) == 0 || ell < 0 ||
        op < ORA_OP_LAPLACIAN || op > ORA_OP_NORMAL || (op == ORA_OP_NORMAL && !Nrm))
        return ORA_EINVAL;
    int M = ora_poly_terms(d, ell, NULL);
    if (M > n) return ORA_EINVAL;
    int K = n + M;
    int* alpha = (int*)malloc(sizeof(int) * M * d);
    double* A = (double*)calloc((size_t)K * K, sizeof(double));
    double* B = (double*)calloc((size_t)K * (q > 0 ? q : 1), sizeof(double));
    double* xi = (double*)malloc(sizeof(double) * n * d);
    double* eta = (double*)malloc(sizeof(double) * (q > 0 ? q : 1) * d);
    double* col = (double*)malloc(sizeof(double) * K);
    int* piv = (int*)malloc(sizeof(int) * K);
    int rc = ORA_OK;
    if (!alpha || !A || !B || !xi || !eta || !col || !piv) { rc = ORA_ENOMEM; goto done; }
    ora_poly_terms(d, ell, alpha);

    const double* xc = X + (int64_t)idx[0] * d;
    double rho2 = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = sqdist(xc, X + (int64_t)idx[j] * d, d);
        if (s > rho2) rho2 = s;
    }
    if (!(rho2 > 0.0)) rho2 = 1.0; /* single-node stencil: any scale */
    double rho = sqrt(rho2);
    for (int j = 0; j < n; ++j)
        for (int a = 0; a < d; ++a) xi[j * d + a] = (X[(int64_t)idx[j] * d + a] - xc[a]) / rho;
    for (int e = 0; e < q; ++e)
        for (int a = 0; a < d; ++a) eta[e * d + a] = (Y[(int64_t)e * d + a] - xc[a]) / rho;

    /* [ A  P ; P^T 0 ]: A_ij = ||xi_i - xi_j||^m, P_il = psi_l(xi_i) */
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double r2 = sqdist(xi + i * d, xi + j * d, d);
            double r = sqrt(r2);
            A[i * K + j] = odd_power(r, r2, m);
        }
        for (int l = 0; l < M; ++l) {
            double v = mono(xi + i * d, alpha + l * d, d);
            A[i * K + n + l] = v;
            A[(n + l) * K + i] = v;
        }
    }
    /* right-hand sides: L phi(||x - xi_j||) and L psi_l(x) at each evaluation point */
    for (int e = 0; e < q; ++e) {
        for (int j = 0; j < n; ++j) {
            double r2 = sqdist(eta + e * d, xi + j * d, d);
            double r = sqrt(r2);
            double v;
            if (op == ORA_OP_LAPLACIAN) {  /* Laplacian of r^m in d dims: m(m+d-2) r^(m-2) */
                v = (double)(m * (m + d - 2)) * odd_power(r, r2, m - 2);
            } else if (op == ORA_OP_NORMAL) {  /* d/dn r^m = m r^(m-2) (y - xi_j) . n */
                double dot = 0.0;
                for (int a = 0; a < d; ++a) dot = dot + (eta[e * d + a] - xi[j * d + a]) * Nrm[e * d + a];
                v = (double)m * odd_power(r, r2, m - 2) * dot;
            } else {
                v = odd_power(r, r2, m);
            }
            B[j * q + e] = v;
        }
        for (int l = 0; l < M; ++l) {
            double v;
            if (op == ORA_OP_LAPLACIAN) v = lap_mono(eta + e * d, alpha + l * d, d);
            else if (op == ORA_OP_NORMAL) v = dn_mono(eta + e * d, alpha + l * d, Nrm + e * d, d);
            else v = mono(eta + e * d, alpha + l * d, d);
            B[(n + l) * q + e] = v;
        }
    }

    rc = lu_factor(A, K, piv);
    if (rc != ORA_OK) goto done;
    for (int e = 0; e < q; ++e) {
        for (int i = 0; i < K; ++i) col[i] = B[i * q + e];
        lu_solve(A, K, piv, col);
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            s = s + fabs(col[j]);
            W[j * q + e] = (op == ORA_OP_LAPLACIAN) ? col[j] / rho2
                         : (op == ORA_OP_NORMAL) ? col[j] / rho : col[j];
        }
        if (lam) lam[e] = s;
    }
done:
    free(alpha); free(A); free(B); free(xi); free(eta); free(col); free(piv);
    return rc;
}

/* ---------------------------------------------------------------- §4.1/§4.2.1 traversal */

/* Sort row entries by column index (insertion sort; n is small). */
static void sort_row(int32_t* c, double* v, int n) {
    for (int a = 1; a < n; ++a) {
        int32_t ck = c[a];
        double vk = v[a];
        int b = a - 1;
        while (b >= 0 && c[b] > ck) { c[b + 1] = c[b]; v[b + 1] = v[b]; --b; }
        c[b + 1] = ck;
        v[b + 1] = vk;
    }
}

/* Write row i of L from stencil `stencil_idx` (n global indices) and its weights. */
static void put_row(int64_t i, int n, const int32_t* stencil_idx, const double* w, int stride,
                    int32_t* col, double* val) {
    for (int j = 0; j < n; ++j) {
        col[i * n + j] = stencil_idx[j];
        val[i * n + j] = w[(int64_t)j * stride];
    }
    sort_row(col + i * n, val + i * n, n);
}

/* Position t in stencil I (n nodes) of the node nearest the stencil's centroid (§4.2.1, the
 * reference point of the Lebesgue test in its centroid reading); ties go to the lower t.
 * The centroid is the mean of the n nodes: each coordinate summed over the stencil in kNN
 * order starting from 0.0, then divided by n. */
static int centroid_node(const double* X, int d, const int32_t* I, int n) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < d; ++a) {
        double s = 0.0;
        for (int t = 0; t < n; ++t) s = s + X[(int64_t)I[t] * d + a];
        c[a] = s / (double)n;
    }
    int best = 0;
    double bd = sqdist(X + (int64_t)I[0] * d, c, d);
    for (int t = 1; t < n; ++t) {
        double s = sqdist(X + (int64_t)I[t] * d, c, d);
        if (s < bd) { bd = s; best = t; }
    }
    return best;
}

/* Evaluation points of one center: the q retained members cols[0..q) (cols[0] = 0, the
 * center) and, with the centroid reference, the reference node appended when it is not one
 * of them.  Returns the number of points; *e_ref the point whose Lebesgue value the test
 * uses. */
static int eval_points(const double* X, int d, const int32_t* I, int n, int lref, int* cols,
                       int q, int* e_ref) {
    *e_ref = 0;
    if (lref != ORA_LREF_CENTROID) return q;
    const int t_ref = centroid_node(X, d, I, n);
    for (int e = 0; e < q; ++e)
        if (cols[e] == t_ref) { *e_ref = e; return q; }
    cols[q] = t_ref;
    *e_ref = q;
    return q + 1;
}

/* The traversal visits nodes in index order.  A node already given a row is never
 * recomputed (§4.1).  An uncovered node k becomes a center: its retention set R_k is the
 * part of the ball of radius (1-delta) rho_k (closed; the ball is a prefix of the kNN list)
 * not yet covered, k first.  One factorization, one solve per member of R_k.  Then, per
 * mode:
 *   SEQ      (§4.2.1) keep member i iff Lambda(x_i) <= Lambda(x_ref), Lambda = ||w||_1 of
 *            its column; rejected members stay uncovered and are reached later by the
 *            traversal (as a member of a later ball or as a center).  The reference point
 *            x_ref of the test is the stencil's own center x_k (ora_assemble), or the
 *            stencil node nearest the stencil's centroid (ora_assemble_bc with
 *            ORA_LREF_CENTROID); the center keeps its own row either way.
 *   OFF      keep every member.
 *   FALLBACK coverage as OFF; each member failing the test gets its row from its own
 *            delta = 1 stencil afterwards. */
int ora_assemble(const double* X, int64_t N, int d, int n, int ell, int m, double delta, int mode,
                 const int32_t* nbr, const double* d2, int64_t* row_ptr, int32_t* col,
                 double* val, int32_t* owner, uint8_t* is_center, double* lam_row,
                 ora_stats* st) {
    return ora_assemble_bc(X, N, d, n, ell, m, delta, mode, ORA_LREF_CENTER, NULL, NULL, nbr, d2,
                           row_ptr, col, val, owner, is_center, lam_row, st);
}

/* Boundary nodes (§5): bc[i] = 1 (Dirichlet) or 2 (Neumann), 0 for interior nodes.  The
 * overlapped traversal runs over the interior only: a boundary node is never a center of
 * it and never a member of a retention set, so its row is never produced by an interior
 * stencil (the interior block of N_delta = (N_i)_delta + N_b).  Each boundary node then
 * gets its own row B from its own stencil: the identity for Dirichlet (B_bb = I, B_bi = 0),
 * the derivative along its unit normal nrm[i] for Neumann.  Boundary rows have is_center
 * = 3 and are their own owners. */
int ora_assemble_bc(const double* X, int64_t N, int d, int n, int ell, int m, double delta,
                    int mode, int lref, const uint8_t* bc, const double* nrm, const int32_t* nbr,
                    const double* d2, int64_t* row_ptr, int32_t* col, double* val,
                    int32_t* owner, uint8_t* is_center, double* lam_row, ora_stats* st) {
    if (N < 1 || n < 1 || n > N || (d != 2 && d != 3) || m < 3 || (m % 2) == 0 ||
        !(delta > 0.0 && delta <= 1.0) || mode < 0 || mode > 2 || lref < 0 || lref > 1)
        return ORA_EINVAL;
    int M = ora_poly_terms(d, ell, NULL);
    if (M > n) return ORA_EINVAL;
    ora_stats s0;
    memset(&s0, 0, sizeof(s0));
    s0.min_abs_margin = INFINITY;

    int32_t* ball = (int32_t*)malloc(sizeof(int32_t) * N);
    uint8_t* covered = (uint8_t*)calloc((size_t)N, 1);
    uint8_t* redo = (uint8_t*)calloc((size_t)N, 1);
    double* Y = (double*)malloc(sizeof(double) * (n + 1) * d);  /* members + reference */
    double* W = (double*)malloc(sizeof(double) * n * (n + 1));
    double* lam = (double*)malloc(sizeof(double) * (n + 1));
    int* cols = (int*)malloc(sizeof(int) * (n + 1));
    int rc = ORA_OK;
    if (!ball || !covered || !redo || !Y || !W || !lam || !cols) { rc = ORA_ENOMEM; goto done; }
    rc = ora_ball_len(d2, N, n, delta, ball);
    if (rc != ORA_OK) goto done;
    for (int64_t i = 0; i < N; ++i) {
        owner[i] = -1;
        is_center[i] = 0;
        if (bc && bc[i] > 2) { rc = ORA_EINVAL; goto done; }
        if (bc && bc[i] == 2 && !nrm) { rc = ORA_EINVAL; goto done; }
    }

    for (int64_t k = 0; k < N; ++k) {
        if (covered[k] || (bc && bc[k])) continue;
        const int32_t* I = nbr + k * n;
        int q = 0;
        for (int t = 0; t < ball[k]; ++t) /* t = 0 is k itself, never covered here */
            if (!covered[I[t]] && !(bc && bc[I[t]])) cols[q++] = t;
        int e_ref;
        const int qe = eval_points(X, d, I, n, lref, cols, q, &e_ref);
        for (int e = 0; e < qe; ++e)
            for (int a = 0; a < d; ++a) Y[e * d + a] = X[(int64_t)I[cols[e]] * d + a];
        rc = ora_local_weights(X, d, I, n, ell, m, ORA_OP_LAPLACIAN, Y, qe, W, lam);
        if (rc != ORA_OK) goto done;
        is_center[k] = 1;
        s0.n_centers++;
        s0.sum_cols += qe;
        for (int e = 0; e < q; ++e) {
            int64_t i = I[cols[e]];
            int pass = 1;
            if (e > 0 && e != e_ref) {  /* (the reference node passes its own test) */
                double margin = (lam[e_ref] - lam[e]) / lam[e_ref];
                pass = lam[e] <= lam[e_ref];
                s0.n_decisions++;
                if (!pass) s0.n_rejected++;
                if (fabs(margin) < s0.min_abs_margin) s0.min_abs_margin = fabs(margin);
                if (fabs(margin) <= 1e-9) s0.n_near_tie++;
            }
            if (mode == ORA_STAB_SEQ && !pass) continue;
            covered[i] = 1;
            owner[i] = (int32_t)k;
            s0.sum_q++;
            if (lam_row) lam_row[i] = lam[e];
            if (mode == ORA_STAB_FALLBACK && !pass) { redo[i] = 1; continue; }
            put_row(i, n, I, W + e, qe, col, val);
        }
    }
    if (mode == ORA_STAB_FALLBACK) {
        for (int64_t i = 0; i < N; ++i) {
            if (!redo[i]) continue;
            const int32_t* I = nbr + i * n;
            rc = ora_local_weights(X, d, I, n, ell, m, ORA_OP_LAPLACIAN, X + i * d, 1, W, lam);
            if (rc != ORA_OK) goto done;
            owner[i] = (int32_t)i;
            is_center[i] = 2;
            s0.n_fallback++;
            s0.sum_cols++;
            if (lam_row) lam_row[i] = lam[0];
            put_row(i, n, I, W, 1, col, val);
        }
    }
    for (int64_t i = 0; bc && i < N; ++i) {
        if (!bc[i]) continue;
        const int32_t* I = nbr + i * n;
        if (bc[i] == 1) {  /* identity row */
            for (int j = 0; j < n; ++j) W[j] = (j == 0) ? 1.0 : 0.0;
            lam[0] = 1.0;
        } else {
            rc = ora_local_weights_dn(X, d, I, n, ell, m, ORA_OP_NORMAL, X + i * d, nrm + i * d, 1,
                                      W, lam);
            if (rc != ORA_OK) goto done;
            s0.sum_cols++;
        }
        owner[i] = (int32_t)i;
        is_center[i] = 3;
        s0.n_boundary++;
        if (lam_row) lam_row[i] = lam[0];
        put_row(i, n, I, W, 1, col, val);
    }
    for (int64_t i = 0; i <= N; ++i) row_ptr[i] = i * n;
done:
    if (st) *st = s0;
    free(ball); free(covered); free(redo); free(Y); free(W); free(lam); free(cols);
    return rc;
}

/* ---------------------------------------------------------------- mixed stencils */

/* The same traversal for node sets whose nodes carry their own stencil size n_k,
 * polynomial degree ell_k and PHS exponent m_k (e.g. a higher degree in part of the
 * domain).  nbr/d2 are the kNN lists of length n_max = max n_k (ora_knn); node k's stencil
 * is the first n_k entries of its list, its width rho_k the distance of the n_k-th.  A row
 * takes the stencil that produced it, so rows have the length n of that stencil; they are
 * stored by row_ptr (N+1), col/val hold up to N*n_max entries. */
int ora_assemble_mixed(const double* X, int64_t N, int d, const int32_t* n_node,
                       const int32_t* ell_node, const int32_t* m_node, int n_max, double delta,
                       int mode, int lref, const int32_t* nbr, const double* d2,
                       int64_t* row_ptr, int32_t* col, double* val, int32_t* owner,
                       uint8_t* is_center, double* lam_row, ora_stats* st) {
    if (N < 1 || n_max < 1 || n_max > N || (d != 2 && d != 3) || !(delta > 0.0 && delta <= 1.0) ||
        mode < 0 || mode > 2 || lref < 0 || lref > 1)
        return ORA_EINVAL;
    for (int64_t k = 0; k < N; ++k) {
        if (n_node[k] < 1 || n_node[k] > n_max || m_node[k] < 3 || (m_node[k] % 2) == 0 ||
            ell_node[k] < 0 || ora_poly_terms(d, ell_node[k], NULL) > n_node[k])
            return ORA_EINVAL;
    }
    ora_stats s0;
    memset(&s0, 0, sizeof(s0));
    s0.min_abs_margin = INFINITY;
    const double f = (1.0 - delta) * (1.0 - delta);
    int32_t* ball = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* src = (int32_t*)malloc(sizeof(int32_t) * N);   /* stencil of each row */
    int32_t* rcol = (int32_t*)malloc(sizeof(int32_t) * N * n_max);
    double* rval = (double*)malloc(sizeof(double) * N * n_max);
    uint8_t* covered = (uint8_t*)calloc((size_t)N, 1);
    uint8_t* redo = (uint8_t*)calloc((size_t)N, 1);
    double* Y = (double*)malloc(sizeof(double) * (n_max + 1) * d);  /* members + reference */
    double* W = (double*)malloc(sizeof(double) * n_max * (n_max + 1));
    double* lam = (double*)malloc(sizeof(double) * (n_max + 1));
    int* cols = (int*)malloc(sizeof(int) * (n_max + 1));
    int rc = ORA_OK;
    if (!ball || !src || !rcol || !rval || !covered || !redo || !Y || !W || !lam || !cols) {
        rc = ORA_ENOMEM;
        goto done;
    }
    for (int64_t k = 0; k < N; ++k) {  /* retention balls with each node's own width */
        const int nk = n_node[k];
        const double r2 = f * d2[k * n_max + nk - 1];
        int len = 0;
        for (int t = 0; t < nk; ++t)
            if (d2[k * n_max + t] <= r2) len = t + 1;
        ball[k] = len;
        owner[k] = -1;
        is_center[k] = 0;
    }
    for (int64_t k = 0; k < N; ++k) {
        if (covered[k]) continue;
        const int32_t* I = nbr + k * n_max;
        const int nk = n_node[k];
        int q = 0;
        for (int t = 0; t < ball[k]; ++t)
            if (!covered[I[t]]) cols[q++] = t;
        int e_ref;
        const int qe = eval_points(X, d, I, nk, lref, cols, q, &e_ref);
        for (int e = 0; e < qe; ++e)
            for (int a = 0; a < d; ++a) Y[e * d + a] = X[(int64_t)I[cols[e]] * d + a];
        rc = ora_local_weights(X, d, I, nk, ell_node[k], m_node[k], ORA_OP_LAPLACIAN, Y, qe, W,
                               lam);
        if (rc != ORA_OK) goto done;
        is_center[k] = 1;
        s0.n_centers++;
        s0.sum_cols += qe;
        for (int e = 0; e < q; ++e) {
            int64_t i = I[cols[e]];
            int pass = 1;
            if (e > 0 && e != e_ref) {  /* (the reference node passes its own test) */
                double margin = (lam[e_ref] - lam[e]) / lam[e_ref];
                pass = lam[e] <= lam[e_ref];
                s0.n_decisions++;
                if (!pass) s0.n_rejected++;
                if (fabs(margin) < s0.min_abs_margin) s0.min_abs_margin = fabs(margin);
                if (fabs(margin) <= 1e-9) s0.n_near_tie++;
            }
            if (mode == ORA_STAB_SEQ && !pass) continue;
            covered[i] = 1;
            owner[i] = (int32_t)k;
            s0.sum_q++;
            if (lam_row) lam_row[i] = lam[e];
            if (mode == ORA_STAB_FALLBACK && !pass) { redo[i] = 1; continue; }
            src[i] = (int32_t)k;
            for (int j = 0; j < nk; ++j) {
                rcol[i * n_max + j] = I[j];
                rval[i * n_max + j] = W[(int64_t)j * qe + e];
            }
        }
    }
    if (mode == ORA_STAB_FALLBACK) {
        for (int64_t i = 0; i < N; ++i) {
            if (!redo[i]) continue;
            const int32_t* I = nbr + i * n_max;
            const int ni = n_node[i];
            rc = ora_local_weights(X, d, I, ni, ell_node[i], m_node[i], ORA_OP_LAPLACIAN,
                                   X + i * d, 1, W, lam);
            if (rc != ORA_OK) goto done;
            owner[i] = (int32_t)i;
            is_center[i] = 2;
            s0.n_fallback++;
            s0.sum_cols++;
            if (lam_row) lam_row[i] = lam[0];
            src[i] = (int32_t)i;
            for (int j = 0; j < ni; ++j) {
                rcol[i * n_max + j] = I[j];
                rval[i * n_max + j] = W[j];
            }
        }
    }
    row_ptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        const int len = n_node[src[i]];
        row_ptr[i + 1] = row_ptr[i] + len;
        for (int j = 0; j < len; ++j) {
            col[row_ptr[i] + j] = rcol[i * n_max + j];
            val[row_ptr[i] + j] = rval[i * n_max + j];
        }
        sort_row(col + row_ptr[i], val + row_ptr[i], len);
    }
done:
    if (st) *st = s0;
    free(ball); free(src); free(rcol); free(rval); free(covered); free(redo);
    free(Y); free(W); free(lam); free(cols);
    return rc;
}
