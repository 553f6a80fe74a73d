/* rbffd_oracle.h -- TEST INFRASTRUCTURE, not part of the library.
 *
 * A plain, slow, single-threaded CPU restatement in FP64 of the overlapped RBF-FD
 * construction of the sparse Laplacian differentiation matrix (Shankar, "The Overlapped
 * RBF-FD Method", §2 and §4.1-§4.2.1).  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the CUDA library never does.
 *
 * Every structural quantity (squared distances, retention radii, comparisons) is evaluated
 * in a fixed left-to-right order with no fused multiply-add (compile with
 * -ffp-contract=off), so the CUDA path can reproduce kNN tables and retention balls
 * bit-for-bit.
 */
#ifndef RBFFD_ORACLE_H
#define RBFFD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_OK = 0, ORA_EINVAL = -1, ORA_EDUPLICATE = -2, ORA_ENOMEM = -3, ORA_ESINGULAR = -4 };
enum { ORA_OP_LAPLACIAN = 0, ORA_OP_IDENTITY = 1, ORA_OP_NORMAL = 2 };
enum { ORA_STAB_SEQ = 0, ORA_STAB_OFF = 1, ORA_STAB_FALLBACK = 2 };
/* Reference point of the Lebesgue test (§4.2.1): the stencil's own center, or the stencil
 * node nearest the centroid of the stencil. */
enum { ORA_LREF_CENTER = 0, ORA_LREF_CENTROID = 1 };

typedef struct {
    int64_t n_centers;      /* N_delta: stencils whose weights were kept (fallback stencils excluded) */
    int64_t n_fallback;     /* rows recomputed by their own delta=1 stencil (FALLBACK mode) */
    int64_t n_decisions;    /* Lebesgue tests made for non-center retained nodes */
    int64_t n_rejected;     /* of which failed  Lambda_i <= Lambda_ref */
    int64_t n_near_tie;     /* of which |margin| <= 1e-9 */
    int64_t sum_q;          /* rows written by centers (== N in SEQ/OFF) */
    int64_t sum_cols;       /* right-hand sides solved in total (reference points included) */
    double min_abs_margin;  /* min over decisions of |(L_ref - L_i) / L_ref| (inf if none) */
    int64_t n_boundary;     /* boundary rows (ora_assemble_bc) */
} ora_stats;

/* Degree rule of §2: 2D closed form s = floor((sqrt(4n+1)-3)/2); 3D: largest s with
 * C(s+3,3) <= n/2.  Returns s, and the number of monomials M through *M_out. */
int ora_degree_for_n(int n, int d, int* M_out);

/* Number of total-degree-<=ell monomials in d dimensions, and their exponents in graded
 * order (degree 0,1,...,ell; within a degree the first exponent descending, then the
 * second).  exps has room for M*d ints (may be NULL). */
int ora_poly_terms(int d, int ell, int* exps);

/* Brute-force exact kNN (§2, §4.1): for every node k the n nodes nearest to x_k ordered by
 * (squared distance, index); nbr[k*n+0] == k.  d2[k*n+t] is the squared distance of the
 * t-th neighbour.  Returns ORA_EDUPLICATE if some other node sits at distance 0. */
int ora_knn(const double* X, int64_t N, int d, int n, int32_t* nbr, double* d2);

/* Retention-ball sizes (§4.1): ball_len[k] = #{t : d2[k*n+t] <= ((1-delta)(1-delta)) rho_k^2},
 * rho_k^2 = d2[k*n+n-1]; always >= 1. */
int ora_ball_len(const double* d2, int64_t N, int n, double delta, int32_t* ball_len);

/* One local system (§4.1, the block system of the augmented method and its overlapped
 * multi-right-hand-side form): stencil nodes X[idx[0..n)] with idx[0] the center,
 * PHS r^m plus monomials of degree <= ell, operator `op` evaluated at the q points
 * Y[e*d..], e < q.  W[j*q+e] receives the weight of stencil node j for point e in the
 * original (unscaled) coordinates; lam[e] (may be NULL) the local L-Lebesgue value
 * sum_j |w| in the stencil's scaled coordinates. */
int ora_local_weights(const double* X, int d, const int32_t* idx, int n, int ell, int m, int op,
                      const double* Y, int q, double* W, double* lam);

/* As ora_local_weights, also for op = ORA_OP_NORMAL: the derivative along the unit normal
 * Nrm[e*d..] at evaluation point e (Nrm may be NULL for the other operators). */
int ora_local_weights_dn(const double* X, int d, const int32_t* idx, int n, int ell, int m,
                         int op, const double* Y, const double* Nrm, int q, double* W,
                         double* lam);

/* Full sequential construction of L (§4.1 traversal in index order, §4.2.1 stabilization).
 * Inputs: nodes X [N][d], the kNN table from ora_knn.  Outputs (all caller-allocated):
 * CSR row_ptr[N+1], col[N*n], val[N*n] with columns ascending; owner[N] = stencil that
 * produced each row; is_center[N] = 1 for centers, 2 for FALLBACK stencils, 0 otherwise;
 * lam_row[N] (may be NULL) = scaled Lebesgue value of each row under its stencil. */
int ora_assemble(const double* X, int64_t N, int d, int n, int ell, int m, double delta, int mode,
                 const int32_t* nbr, const double* d2, int64_t* row_ptr, int32_t* col,
                 double* val, int32_t* owner, uint8_t* is_center, double* lam_row,
                 ora_stats* stats);

/* ora_assemble with boundary nodes (§5): bc[i] = 0 interior, 1 Dirichlet, 2 Neumann (unit
 * outward normal nrm[i*d..], may be NULL without Neumann nodes).  The overlapped traversal
 * covers the interior only; every boundary node gets its own-stencil row: the identity
 * (Dirichlet) or the normal derivative (Neumann); is_center = 3 for those rows.  bc may be
 * NULL (no boundary: ora_assemble).  lref (ORA_LREF_*) picks the reference point of the
 * Lebesgue test: with ORA_LREF_CENTROID a retained member passes iff its value is <= the
 * value at the stencil node nearest the stencil's centroid (solved as one more point when it
 * is not a retained member); the center itself keeps its row either way. */
int ora_assemble_bc(const double* X, int64_t N, int d, int n, int ell, int m, double delta,
                    int mode, int lref, const uint8_t* bc, const double* nrm, const int32_t* nbr,
                    const double* d2, int64_t* row_ptr, int32_t* col, double* val,
                    int32_t* owner, uint8_t* is_center, double* lam_row, ora_stats* stats);

/* Mixed stencils: node k has its own n_k <= n_max, ell_k and m_k.  nbr/d2 from ora_knn with
 * n = n_max; node k's stencil is the first n_k entries.  Rows take the length of the stencil
 * that produced them: row_ptr[N+1], col/val with room for N*n_max entries. */
int ora_assemble_mixed(const double* X, int64_t N, int d, const int32_t* n_node,
                       const int32_t* ell_node, const int32_t* m_node, int n_max, double delta,
                       int mode, int lref, const int32_t* nbr, const double* d2, int64_t* row_ptr,
                       int32_t* col, double* val, int32_t* owner, uint8_t* is_center,
                       double* lam_row, ora_stats* stats);

#ifdef __cplusplus
}
#endif
#endif
