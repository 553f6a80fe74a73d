/* rbffd.h -- C ABI of the GB300 library that forms the sparse Laplacian differentiation
 * matrix L of the overlapped RBF-FD method (V. Shankar, "The Overlapped Radial Basis
 * Function-Finite Difference (RBF-FD) Method: A Generalization of RBF-FD").
 *
 * The method (§4.1): every node x_k has a stencil P_k = x_k and its n-1 nearest
 * neighbours.  Visiting nodes in index order, a node not yet given a row becomes a stencil
 * center; its retention ball of radius (1-delta) rho_k (rho_k = stencil width) selects
 * the nodes whose Laplacian weights this one stencil computes: one factorization of the
 * (n+M) x (n+M) block system [Phi P; P^T 0] (polyharmonic spline r^m, monomials of total
 * degree <= ell, M of them) and one solve per retained node.  §4.2.1 keeps a retained
 * node only if its local L-Lebesgue value ||w||_1 does not exceed that of the center.
 * Rows are never recomputed by a later stencil.  The result is CSR.
 *
 * Conventions for every entry point:
 *   - Return 0 on success or a negative RBFFD_E* code; nothing throws, traps or exits.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is enqueued on it; device outputs are valid once the stream has completed.
 *   - Device pointers are plain CUDA device (or managed) pointers on the current device.
 *   - Nodes are row-major [N][d] FP64; all indices are 0-based int32.
 *   - One plan may be used by one host thread at a time; distinct plans may run
 *     concurrently on distinct streams.
 */
#ifndef RBFFD_H
#define RBFFD_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ error codes */
#define RBFFD_OK 0
#define RBFFD_EINVAL -1      /* bad argument (see each call) */
#define RBFFD_EDUPLICATE -2  /* two nodes coincide: some stencil system is singular */
#define RBFFD_ENOMEM -3      /* device allocation failed */
#define RBFFD_ESINGULAR -4   /* an exactly zero pivot in some local system */
#define RBFFD_ETIMEOUT -5    /* a bounded device-side wait ran out (work queue stalled) */
#define RBFFD_ECUDA -6       /* a CUDA runtime call failed */
#define RBFFD_ESTATE -7      /* call out of order (e.g. apply before assemble) */

/* ------------------------------------------------------------------ options */
#define RBFFD_STAB_SEQ 0      /* §4.2.1 test as printed; rejected nodes stay uncovered and are
                                 reached later by the traversal (default) */
#define RBFFD_STAB_OFF 1      /* no Lebesgue test: every retained node is kept */
#define RBFFD_STAB_FALLBACK 2 /* coverage as OFF; a node failing the test gets its row from
                                 its own delta = 1 stencil */

/* Factorization of the local symmetric saddle-point system (§4.1, §4.3 "one matrix
 * decomposition").  LDLT: symmetric indefinite LDL^T with Bunch-Kaufman pivoting,
 * (1/3) K^3 flops; LU: partial-pivot LU, (2/3) K^3 flops.  Same weights up to rounding. */
#define RBFFD_FACTOR_LDLT 0
#define RBFFD_FACTOR_LU 1

/* Reference point of the Lebesgue test (§4.2.1): the stencil's own center (default), or the
 * stencil node nearest the stencil's centroid (the centroid is the sum of the n stencil nodes
 * in kNN order divided by n; ties to the nearer kNN position).  With the centroid a retained
 * node passes iff its value is <= the value at that node, which is solved as one more
 * right-hand side when it is not a retained node; the center keeps its own row either way. */
#define RBFFD_LREF_CENTER 0
#define RBFFD_LREF_CENTROID 1

typedef struct {
    int stab_mode;      /* RBFFD_STAB_* */
    int nodes_on_host;  /* 1: `nodes` is a host pointer, copied to the device by rbffd_plan */
    int timeout_ms;     /* limit for any single device-side wait; <= 0 means 5000 */
    int sync;           /* 1 (default): rbffd_assemble waits for the stream and reports device
                           errors; 0: fully asynchronous, errors surface in rbffd_stats */
    int fault_inject;   /* tests only: 1 = seed no work, so every traversal wait runs out and
                           rbffd_assemble returns RBFFD_ETIMEOUT after timeout_ms; 0 = off */
    int factor;         /* RBFFD_FACTOR_LDLT (default) or RBFFD_FACTOR_LU */
    int max_ctas;       /* cap on the persistent traversal grid, so that plans assembled
                           concurrently on several streams share the GPU; 0 = fill the GPU */
    int team;           /* threads per stencil team: 0 = chosen from the shared-memory
                           footprint (96 for LDL^T, or 128 if that keeps more stencils
                           resident, when more than 4 fit an SM and the plan does not
                           refine; 256 when 2 to 4 fit, or more for a plan that refines;
                           512 when one fits), or 32 (one warp per stencil), 64, 96, 128,
                           256 or 512 to force one (used by the schedule autotuner); 32, 64,
                           96 and 256 need RBFFD_FACTOR_LDLT, else RBFFD_EINVAL; 96 and 128
                           are refused for plans that refine (see refine) */
    int rhs_chunk;      /* right-hand sides carried through one factorization (RBFFD_FACTOR_LDLT):
                           a center with more columns solves the rest afterwards, this many at
                           a time, with the stored factors (same results, bit for bit).  0 = all
                           columns of the largest retention ball when that system fits shared
                           memory, else the largest count that fits; k >= 1 = at most k (fewer
                           columns per CTA can keep more stencils resident per SM: a tuning
                           knob, see autotune).  Values < 0, or > 0 with RBFFD_FACTOR_LU, give
                           RBFFD_EINVAL */
    int lebesgue_ref;   /* RBFFD_LREF_CENTER (default) or RBFFD_LREF_CENTROID; the centroid
                           reference solves no center ahead of its turn */
    int refine;         /* one step of iterative refinement of the LDL^T local solves of plans
                           whose largest system has K >= RBFFD_REFINE_MIN_K (degree-4 and -5
                           stencils in 3D reach condition numbers near 1e10, where the first
                           solution's error is dominated by the symmetric-pivoting
                           factorization): RBFFD_REFINE_AUTO (default) refines a system when its
                           pivots span at least 2^16 (max |d| / min |d| over the D blocks, a
                           lower bound of its condition number); RBFFD_REFINE_ALL refines every
                           system of every plan; RBFFD_REFINE_NONE none.  The residual b - A x0 is formed
                           in FP64 with the assembled system (copied to the plan's assembly
                           memory before the factorization: one full K x K copy per resident
                           CTA) and the correction is solved with
                           the stored factors (about 4 K^2 flops per refined column).  With a
                           Lebesgue test (SEQ, FALLBACK) a column whose first Lebesgue value
                           exceeds the test's reference by more than 2^-10 of it is not
                           refined: it fails the test either way and its weights are
                           discarded; the matrix is the same as with every column refined.  The
                           traversal's 96- and 128-thread teams have no refinement step, so
                           forcing them (opts.team) on a plan that refines is RBFFD_EINVAL.
                           RBFFD_FACTOR_LU is never refined.  Other values: RBFFD_EINVAL */
    int elastic;        /* 0 (default): the persistent traversal grid keeps every CTA until the
                           traversal is done; T > 0: a CTA that has finished a center leaves
                           instead of claiming the next queue entry when at least T others are
                           already waiting for entries (the dependency tail of delta < 1), so a
                           kernel launched beside it (another plan's assembly on another stream)
                           takes over its SM.  The matrix does not change.  Fewer waiting CTAs
                           also means fewer solves made ahead, so a plan assembled alone is not
                           faster with it.  < 0: RBFFD_EINVAL */
} rbffd_opts;

#define RBFFD_REFINE_AUTO 0
#define RBFFD_REFINE_ALL 1
#define RBFFD_REFINE_NONE 2
#define RBFFD_REFINE_MIN_K 100

typedef struct rbffd_plan_s* rbffd_plan_t; /* opaque; owned by the library */

/* CSR of L.  Device pointers owned by the plan; valid until the next rbffd_assemble on
 * the same plan or rbffd_destroy.  Each row has n entries (the size of the stencil that
 * produced it, for rbffd_plan_mixed), columns ascending.  nnz is -1 when it is not known yet
 * (per-node stencils assembled with opts.sync = 0: read it from rbffd_stats). */
typedef struct {
    int64_t n_rows;
    int64_t nnz;
    const int64_t* row_ptr; /* [n_rows + 1] */
    const int32_t* col;     /* [nnz] */
    const double* val;      /* [nnz] */
} rbffd_csr;

typedef struct {
    int64_t n_nodes;        /* N */
    int64_t n_centers;      /* N_delta: stencils factored for the final matrix */
    int64_t n_fallback;     /* rows recomputed by their own delta = 1 stencil */
    int64_t n_rejected;     /* retained nodes that failed the Lebesgue test at their
                               final owner-candidate stencils (all solved columns) */
    int64_t sum_cols;       /* right-hand sides solved in total */
    int64_t max_ball;       /* largest retention ball (columns per stencil, upper bound) */
    int64_t n_singular;     /* stencils with an exactly zero pivot */
    int32_t status;         /* device status of the last assemble (RBFFD_OK or an error) */
    int32_t n, M, K, d;     /* stencil size, monomials, n + M, dimension */
    double alg_flops;       /* §4.3 cost model for the result: sum over factored stencils of
                               c K^3 + 2 K^2 q_k, q_k = rows the stencil kept, c = 1/3 (LDLT)
                               or 2/3 (LU) */
    int64_t n_launches;     /* kernels this plan has launched so far (cumulative) */
    float ms_stencils;      /* device time of the kNN/retention-ball phase of rbffd_plan */
    float ms_traversal;     /* device time of the traversal + local-solve kernel */
    float ms_fallback;      /* device time of the FALLBACK re-solves (0 otherwise) */
    float ms_finalize;      /* device time of the CSR scatter */
    int64_t nnz;            /* entries of L (N n for uniform stencils) */
    int64_t plan_bytes;     /* device memory the plan holds after rbffd_plan */
    int64_t assemble_bytes; /* device memory rbffd_assemble adds (exact, known after plan) */
    int64_t n_boundary;      /* boundary rows (rbffd_set_boundary) */
    int64_t n_speculated;    /* solves made ahead by CTAs that found no ready center */
    int64_t n_spec_used;     /* centers whose solve had been made ahead */
    int64_t rhs_chunk;       /* right-hand sides carried per factorization (opts.rhs_chunk as
                                chosen by rbffd_plan) */
    double sum_k3;           /* sum over factored stencils of K^3 */
    double sum_k2_cols;      /* sum over factored stencils of K^2 q_k, q_k = the columns the
                                result needed (every retained node solved, kept or not) */
    double flops_refine;     /* refinement work executed: 4 K^2 per refined column */
    int32_t refine_min_K;    /* systems with K >= this are refined (INT32_MAX: none) */
    int32_t pad0;
} rbffd_stats_t;

/* rbffd_plan -- build the stencils of §4.1 for one node set.
 *   nodes   [N][d] FP64, device pointer (or host if opts->nodes_on_host); copied, so the
 *           caller may free it once the stream has completed.
 *   N       number of nodes, n <= N <= 2^31 - 1.
 *   d       2 or 3.
 *   n       stencil size (x_k and its n-1 nearest neighbours by (squared distance,
 *           index)), M <= n <= 128.
 *   ell     degree of the appended polynomial (§2), 0 <= ell <= 8; M = C(ell+d, d).
 *   m       PHS exponent, odd, 3 <= m <= 15.
 *   delta   overlap parameter (§4.1), 0 < delta <= 1; delta = 1 is standard RBF-FD.
 *   opts    NULL for defaults.
 *   out     receives the plan.
 * Runs the exact kNN search and the retention balls on the device and waits for the
 * stream once (to size the local systems).  Each local system lives in one SM's shared
 * memory with q of its right-hand sides: with K = n + M, about 8 (K (K + 1) / 2 + K q + 6 K)
 * bytes (LU option: 8 K (K + q + 4)) must fit the device's per-block limit (227 KB on GB300).
 * LU carries every column (q = the largest retention ball); LDL^T carries opts->rhs_chunk
 * columns and solves the rest in chunks of that many, so its limit is q = 1: in 3D,
 * n = 128 with degree 7 (K = 248) is too large.  Else RBFFD_EINVAL.  Errors: RBFFD_EINVAL,
 * RBFFD_EDUPLICATE, RBFFD_ENOMEM, RBFFD_ECUDA.  On error *out is NULL and nothing leaks. */
int rbffd_plan(const double* nodes, int64_t N, int d, int n, int ell, int m, double delta,
               const rbffd_opts* opts, void* stream, rbffd_plan_t* out);

/* rbffd_plan_mixed -- as rbffd_plan, for node sets whose nodes carry their own stencil size
 * n_node[k], polynomial degree ell_node[k] and PHS exponent m_node[k] (host arrays of N
 * int32, copied; same limits as rbffd_plan's scalars, M_k <= n_k).  Node k's stencil is x_k
 * and its n_k - 1 nearest neighbours, its width and retention ball follow from that
 * stencil, and a row of L takes the stencil that produced it, so rows have the length n of
 * that stencil (row_ptr gives them; nnz is known once rbffd_assemble has completed).  The
 * paper uses one n and ell everywhere (§4.1); this extends the traversal unchanged. */
int rbffd_plan_mixed(const double* nodes, int64_t N, int d, const int32_t* n_node,
                     const int32_t* ell_node, const int32_t* m_node, double delta,
                     const rbffd_opts* opts, void* stream, rbffd_plan_t* out);

/* rbffd_plan_delta -- a plan for the node set, stencil sizes, degrees and PHS exponents of
 * base (built by rbffd_plan or rbffd_plan_mixed) with another overlap parameter delta (§4.1)
 * and options opts (NULL for defaults).  The kNN stencils and widths do not depend on delta,
 * so they are copied from base on the device instead of searched again; the retention balls
 * (closed, radius (1 - delta) rho_k, squared distances formed as rbffd_plan forms them) and the
 * traversal's in-degrees are recomputed.  The result is the plan rbffd_plan would build for
 * these arguments: the same stencils, balls and, after rbffd_assemble, the same matrix bit for
 * bit.  base's stencils are complete when rbffd_plan returns, so base may be assembling on
 * another stream meanwhile; it must stay alive until this call returns and may be destroyed
 * after it (the copies are done by then).  Boundary nodes (rbffd_set_boundary) are not
 * carried over.  Like rbffd_plan, waits for the stream once; for a per-node plan it also
 * copies the per-node parameters back to the host first.  Errors: RBFFD_EINVAL (base or out
 * NULL, delta outside (0, 1], bad opts), RBFFD_ENOMEM, RBFFD_ECUDA.  On error *out is NULL. */
int rbffd_plan_delta(rbffd_plan_t base, double delta, const rbffd_opts* opts, void* stream,
                     rbffd_plan_t* out);

/* rbffd_assemble -- the traversal of §4.1 with the stabilization of §4.2.1: greedy center
 * selection, one factorization per center, multi-right-hand-side solves, Lebesgue test
 * and scatter into CSR (owned by the plan, described through *out, which may be NULL).
 * With opts.sync = 1 it waits for the stream and returns RBFFD_ESINGULAR / RBFFD_ETIMEOUT
 * from the device; the CSR pointers are valid either way once the stream completes. */
int rbffd_assemble(rbffd_plan_t plan, void* stream, rbffd_csr* out);

/* rbffd_apply -- y = L u (§5 use of L).  u [N], y [N]: FP64 device pointers owned by the
 * caller; must not overlap.  RBFFD_ESTATE before the first assemble. */
int rbffd_apply(rbffd_plan_t plan, const double* u, double* y, void* stream);

/* rbffd_stats -- counters of the last plan/assemble (waits for nothing; values produced by
 * an asynchronous assemble are complete once its stream has completed and a later call
 * refreshed them: rbffd_stats itself synchronises the plan's last stream). */
int rbffd_stats(rbffd_plan_t plan, rbffd_stats_t* out);

/* rbffd_export -- copy L and the stencil ownership to host memory (tests, serving).
 * row_ptr [N+1], col [nnz], val [nnz], owner [N] (stencil that produced each row;
 * a FALLBACK row names itself).  Any pointer may be NULL to skip it.  Synchronous. */
int rbffd_export(rbffd_plan_t plan, int64_t* row_ptr, int32_t* col, double* val,
                 int32_t* owner);

/* rbffd_export_async -- rbffd_export enqueued on `stream` (a CUDA stream, NULL for the legacy
 * default stream) without waiting: the copies start once the plan's last assembly has
 * finished and are complete when `stream` reaches them, so one plan's copies can overlap
 * another plan's assembly (host buffers should be pinned for that).  Later work on the plan
 * (an assembly, rbffd_stats, rbffd_destroy) waits for the copies.  nnz must be known without
 * waiting: always for uniform stencils (N n); for per-node stencils assembled with
 * opts.sync = 0, only once rbffd_stats has been called after the assembly, else
 * RBFFD_ESTATE.  Other errors: RBFFD_EINVAL, RBFFD_ECUDA. */
int rbffd_export_async(rbffd_plan_t plan, int64_t* row_ptr, int32_t* col, double* val,
                       int32_t* owner, void* stream);

/* rbffd_export_stencils -- copy the kNN stencils to host memory: nbr [N][n] (nbr[k][0] ==
 * k, ordered by (squared distance, index); n is the largest stencil size of the plan; for
 * rbffd_plan_mixed row k holds node k's n_k nearest and -1 after them), rho2 [N] (squared
 * stencil width), ball_len [N] (retention-ball size; the ball is the prefix
 * nbr[k][0..ball_len)).  NULL skips. */
int rbffd_export_stencils(rbffd_plan_t plan, int32_t* nbr, double* rho2, int32_t* ball_len);

/* rbffd_export_lambda -- scaled local Lebesgue value of every row under the stencil that
 * produced it (§4.2.1), and is_center [N] (1 center, 2 fallback stencil, 0 otherwise). */
int rbffd_export_lambda(rbffd_plan_t plan, double* lam_row, uint8_t* is_center);

/* rbffd_stencils_noalloc -- the stencil step of rbffd_plan (kNN by (squared distance,
 * index), stencil width, retention-ball size) for callers that cannot allocate device
 * memory while they run: for example a solver that hands all device memory to its own pool
 * before the run starts, or a loop with a fixed time budget that must not wait on the
 * allocator.  The paper has no counterpart; this is a service of the library.
 *   nodes    [N][d] FP64 device pointer; nbr [N][n] int32, rho2 [N] FP64, ball_len [N] int32
 *            device pointers to caller-owned outputs (same contents as rbffd_export_stencils
 *            of a plan built with the same arguments).
 *   N        1 <= n <= N <= RBFFD_NOALLOC_MAX_NODES; larger N returns RBFFD_EINVAL and
 *            writes nothing.  d, n, delta as for rbffd_plan.
 * It allocates nothing: its working memory is one fixed array in the library's device
 * memory (about 2 MB, held on every GPU that loads the library until the process exits).
 * The first call on a device looks that array's device address up for the current device
 * and keeps it for the process; after cudaDeviceReset of that device the kept address is no
 * longer valid, so the call must not be used on that device again in the process.  All calls
 * share the array, so calls that overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller; each call clears the status it reads.  Every call
 * ends by copying the device status to the host and waiting for `stream`
 * (RBFFD_EDUPLICATE for coincident nodes), so no call can be made while `stream` is being
 * captured into a CUDA graph. */
#define RBFFD_NOALLOC_MAX_NODES 32768
int rbffd_stencils_noalloc(const double* nodes, int64_t N, int d, int n, double delta,
                           int32_t* nbr, double* rho2, int32_t* ball_len, void* stream);

/* rbffd_set_boundary -- mark boundary nodes (§5: the method-of-lines system, whose boundary
 * block B replaces the Laplacian rows of the boundary nodes).
 *   plan     a plan from rbffd_plan (per-node plans: RBFFD_EINVAL)
 *   bc       host array [N]: 0 interior, 1 Dirichlet, 2 Neumann (other values: RBFFD_EINVAL);
 *            NULL removes the boundary
 *   normals  host array [N][d] row-major: the unit outward normal of each Neumann node (other
 *            rows are ignored); may be NULL when no node is Neumann (else RBFFD_EINVAL);
 *            non-finite entries of Neumann rows: RBFFD_EINVAL
 * Takes effect at the next rbffd_assemble: the overlapped traversal then runs over the
 * interior only (a boundary node is never a center and never in a retention set, so
 * N_delta = (N_i)_delta + N_b), and every boundary node gets its own-stencil row: the identity
 * for Dirichlet (B_bb = I, B_bi = 0), the derivative along its normal for Neumann.  Those rows
 * have is_center = 3 (rbffd_export_lambda) and are their own owners.  Both arrays are copied;
 * the call waits for the plan's last stream. */
int rbffd_set_boundary(rbffd_plan_t plan, const uint8_t* bc, const double* normals);

/* rbffd_timestep_matrix -- values of the time-stepping matrix of §5 on L's sparsity pattern:
 * interior row i: e_i - c L_i (c = nu dt for backward Euler, (12/25) nu dt for BDF4), boundary
 * row: B_i unchanged.
 *   val_out  device array of nnz doubles (the count rbffd_assemble reported), caller-owned;
 *            entry k pairs with L's col[k]
 * Needs an assembled plan (else RBFFD_ESTATE).  Asynchronous on `stream`. */
int rbffd_timestep_matrix(rbffd_plan_t plan, double c, double* val_out, void* stream);

/* rbffd_destroy -- free the plan and everything it owns (waits for its last stream). */
void rbffd_destroy(rbffd_plan_t plan);

/* rbffd_strerror -- static description of an error code. */
const char* rbffd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
