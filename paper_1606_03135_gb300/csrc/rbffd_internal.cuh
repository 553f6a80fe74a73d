// rbffd_internal.cuh -- shared declarations of the GB300 overlapped RBF-FD library.
//
// Device memory layout of one plan (N nodes, stencil size n, dimension D):
//   X        [N][D]  f64   node coordinates (copied from the caller)
//   nbr      [N][n]  i32   kNN stencil of every node, ordered by (squared distance, index)
//   rho2     [N]     f64   squared stencil width rho_k^2 (distance of the n-th neighbour)
//   ball_len [N]     i32   retention-ball size; the ball is the prefix nbr[k][0..ball_len)
//   indeg    [N]     i32   #{j < k : k in ball(j)}  (dependencies of k in the traversal)
//   slot_off [N+1]   i64   exclusive prefix sum of ball_len: weight slot of (stencil j, ball
//                          position t) is slot_off[j] + t
//   slot_w   [S][n]  f64   weights of a solved column (S = slot_off[N])
//   CSR      row_ptr [N+1] i64, col [N n] i32, val [N n] f64
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rbffd.h"

namespace rbffd {

constexpr int kMaxStencil = 128;  // n
constexpr int kMaxEll = 8;
constexpr int kMaxTerms = 165;    // C(8 + 3, 3)
constexpr int kWarp = 32;

// node states of the traversal
constexpr int kUndecided = 0;
constexpr int kCenter = 1;
constexpr int kCovered = 2;
constexpr int kBoundary = 3;  // boundary node: outside the overlapped traversal
constexpr int kNoOwner = 0x7fffffff;

struct GridParams {
    double lo[3];
    double h;      // cell edge
    double inv_h;  // 1 / h
    int dims[3];
    int ncell;
    int r0;        // first search ring (in cells)
    float xerr;    // FP32 screen of the kNN: bound on |fl32(fl32(a) - fl32(b))| - |a - b|
};

// Bounding-box accumulators of the grid build (zeroed before the launch): nlo holds the
// complement of the smallest order-preserving key, so both bounds grow by atomicMax from zero.
struct BBoxAcc {
    unsigned long long nlo[3];
    unsigned long long hi[3];
    unsigned int done;
};

// Device-side counters and status of one plan (one 256-byte block; zeroed per call).
struct DevCounters {
    int status;              // first error code (RBFFD_*), 0 = OK
    int n_singular;
    int max_ball;
    int q_head;              // next queue slot to claim
    int q_tail;              // next queue slot to fill
    int fb_count;            // fallback rows
    int done;                // nodes whose traversal state is final
    int abort;               // set when a bounded wait ran out: every worker leaves
    unsigned long long n_centers;
    unsigned long long n_rejected;
    unsigned long long sum_cols;
    unsigned long long n_fallback;
    unsigned long long sum_k3;   // sum over factored stencils of K^3
    unsigned long long sum_k2q;  // sum over factored stencils of K^2 (rows they own)
    unsigned long long n_spec;       // speculative solves made by idle CTAs
    unsigned long long n_spec_used;  // centers that found their solve already made
    int spec_next;                   // next node an idle CTA considers for speculation
    int pad_i;
    unsigned long long sum_k2c;      // sum over factored stencils of K^2 (columns solved)
    unsigned long long sum_k2r;      // sum over refined solves of K^2 (columns refined)
    unsigned long long pad[15];
};

// Map a CUDA status to an RBFFD code; with RBFFD_DEBUG set in the environment the failing
// call is named on stderr.
int cuda_status(cudaError_t e, const char* what, int line);
#define RB_CUDA(call) ::rbffd::cuda_status((call), #call, __LINE__)
#define RB_LAUNCHED(what) ::rbffd::cuda_status(cudaGetLastError(), what, __LINE__)

__device__ __forceinline__ void set_error(DevCounters* c, int code) {
    atomicCAS(&c->status, 0, code);
}

// ((dx*dx + dy*dy) + dz*dz), every operation rounded separately (no FMA), x_a - y_a order.
template <int D>
__device__ __forceinline__ double sqdist_rn(const double* a, const double* b) {
    double t = __dsub_rn(a[0], b[0]);
    double s = __dmul_rn(t, t);
    t = __dsub_rn(a[1], b[1]);
    s = __dadd_rn(s, __dmul_rn(t, t));
    if (D == 3) {
        t = __dsub_rn(a[2], b[2]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// squared distances are >= 0, so their IEEE bit patterns order like the values
__device__ __forceinline__ unsigned long long dkey(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ host-side launchers
struct PlanDev;  // defined in api.cu

// Exact kNN with n neighbours per node; with node_n (device, may be NULL) node q's stencil,
// width and ball use only its first node_n[q] neighbours.
int launch_grid_and_knn(int D, const double* X, int N, int n, double omd2, void* scratch_grid,
                        size_t scratch_bytes, int ncell_max, int* nbr, double* rho2, int* ball_len,
                        int* indeg, const int* node_n, DevCounters* ctr, cudaStream_t s,
                        int* launches);
size_t grid_scratch_bytes(int N, int D, int ncell_max);
// Retention balls, in-degrees and max_ball (ctr) of another delta from an existing plan's
// stencils nbr / rho2 (k_balls).
int launch_balls(int D, const double* X, int N, int n, double omd2, const int* nbr,
                 const double* rho2, const int* node_n, int* ball_len, int* indeg,
                 DevCounters* ctr, cudaStream_t s, int* launches);

int launch_scan_i32_to_i64(const int* in, long long* out, int count, cudaStream_t s,
                           int* launches);

struct SolveArgs {
    const double* X;
    const int* nbr;
    const double* rho2;
    const int* ball_len;
    const long long* slot_off;
    const short* basis;        // monomial recurrence and Laplacian tables (see assemble.cu)
    int basis_count;           // shorts in `basis` (tables of every degree in use)
    int boff[kMaxEll + 1];     // offset of degree ell's tables in `basis`
    int Mof[kMaxEll + 1];      // number of monomials of degree <= ell
    // Per-node stencil parameters (NULL: every node uses n, ell, m).  n is also the row stride
    // of nbr and of a weight slot (the largest stencil size); M and K are the largest.
    const int* node_n;
    const signed char* node_ell;
    const signed char* node_m;
    const unsigned char* bc;   // boundary kind per node (0 interior, 1 Dirichlet, 2 Neumann) or null
    int* spec;                 // per node: 0 none, 1 speculative solve running, 2 made, 3 singular
    const double* nrm;         // unit normals [N][d] of Neumann nodes (or null)
    int N, n, M, K, m, ell;
    int qcap;                  // right-hand-side columns carried per factorization
    int qmax;                  // columns of the largest ball
    int stride;                // row stride of the full matrix (LU) or of the RHS block (LDL^T)
    int mode;                  // RBFFD_STAB_*
    const unsigned char* ref_pos;  // centroid reference of the Lebesgue test: its stencil
                                   // position per node (nullptr: the stencil's center)
    double coef;               // m (m + D - 2)
    int no_seed;               // fault injection: push no initial center (waits run out)
    int factor;                // RBFFD_FACTOR_LDLT (packed layout) or RBFFD_FACTOR_LU (full)
    int max_ctas;              // cap on the persistent grid (0 = fill the GPU)
    int elastic;               // > 0: a CTA holding no queue slot leaves when this many wait
    int fma_r2;                // 1: squared distances of the local systems with FMA (plans
                               // that refine nothing), 0: rounded like the oracle's
    // One step of iterative refinement of ill-conditioned LDL^T local solves, in plans whose
    // largest system has K >= refine_min_K: per-CTA scratch of rs_stride doubles at
    // rs + blockIdx.x rs_stride holding the assembled matrix in full (K x K) and, from offset
    // rs_x0, the first solution of a chunk of right-hand sides and the residual's partial sums
    // (K x q each, 5 in all; rs == nullptr: the plan refines nothing).
    double* rs;
    long long rs_stride;
    int rs_x0;
    int refine_min_K;
    int refine_all;            // 1: refine every system; 0: only those whose pivot ratio
                               // max |d| / min |d| reaches 2^16 (ill-conditioned)

    unsigned long long timeout_ns;
    // traversal state
    int* state;
    int* pending;
    int* owner;
    int* queue;
    unsigned char* fb_flag;
    int* fb_list;
    // results
    double* slot_w;
    double* slot_lam;
    unsigned char* slot_pass;
    DevCounters* ctr;
};

size_t solve_smem_per_cta(int n, int K, int qcap, int qmax, int D, int packed,
                          int* stride_out);
size_t basis_smem_bytes(int count);

// Launch geometry decided once per plan.  Fallback re-solves run per stencil class (one
// class per polynomial degree for per-node stencils, one class otherwise).
struct FallbackClass {
    int cls;        // degree handled (-1: every node)
    int n, K, xs;   // largest stencil / system of the class, right-hand-side stride
    int nt, grid;
    size_t smem;
    long long rs_stride;  // refinement scratch per CTA of this class's launch (doubles)
    int rs_x0;
};
struct LaunchPlan {
    int force_nt = 0;  // 0: choose; 32 .. 512: forced team size of the traversal
    int refine_min_K = 0x7fffffff;  // systems this large are refined (their teams carry the step)
    int nt = 128, grid = 0;
    bool chunked = false;  // some balls have more columns than one factorization carries
    size_t smem = 0;
    int n_fb = 0;
    FallbackClass fb[kMaxEll + 1];
};
int prepare_solve_kernels(int D, int packed, int n, int K, int qcap, int qmax, int basis_count,
                          LaunchPlan* lp);
int launch_centroid_ref(int D, const double* X, const int* nbr, const int* node_n, int N, int ns,
                        unsigned char* ref_pos, cudaStream_t s, int* launches);
int launch_traversal(int D, const SolveArgs& a, const LaunchPlan& lp, const int* indeg,
                     cudaStream_t s, int* launches, cudaEvent_t ev0, cudaEvent_t ev1);
int launch_fallback(int D, const SolveArgs& a, const LaunchPlan& lp, cudaStream_t s,
                    int* launches);
int launch_finalize(const SolveArgs& a, long long* row_ptr, int* col, double* val,
                    double* lam_row, unsigned char* is_center, cudaStream_t s, int* launches);
int launch_spmv(int N, int n, const long long* row_ptr, const int* col, const double* val,
                const double* u, double* y, cudaStream_t s, int* launches);
int launch_timestep(int N, const long long* row_ptr, const int* col, const double* val,
                    const unsigned char* bc, double c, double* out, cudaStream_t s, int* launches);

}  // namespace rbffd
