// assemble.cu -- the overlapped RBF-FD traversal (§4.1) with local L-Lebesgue stabilization
// (§4.2.1), the local FP64 solves, the CSR scatter and y = L u.
//
// Traversal as a dataflow.  The sequential rule "visit k = 0..N-1; an uncovered k becomes a
// center and keeps the members of its retention ball that pass the Lebesgue test" has a
// unique outcome: k is a center iff no earlier center keeps it, and a row belongs to the
// earliest center keeping it.  Whether center j keeps node i depends only on stencil j and
// x_i, so node k's fate is final as soon as every earlier node whose ball contains k (its
// in-neighbours, counted in `indeg`) is final.  A persistent kernel runs this: a node whose
// in-neighbours are all final and none kept it is pushed to a work queue as a center; a CTA
// pops it, factors its local system once, solves the right-hand sides of its still-open
// ball members, and then (i) marks the members it keeps as covered and (ii) releases one
// dependency of each later ball member.  Every device-side wait is bounded by a timeout and
// ends the kernel with RBFFD_ETIMEOUT.
//
// Local solve (one team of 32 to 512 threads per stencil).  The (n+M) x (n+M) saddle-point
// matrix [A P; P^T 0] of §4.1 and the q right-hand sides of the overlapped system (one per
// solved ball member) are assembled in shared memory.  The matrix is symmetric, so by
// default its lower triangle is stored packed and factored as L D L^T with Bunch-Kaufman
// pivoting, the right-hand sides carried along ((1/3) K^3 + 2 K^2 q flops); the paper's
// partial-pivot LU of the full [A_hat | B_hat] array ((2/3) K^3 + 2 K^2 q) is the
// RBFFD_FACTOR_LU option.  Every FP64 warp instruction occupies all 32 lanes of the narrow
// FP64 pipe whatever its active mask, so the updates are flattened over (row, column) pairs
// to keep lanes busy, and scalar work (pivot tests, reciprocals, square roots) is moved to
// the integer and FP32 pipes where it can be.
//
// Own-stencil rows (one right-hand side): FALLBACK re-solves of rows that failed the test,
// and the boundary rows of §5 (Dirichlet identity, Neumann normal derivative).
#include <cuda_runtime.h>

#include <mutex>

#include "fp64_int.cuh"
#include "rbffd_internal.cuh"

namespace rbffd {

constexpr int kNT = 128;     // default stencil team: one warp per SM sub-partition
constexpr int kMaxNT = 512;  // largest team (big systems, when few fit in shared memory)
constexpr int kMidNT = 256;  // fallback solves with two to four systems per SM
// Device code is compiled for a team size NT of 128 (small systems, many per SM) or 512
// (large systems, one or a few per SM); the LDL^T traversal also for 96, 64 and 32 (one warp
// per stencil), the fallback solves also for 256 (two to four systems per SM).  The host
// picks the instantiation per launch.

// CTAs per SM the register allocation must allow for a team size (the shared-memory limit of
// small systems): 40 registers for 96- and 128-thread teams, 64 for 32-, 64- and 256-thread
// teams.
__host__ __device__ constexpr int team_min_blocks(int nt) {
    return nt == 32 ? 32 : (nt == 64 ? 16 : (nt == 96 ? 16 : (nt == 128 ? 12 : (nt == 256 ? 4 : 1))));
}

// Per-CTA shared-memory views of one local system.  Two layouts:
//   full   (LU):     A is K x S row-major holding [A_hat | B_hat]; X = A + K, xs = S
//   packed (LDL^T):  T holds the lower triangle of A_hat by rows (row i starts at i(i+1)/2);
//                    X is the K x q right-hand-side block with row stride xs (odd)
struct StencilSmem {
    double* A;
    double* T;
    double* X;
    int xs;
    double* xi;     // n x D scaled stencil coordinates
    double* rdiag;  // K reciprocal pivots (LDL^T: 1x1 reciprocal; for a 2x2 block at rows p,
                    //   p+1 the inverse's entry 00 at p and entry 11 at p+1)
    double* dinv1;  // K  LDL^T 2x2 inverse entry 01 (at the block's first row)
    double* wv;     // K  unscaled pivot column(s) of the current LDL^T step
    double* wv2;    // K
    int* perm;      // K  original unknown held by each row (symmetric pivoting)
    int* rowof;     // K  row holding each original unknown
    unsigned char* pk;  // K  1: 1x1 pivot, 2: first row of a 2x2 pivot, 0: its second row
    double* lam;    // qmax Lebesgue values of the solved columns (all chunks)
    int* cols;      // qmax ball position of each solved column
    int* colof;     // n column of each ball position, or -1
    unsigned char* keep;  // qmax kept-for-coverage flags
};

__host__ __device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }

// Squared distance of two scaled stencil nodes inside a local system, with FMA:
// fma(t_D, t_D, ... fma(t_1, t_1, t_0 t_0)), t_c = a_c - b_c (6 FP64 operations in 3D instead
// of 8).  Symmetric in a and b (b - a = -(a - b) exactly).  Only the local systems of plans
// that refine nothing use it (a.fma_r2): ill-conditioned systems amplify its different
// rounding, so plans that refine keep sqdist_rn (no FMA, as the oracle forms it), and so do
// the stencils, balls and every structural comparison.
template <int D>
__device__ __forceinline__ double sqdist_local(const double* a, const double* b) {
    double t = __dsub_rn(a[0], b[0]);
    double s = __dmul_rn(t, t);
#pragma unroll
    for (int c = 1; c < D; ++c) {
        t = __dsub_rn(a[c], b[c]);
        s = __fma_rn(t, t, s);
    }
    return s;
}

// Monomial basis tables in shared memory (built on the host in graded order):
//   psi_l = psi_parent[l] * xi_var[l]            (l >= 1; psi_0 = 1)
//   Laplacian psi_l = sum_a lap_coef[l][a] * psi_lap_child[l][a]
struct Basis {
    const short* parent;
    const short* var;
    const short* lap_child;
    const short* lap_coef;
};

// The parameters of one stencil: size n, monomials M, system size K = n + M, PHS exponent m,
// right-hand-side factor m (m + D - 2) and the basis tables of its degree.
struct Shape {
    int n, M, K, m;
    double coef;
    Basis bs;
};

template <int D>
__device__ __forceinline__ Shape shape_of(const SolveArgs& a, const short* sbasis, int j) {
    const int ell = a.node_ell ? (int)a.node_ell[j] : a.ell;
    Shape s;
    s.n = a.node_n ? a.node_n[j] : a.n;
    s.M = a.Mof[ell];
    s.K = s.n + s.M;
    s.m = a.node_m ? (int)a.node_m[j] : a.m;
    s.coef = exact_double(s.m * (s.m + D - 2));
    const short* b = sbasis + a.boff[ell];
    s.bs.parent = b;
    s.bs.var = b + s.M;
    s.bs.lap_child = b + 2 * s.M;
    s.bs.lap_coef = b + 2 * s.M + s.M * D;
    return s;
}

// Bytes of one CTA's local system; *stride_out is S (full) or xs (packed).
size_t solve_smem_per_cta(int n, int K, int qcap, int qmax, int D, int packed,
                          int* stride_out) {
    int stride = packed ? qcap : K + qcap;
    if ((stride & 1) == 0) ++stride;  // odd row stride: column walks hit distinct banks
    if (stride_out) *stride_out = stride;
    const size_t mat = packed ? ((size_t)tri(K) + 1) / 2 * 2 + (size_t)K * stride
                              : (size_t)K * stride;
    size_t b = mat * 8 + (size_t)n * D * 8 + (size_t)K * 4 * 8 + (size_t)qmax * 8 +
               (size_t)(qmax + n) * 4 + (size_t)K * 2 * 4 + (size_t)K + (size_t)qmax;
    return (b + 15) & ~size_t(15);
}

size_t basis_smem_bytes(int count) { return ((size_t)count * sizeof(short) + 15) & ~size_t(15); }

template <int D, bool PACKED>
__device__ __forceinline__ void carve(char* p, int n, int K, int qmax, int S, StencilSmem& sm) {
    if (PACKED) {
        sm.A = nullptr;
        sm.T = reinterpret_cast<double*>(p);
        p += ((size_t)tri(K) + 1) / 2 * 2 * 8;
        sm.X = reinterpret_cast<double*>(p);
        sm.xs = S;
        p += (size_t)K * S * 8;
    } else {
        sm.A = reinterpret_cast<double*>(p);
        sm.T = nullptr;
        sm.X = sm.A + K;
        sm.xs = S;
        p += (size_t)K * S * 8;
    }
    sm.xi = reinterpret_cast<double*>(p);
    p += (size_t)n * D * 8;
    sm.rdiag = reinterpret_cast<double*>(p);
    p += (size_t)K * 8;
    sm.dinv1 = reinterpret_cast<double*>(p);
    p += (size_t)K * 8;
    sm.wv = reinterpret_cast<double*>(p);
    p += (size_t)K * 8;
    sm.wv2 = reinterpret_cast<double*>(p);
    p += (size_t)K * 8;
    sm.lam = reinterpret_cast<double*>(p);
    p += (size_t)qmax * 8;
    sm.cols = reinterpret_cast<int*>(p);
    p += (size_t)qmax * 4;
    sm.colof = reinterpret_cast<int*>(p);
    p += (size_t)n * 4;
    sm.perm = reinterpret_cast<int*>(p);
    p += (size_t)K * 4;
    sm.rowof = reinterpret_cast<int*>(p);
    p += (size_t)K * 4;
    sm.pk = reinterpret_cast<unsigned char*>(p);
    p += (size_t)K;
    sm.keep = reinterpret_cast<unsigned char*>(p);
}

__device__ __forceinline__ const short* load_basis(char* smem, const short* g, int count) {
    short* s = reinterpret_cast<short*>(smem);
    for (int e = threadIdx.x; e < count; e += blockDim.x) s[e] = g[e];
    return s;
}

// Assemble the local system of stencil j (§4.1) and its q right-hand sides (the columns in
// sm.cols) in shared memory, with the whole CTA.  Full layout: both triangles of A_hat and
// B_hat beside it.  Packed layout: the lower triangle of A_hat and B_hat apart.
template <int D, bool PACKED, int NT>
__device__ void assemble_local(const SolveArgs& a, const Shape& sh, int j, int q,
                               const StencilSmem& sm) {
    const int tid = threadIdx.x;
    const int n = sh.n, M = sh.M, K = sh.K, m = sh.m;
    const Basis& bs = sh.bs;
    double* X = sm.X;
    const int xs = sm.xs;
    const double* xc = a.X + (size_t)j * D;
    // Scaled coordinates (x - x_c) / rho_j, correctly rounded: the weights of ill-conditioned
    // stencils are as sensitive to the node positions as to the solve, so these match the
    // oracle's exactly.  Only the threads that hold a node compute rho_j.
    if (tid < n) {
        double r2c = a.rho2[j];
        if (__double_as_longlong(r2c) <= 0) r2c = 1.0;
        const double rho = sqrt(r2c);
        for (int t = tid; t < n; t += NT) {
            const int id = a.nbr[(size_t)j * a.n + t];
            for (int c = 0; c < D; ++c)
                sm.xi[t * D + c] = __ddiv_rn(__dsub_rn(a.X[(size_t)id * D + c], xc[c]), rho);
        }
    }
    if (PACKED) {
        for (int e = tid; e < tri(K); e += NT) sm.T[e] = 0.0;
        for (int e = tid; e < K * q; e += NT) {
            const int r = e / q, c = e - r * q;
            X[r * xs + c] = 0.0;
        }
    } else {
        const int Wd = K + q, S = xs;
        for (int e = tid; e < K * Wd; e += NT) {
            const int r = e / Wd, c = e - r * Wd;
            sm.A[r * S + c] = 0.0;
        }
    }
    __syncthreads();
    // A_ab = r^m and, for solved ball members, the phi-part of the right-hand side
    // m (m + D - 2) r^(m-2) (Laplacian of r^m in D dimensions), pair by pair
    // (pairs a < b; row a of the strict upper triangle has n-1-a entries, and rows a and
    // n-2-a together have n, so the flattened index steps in O(1))
    if (n > 1) {
        const int rows = n - 1, L2 = n;
        const int total = ((rows + 1) >> 1) * L2;
        int pr = tid / L2, off = tid - (tid / L2) * L2;
        const int di = NT / L2, dj = NT - di * L2;
        for (int e = tid; e < total; e += NT) {
            const int len0 = rows - pr;
            const bool first = off < len0;
            const int ra = first ? pr : rows - 1 - pr;
            const int t = first ? off : off - len0;
            if (first || ra != pr) {
                const int rb = ra + 1 + t;
                const double r2 = a.fma_r2 ? sqdist_local<D>(sm.xi + ra * D, sm.xi + rb * D)
                                           : sqdist_rn<D>(sm.xi + ra * D, sm.xi + rb * D);
                const double r = sqrt_fast(r2);
                double pm2 = r;
                for (int s = 0; s < (m - 3) / 2; ++s) pm2 = __dmul_rn(pm2, r2);
                const double pm = __dmul_rn(pm2, r2);
                if (PACKED) {
                    sm.T[tri(rb) + ra] = pm;
                } else {
                    sm.A[ra * xs + rb] = pm;
                    sm.A[rb * xs + ra] = pm;
                }
                const int ca = sm.colof[ra], cb = sm.colof[rb];
                if (cb >= 0 && cb < q) X[ra * xs + cb] = __dmul_rn(sh.coef, pm2);
                if (ca >= 0 && ca < q) X[rb * xs + ca] = __dmul_rn(sh.coef, pm2);
            }
            pr += di;
            off += dj;
            if (off >= L2) { off -= L2; ++pr; }
        }
    }
    // P: one stencil point per thread, each monomial = an earlier one times one coordinate
    for (int r = tid; r < n; r += NT) {
        if (PACKED) {
            sm.T[tri(n) + r] = 1.0;
            for (int l = 1; l < M; ++l)
                sm.T[tri(n + l) + r] = sm.T[tri(n + bs.parent[l]) + r] * sm.xi[r * D + bs.var[l]];
        } else {
            double* row = sm.A + r * xs + n;
            row[0] = 1.0;
            sm.A[n * xs + r] = 1.0;
            for (int l = 1; l < M; ++l) {
                const double v = row[bs.parent[l]] * sm.xi[r * D + bs.var[l]];
                row[l] = v;
                sm.A[(n + l) * xs + r] = v;
            }
        }
    }
    __syncthreads();
    // psi-part of the right-hand sides: Laplacian of each monomial at each solved member,
    // from the monomial values already computed for that member
    for (int e = tid; e < M * q; e += NT) {
        const int l = e / q, c = e - l * q;
        const int t = sm.cols[c];
        double s = 0.0;
        for (int d = 0; d < D; ++d) {
            const int ch = bs.lap_child[l * D + d];
            if (ch >= 0) {
                const double pv = PACKED ? sm.T[tri(n + ch) + t] : sm.A[t * xs + n + ch];
                s = fma(exact_double(bs.lap_coef[l * D + d]), pv, s);
            }
        }
        X[(n + l) * xs + c] = s;
    }
    __syncthreads();
}

// LU with partial pivoting of [A_hat | B_hat] in the full layout (the paper's decomposition,
// §4.3 cost model (2/3) K^3 + 2 K^2 q), then back substitution.  Returns false (uniformly)
// on an exactly zero pivot; on success row r of the right-hand-side block holds unknown r.
template <int NT>
__device__ bool factor_solve_lu(int K, int q, const StencilSmem& sm) {
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int S = sm.xs;
    const int Wd = K + q;
    for (int r = tid; r < K; r += NT) { sm.rowof[r] = r; sm.perm[r] = r; }  // unknowns stay in place
    // the pivot search, row swap, reciprocal and multipliers are done by warp 0 alone (FP64
    // work counts per warp instruction, so the other warps must not repeat it)
    for (int p = 0; p < K; ++p) {
        if (wid == 0) {
            unsigned long long bv = 0ull;
            int bi = 0x7fffffff;
            for (int i = p + lane; i < K; i += 32) {
                const unsigned long long v = abs_bits(sm.A[i * S + p]);
                if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (bv == 0ull) {
                if (lane == 0) s_ok = 0;
            } else {
                if (bi != p) {
                    for (int c = p + lane; c < Wd; c += 32) {
                        const double t = sm.A[p * S + c];
                        sm.A[p * S + c] = sm.A[bi * S + c];
                        sm.A[bi * S + c] = t;
                    }
                    __syncwarp();
                }
                const double rcp = rcp_fixed(sm.A[p * S + p]);
                if (lane == 0) { sm.rdiag[p] = rcp; s_ok = 1; }
                for (int i = p + 1 + lane; i < K; i += 32) sm.A[i * S + p] *= rcp;
            }
        }
        __syncthreads();
        if (!s_ok) return false;
        const int wr = K - p - 1, wc = Wd - p - 1;
        const int total = wr * wc;
        if (tid < total) {
            int ii = tid / wc, jj = tid - (tid / wc) * wc;
            const int di = NT / wc, dj = NT - di * wc;
            const double* Ap = sm.A + p * S + p + 1;
            double* Ab = sm.A + (p + 1) * S;
#pragma unroll 4
            for (int e = tid; e < total; e += NT) {
                double* row = Ab + ii * S;
                row[p + 1 + jj] = fma(-row[p], Ap[jj], row[p + 1 + jj]);
                ii += di;
                jj += dj;
                if (jj >= wc) { jj -= wc; ++ii; }
            }
        }
        __syncthreads();
    }
    // back substitution, q columns at once
    for (int p = K - 1; p >= 0; --p) {
        for (int c = tid; c < q; c += NT) sm.A[p * S + K + c] *= sm.rdiag[p];
        __syncthreads();
        const int total = p * q;
        if (tid < total) {
            int ii = tid / q, jj = tid - (tid / q) * q;
            const int di = NT / q, dj = NT - di * q;
            const double* xp = sm.A + p * S + K;
#pragma unroll 4
            for (int e = tid; e < total; e += NT) {
                double* row = sm.A + ii * S;
                row[K + jj] = fma(-row[p], xp[jj], row[K + jj]);
                ii += di;
                jj += dj;
                if (jj >= q) { jj -= q; ++ii; }
            }
        }
        __syncthreads();
    }
    return true;
}

// Forward substitution with the unit lower factor of one column Xc (row stride xs) by one
// warp, 32 rows at a time (2x2 pivots update a row with both columns in one expression, as in
// the factorization; a block never splits a 2x2 pivot): inside a block the lanes keep x in
// registers and take each pivot's value by a shuffle; below the block every lane applies the
// block's updates to its rows in pivot order.  Each entry receives the same FMAs in the same
// order as in forward_subst, with one warp synchronisation per block instead of per pivot.
__device__ __forceinline__ void forward_subst_warp(int K, const StencilSmem& sm, double* Xc, int xs) {
    const int lane = threadIdx.x & 31;
    for (int b0 = 0; b0 < K;) {
        int b1 = min(b0 + 32, K);
        if (b1 < K && sm.pk[b1 - 1] == 2) --b1;
        const int i = b0 + lane;
        double x = i < b1 ? Xc[i * xs] : 0.0;
        for (int p = b0; p < b1;) {
            const int k = sm.pk[p];
            const double xp = __shfl_sync(0xffffffffu, x, p - b0);
            const double xq = __shfl_sync(0xffffffffu, x, min(p + 1 - b0, 31));
            if (i > p + k - 1 && i < b1) {
                const double* Ti = sm.T + tri(i);
                x = k == 1 ? fma(-Ti[p], xp, x) : fma(-Ti[p + 1], xq, fma(-Ti[p], xp, x));
            }
            p += k;
        }
        if (i < b1) Xc[i * xs] = x;
        __syncwarp();
        for (int r = b1 + lane; r < K; r += 32) {
            const double* Tr = sm.T + tri(r);
            double xr = Xc[r * xs];
            for (int p = b0; p < b1;) {
                const int k = sm.pk[p];
                xr = k == 1 ? fma(-Tr[p], Xc[p * xs], xr)
                            : fma(-Tr[p + 1], Xc[(p + 1) * xs], fma(-Tr[p], Xc[p * xs], xr));
                p += k;
            }
            Xc[r * xs] = xr;
        }
        __syncwarp();
        b0 = b1;
    }
}

// Blocked triangular solves of the columns 0 .. q-1 of sm.X with the whole team, 32 unknowns
// at a time, for teams that hold one to four systems per SM (256 and 512 threads): a warp
// solves a column's diagonal block (lanes keep x in registers, each pivot's value by a
// shuffle), then every thread updates the column's remaining rows with that block in pivot
// order.  On GB300 a warp issues FP64 instructions to one quarter of the SM's FP64 units
// only, so a triangular solve by a single warp runs at a quarter of the SM's rate when few
// systems share the SM; here the rows' updates spread over all four.  (With ten or more
// systems per SM the step-by-step forms keep the pipe busier.)  Each entry receives the same
// FMAs in the same order as in the step-by-step forms (forward_subst; the back substitution
// of ldlt_solve_tail), so results are bit-identical.

// Forward substitution with the unit lower factor (a block never splits a 2x2 pivot).
template <int NT>
__device__ void forward_subst_blocked(int K, int q, const StencilSmem& sm) {
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int xs = sm.xs;
    for (int b0 = 0; b0 < K;) {
        int b1 = min(b0 + 32, K);
        if (b1 < K && sm.pk[b1 - 1] == 2) --b1;
        for (int c = wid; c < q; c += NW) {
            double* Xc = sm.X + c;
            const int i = b0 + lane;
            double x = i < b1 ? Xc[i * xs] : 0.0;
            for (int p = b0; p < b1;) {
                const int k = sm.pk[p];
                const double xp = __shfl_sync(0xffffffffu, x, p - b0);
                const double xq = __shfl_sync(0xffffffffu, x, min(p + 1 - b0, 31));
                if (i > p + k - 1 && i < b1) {
                    const double* Ti = sm.T + tri(i);
                    x = k == 1 ? fma(-Ti[p], xp, x) : fma(-Ti[p + 1], xq, fma(-Ti[p], xp, x));
                }
                p += k;
            }
            if (i < b1) Xc[i * xs] = x;
        }
        __syncthreads();
        for (int e = tid; e < (K - b1) * q; e += NT) {
            const int r = b1 + e / q, c = e - (e / q) * q;
            const double* Tr = sm.T + tri(r);
            const double* Xc = sm.X + c;
            double xr = Xc[r * xs];
            for (int p = b0; p < b1;) {
                const int k = sm.pk[p];
                xr = k == 1 ? fma(-Tr[p], Xc[p * xs], xr)
                            : fma(-Tr[p + 1], Xc[(p + 1) * xs], fma(-Tr[p], Xc[p * xs], xr));
                p += k;
            }
            sm.X[r * xs + c] = xr;
        }
        __syncthreads();
        b0 = b1;
    }
}

// Back substitution with L^T (after the D solve): x_j -= L[i][j] x_i for j < i, i descending.
template <int NT>
__device__ void back_subst_blocked(int K, int q, const StencilSmem& sm) {
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int xs = sm.xs;
    for (int b1 = K; b1 > 0;) {
        const int b0 = max(b1 - 32, 0);
        for (int c = wid; c < q; c += NW) {
            double* Xc = sm.X + c;
            const int j = b0 + lane;
            double x = j < b1 ? Xc[j * xs] : 0.0;
            for (int i = b1 - 1; i > b0; --i) {
                const double xi = __shfl_sync(0xffffffffu, x, i - b0);
                if (j < i) x = fma(-sm.T[tri(i) + j], xi, x);
            }
            if (j < b1) Xc[j * xs] = x;
        }
        __syncthreads();
        for (int e = tid; e < b0 * q; e += NT) {
            const int r = e / q, c = e - (e / q) * q;
            const double* Xc = sm.X + c;
            double xr = Xc[r * xs];
            for (int i = b1 - 1; i >= b0; --i) xr = fma(-sm.T[tri(i) + r], Xc[i * xs], xr);
            sm.X[r * xs + c] = xr;
        }
        __syncthreads();
        b1 = b0;
    }
}

// D solve and back substitution of the right-hand-side columns 0 .. q-1 held in sm.X, after
// the forward substitution (carried through the factorization, or forward_subst).
template <int NT>
__device__ __forceinline__ void ldlt_solve_tail(int K, int q, const StencilSmem& sm) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int xs = sm.xs;
    double* T = sm.T;
    double* X = sm.X;
    // D solve: 1x1 rows scale by the reciprocal pivot, 2x2 blocks multiply by their inverse;
    // then back substitution with L^T: once x_i is final, x_j -= L[i][j] x_i for j < i.
    // With at most one column per warp (q <= NW), warp w owns column w and its K sequential
    // steps need only warp synchronisation; otherwise all threads share every step (the
    // flattened (row, column) pairs keep the lanes busy) with a barrier per step.  Both do
    // the same operations on every element.
    constexpr int NW = NT / 32;
    if (q <= NW && NT < 256) {
        if (wid < q) {
            double* Xc = X + wid;
            for (int i = lane; i < K; i += 32) {
                const int k = sm.pk[i];
                double* Bi = Xc + i * xs;
                if (k == 1) {
                    *Bi *= sm.rdiag[i];
                } else if (k == 2) {  // rows i, i + 1 form a 2x2 block
                    double* Bn = Bi + xs;
                    const double y0 = *Bi, y1 = *Bn;
                    *Bi = fma(sm.rdiag[i], y0, sm.dinv1[i] * y1);
                    *Bn = fma(sm.dinv1[i], y0, sm.rdiag[i + 1] * y1);
                }
            }
            __syncwarp();
            for (int i = K - 1; i > 0; --i) {
                const double* Li = T + tri(i);
                const double xv = Xc[i * xs];
                for (int jj = lane; jj < i; jj += 32) Xc[jj * xs] = fma(-Li[jj], xv, Xc[jj * xs]);
                __syncwarp();
            }
        }
        return;
    }
    for (int e = tid; e < K * q; e += NT) {
        const int i = e / q, c = e - (e / q) * q;
        const int k = sm.pk[i];
        double* Bi = X + i * xs + c;
        if (k == 1) {
            *Bi *= sm.rdiag[i];
        } else if (k == 2) {
            double* Bn = Bi + xs;
            const double y0 = *Bi, y1 = *Bn;
            *Bi = fma(sm.rdiag[i], y0, sm.dinv1[i] * y1);
            *Bn = fma(sm.dinv1[i], y0, sm.rdiag[i + 1] * y1);
        }
    }
    __syncthreads();
    if constexpr (NT >= 256) {
        back_subst_blocked<NT>(K, q, sm);
        return;
    }
    for (int i = K - 1; i > 0; --i) {
        const int total = i * q;
        if (tid < total) {
            int jj = tid / q, cc = tid - (tid / q) * q;
            const int dj = NT / q, dc = NT - dj * q;
            const double* Li = T + tri(i);
            const double* xi = X + i * xs;
#pragma unroll 4
            for (int e = tid; e < total; e += NT) {
                double* xj = X + jj * xs;
                xj[cc] = fma(-Li[jj], xi[cc], xj[cc]);
                jj += dj;
                cc += dc;
                if (cc >= q) { cc -= q; ++jj; }
            }
        }
        __syncthreads();
    }
}

// Symmetric indefinite LDL^T factorization with Bunch-Kaufman partial pivoting (J. R. Bunch
// and L. Kaufman, "Some stable methods for calculating inertia and solving symmetric linear
// systems", Math. Comp. 31 (1977)) of the symmetric saddle-point matrix [A P; P^T 0] in the
// packed layout, with the right-hand sides carried along; (1/3) K^3 + 2 K^2 q flops.  1x1
// and 2x2 pivots with alpha = (1 + sqrt(17)) / 8; symmetric swaps are tracked in sm.perm.
// Returns false (uniformly) on an exactly singular pivot column.  On success sm.rowof[u] is
// the row of the right-hand-side block that holds unknown u.
// Pivot ratio of the factorization, written by factor_solve_ldlt<NT, true>: floor(log2) of
// max |D block entry| times floor(log2) of max |D^-1 block entry|, i.e. an estimate (within a
// factor 4) of log2 of max |d| / min |d| over the pivots, a lower bound of the system's
// condition number.  Read after a barrier.
__shared__ int s_pivot_log2_ratio;
constexpr int kRefinePivotLog2 = 16;  // refine systems whose pivots span at least 2^16

// Biased IEEE exponent of |v| (an integer-pipe floor(log2 |v|) + 1023).
__device__ __forceinline__ int exp_bits(double v) { return (int)((abs_bits(v) >> 52) & 0x7ff); }

// One pivot step at p of the factorization below, by warp 0: the Bunch-Kaufman choice (1x1,
// possibly after a symmetric swap, or 2x2), the reciprocal pivot or the 2x2 inverse, and the
// scaled column(s) of L in place; the unscaled pivot column is kept in wb (a 1x1 step) or in
// sm.wv and sm.wv2 (a 2x2 step) for the trailing update.  Lane 0 publishes s_ok and s_kind.
__shared__ int s_ok, s_kind;

template <bool TRACK>
__device__ __forceinline__ void pivot_step(int K, int q, int p, const StencilSmem& sm, double* wb,
                                           int& e_d, int& e_r) {
    const int lane = threadIdx.x & 31;
    const int xs = sm.xs;
    double* T = sm.T;
    double* X = sm.X;
    // The lane's first two entries of the pivot column and the reciprocal of the
    // diagonal, in one straight-line block so the reciprocal's integer chain overlaps
    // the loads and the search; the usual 1x1 step without a swap then scales these
    // registers directly.
    const double dpp = T[tri(p) + p];
    const int i0 = p + 1 + lane, i1 = i0 + 32;
    const double w0 = i0 < K ? T[tri(i0) + p] : 0.0;
    const double w1 = i1 < K ? T[tri(i1) + p] : 0.0;
    bool slow;
    const double rcp_p = rcp_core(dpp, &slow);
    // lambda = max |A[i][p]|, i > p, on magnitude keys (the top 32 bits of |A[i][p]|,
    // an order-preserving truncation), lowest index among equal keys; two warp
    // reductions instead of a shuffle tree
    unsigned lk = 0u;
    int r = 0x7fffffff;
    {
        const unsigned k0 = i0 < K ? mag_key(w0) : 0u;
        const unsigned k1 = i1 < K ? mag_key(w1) : 0u;
        if (k0 > lk) { lk = k0; r = i0; }
        if (k1 > lk) { lk = k1; r = i1; }
    }
    for (int i = i1 + 32; i < K; i += 32) {  // columns longer than 64
        const unsigned v = mag_key(T[tri(i) + p]);
        if (v > lk) { lk = v; r = i; }
    }
    const unsigned lmax = __reduce_max_sync(0xffffffffu, lk);
    r = (int)__reduce_min_sync(0xffffffffu,
                               (lk == lmax && lmax != 0u) ? (unsigned)r : 0x7fffffffu);
    const unsigned long long lv = (unsigned long long)lmax << 32;
    // the pivot choice only has to be a valid Bunch-Kaufman choice, so the tests run in
    // FP32 on values rebuilt from the FP64 bit patterns (no FP64 instructions)
    const unsigned long long pv = abs_bits(dpp);
    const float lam = approx_f32(lv), app = approx_f32(pv);
    const float af = 0.6403882f;
    int kind = 1, swap_a = p, swap_b = p;
    bool ok = true;
    if (lv == 0ull) {
        ok = pv != 0ull;  // column already eliminated: 1x1 pivot if nonzero
    } else if (!(app >= af * lam)) {
        // sigma = max |A_rj| over the active part of row/column r, j != r
        unsigned sk = 0u;
        for (int jj = p + lane; jj < K; jj += 32) {
            if (jj == r) continue;
            const unsigned b = mag_key(jj < r ? T[tri(r) + jj] : T[tri(jj) + r]);
            sk = b > sk ? b : sk;
        }
        sk = __reduce_max_sync(0xffffffffu, sk);
        const float sig = approx_f32((unsigned long long)sk << 32),
                    arr = approx_f32(abs_bits(T[tri(r) + r]));
        if (app * sig >= af * lam * lam) {
            kind = 1;
        } else if (arr >= af * sig) {
            kind = 1; swap_a = p; swap_b = r;
        } else {
            kind = 2; swap_a = p + 1; swap_b = r;
        }
    }
    if (ok && swap_a != swap_b) {
        // symmetric swap of unknowns ua < ub in the packed lower triangle, one uniform
        // loop per segment (row parts left of ua, the part between, the columns below
        // ub, the right-hand-side rows, the diagonal pair)
        const int ua = swap_a, ub = swap_b;
        auto exch = [](double* x, double* y) { const double t = *x; *x = *y; *y = t; };
        for (int e = lane; e < ua; e += 32) exch(T + tri(ua) + e, T + tri(ub) + e);
        for (int i = ua + 1 + lane; i < ub; i += 32) exch(T + tri(i) + ua, T + tri(ub) + i);
        for (int i = ub + 1 + lane; i < K; i += 32) exch(T + tri(i) + ua, T + tri(i) + ub);
        for (int c = lane; c < q; c += 32) exch(X + ua * xs + c, X + ub * xs + c);
        if (lane == 0) {
            exch(T + tri(ua) + ua, T + tri(ub) + ub);
            const int t = sm.perm[ua]; sm.perm[ua] = sm.perm[ub]; sm.perm[ub] = t;
        }
        __syncwarp();
    }
    if (ok) {
        if (kind == 1 && swap_a == swap_b && !slow) {  // the usual step: all in registers
            if (lane == 0) { sm.rdiag[p] = rcp_p; sm.pk[p] = 1; }
            if (TRACK && lane == 0) {
                e_d = max(e_d, exp_bits(dpp));
                e_r = max(e_r, exp_bits(rcp_p));
            }
            const double s0 = w0 * rcp_p, s1 = w1 * rcp_p;
            if (i0 < K) { wb[i0] = w0; T[tri(i0) + p] = s0; }
            if (i1 < K) { wb[i1] = w1; T[tri(i1) + p] = s1; }
            for (int i = i1 + 32; i < K; i += 32) {
                const double w = T[tri(i) + p];
                wb[i] = w;
                T[tri(i) + p] = w * rcp_p;
            }
        } else if (kind == 1) {  // after a swap (or an extreme pivot): reload
            const double rcp = rcp_fixed(T[tri(p) + p]);
            if (lane == 0) { sm.rdiag[p] = rcp; sm.pk[p] = 1; }
            if (TRACK && lane == 0) {
                e_d = max(e_d, exp_bits(T[tri(p) + p]));
                e_r = max(e_r, exp_bits(rcp));
            }
            for (int i = p + 1 + lane; i < K; i += 32) {
                const double w = T[tri(i) + p];
                wb[i] = w;
                T[tri(i) + p] = w * rcp;
            }
        } else {
            const double d0 = T[tri(p) + p], d1 = T[tri(p + 1) + p], d2 = T[tri(p + 1) + p + 1];
            const double rdet = rcp_fixed(fma(d0, d2, -d1 * d1));
            const double i00 = d2 * rdet, i01 = -d1 * rdet, i11 = d0 * rdet;
            if (lane == 0) {
                sm.rdiag[p] = i00; sm.dinv1[p] = i01; sm.rdiag[p + 1] = i11;
                sm.pk[p] = 2; sm.pk[p + 1] = 0;
                T[tri(p + 1) + p] = 0.0;  // L has no entry inside a 2x2 pivot block
                if (TRACK) {
                    e_d = max(e_d, max(exp_bits(d0), max(exp_bits(d1), exp_bits(d2))));
                    e_r = max(e_r, max(exp_bits(i00), max(exp_bits(i01), exp_bits(i11))));
                }
            }
            for (int i = p + 2 + lane; i < K; i += 32) {
                const double w1 = T[tri(i) + p], w2 = T[tri(i) + p + 1];
                sm.wv[i] = w1;
                sm.wv2[i] = w2;
                T[tri(i) + p] = fma(w1, i00, w2 * i01);
                T[tri(i) + p + 1] = fma(w1, i01, w2 * i11);
            }
        }
    }
    if (lane == 0) { s_ok = ok ? 1 : 0; s_kind = kind; }
}

// Trailing update after the pivot step at p (kind 1 or 2) by the threads U0 .. NT-1; wb holds a
// 1x1 step's unscaled pivot column (sm.wv for a 2x2 step, with sm.wv2).
template <int NT, int U0>
__device__ __forceinline__ void trailing_update(int K, int q, int p, int kind, const StencilSmem& sm,
                                                const double* wb, bool skip_next) {
    constexpr int UT = NT - U0;
    const int ut = (int)threadIdx.x - U0;
    const int xs = sm.xs;
    double* T = sm.T;
    double* X = sm.X;
    // Trailing update of the lower triangle and of the right-hand sides: row i (> p0)
    // has (i - p0) triangle entries followed by q right-hand-side entries.  Rows r and
    // rows-1-r are paired into one virtual row of constant length rows + 1 + 2q, so the
    // flattened index steps in O(1).  The FP64 work is branch-free: source operands are
    // selected with integer arithmetic so every lane issues the same FMA (a divergent
    // FP64 instruction costs the whole warp on the FP64 pipe).
    const int p0 = p + kind - 1;
    const int rows = K - p0 - 1;
    if (rows > 0) {
        const int L2 = rows + 1 + 2 * q;
        const int total = ((rows + 1) >> 1) * L2;
        if (ut < total) {
            int pr = ut / L2, off = ut - (ut / L2) * L2;
            const int di = UT / L2, dj = UT - di * L2;
            for (int e = ut; e < total; e += UT) {
                const int len0 = pr + 1 + q;
                const bool first = off < len0;
                const int r = first ? pr : rows - 1 - pr;
                const int t = first ? off : off - len0;
                // an odd middle row pairs with itself: once only; with skip_next column p0 + 1 is
                // left to warp 0
                if ((first || r != pr) && (t != 0 || !skip_next)) {
                    const int i = p0 + 1 + r;
                    double* Ti = T + tri(i);
                    const bool trin = t <= r;
                    const int jj = p0 + 1 + t;      // triangle column
                    const int c = t - (r + 1);      // right-hand-side column
                    double* dst = trin ? Ti + jj : X + i * xs + c;
                    const double* s1 = trin ? wb + jj : X + p * xs + c;
                    if (kind == 1) {
                        *dst = fma(-Ti[p], *s1, *dst);
                    } else {
                        const double* s2 = trin ? sm.wv2 + jj : X + (p + 1) * xs + c;
                        *dst = fma(-Ti[p + 1], *s2, fma(-Ti[p], *s1, *dst));
                    }
                }
                pr += di;
                off += dj;
                if (off >= L2) { off -= L2; ++pr; }
            }
        }
    }
}

// Look-ahead of the next pivot for 512-thread teams (one system per SM, where nothing hides
// the serial pivot step): while the other warps apply the 1x1 step at p, warp 0 applies it
// to column pn = p + 1 (the FMA every entry of the trailing update gets) and tries the usual
// next step there, a 1x1 pivot without a swap, which the column alone decides.  If it holds
// (and the pivot is not extreme), the step is stored exactly as pivot_step would store it,
// its unscaled column in wn (the other buffer: the update running now reads wc); otherwise
// the updated column stays unscaled for pivot_step.  Results are bit-identical either way.
template <bool TRACK>
__device__ __forceinline__ bool lookahead_pivot(int K, int p, const StencilSmem& sm, const double* wc,
                                                double* wn, int& e_d, int& e_r) {
    const int lane = threadIdx.x & 31;
    double* T = sm.T;
    const int pn = p + 1;
    const double f = wc[pn];
    const double dpp = fma(-T[tri(pn) + p], f, T[tri(pn) + pn]);
    const int i0 = pn + 1 + lane, i1 = i0 + 32;
    const double w0 = i0 < K ? fma(-T[tri(i0) + p], f, T[tri(i0) + pn]) : 0.0;
    const double w1 = i1 < K ? fma(-T[tri(i1) + p], f, T[tri(i1) + pn]) : 0.0;
    bool slow;
    const double rcp_p = rcp_core(dpp, &slow);
    unsigned lk = 0u;
    {
        const unsigned k0 = i0 < K ? mag_key(w0) : 0u;
        const unsigned k1 = i1 < K ? mag_key(w1) : 0u;
        lk = k0 > k1 ? k0 : k1;
    }
    for (int i = i1 + 32; i < K; i += 32) {
        const double w = fma(-T[tri(i) + p], f, T[tri(i) + pn]);
        T[tri(i) + pn] = w;
        const unsigned v = mag_key(w);
        lk = v > lk ? v : lk;
    }
    const unsigned long long lv = (unsigned long long)__reduce_max_sync(0xffffffffu, lk) << 32;
    const unsigned long long pv = abs_bits(dpp);
    const float lam = approx_f32(lv), app = approx_f32(pv);
    const float af = 0.6403882f;
    const bool take = lv != 0ull && app >= af * lam && !slow;
    if (lane == 0) T[tri(pn) + pn] = dpp;
    if (take) {
        if (lane == 0) { sm.rdiag[pn] = rcp_p; sm.pk[pn] = 1; }
        if (TRACK && lane == 0) {
            e_d = max(e_d, exp_bits(dpp));
            e_r = max(e_r, exp_bits(rcp_p));
        }
        if (i0 < K) { wn[i0] = w0; T[tri(i0) + pn] = w0 * rcp_p; }
        if (i1 < K) { wn[i1] = w1; T[tri(i1) + pn] = w1 * rcp_p; }
        for (int i = i1 + 32; i < K; i += 32) {
            const double w = T[tri(i) + pn];
            wn[i] = w;
            T[tri(i) + pn] = w * rcp_p;
        }
    } else {
        if (i0 < K) T[tri(i0) + pn] = w0;
        if (i1 < K) T[tri(i1) + pn] = w1;
    }
    return take;
}

template <int NT, bool TRACK = false>
__device__ bool factor_solve_ldlt(int K, int q, const StencilSmem& sm) {
    const int tid = threadIdx.x, wid = tid >> 5;
    int e_d = 0, e_r = 0;  // (thread 0, TRACK) largest exponents of |D| and |D^-1| entries
    for (int r = tid; r < K; r += NT) sm.perm[r] = r;
    __syncthreads();
    int p = 0;
    if constexpr (NT == 512) {
        // Warp 0 looks one pivot ahead (lookahead_pivot) while warps 1-15 update; the 1x1
        // steps alternate their unscaled column between sm.wv and sm.wv + K (= sm.wv2, which
        // only 2x2 steps use otherwise), and the look-ahead's outcome alternates between two
        // flags, so no flag or column is rewritten while another warp may still read it.
        __shared__ int s_took[2];
        int cur = 0, it = 0;
        bool have_pivot = false;
        while (p < K) {
            if (!have_pivot) {
                if (wid == 0) pivot_step<TRACK>(K, q, p, sm, sm.wv + cur * K, e_d, e_r);
                __syncthreads();
                if (!s_ok) return false;
            }
            const int kind = have_pivot ? 1 : s_kind;
            const double* wb = kind == 2 ? sm.wv : sm.wv + cur * K;
            const bool look = kind == 1 && p + 1 < K;
            if (wid == 0) {
                if (look) {
                    const bool took = lookahead_pivot<TRACK>(K, p, sm, wb, sm.wv + (cur ^ 1) * K, e_d, e_r);
                    if ((tid & 31) == 0) s_took[it & 1] = took ? 1 : 0;
                }
            } else {
                trailing_update<NT, 32>(K, q, p, kind, sm, wb, look);
            }
            __syncthreads();
            have_pivot = look && s_took[it & 1] != 0;
            if (have_pivot) cur ^= 1;
            ++it;
            p += kind;
        }
    } else {
        while (p < K) {
            if (wid == 0) pivot_step<TRACK>(K, q, p, sm, sm.wv, e_d, e_r);
            __syncthreads();
            if (!s_ok) return false;
            const int kind = s_kind;
            trailing_update<NT, 0>(K, q, p, kind, sm, sm.wv, false);
            __syncthreads();
            p += kind;
        }
    }
    // The inverse permutation (read after the caller's next barrier).
    for (int r = tid; r < K; r += NT) sm.rowof[sm.perm[r]] = r;
    if (TRACK && tid == 0) s_pivot_log2_ratio = e_d + e_r - 2 * 1023;
    ldlt_solve_tail<NT>(K, q, sm);
    return true;
}

// ------------------------------------------------------------------ right-hand sides in chunks
// The factorization carries at most a.qcap right-hand sides (shared memory is sized for that
// many); a center with more solves the rest afterwards, a.qcap at a time, with the stored
// factors.  Every column gets the same operations, in the same order, as it would have had
// in the first chunk, so the weights do not depend on the chunk a column falls in.

// psi_l(x) by the parent recurrence, multiplied in the order the monomial block is built.
template <int D>
__device__ __forceinline__ double mono_value(const Basis& bs, int l, const double* x) {
    unsigned code = 0;  // the variables from l up to the constant, 2 bits each
    int depth = 0;
    while (l > 0) {
        code = (code << 2) | (unsigned)bs.var[l];
        ++depth;
        l = bs.parent[l];
    }
    double v = 1.0;
    for (int i = 0; i < depth; ++i) {
        v = v * x[code & 3u];
        code >>= 2;
    }
    return v;
}

// Right-hand-side entry of unknown u for the column of stencil position t: m (m + D - 2)
// r^(m-2) (as in the pair loop) for a stencil node, the Laplacian of psi_(u-n) at node t for a
// monomial.
template <int D>
__device__ __forceinline__ double rhs_entry(const Shape& sh, int u, int t, const StencilSmem& sm,
                                            bool fma_r2) {
    const int n = sh.n;
    double v = 0.0;
    if (u < n) {
        if (u != t) {
            const double r2 = fma_r2 ? sqdist_local<D>(sm.xi + u * D, sm.xi + t * D)
                                     : sqdist_rn<D>(sm.xi + u * D, sm.xi + t * D);
            double pm2 = sqrt_fast(r2);
            for (int k = 0; k < (sh.m - 3) / 2; ++k) pm2 = __dmul_rn(pm2, r2);
            v = __dmul_rn(sh.coef, pm2);
        }
    } else {
        const int l = u - n;
        for (int d = 0; d < D; ++d) {
            const int ch = sh.bs.lap_child[l * D + d];
            if (ch >= 0)
                v = fma(exact_double(sh.bs.lap_coef[l * D + d]), mono_value<D>(sh.bs, ch, sm.xi + t * D), v);
        }
    }
    return v;
}

// Right-hand sides of columns c0 .. c0+qk-1 into sm.X, rows in the factorization's permuted
// order (row r holds unknown perm[r]).
template <int D, int NT>
__device__ void chunk_rhs(const Shape& sh, int c0, int qk, const StencilSmem& sm, bool fma_r2) {
    const int K = sh.K;
    for (int e = threadIdx.x; e < K * qk; e += NT) {
        const int r = e / qk, c = e - (e / qk) * qk;
        sm.X[r * sm.xs + c] = rhs_entry<D>(sh, sm.perm[r], sm.cols[c0 + c], sm, fma_r2);
    }
}

// Forward substitution with the unit lower factor, step by step as the factorization applied
// it to the carried columns (a 2x2 pivot's two columns update a row in one expression).
template <int NT>
__device__ void forward_subst(int K, int q, const StencilSmem& sm) {
    const int xs = sm.xs;
    for (int p = 0; p < K;) {
        const int k = sm.pk[p];
        const int p0 = p + k - 1;
        const int total = (K - p0 - 1) * q;
        for (int e = threadIdx.x; e < total; e += NT) {
            const int r = e / q, c = e - (e / q) * q;
            const int i = p0 + 1 + r;
            const double* Ti = sm.T + tri(i);
            double* dst = sm.X + i * xs + c;
            if (k == 1) *dst = fma(-Ti[p], sm.X[p * xs + c], *dst);
            else *dst = fma(-Ti[p + 1], sm.X[(p + 1) * xs + c], fma(-Ti[p], sm.X[p * xs + c], *dst));
        }
        __syncthreads();
        p += k;
    }
}

template <int NT>
__device__ __forceinline__ void lebesgue_values(int n, int K, int q, const StencilSmem& sm,
                                                int off = 0);

// Right-hand side of the normal derivative at the stencil center (the origin of the scaled
// coordinates) for unknown u of node i's own stencil (§5, a Neumann row): d/dn ||y - xi_u||^m
// at y = 0 is -m ||xi_u||^(m-2) (xi_u . n), and of the monomials only the linear ones have a
// nonzero gradient there (d/dn xi_a = n_a).
template <int D>
__device__ __forceinline__ double neumann_value(const SolveArgs& a, const Shape& sh, int i, int u,
                                                const StencilSmem& sm) {
    const double* nv = a.nrm + (size_t)i * D;
    if (u < sh.n) {
        const double mm = exact_double(sh.m);
        const double* xj = sm.xi + u * D;
        double r2 = xj[0] * xj[0], dot = xj[0] * nv[0];
        for (int c = 1; c < D; ++c) {
            r2 = fma(xj[c], xj[c], r2);
            dot = fma(xj[c], nv[c], dot);
        }
        double pm2 = sqrt_fast(r2);  // r^(m-2), m odd
        for (int t = 0; t < (sh.m - 3) / 2; ++t) pm2 *= r2;
        return -mm * pm2 * dot;
    }
    const int l = u - sh.n;
    return (l > 0 && sh.bs.parent[l] == 0) ? nv[sh.bs.var[l]] : 0.0;
}

// Team sizes whose traversal kernels carry the refinement step: the 96- and 128-thread teams
// run with 40 registers for small systems (many per SM), and the planner gives plans that
// refine (largest system K >= 100, at most a few per SM) 256- or 512-thread teams, or 32 or
// 64 when forced.  The fallback kernel carries it at every team size (ALL_TEAMS).
__host__ __device__ constexpr bool team_refines(int nt) { return nt != 96 && nt != 128; }

// Per-CTA scratch of the refinement step of this launch, or nullptr when the plan refines
// nothing.  (Whether a system is refined is decided after its factorization.)
template <int NT, bool ALL_TEAMS = false>
__device__ __forceinline__ double* refine_scratch(const SolveArgs& a) {
    if constexpr (!ALL_TEAMS && !team_refines(NT)) {
        return nullptr;
    } else {
        return a.rs != nullptr ? a.rs + (size_t)blockIdx.x * a.rs_stride : nullptr;
    }
}

// The residual's dot products sum_v A_uv x0_v are split into kRefineSegs fixed ranges of v
// (the same for every team size), summed in order within a range and then combined in a
// fixed order, so every thread of a team has short independent chains and the bits do not
// depend on the team.
constexpr int kRefineSegs = 4;

// Partial sum over v in segment g of A_uv x0_v: gA is the full assembled matrix (row v at
// v K, so the threads of a warp, holding consecutive u, read one contiguous row), gX0 holds
// x0 by unknown (unknown v of column c at v qk + c: one address for the whole warp).
__device__ __forceinline__ double residual_part(int u, int c, int g, int K, int qk,
                                                const double* __restrict__ gA,
                                                const double* __restrict__ gX0) {
    const int len = (K + kRefineSegs - 1) / kRefineSegs;
    const int v0 = g * len, v1 = min(K, v0 + len);
    double s = 0.0;
#pragma unroll 8
    for (int v = v0; v < v1; ++v) s = fma(__ldcg(gA + (size_t)v * K + u), __ldcg(gX0 + v * qk + c), s);
    return s;
}

// One step of iterative refinement (J. H. Wilkinson, "Rounding Errors in Algebraic Processes",
// 1963) of the columns c0 .. c0+qk-1 held in sm.X after their LDL^T solve:
// x1 = x0 + (L D L^T)^-1 (b - A x0), the residual formed in FP64 with the assembled matrix A
// (gA, copied in full before the factorization overwrote it) and the right-hand sides rebuilt
// bit for bit.  On the ill-conditioned systems of large stencils (condition
// numbers up to ~1e10) the first solution's forward error is dominated by the symmetric-
// pivoting factorization; one step brings it down to that of the assembled system itself.
// Only systems whose pivot ratio (s_pivot_log2_ratio) reaches 2^kRefinePivotLog2 are refined,
// unless a.refine_all: the well-conditioned majority keeps its first solution.  kind: 0 the
// Laplacian right-hand sides of the columns in sm.cols, 2 the normal derivative at the center
// of node i (one column).  gX0 holds x0 (K x qk).  With at most one column per warp each warp
// forward-substitutes its own column; the arithmetic of an entry is the same either way, so
// every team size gives the same bits.
template <int D, int NT>
__device__ void refine_columns(const SolveArgs& a, const Shape& sh, int c0, int qk,
                               const StencilSmem& sm, const double* __restrict__ gA,
                               double* __restrict__ gX0, int kind, int i) {
    constexpr int NW = NT / 32;
    const int K = sh.K, xs = sm.xs, tid = threadIdx.x, wid = tid >> 5;
    double* gP = gX0 + (size_t)K * qk;  // kRefineSegs partial sums per entry
    __syncthreads();  // (the last solve steps may have been warp-synchronous)
    // adaptive: only systems whose pivots span at least 2^16 (unless every system is refined)
    if (a.refine_all == 0 && s_pivot_log2_ratio < kRefinePivotLog2) return;
    for (int e = tid; e < K * qk; e += NT) {  // x0 by unknown
        const int r = e / qk, c = e - r * qk;
        gX0[sm.perm[r] * qk + c] = sm.X[r * xs + c];
    }
    if (kind == 2) {
        for (int r = tid; r < K; r += NT) sm.X[r * xs] = neumann_value<D>(a, sh, i, sm.perm[r], sm);
    } else {
        chunk_rhs<D, NT>(sh, c0, qk, sm, a.fma_r2 != 0);
    }
    __syncthreads();
    for (int e = tid; e < K * qk * kRefineSegs; e += NT) {  // (unknown, column, segment) items
        const int g = e / (K * qk), uc = e - g * (K * qk);
        const int u = uc / qk, c = uc - u * qk;
        gP[e] = residual_part(u, c, g, K, qk, gA, gX0);
    }
    __syncthreads();
    for (int e = tid; e < K * qk; e += NT) {  // r = b - ((p0 + p1) + (p2 + p3)), rows permuted
        const int r = e / qk, c = e - r * qk;
        const int uc = sm.perm[r] * qk + c;
        const double* P = gP + uc;
        const size_t st = (size_t)K * qk;
        sm.X[r * xs + c] = sm.X[r * xs + c] - ((__ldcg(P) + __ldcg(P + st)) + (__ldcg(P + 2 * st) + __ldcg(P + 3 * st)));
    }
    __syncthreads();
    if (NT >= 256) {  // forward substitution
        forward_subst_blocked<NT>(K, qk, sm);
    } else if (qk <= NW) {  // a warp per column with warp synchronisation only
        if (wid < qk) forward_subst_warp(K, sm, sm.X + wid, xs);
    } else {
        forward_subst<NT>(K, qk, sm);
    }
    ldlt_solve_tail<NT>(K, qk, sm);
    __syncthreads();
    for (int e = tid; e < K * qk; e += NT) {
        const int r = e / qk, c = e - r * qk;
        sm.X[r * xs + c] += __ldcg(gX0 + sm.perm[r] * qk + c);
    }
    if (tid == 0) atomicAdd(&a.ctr->sum_k2r, (unsigned long long)K * K * qk);
    __syncthreads();
}

// The refinement step for the columns that can be kept (refine_columns on a subset).  With a
// Lebesgue test (SEQ, FALLBACK) a column whose first solution's Lebesgue value exceeds the
// test's reference value by more than 2^-10 of it fails the test whatever the refinement does
// (a step changes the values by far less on the systems it is for: about the condition number
// times the rounding, below 1e-5), and its weights are discarded; only the center, the
// reference column and the other columns are refined.  They are moved to the front of the
// right-hand-side block (and sm.cols with them), refined there and moved back; each column's
// arithmetic does not depend on the others, so a kept column gets the same bits as when every
// column is refined.  cref is the reference column (0, or 1 with the centroid option); the
// chunk's unrefined Lebesgue values are left in sm.lam for the caller to recompute.  The
// scratch slot holds the moved block after the refinement's own arrays (6 K q_cap + q_cap).
template <int D, int NT>
__device__ void refine_kept_columns(const SolveArgs& a, const Shape& sh, int c0, int qk,
                                    const StencilSmem& sm, double* __restrict__ gA, int cref,
                                    int j) {
    __syncthreads();
    if (a.refine_all == 0 && s_pivot_log2_ratio < kRefinePivotLog2) return;
    double* gX0 = gA + a.rs_x0;
    if (a.mode == RBFFD_STAB_OFF || qk == 1) {
        refine_columns<D, NT>(a, sh, c0, qk, sm, gA, gX0, 0, j);
        return;
    }
    const int K = sh.K, xs = sm.xs, tid = threadIdx.x;
    lebesgue_values<NT>(sh.n, K, qk, sm, c0);
    __syncthreads();
    // the selection, in column order, by warp 0: kept columns first (map[c'] = column of
    // position c'); sm.keep[c0 ..] serves as the map (the test writes it afterwards)
    __shared__ int s_qr;
    unsigned char* map = sm.keep + c0;
    if (tid < 32) {
        const double lref = sm.lam[cref];
        const double lim = lref * (1.0 + 0x1p-10);
        int nsel = 0;
        for (int b = 0; b < qk; b += 32) {  // selected columns, in order
            const int c = b + tid;
            const bool sel = c < qk && (c0 + c == 0 || c0 + c == cref || sm.lam[c0 + c] <= lim);
            const unsigned bal = __ballot_sync(0xffffffffu, sel);
            if (sel) map[nsel + __popc(bal & ((1u << tid) - 1u))] = (unsigned char)c;
            nsel += __popc(bal);
        }
        int nrest = nsel;
        for (int b = 0; b < qk; b += 32) {  // then the others, in order
            const int c = b + tid;
            const bool sel = c < qk && (c0 + c == 0 || c0 + c == cref || sm.lam[c0 + c] <= lim);
            const bool other = c < qk && !sel;
            const unsigned bal = __ballot_sync(0xffffffffu, other);
            if (other) map[nrest + __popc(bal & ((1u << tid) - 1u))] = (unsigned char)c;
            nrest += __popc(bal);
        }
        if (tid == 0) s_qr = nsel;
    }
    __syncthreads();
    const int qr = s_qr;
    if (qr == qk) {
        refine_columns<D, NT>(a, sh, c0, qk, sm, gA, gX0, 0, j);
        return;
    }
    double* gT = gX0 + (size_t)5 * K * qk;   // the block in the new column order
    int* gC = reinterpret_cast<int*>(gT + (size_t)K * qk);  // sm.cols of the chunk, saved
    for (int e = tid; e < K * qk; e += NT) {
        const int c = e / K, r = e - c * K;
        gT[e] = sm.X[r * xs + map[c]];
    }
    for (int c = tid; c < qk; c += NT) gC[c] = sm.cols[c0 + c];
    __syncthreads();
    for (int e = tid; e < K * qr; e += NT) {
        const int c = e / K, r = e - c * K;
        sm.X[r * xs + c] = __ldcg(gT + e);
    }
    for (int c = tid; c < qk; c += NT) sm.cols[c0 + c] = __ldcg(gC + map[c]);
    __syncthreads();
    refine_columns<D, NT>(a, sh, c0, qr, sm, gA, gX0, 0, j);  // (ends with a barrier)
    for (int e = tid; e < K * qr; e += NT) {  // the refined columns over their first solutions
        const int c = e / K, r = e - c * K;
        gT[e] = sm.X[r * xs + c];
    }
    __syncthreads();
    for (int e = tid; e < K * qk; e += NT) {  // back to the original order
        const int c = e / K, r = e - c * K;
        sm.X[r * xs + map[c]] = __ldcg(gT + e);
    }
    for (int c = tid; c < qk; c += NT) sm.cols[c0 + c] = __ldcg(gC + c);
    __syncthreads();
}

// The assembled symmetric matrix (packed lower triangle in shared memory) to gA in full,
// row-major K x K, before the factorization overwrites it.
template <int NT>
__device__ __forceinline__ void copy_full_matrix(int K, const StencilSmem& sm, double* __restrict__ gA) {
    for (int e = threadIdx.x; e < K * K; e += NT) {
        const int r = e / K, c = e - r * K;
        gA[e] = r >= c ? sm.T[tri(r) + c] : sm.T[tri(c) + r];
    }
}

// Columns c0 .. c0+qk-1 with the stored LDL^T factors: right-hand sides, forward substitution,
// D solve, back substitution (refined like the first chunk) and Lebesgue values (a chunk after
// the first of a center).
template <int D, int NT>
__device__ __forceinline__ void solve_chunk(const SolveArgs& a, const Shape& sh, int c0, int qk,
                                            const StencilSmem& sm, int j, int cref) {
    chunk_rhs<D, NT>(sh, c0, qk, sm, a.fma_r2 != 0);
    __syncthreads();
    if constexpr (NT >= 256) forward_subst_blocked<NT>(sh.K, qk, sm);
    else forward_subst<NT>(sh.K, qk, sm);
    ldlt_solve_tail<NT>(sh.K, qk, sm);
    if constexpr (team_refines(NT)) {
        if (double* gA = refine_scratch<NT>(a))
            refine_kept_columns<D, NT>(a, sh, c0, qk, sm, gA, cref, j);
    }
    __syncthreads();
    lebesgue_values<NT>(sh.n, sh.K, qk, sm, c0);
}

// Assemble, factor and solve the first q columns of stencil j (refined when its shape asks).
template <int D, bool PACKED, int NT>
__device__ bool solve_local(const SolveArgs& a, const Shape& sh, int j, int q,
                            const StencilSmem& sm, int cref) {
    assemble_local<D, PACKED, NT>(a, sh, j, q, sm);
    if constexpr (!PACKED) {
        return factor_solve_lu<NT>(sh.K, q, sm);
    } else {
        double* gA = refine_scratch<NT>(a);
        if (gA) copy_full_matrix<NT>(sh.K, sm, gA);
        if (!factor_solve_ldlt<NT, team_refines(NT)>(sh.K, q, sm)) return false;
        if constexpr (team_refines(NT)) {
            if (gA) refine_kept_columns<D, NT>(a, sh, 0, q, sm, gA, cref, j);
        }
        return true;
    }
}

// Local L-Lebesgue value sum_r |w_r| of every solved column: warp w sums the columns w, w + NW,
// ... (the columns it back-substituted), over the unknowns u whose original index perm[u] is
// a stencil node (not a polynomial coefficient).
template <int NT>
__device__ __forceinline__ void lebesgue_values(int n, int K, int q, const StencilSmem& sm,
                                                int off) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = wid; c < q; c += (NT / 32)) {
        double s = 0.0;
        for (int u = lane; u < K; u += 32) {
            const double v = sm.X[u * sm.xs + c];
            s += sm.perm[u] < n ? fabs(v) : 0.0;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sm.lam[off + c] = s;
    }
}

// ------------------------------------------------------------------ traversal state machine
// Acquire-release fence at device scope: orders this thread's earlier memory operations, and
// those of its CTA that a barrier made visible to it, before its later ones, as seen by every
// thread of the device.  Only threads that publish (or consume) traversal state execute it.
__device__ __forceinline__ void fence_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void push_center(const SolveArgs& a, int k) {
    fence_gpu();
    const int slot = atomicAdd(&a.ctr->q_tail, 1);
    atomicExch(&a.queue[slot], k);
}

__device__ __forceinline__ void release(const SolveArgs& a, int k) {
    const int old = atomicSub(&a.pending[k], 1);
    if (old == 1) {
        fence_gpu();
        if (atomicCAS(&a.state[k], kUndecided, kCenter) == kUndecided) {
            atomicMin(&a.owner[k], k);
            push_center(a, k);
        }
    }
}

// node i has just become covered: its own ball releases its later members
__device__ void on_covered(const SolveArgs& a, int i) {
    atomicAdd(&a.ctr->done, 1);
    const int L = a.ball_len[i];
    const int* nb = a.nbr + (size_t)i * a.n;
    for (int t = 1; t < L; ++t) {
        const int k = nb[t];
        if (k > i) release(a, k);
    }
}

__global__ void k_traversal_init(int N, const int* __restrict__ indeg,
                                 const unsigned char* __restrict__ bc, int* state, int* pending,
                                 int* owner, int* queue, unsigned char* fb_flag, int* spec) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        state[i] = (bc && bc[i]) ? kBoundary : kUndecided;
        if (spec) spec[i] = 0;
        pending[i] = indeg[i];
        owner[i] = kNoOwner;
        queue[i] = -1;
        fb_flag[i] = 0;
    }
}

// Boundary nodes (§5) take no part in the overlapped traversal: each releases the later
// members of its ball (which counted it as a possible center), is done at once, and is queued
// for its own-stencil row with the fallback rows.
__global__ void k_boundary_release(SolveArgs a) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.N; q += gridDim.x * blockDim.x) {
        if (!a.bc[q]) continue;
        const int* nb = a.nbr + (size_t)q * a.n;
        for (int t = 1; t < a.ball_len[q]; ++t)
            if (nb[t] > q) atomicSub(&a.pending[nb[t]], 1);
        a.owner[q] = q;
        a.fb_flag[q] = 1;
        a.fb_list[atomicAdd(&a.ctr->fb_count, 1)] = q;
        atomicAdd(&a.ctr->done, 1);
    }
}

__global__ void k_traversal_seed(SolveArgs a) {
    if (a.no_seed) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        if (a.pending[i] == 0 && a.state[i] == kUndecided) {
            a.state[i] = kCenter;
            a.owner[i] = i;
            push_center(a, i);
        }
    }
}

// Speculation.  At delta < 1 a center can wait on earlier centers (a chain of dependency
// levels), so CTAs can find the queue empty.  Such a CTA solves ahead the lowest-index node
// that is still undecided: its center column and every later ball member not owned by an
// earlier center at that moment, all written to the node's own weight slots.  Ownership only
// moves to earlier centers, so the columns the node needs if it does become a center are a
// subset of these, and their arithmetic is the same as in a regular solve (the columns of a
// factorization are independent); the center then only runs the test and publishes.  A node
// that ends up covered wastes its speculative solve, done while the CTA would have been idle.
__device__ int pick_spec(const SolveArgs& a) {
    const int k = atomicAdd(&a.ctr->spec_next, 1);  // one candidate per idle poll
    if (k >= a.N || *((volatile int*)&a.state[k]) != kUndecided) return -1;
    return atomicCAS(&a.spec[k], 0, 1) == 0 ? k : -1;
}

// Reference point of the Lebesgue test in its centroid reading (§4.2.1): for every node j,
// the position in its stencil (n_j nodes) of the node nearest the stencil's centroid; one warp
// per node.  The centroid is the mean of the stencil's nodes: lane 0 sums each coordinate in
// kNN order from 0.0 and divides by n_j (at most 128 additions per coordinate, once per plan),
// then broadcasts it; ties in the distance go to the lower position.  It depends on the
// stencil only, so it runs once per plan, before the traversal.
template <int D>
__global__ void k_centroid_ref(const double* X, const int* nbr, const int* node_n, int N, int ns,
                               unsigned char* ref_pos) {
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (j >= N) return;  // (warp-uniform)
    const int n = node_n ? node_n[j] : ns;
    const int* nb = nbr + (size_t)j * ns;
    double c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        double s = 0.0;
        if (lane == 0) {
            for (int t = 0; t < n; ++t) s = __dadd_rn(s, __ldg(&X[(size_t)nb[t] * D + d]));
            s = __ddiv_rn(s, exact_double(n));
        }
        c[d] = __shfl_sync(0xffffffffu, s, 0);
    }
    unsigned long long best = ~0ull;  // this lane's smallest squared distance (bits; r2 >= 0)
    int tb = 0x7fffffff;              // and its lowest position
    for (int t = lane; t < n; t += 32) {
        const unsigned long long k =
            (unsigned long long)__double_as_longlong(sqdist_rn<D>(X + (size_t)nb[t] * D, c));
        if (k < best) { best = k; tb = t; }
    }
    unsigned long long m = best;
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v < m ? v : m;
    }
    const unsigned t = __reduce_min_sync(0xffffffffu, best == m ? (unsigned)tb : 0x7fffffffu);
    if (lane == 0) ref_pos[j] = (unsigned char)t;
}

// One CTA per center.  Thread 0 claims the next queue slot and waits (bounded) for it to be
// filled; the CTA then solves the center, tests and writes its columns, and resolves the
// traversal state of its ball members.
// Registers are capped per team size (team_min_blocks) so that the CTAs that fit an SM's
// shared memory also fit its register file.  CHUNKED (LDL^T only) is the instantiation for
// plans whose largest ball has more columns than one factorization carries; the other one
// has no code for later chunks, so it keeps the registers of the one-chunk path.
template <int D, bool PACKED, int NT, bool CHUNKED>
__global__ void __launch_bounds__(NT, team_min_blocks(NT)) k_traversal(SolveArgs a, size_t per_cta, int basis_bytes) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_j, s_q, s_rej, s_own, s_k, s_sp, s_ref, s_refonly;
    const short* sbasis = load_basis(smem, a.basis, a.basis_count);
    StencilSmem sm;
    carve<D, PACKED>(smem + basis_bytes, a.n, a.K, a.qmax, a.stride, sm);
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ns = a.n, N = a.N;  // ns: row stride of nbr and of a weight slot
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    int slot = -1;  // thread 0: the claimed queue slot, kept while the CTA speculates

    for (;;) {
        if (tid == 0) {
            int j = -1, k = -1, sp = 0;
            bool leave = false;
            if (slot < 0 && a.elastic > 0) {
                // Elastic grid: holding no slot, this CTA may leave; the CTAs that hold the
                // unfilled slots (at least a.elastic of them) process every entry still to
                // come, and none of them leaves while it holds one.
                const int waiting = *((volatile int*)&a.ctr->q_head) - *((volatile int*)&a.ctr->q_tail);
                leave = waiting >= a.elastic;
            }
            if (slot < 0 && !leave) slot = atomicAdd(&a.ctr->q_head, 1);
            if (!leave && slot < N) {
                const unsigned long long t0 = globaltimer_ns();
                unsigned nsl = 32;
                for (;;) {
                    j = *((volatile int*)&a.queue[slot]);
                    if (j >= 0) break;
                    if (*((volatile int*)&a.ctr->done) >= N || *((volatile int*)&a.ctr->abort) != 0) {
                        j = -1;
                        break;
                    }
                    if (globaltimer_ns() - t0 > a.timeout_ns) {
                        set_error(a.ctr, RBFFD_ETIMEOUT);
                        atomicExch(&a.ctr->abort, 1);
                        j = -1;
                        break;
                    }
                    if (a.spec && (k = pick_spec(a)) >= 0) break;  // idle: solve ahead
                    __nanosleep(nsl);
                    if (nsl < 2048) nsl <<= 1;
                }
            }
            if (j >= 0) {
                slot = -1;
                if (a.spec) sp = *((volatile int*)&a.spec[j]);
                fence_gpu();  // acquire what the centers that released j (or its solve) published
            }
            s_j = j;
            s_k = k;
            s_sp = sp;
            s_rej = 0;
            s_own = 0;
        }
        __syncthreads();
        const int jc = s_j, ks = s_k;
        if (jc < 0 && ks < 0) break;
        const bool ahead = jc < 0;           // a speculative solve of node ks
        const bool made = !ahead && s_sp == 2;  // center jc whose solve was made ahead
        const int j = ahead ? ks : jc;
        const Shape sh = shape_of<D>(a, sbasis, j);
        const int n = sh.n;

        // columns: the center and every later ball member not already kept by an earlier center.
        // With the centroid reference of the Lebesgue test, the reference node's column goes to
        // position 1 (after the center), and is solved as one more column when it is not such
        // a member (reference only: never kept).
        const int L = a.ball_len[j];
        if (wid == 0) {
            int q = 0;
            for (int t0 = 0; t0 < n; t0 += 32) {
                const int t = t0 + lane;
                bool inc = false;
                if (t < L) {
                    if (t == 0) inc = true;
                    else {
                        const int i = a.nbr[(size_t)j * ns + t];
                        inc = (i > j) && (__ldcg(&a.owner[i]) >= j) && !(a.bc && a.bc[i]);
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, inc);
                const int pos = q + __popc(bal & ((1u << lane) - 1u));
                if (inc) sm.cols[pos] = t;
                if (t < n) sm.colof[t] = inc ? pos : -1;
                q += __popc(bal);
            }
            __syncwarp();
            if (lane == 0) {
                int ref = 0, only = 0;
                if (a.ref_pos) {
                    const int tref = a.ref_pos[j];
                    if (tref > 0) {  // the reference column to position 1
                        int p = sm.colof[tref];
                        if (p < 0) { p = q++; sm.cols[p] = tref; only = 1; }
                        const int t1 = sm.cols[1];
                        sm.cols[1] = tref; sm.colof[tref] = 1;
                        sm.cols[p] = t1; sm.colof[t1] = p;
                        ref = 1;
                    }
                }
                s_q = q;
                s_ref = ref;
                s_refonly = only;
            }
        }
        __syncthreads();
        const int q = s_q;
        const long long base = a.slot_off[j];
        double r2c = a.rho2[j];
        if (__double_as_longlong(r2c) <= 0) r2c = 1.0;
        const double inv_r2 = rcp_fixed(r2c);
        bool ok = true;
        // The columns pass through the right-hand-side block a.qcap at a time: the first chunk
        // is carried through the factorization, later ones use the stored factors (LDL^T only;
        // with LU a.qcap covers every ball).  A center whose solve was made ahead only reads
        // its Lebesgue values.  A ball always holds its center, so q >= 1.
        if (made) {
            for (int c = tid; c < q; c += NT) sm.lam[c] = __ldcg(&a.slot_lam[base + sm.cols[c]]);
        } else {
            const int q1 = CHUNKED ? min(q, a.qcap) : q;
            ok = solve_local<D, PACKED, NT>(a, sh, j, q1, sm, s_ref);
            if (ok) lebesgue_values<NT>(n, sh.K, q1, sm);
        }
        __syncthreads();
        const int qc = (CHUNKED && !made) ? min(q, a.qcap) : q;
        // the solved columns c0 .. c0+qk-1 (held in sm.X as 0 .. qk-1) to the weight slots
        auto emit = [&](int c0, int qk) {
            const int cref = s_ref;                       // the test's reference column
            const int conly = s_refonly ? cref : -1;      // a reference-only column
            if (ahead) {  // every column goes to the node's own slots
                if (!ok) return;
                for (int e = tid; e < qk * n; e += NT) {
                    const int c = e / n, r = e - c * n;
                    if (c0 + c == conly) continue;
                    a.slot_w[(base + sm.cols[c0 + c]) * ns + r] = sm.X[sm.rowof[r] * sm.xs + c] * inv_r2;
                }
                for (int c = tid; c < qk; c += NT)
                    if (c0 + c != conly) a.slot_lam[base + sm.cols[c0 + c]] = sm.lam[c0 + c];
                return;
            }
            // Lebesgue test (§4.2.1) per column; the center keeps its own row
            int failed = 0, own = 0;
            for (int c = c0 + tid; c < c0 + qk; c += NT) {
                if (c == conly) { sm.keep[c] = 0; continue; }
                const double lam = ok ? sm.lam[c] : nan;
                const bool test_ok =
                    ok && (c == 0 || __double_as_longlong(lam) <= __double_as_longlong(sm.lam[cref]));
                bool keep;
                if (!ok) keep = (c == 0);
                else if (a.mode != RBFFD_STAB_SEQ) keep = true;
                else keep = test_ok;
                sm.keep[c] = keep ? 1 : 0;
                a.slot_lam[base + sm.cols[c]] = lam;
                a.slot_pass[base + sm.cols[c]] = (c == 0 || test_ok) ? 1 : 0;
                failed += c > 0 && !test_ok;
                own += keep && (a.mode != RBFFD_STAB_FALLBACK || c == 0 || test_ok);
            }
            if (failed) atomicAdd_block(&s_rej, failed);
            if (own) atomicAdd_block(&s_own, own);
            __syncthreads();
            for (int e = tid; !made && e < qk * n; e += NT) {  // (made ahead: already in the slots)
                const int c = e / n, r = e - c * n;
                if (!sm.keep[c0 + c]) continue;
                a.slot_w[(base + sm.cols[c0 + c]) * ns + r] =
                    ok ? sm.X[sm.rowof[r] * sm.xs + c] * inv_r2 : nan;
            }
        };
        emit(0, qc);
        if constexpr (CHUNKED) {
            for (int c0 = qc; c0 < q; c0 += qc) {  // later chunks (more columns than a.qcap)
                const int qk = min(qc, q - c0);
                __syncthreads();  // sm.X is read until here
                // (the shape is read again rather than kept in registers)
                if (ok) solve_chunk<D, NT>(a, shape_of<D>(a, sbasis, j), c0, qk, sm, j, s_ref);
                __syncthreads();
                emit(c0, qk);
            }
        }
        if (ahead) {  // publish every column, then the node's flag
            __syncthreads();
            if (tid == 0) {
                fence_gpu();
                atomicExch(&a.spec[j], ok ? 2 : 3);
                atomicAdd(&a.ctr->n_spec, 1ull);
            }
            continue;
        }
        // ownership: the earliest center keeping a row owns it
        for (int c = tid; c < q; c += NT) {
            if (c > 0 && sm.keep[c]) atomicMin(&a.owner[a.nbr[(size_t)j * ns + sm.cols[c]]], j);
        }
        __syncthreads();
        // resolve: kept members become covered; every later ball member loses a dependency.
        // Each publishing thread fences first, so the CTA's ownership updates (ordered before
        // it by the barrier) are visible wherever its state changes are.
        for (int t = 1 + tid; t < L; t += NT) {
            const int i = a.nbr[(size_t)j * ns + t];
            if (i <= j) continue;
            const int c = sm.colof[t];
            const bool kept = c >= 0 && sm.keep[c];
            fence_gpu();
            if (kept && atomicCAS(&a.state[i], kUndecided, kCovered) == kUndecided) on_covered(a, i);
            release(a, i);
        }
        if (tid == 0) {
            if (!ok) {
                atomicAdd(&a.ctr->n_singular, 1);
                set_error(a.ctr, RBFFD_ESINGULAR);
            }
            const unsigned long long K = (unsigned long long)sh.K;
            atomicAdd(&a.ctr->sum_k3, K * K * K);
            atomicAdd(&a.ctr->sum_k2q, K * K * (unsigned long long)s_own);
            atomicAdd(&a.ctr->sum_k2c, K * K * (unsigned long long)q);
            atomicAdd(&a.ctr->n_centers, 1ull);
            atomicAdd(&a.ctr->sum_cols, (unsigned long long)q);
            atomicAdd(&a.ctr->n_rejected, (unsigned long long)s_rej);
            if (made) atomicAdd(&a.ctr->n_spec_used, 1ull);
            atomicAdd(&a.ctr->done, 1);
        }
        __syncthreads();
    }
}

// FALLBACK mode: rows whose owner column failed the test get their own delta = 1 stencil.
__global__ void k_fallback_collect(SolveArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        const int s = a.owner[i];
        if (s == i || s == kNoOwner) continue;
        const int* nb = a.nbr + (size_t)s * a.n;
        const int L = a.ball_len[s];
        int t = -1;
        for (int u = 1; u < L; ++u)
            if (nb[u] == i) { t = u; break; }
        if (t < 0) { set_error(a.ctr, RBFFD_ECUDA); continue; }
        if (!a.slot_pass[a.slot_off[s] + t]) {
            a.fb_flag[i] = 1;
            a.fb_list[atomicAdd(&a.ctr->fb_count, 1)] = i;
        }
    }
}

// Normal-derivative right-hand side of node i's own stencil, replacing column 0 of the
// right-hand-side block (unknowns in index order, before the factorization).
template <int D, int NT>
__device__ void neumann_rhs(const SolveArgs& a, const Shape& sh, int i, const StencilSmem& sm) {
    for (int j = threadIdx.x; j < sh.n + sh.M; j += NT) sm.X[j * sm.xs] = neumann_value<D>(a, sh, i, j, sm);
}

// FALLBACK re-solves (one right-hand side each), one launch per stencil class: `cls` is the
// degree this launch handles (-1: all), n_cls/K_cls the largest stencil/system of the class,
// so shared memory is sized for the class and a single column.
template <int D, bool PACKED, int NT>
__global__ void __launch_bounds__(NT, team_min_blocks(NT)) k_fallback_solve(SolveArgs a, int cls, int n_cls,
                                                           int K_cls, int xs_cls,
                                                           int basis_bytes) {
    extern __shared__ __align__(16) char smem[];
    const short* sbasis = load_basis(smem, a.basis, a.basis_count);
    StencilSmem sm;
    carve<D, PACKED>(smem + basis_bytes, n_cls, K_cls, 1, xs_cls, sm);
    __syncthreads();
    const int tid = threadIdx.x;
    const int count = *((volatile int*)&a.ctr->fb_count);
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int w = blockIdx.x; w < count; w += gridDim.x) {
        const int i = a.fb_list[w];
        if (cls >= 0 && (int)a.node_ell[i] != cls) continue;  // another class's launch
        const int kind = a.bc ? (int)a.bc[i] : 0;  // boundary rows (§5) share this launch
        const Shape sh = shape_of<D>(a, sbasis, i);
        const long long slot = a.slot_off[i];
        if (kind == 1) {  // Dirichlet: the identity row, exactly
            for (int r = tid; r < sh.n; r += NT) a.slot_w[slot * a.n + r] = (r == 0) ? 1.0 : 0.0;
            if (tid == 0) a.slot_lam[slot] = 1.0;
            continue;
        }
        for (int t = tid; t < sh.n; t += NT) sm.colof[t] = (t == 0) ? 0 : -1;
        if (tid == 0) sm.cols[0] = 0;
        __syncthreads();
        assemble_local<D, PACKED, NT>(a, sh, i, 1, sm);
        if (kind == 2) {
            neumann_rhs<D, NT>(a, sh, i, sm);
            __syncthreads();
        }
        bool ok;
        if constexpr (PACKED) {
            double* gA = refine_scratch<NT, true>(a);
            if (gA) copy_full_matrix<NT>(sh.K, sm, gA);
            ok = factor_solve_ldlt<NT, true>(sh.K, 1, sm);
            if (ok && gA) refine_columns<D, NT>(a, sh, 0, 1, sm, gA, gA + a.rs_x0, kind, i);
        } else {
            ok = factor_solve_lu<NT>(sh.K, 1, sm);
        }
        if (ok) lebesgue_values<NT>(sh.n, sh.K, 1, sm);
        __syncthreads();
        double r2c = a.rho2[i];
        if (__double_as_longlong(r2c) <= 0) r2c = 1.0;
        // weights of the scaled problem times rho^-2 (Laplacian) or rho^-1 (normal derivative)
        const double scale = kind == 2 ? rcp_fixed(sqrt(r2c)) : rcp_fixed(r2c);
        for (int r = tid; r < sh.n; r += NT)
            a.slot_w[slot * a.n + r] = ok ? sm.X[sm.rowof[r] * sm.xs] * scale : nan;
        if (tid == 0) {
            a.slot_lam[slot] = ok ? sm.lam[0] : nan;
            if (!ok) {
                atomicAdd(&a.ctr->n_singular, 1);
                set_error(a.ctr, RBFFD_ESINGULAR);
            }
            const unsigned long long K = (unsigned long long)sh.K;
            atomicAdd(&a.ctr->sum_k3, K * K * K);
            atomicAdd(&a.ctr->sum_k2q, K * K);
            atomicAdd(&a.ctr->sum_k2c, K * K);
            if (kind == 0) atomicAdd(&a.ctr->n_fallback, 1ull);
            atomicAdd(&a.ctr->sum_cols, 1ull);
        }
        __syncthreads();
    }
}

// Per-node stencils only: the length of every row (the size of the stencil that produced
// it), into `len`, for the row-pointer scan.
__global__ void k_row_len(SolveArgs a, int* __restrict__ len) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        const int s = a.fb_flag[i] ? i : a.owner[i];
        len[i] = (s == kNoOwner) ? 0 : a.node_n[s];
    }
}

// CSR: row i takes the weights of the column computed for it by its owner stencil (or its
// own fallback stencil), with the columns sorted ascending.  Uniform stencils: row i starts
// at i n; per-node stencils: row_ptr was scanned from the row lengths.
__global__ void __launch_bounds__(256) k_finalize(SolveArgs a, long long* __restrict__ row_ptr,
                                                  int* __restrict__ col, double* __restrict__ val,
                                                  double* __restrict__ lam_row,
                                                  unsigned char* __restrict__ is_center) {
    extern __shared__ int fin_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int ns = a.n;
    const bool uniform = a.node_n == nullptr;
    int* cs = fin_smem + wib * ns;
    for (int i = blockIdx.x * wpb + wib; i < a.N; i += gridDim.x * wpb) {
        const bool fb = a.fb_flag[i] != 0;
        const int s = fb ? i : a.owner[i];
        if (s == kNoOwner) {
            if (lane == 0) set_error(a.ctr, RBFFD_ECUDA);
            continue;
        }
        const int n = uniform ? ns : a.node_n[s];
        int t = 0;
        if (s != i) {
            const int L = a.ball_len[s];
            int found = -1;
            for (int u0 = 1; u0 < L; u0 += 32) {
                const int u = u0 + lane;
                const bool hit = u < L && a.nbr[(size_t)s * ns + u] == i;
                const unsigned b = __ballot_sync(0xffffffffu, hit);
                if (b && found < 0) found = u0 + __ffs(b) - 1;
            }
            t = found;
            if (t < 0) {
                if (lane == 0) set_error(a.ctr, RBFFD_ECUDA);
                continue;
            }
        }
        const long long slot = a.slot_off[s] + t;
        const long long rp = uniform ? (long long)i * ns : row_ptr[i];
        for (int r = lane; r < n; r += 32) cs[r] = a.nbr[(size_t)s * ns + r];
        __syncwarp();
        for (int r = lane; r < n; r += 32) {
            const int c = cs[r];
            int rank = 0;
            for (int u = 0; u < n; ++u) rank += cs[u] < c;
            col[rp + rank] = c;
            val[rp + rank] = a.slot_w[slot * ns + r];
        }
        if (lane == 0) {
            if (fb) a.owner[i] = i;  // a fallback row names its own stencil
            if (uniform) {
                row_ptr[i] = rp;
                if (i == a.N - 1) row_ptr[a.N] = (long long)a.N * ns;
            }
            lam_row[i] = a.slot_lam[slot];
            is_center[i] = fb ? ((a.bc && a.bc[i]) ? 3 : 2) : (s == i ? 1 : 0);
        }
        __syncwarp();
    }
}

// y = L u, one warp per row
__global__ void __launch_bounds__(256) k_spmv(int N, const long long* __restrict__ row_ptr,
                                              const int* __restrict__ col,
                                              const double* __restrict__ val,
                                              const double* __restrict__ u, double* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < N; i += gridDim.x * wpb) {
        const long long b = row_ptr[i], e = row_ptr[i + 1];
        double s = 0.0;
        for (long long k = b + lane; k < e; k += 32) s = fma(val[k], __ldg(&u[col[k]]), s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) y[i] = s;
    }
}

// Values of the time-stepping matrix of §5 on L's pattern, one warp per row: interior rows
// e_i - c L_i, boundary rows unchanged.  Rounded as 1 - c v and -(c v).
__global__ void __launch_bounds__(256) k_timestep(int N, const long long* __restrict__ row_ptr,
                                                  const int* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const unsigned char* __restrict__ bc, double c,
                                                  double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < N; i += gridDim.x * wpb) {
        const bool boundary = bc && bc[i];
        for (long long k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) {
            const double v = val[k];
            const double cv = __dmul_rn(c, v);
            out[k] = boundary ? v : (col[k] == i ? __dsub_rn(1.0, cv) : -cv);
        }
    }
}

// ------------------------------------------------------------------ launchers
static int sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// The dynamic shared-memory limit is a per-kernel setting shared by every host thread, so it
// is always raised to the device maximum (never lowered to one plan's need): plans assembled
// concurrently on other streams cannot undercut each other's launches.  Raised once per
// (device, kernel); occupancy answers are cached per (device, kernel, block, shared memory),
// so planning does not repeat these driver queries while the GPU waits.
namespace {
struct SmemRaised { int dev; const void* k; };
struct OccEntry { int dev; const void* k; int nt; size_t smem; int per_sm; };
std::mutex g_attr_mu;
SmemRaised g_raised[128];
int g_n_raised = 0;
OccEntry g_occ[512];
int g_n_occ = 0;
}  // namespace

static cudaError_t allow_max_smem(const void* kern) {
    int dev = 0, mx = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    for (int i = 0; i < g_n_raised; ++i)
        if (g_raised[i].dev == dev && g_raised[i].k == kern) return cudaSuccess;
    cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             mx - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess && g_n_raised < 128) g_raised[g_n_raised++] = {dev, kern};
    return e;
}

static cudaError_t occupancy(int* per_sm, const void* kern, int nt, size_t smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        for (int i = 0; i < g_n_occ; ++i)
            if (g_occ[i].dev == dev && g_occ[i].k == kern && g_occ[i].nt == nt &&
                g_occ[i].smem == smem) {
                *per_sm = g_occ[i].per_sm;
                return cudaSuccess;
            }
    }
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, nt, smem);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        if (g_n_occ < 512) g_occ[g_n_occ++] = {dev, kern, nt, smem, *per_sm};
    }
    return e;
}

// Resident CTAs per SM of the traversal kernel at team size nt (0 if nt has no instantiation
// for this factorization).
// The traversal kernel for a team size, or nullptr (teams below 128 and chunked right-hand
// sides exist for LDL^T only).
template <int D, bool PACKED, bool CH>
static const void* traversal_kernel(int nt) {
    if constexpr (!PACKED && CH) {
        return nullptr;
    } else {
        switch (nt) {
            case 32: if constexpr (PACKED) return (const void*)k_traversal<D, PACKED, 32, CH>; break;
            case 64: if constexpr (PACKED) return (const void*)k_traversal<D, PACKED, 64, CH>; break;
            case 96: if constexpr (PACKED) return (const void*)k_traversal<D, PACKED, 96, CH>; break;
            case kNT: return (const void*)k_traversal<D, PACKED, kNT, CH>;
            case kMidNT: if constexpr (PACKED) return (const void*)k_traversal<D, PACKED, kMidNT, CH>; break;
            case kMaxNT: return (const void*)k_traversal<D, PACKED, kMaxNT, CH>;
            default: break;
        }
        return nullptr;
    }
}

template <int D, bool PACKED>
static int traversal_occupancy(int nt, size_t smem, bool chunked, int* per_sm) {
    *per_sm = 0;
    const void* k = chunked ? traversal_kernel<D, PACKED, true>(nt)
                            : traversal_kernel<D, PACKED, false>(nt);
    if (!k) return RBFFD_EINVAL;
    if (RB_CUDA(allow_max_smem(k)) ||
        RB_CUDA(occupancy(per_sm, k, nt, smem)) || *per_sm < 1)
        return RBFFD_EINVAL;
    return RBFFD_OK;
}

template <int D, bool PACKED>
static int fallback_occupancy(int nt, size_t smem, int* per_sm) {
    *per_sm = 0;
    const void* k = nt == kMaxNT ? (const void*)k_fallback_solve<D, PACKED, kMaxNT>
                                 : (const void*)k_fallback_solve<D, PACKED, kNT>;
    if constexpr (PACKED) {
        if (nt == kMidNT) k = (const void*)k_fallback_solve<D, PACKED, kMidNT>;
    }
    if (RB_CUDA(allow_max_smem(k)) ||
        RB_CUDA(occupancy(per_sm, k, nt, smem)) || *per_sm < 1)
        return RBFFD_EINVAL;
    return RBFFD_OK;
}

// Team size for a launch when none is forced: 128 threads when more than four stencils fit an
// SM's shared memory, 256 when two to four fit (LDL^T), else 512 so that the one resident
// stencil still keeps enough warps busy.  The LDL^T traversal takes 96 threads instead of 128
// unless that keeps fewer stencils resident: more stencils in flight hide more of each one's
// serial pivot steps (2D, K = 46,
// 13 columns: 13 stencils of 96 threads beat 12 of 128 by 7%), and at equal residency the
// smaller team wastes fewer lanes in its short steps (2D, 21 columns: 1.11 against 1.17 ms;
// 3D, K = 65, one column: 15.5 against 15.7 ms).  A
// forced size (32, 64, 96 and 256 exist for LDL^T only) is taken as given.
template <int D, bool PACKED, bool TRAVERSAL>
static int pick_team(size_t smem, int force, int* nt_out, int* per_sm_out, bool chunked = false,
                     bool refined = false) {
    auto occ = [&](int nt, int* ps) {
        return TRAVERSAL ? traversal_occupancy<D, PACKED>(nt, smem, chunked, ps)
                         : fallback_occupancy<D, PACKED>(nt, smem, ps);
    };
    int nt = force, rc;
    if (refined && nt != 0 && !team_refines(nt)) return RBFFD_EINVAL;  // no refinement step there
    if (nt == 0) {
        int per_sm = 0;
        if ((rc = occ(kNT, &per_sm))) return rc;
        // The fallback's one-column systems hide each other's serial pivot steps when two or
        // more share an SM (512-thread teams run one per SM: their registers fill it); two to
        // four per SM take 256-thread teams (mixed cube, K = 106, four per SM: 315 -> 302 ms
        // of fallback solves against 128-thread teams).
        // 256-thread teams exist for LDL^T only; their 64 registers let four share an SM,
        // where the 512-thread teams' registers allow one.
        const int mid = PACKED ? kMidNT : kMaxNT;
        nt = TRAVERSAL ? (per_sm <= 1 ? kMaxNT : ((per_sm <= 4 || refined) ? mid : kNT))
                       : (per_sm <= 1 ? kMaxNT : (per_sm <= 4 ? mid : kNT));
        if (TRAVERSAL && PACKED && nt == kNT) {
            int p96 = 0;
            if ((rc = occ(96, &p96))) return rc;
            if (p96 >= per_sm) nt = 96;
        }
    }
    if ((rc = occ(nt, per_sm_out))) return rc;
    *nt_out = nt;
    return RBFFD_OK;
}

// Host-side preparation, done once per plan (not per assembly, so that rbffd_assemble only
// enqueues stream work and can be captured in a CUDA graph): raise the kernels' shared-memory
// limit, choose team sizes and size the persistent grid from the occupancy.  fb[c] holds the
// fallback launch of stencil class c.
template <int D, bool PACKED>
static int prepare(int n, int K, int qcap, int qmax, int basis_count, LaunchPlan* lp) {
    int stride = 0;
    const size_t bb = basis_smem_bytes(basis_count);
    const size_t smem = bb + solve_smem_per_cta(n, K, qcap, qmax, D, PACKED, &stride);
    int per_sm = 0, rc;
    lp->chunked = PACKED && qcap < qmax;
    if ((rc = pick_team<D, PACKED, true>(smem, lp->force_nt, &lp->nt, &per_sm, lp->chunked,
                                         PACKED && K >= lp->refine_min_K)))
        return rc;
    lp->grid = per_sm * sm_count();
    lp->smem = smem;
    for (int c = 0; c < lp->n_fb; ++c) {
        FallbackClass& f = lp->fb[c];
        const size_t fs = bb + solve_smem_per_cta(f.n, f.K, 1, 1, D, PACKED, &f.xs);
        if ((rc = pick_team<D, PACKED, false>(fs, 0, &f.nt, &per_sm))) return rc;
        f.grid = per_sm * sm_count();
        f.smem = fs;
    }
    return RBFFD_OK;
}

int prepare_solve_kernels(int D, int packed, int n, int K, int qcap, int qmax, int basis_count,
                          LaunchPlan* lp) {
    if (D == 2)
        return packed ? prepare<2, true>(n, K, qcap, qmax, basis_count, lp)
                      : prepare<2, false>(n, K, qcap, qmax, basis_count, lp);
    return packed ? prepare<3, true>(n, K, qcap, qmax, basis_count, lp)
                  : prepare<3, false>(n, K, qcap, qmax, basis_count, lp);
}

template <int D, bool PACKED>
static int traversal(const SolveArgs& a, const LaunchPlan& lp, const int* indeg, cudaStream_t s,
                     int* launches, cudaEvent_t ev0, cudaEvent_t ev1) {
    const int basis_bytes = (int)basis_smem_bytes(a.basis_count);
    const int tb = 256, nb = (a.N + tb - 1) / tb;
    k_traversal_init<<<nb, tb, 0, s>>>(a.N, indeg, a.bc, a.state, a.pending, a.owner, a.queue,
                                       a.fb_flag, a.spec);
    if (a.bc) {
        k_boundary_release<<<nb, tb, 0, s>>>(a);
        ++*launches;
    }
    k_traversal_seed<<<nb, tb, 0, s>>>(a);
    *launches += 2;
    int grid = min(lp.grid, a.N);
    if (a.max_ctas > 0) grid = min(grid, a.max_ctas);
    // A plain launch suffices: a worker only waits for queue entries that workers already
    // running will push (the smallest unresolved node is always ready once every center
    // that holds a claimed entry is solved), so progress needs no co-residency, and plans
    // on other streams can run beside this grid.
    if (ev0) cudaEventRecord(ev0, s);
    size_t per_cta = lp.smem - basis_bytes;
    int bb = basis_bytes;
    SolveArgs args = a;
    const void* k = lp.chunked ? traversal_kernel<D, PACKED, true>(lp.nt)
                               : traversal_kernel<D, PACKED, false>(lp.nt);
    if (!k) return RBFFD_EINVAL;
    void* params[] = {&args, &per_cta, &bb};
    const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(lp.nt), params, lp.smem, s);
    if (ev1) cudaEventRecord(ev1, s);
    ++*launches;
    if (e != cudaSuccess) return RB_CUDA(e);
    return RB_LAUNCHED(__func__);
}

int launch_centroid_ref(int D, const double* X, const int* nbr, const int* node_n, int N, int ns,
                        unsigned char* ref_pos, cudaStream_t s, int* launches) {
    const int tb = 256, nb = (int)(((size_t)N * 32 + tb - 1) / tb);
    if (D == 2) k_centroid_ref<2><<<nb, tb, 0, s>>>(X, nbr, node_n, N, ns, ref_pos);
    else k_centroid_ref<3><<<nb, tb, 0, s>>>(X, nbr, node_n, N, ns, ref_pos);
    ++*launches;
    return RB_LAUNCHED(__func__);
}

int launch_traversal(int D, const SolveArgs& a, const LaunchPlan& lp, const int* indeg,
                     cudaStream_t s, int* launches, cudaEvent_t ev0, cudaEvent_t ev1) {
    const bool packed = a.factor == RBFFD_FACTOR_LDLT;
    if (D == 2)
        return packed ? traversal<2, true>(a, lp, indeg, s, launches, ev0, ev1)
                      : traversal<2, false>(a, lp, indeg, s, launches, ev0, ev1);
    return packed ? traversal<3, true>(a, lp, indeg, s, launches, ev0, ev1)
                  : traversal<3, false>(a, lp, indeg, s, launches, ev0, ev1);
}

template <int D, bool PACKED>
static void launch_fallback_mid(const SolveArgs& af, const FallbackClass& f, int basis_bytes,
                                cudaStream_t s) {
    if constexpr (PACKED)
        k_fallback_solve<D, PACKED, kMidNT><<<f.grid, kMidNT, f.smem, s>>>(af, f.cls, f.n, f.K, f.xs, basis_bytes);
}

template <int D, bool PACKED>
static int fallback(const SolveArgs& a, const LaunchPlan& lp, cudaStream_t s, int* launches) {
    const int tb = 256, nb = (a.N + tb - 1) / tb;
    if (a.mode == RBFFD_STAB_FALLBACK) {  // rows that failed the test (boundary rows are queued)
        k_fallback_collect<<<nb, tb, 0, s>>>(a);
        ++*launches;
    }
    const int basis_bytes = (int)basis_smem_bytes(a.basis_count);
    for (int c = 0; c < lp.n_fb; ++c) {
        const FallbackClass& f = lp.fb[c];
        SolveArgs af = a;  // refinement scratch laid out for this class's systems
        af.rs_stride = f.rs_stride;
        af.rs_x0 = f.rs_x0;
        if (f.nt == kMaxNT)
            k_fallback_solve<D, PACKED, kMaxNT><<<f.grid, kMaxNT, f.smem, s>>>(af, f.cls, f.n, f.K, f.xs, basis_bytes);
        else if (PACKED && f.nt == kMidNT)
            launch_fallback_mid<D, PACKED>(af, f, basis_bytes, s);
        else
            k_fallback_solve<D, PACKED, kNT><<<f.grid, kNT, f.smem, s>>>(af, f.cls, f.n, f.K, f.xs, basis_bytes);
        ++*launches;
    }
    return RB_LAUNCHED(__func__);
}

int launch_fallback(int D, const SolveArgs& a, const LaunchPlan& lp, cudaStream_t s,
                    int* launches) {
    const bool packed = a.factor == RBFFD_FACTOR_LDLT;
    if (D == 2)
        return packed ? fallback<2, true>(a, lp, s, launches) : fallback<2, false>(a, lp, s, launches);
    return packed ? fallback<3, true>(a, lp, s, launches) : fallback<3, false>(a, lp, s, launches);
}

int launch_finalize(const SolveArgs& a, long long* row_ptr, int* col, double* val,
                    double* lam_row, unsigned char* is_center, cudaStream_t s, int* launches) {
    if (a.node_n) {  // rows of different lengths: scan their lengths into row_ptr first
        const int tb = 256, nb = (a.N + tb - 1) / tb;
        k_row_len<<<nb, tb, 0, s>>>(a, a.fb_list);
        ++*launches;
        int rc = launch_scan_i32_to_i64(a.fb_list, row_ptr, a.N, s, launches);
        if (rc) return rc;
    }
    const int wpb = 8;
    const int blocks = (a.N + wpb - 1) / wpb;
    k_finalize<<<blocks, wpb * 32, wpb * a.n * sizeof(int), s>>>(a, row_ptr, col, val, lam_row,
                                                                is_center);
    ++*launches;
    return RB_LAUNCHED(__func__);
}

int launch_timestep(int N, const long long* row_ptr, const int* col, const double* val,
                    const unsigned char* bc, double c, double* out, cudaStream_t s, int* launches) {
    const int wpb = 8;
    const int blocks = (N + wpb - 1) / wpb;
    k_timestep<<<blocks, wpb * 32, 0, s>>>(N, row_ptr, col, val, bc, c, out);
    ++*launches;
    return RB_LAUNCHED(__func__);
}

int launch_spmv(int N, int n, const long long* row_ptr, const int* col, const double* val,
                const double* u, double* y, cudaStream_t s, int* launches) {
    (void)n;
    const int wpb = 8;
    const int blocks = (N + wpb - 1) / wpb;
    k_spmv<<<blocks, wpb * 32, 0, s>>>(N, row_ptr, col, val, u, y);
    ++*launches;
    return RB_LAUNCHED(__func__);
}

}  // namespace rbffd
