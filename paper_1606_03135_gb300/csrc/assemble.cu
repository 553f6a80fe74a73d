// assemble.cu -- the overlapped RBF-FD traversal (§4.1) with local L-Lebesgue stabilization
// (§4.2.1), the local FP64 solves, the CSR scatter and y = L u.
//
// Traversal as a dataflow.  The sequential rule "visit k = 0..N-1; an uncovered k becomes a
// center and keeps the members of its retention ball that pass the Lebesgue test" has a
// unique outcome: k is a center iff no earlier center keeps it, and a row belongs to the
// earliest center keeping it.  Whether center j keeps node i depends only on stencil j and
// x_i, so node k's fate is final as soon as every earlier node whose ball contains k (its
// in-neighbours, counted in `indeg`) is final.  A persistent kernel runs this: a node whose
// in-neighbours are all final and none kept it is pushed to a work queue as a center; a warp
// pops it, factors its local system once, solves the right-hand sides of its still-open
// ball members, and then (i) marks the members it keeps as covered and (ii) releases one
// dependency of each later ball member.  Every device-side wait is bounded by a timeout and
// ends the kernel with RBFFD_ETIMEOUT.
//
// Local solve (one warp per stencil).  The (n+M) x (n+M) saddle-point matrix [A P; P^T 0]
// of §4.1 and the q right-hand sides of the overlapped system (one per solved ball member)
// are assembled side by side in shared memory as one K x (K+q) array and reduced by
// Gaussian elimination with partial pivoting (the forward substitution rides along with
// the factorization), followed by back substitution for the q columns.  This is exactly
// the paper's cost model (2/3) K^3 + 2 K^2 q flops.  Every FP64 warp instruction occupies
// all 32 lanes of the narrow FP64 pipe whatever its active mask, so the updates are
// flattened over (row, column) pairs to keep lanes busy.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "rbffd_internal.cuh"

namespace rbffd {

struct WarpSmem {
    double* A;     // K rows x stride, [A P | B ; P^T 0 | B_psi]
    double* xi;    // n x D scaled stencil coordinates
    double* rdiag; // K reciprocal pivots
    int* cols;     // qcap: ball position of each solved column
    int* colof;    // n: column of each ball position or -1
};

size_t solve_smem_per_warp(int n, int K, int qcap, int D, int* stride_out) {
    int stride = K + qcap;
    if ((stride & 1) == 0) ++stride;  // odd row stride: column walks hit distinct banks
    if (stride_out) *stride_out = stride;
    size_t b = (size_t)K * stride * 8 + (size_t)n * D * 8 + (size_t)K * 8 +
               (size_t)(qcap + n) * 4;
    return (b + 15) & ~size_t(15);
}

__device__ __forceinline__ double ipow_rn(double x, int e) {
    double p = 1.0;
    for (int s = 0; s < e; ++s) p = __dmul_rn(p, x);
    return p;
}

// psi(x) = prod_a x_a^alpha_a (same multiplication order as the definition, no FMA)
template <int D>
__device__ __forceinline__ double mono_rn(const double* x, const signed char* al) {
    double p = 1.0;
    for (int a = 0; a < D; ++a) p = __dmul_rn(p, ipow_rn(x[a], al[a]));
    return p;
}

// Laplacian of psi: sum_a alpha_a (alpha_a - 1) x^(alpha - 2 e_a)
template <int D>
__device__ __forceinline__ double lap_mono_rn(const double* x, const signed char* al) {
    double s = 0.0;
    for (int a = 0; a < D; ++a) {
        if (al[a] < 2) continue;
        double p = (double)(al[a] * (al[a] - 1));
        for (int b = 0; b < D; ++b) p = __dmul_rn(p, ipow_rn(x[b], b == a ? al[b] - 2 : al[b]));
        s = __dadd_rn(s, p);
    }
    return s;
}

// Assemble and solve the local system of stencil j for the q columns in sm.cols.
// Returns false on an exactly zero pivot.  On return (true) the first n rows of the
// right-hand-side block of sm.A hold the scaled weights.
template <int D>
__device__ bool solve_local(const SolveArgs& a, const signed char* alpha, int j, int q,
                            const WarpSmem& sm, int lane) {
    const int n = a.n, M = a.M, K = a.K, S = a.stride, m = a.m;
    const int Wd = K + q;
    double r2c = a.rho2[j];
    if (!(r2c > 0.0)) r2c = 1.0;
    const double rho = sqrt(r2c);
    const double* xc = a.X + (size_t)j * D;
    for (int t = lane; t < n; t += 32) {
        const int id = a.nbr[(size_t)j * n + t];
        for (int c = 0; c < D; ++c)
            sm.xi[t * D + c] = __ddiv_rn(__dsub_rn(a.X[(size_t)id * D + c], xc[c]), rho);
    }
    for (int e = lane; e < K * Wd; e += 32) {
        const int r = e / Wd, c = e - r * Wd;
        sm.A[r * S + c] = 0.0;
    }
    __syncwarp();
    // A_ab = r^m and, for solved ball members, the phi-part of the right-hand side
    // m (m + D - 2) r^(m-2) (Laplacian of r^m in D dimensions), pair by pair
    {
        int ra = 0, off = lane;
        while (ra < n - 1 && off >= n - 1 - ra) { off -= n - 1 - ra; ++ra; }
        while (ra < n - 1) {
            const int rb = ra + 1 + off;
            const double r2 = sqdist_rn<D>(sm.xi + ra * D, sm.xi + rb * D);
            const double r = sqrt(r2);
            double pm2 = r;
            for (int s = 0; s < (m - 3) / 2; ++s) pm2 = __dmul_rn(pm2, r2);
            const double pm = __dmul_rn(pm2, r2);
            sm.A[ra * S + rb] = pm;
            sm.A[rb * S + ra] = pm;
            const int ca = sm.colof[ra], cb = sm.colof[rb];
            if (cb >= 0) sm.A[ra * S + K + cb] = __dmul_rn(a.coef, pm2);
            if (ca >= 0) sm.A[rb * S + K + ca] = __dmul_rn(a.coef, pm2);
            off += 32;
            while (ra < n - 1 && off >= n - 1 - ra) { off -= n - 1 - ra; ++ra; }
        }
    }
    // polynomial blocks P and P^T
    for (int e = lane; e < n * M; e += 32) {
        const int r = e / M, l = e - r * M;
        const double v = mono_rn<D>(sm.xi + r * D, alpha + l * D);
        sm.A[r * S + n + l] = v;
        sm.A[(n + l) * S + r] = v;
    }
    // psi-part of the right-hand sides: Laplacian of each monomial at each solved member
    for (int e = lane; e < M * q; e += 32) {
        const int l = e / q, c = e - l * q;
        sm.A[(n + l) * S + K + c] = lap_mono_rn<D>(sm.xi + sm.cols[c] * D, alpha + l * D);
    }
    __syncwarp();

    // Gaussian elimination with partial pivoting on [A_hat | B_hat]
    for (int p = 0; p < K; ++p) {
        unsigned long long bv = 0ull;
        int bi = 0x7fffffff;
        for (int i = p + lane; i < K; i += 32) {
            const unsigned long long v =
                (unsigned long long)__double_as_longlong(sm.A[i * S + p]) & 0x7fffffffffffffffull;
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (bv == 0ull) return false;
        if (bi != p) {
            for (int c = p + lane; c < Wd; c += 32) {
                const double t = sm.A[p * S + c];
                sm.A[p * S + c] = sm.A[bi * S + c];
                sm.A[bi * S + c] = t;
            }
            __syncwarp();
        }
        const double rcp = 1.0 / sm.A[p * S + p];
        if (lane == 0) sm.rdiag[p] = rcp;
        for (int i = p + 1 + lane; i < K; i += 32) sm.A[i * S + p] = sm.A[i * S + p] * rcp;
        __syncwarp();
        const int wr = K - p - 1, wc = Wd - p - 1;
        if (wr > 0 && wc > 0) {
            const int total = wr * wc;
            int ii = lane / wc, jj = lane - (lane / wc) * wc;
            const int di = 32 / wc, dj = 32 - di * wc;
            double* Ap = sm.A + p * S + p + 1;
            double* Ab = sm.A + (p + 1) * S;
#pragma unroll 4
            for (int e = lane; e < total; e += 32) {
                double* row = Ab + ii * S;
                row[p + 1 + jj] = fma(-row[p], Ap[jj], row[p + 1 + jj]);
                ii += di;
                jj += dj;
                if (jj >= wc) { jj -= wc; ++ii; }
            }
        }
        __syncwarp();
    }
    // back substitution, q columns at once
    for (int p = K - 1; p >= 0; --p) {
        const double rcp = sm.rdiag[p];
        for (int c = lane; c < q; c += 32) sm.A[p * S + K + c] *= rcp;
        __syncwarp();
        const int total = p * q;
        if (total > 0) {
            int ii = lane / q, jj = lane - (lane / q) * q;
            const int di = 32 / q, dj = 32 - di * q;
            const double* xp = sm.A + p * S + K;
#pragma unroll 4
            for (int e = lane; e < total; e += 32) {
                double* row = sm.A + ii * S;
                row[K + jj] = fma(-row[p], xp[jj], row[K + jj]);
                ii += di;
                jj += dj;
                if (jj >= q) { jj -= q; ++ii; }
            }
        }
        __syncwarp();
    }
    return true;
}

// ------------------------------------------------------------------ traversal state machine
__device__ __forceinline__ void push_center(const SolveArgs& a, int k) {
    __threadfence();
    const int slot = atomicAdd(&a.ctr->q_tail, 1);
    atomicExch(&a.queue[slot], k);
}

__device__ __forceinline__ void release(const SolveArgs& a, int k) {
    const int old = atomicSub(&a.pending[k], 1);
    if (old == 1) {
        __threadfence();
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

__global__ void k_traversal_init(int N, const int* __restrict__ indeg, int* state, int* pending,
                                 int* owner, int* queue, unsigned char* fb_flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        state[i] = kUndecided;
        pending[i] = indeg[i];
        owner[i] = kNoOwner;
        queue[i] = -1;
        fb_flag[i] = 0;
    }
}

__global__ void k_traversal_seed(SolveArgs a, const int* __restrict__ indeg) {
    if (a.no_seed) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        if (indeg[i] == 0) {
            a.state[i] = kCenter;
            a.owner[i] = i;
            push_center(a, i);
        }
    }
}

template <int D>
__device__ __forceinline__ void carve(char* smem, int wib, size_t per_warp, int n, int K,
                                      int qcap, int S, WarpSmem& sm) {
    char* p = smem + per_warp * wib;
    sm.A = reinterpret_cast<double*>(p);
    p += (size_t)K * S * 8;
    sm.xi = reinterpret_cast<double*>(p);
    p += (size_t)n * D * 8;
    sm.rdiag = reinterpret_cast<double*>(p);
    p += (size_t)K * 8;
    sm.cols = reinterpret_cast<int*>(p);
    p += (size_t)qcap * 4;
    sm.colof = reinterpret_cast<int*>(p);
}

template <int D>
__global__ void __launch_bounds__(128) k_traversal(SolveArgs a, size_t per_warp, int alpha_bytes) {
    extern __shared__ __align__(16) char smem[];
    signed char* alpha = reinterpret_cast<signed char*>(smem);
    for (int e = threadIdx.x; e < a.M * D; e += blockDim.x) alpha[e] = a.alpha[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpSmem sm;
    carve<D>(smem + alpha_bytes, wib, per_warp, a.n, a.K, a.qcap, a.stride, sm);
    const int n = a.n, N = a.N;

    for (;;) {
        int slot = 0;
        if (lane == 0) slot = atomicAdd(&a.ctr->q_head, 1);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= N) break;
        int j = -1;
        if (lane == 0) {
            const unsigned long long t0 = globaltimer_ns();
            unsigned ns = 32;
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
                __nanosleep(ns);
                if (ns < 2048) ns <<= 1;
            }
        }
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j < 0) break;
        __threadfence();

        // columns: the center and every later ball member not already kept by an earlier center
        const int L = a.ball_len[j];
        int q = 0;
        for (int t0 = 0; t0 < n; t0 += 32) {
            const int t = t0 + lane;
            bool inc = false;
            if (t < L) {
                if (t == 0) inc = true;
                else {
                    const int i = a.nbr[(size_t)j * n + t];
                    inc = (i > j) && (__ldcg(&a.owner[i]) >= j);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, inc);
            const int pos = q + __popc(bal & ((1u << lane) - 1u));
            if (inc) sm.cols[pos] = t;
            if (t < n) sm.colof[t] = inc ? pos : -1;
            q += __popc(bal);
        }
        __syncwarp();
        const bool ok = solve_local<D>(a, alpha, j, q, sm, lane);
        if (!ok && lane == 0) {
            atomicAdd(&a.ctr->n_singular, 1);
            set_error(a.ctr, RBFFD_ESINGULAR);
        }
        // Lebesgue test per column (columns beyond 32 are handled in chunks of 32)
        int rejected = 0;
        unsigned keepmask[4] = {0u, 0u, 0u, 0u};
        {
            int done_cols = 0;
            double lam0 = 0.0;
            const int S = a.stride, K = a.K;
            const long long base = a.slot_off[j];
            double r2c = a.rho2[j];
            if (!(r2c > 0.0)) r2c = 1.0;
            const double inv_r2 = 1.0 / r2c;
            while (done_cols < q) {
                const int c = done_cols + lane;
                double lam = 0.0;
                if (ok && c < q) {
                    double s = 0.0;
                    for (int r = 0; r < n; ++r) s = __dadd_rn(s, fabs(sm.A[r * S + K + c]));
                    lam = s;
                }
                if (done_cols == 0) lam0 = __shfl_sync(0xffffffffu, lam, 0);
                bool pass = false;
                if (c < q) {
                    if (!ok) pass = (c == 0);
                    else if (a.mode != RBFFD_STAB_SEQ) pass = true;
                    else pass = __double_as_longlong(lam) <= __double_as_longlong(lam0);
                    a.slot_lam[base + sm.cols[c]] = ok ? lam : __longlong_as_double(0x7ff8000000000000LL);
                    const bool test_ok = ok && __double_as_longlong(lam) <= __double_as_longlong(lam0);
                    a.slot_pass[base + sm.cols[c]] = (c == 0 || test_ok) ? 1 : 0;
                    if (c > 0 && !test_ok) ++rejected;
                }
                const unsigned pm = __ballot_sync(0xffffffffu, pass);
                keepmask[done_cols >> 5] = pm;
                const int w = min(32, q - done_cols);
                for (int e = lane; e < w * n; e += 32) {
                    const int cc = e / n, r = e - cc * n;
                    if (!((pm >> cc) & 1u)) continue;
                    const int col = done_cols + cc;
                    const double v = ok ? sm.A[r * S + K + col] * inv_r2
                                        : __longlong_as_double(0x7ff8000000000000LL);
                    a.slot_w[(base + sm.cols[col]) * n + r] = v;
                }
                done_cols += 32;
            }
        }
        for (int o = 16; o > 0; o >>= 1) rejected += __shfl_xor_sync(0xffffffffu, rejected, o);
        // ownership: the earliest center keeping a row owns it
        for (int c = 1 + lane; c < q; c += 32) {
            if ((keepmask[c >> 5] >> (c & 31)) & 1u) {
                const int i = a.nbr[(size_t)j * n + sm.cols[c]];
                atomicMin(&a.owner[i], j);
            }
        }
        __threadfence();
        // resolve: kept members become covered; every later ball member loses a dependency
        for (int t = 1 + lane; t < L; t += 32) {
            const int i = a.nbr[(size_t)j * n + t];
            if (i <= j) continue;
            const int c = sm.colof[t];
            const bool kept = c >= 0 && ((keepmask[c >> 5] >> (c & 31)) & 1u);
            if (kept && atomicCAS(&a.state[i], kUndecided, kCovered) == kUndecided) on_covered(a, i);
            __threadfence();
            release(a, i);
        }
        if (lane == 0) {
            atomicAdd(&a.ctr->n_centers, 1ull);
            atomicAdd(&a.ctr->sum_cols, (unsigned long long)q);
            atomicAdd(&a.ctr->n_rejected, (unsigned long long)rejected);
            atomicAdd(&a.ctr->done, 1);
        }
        __syncwarp();
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

template <int D>
__global__ void __launch_bounds__(128) k_fallback_solve(SolveArgs a, size_t per_warp, int alpha_bytes) {
    extern __shared__ __align__(16) char smem[];
    signed char* alpha = reinterpret_cast<signed char*>(smem);
    for (int e = threadIdx.x; e < a.M * D; e += blockDim.x) alpha[e] = a.alpha[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpSmem sm;
    carve<D>(smem + alpha_bytes, wib, per_warp, a.n, a.K, a.qcap, a.stride, sm);
    const int count = *((volatile int*)&a.ctr->fb_count);
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int w = blockIdx.x * (blockDim.x >> 5) + wib; w < count; w += nw) {
        const int i = a.fb_list[w];
        for (int t = lane; t < a.n; t += 32) sm.colof[t] = (t == 0) ? 0 : -1;
        if (lane == 0) sm.cols[0] = 0;
        __syncwarp();
        const bool ok = solve_local<D>(a, alpha, i, 1, sm, lane);
        if (!ok && lane == 0) {
            atomicAdd(&a.ctr->n_singular, 1);
            set_error(a.ctr, RBFFD_ESINGULAR);
        }
        double lam = 0.0;
        if (ok)
            for (int r = 0; r < a.n; ++r) lam = __dadd_rn(lam, fabs(sm.A[r * a.stride + a.K]));
        double r2c = a.rho2[i];
        if (!(r2c > 0.0)) r2c = 1.0;
        const double inv_r2 = 1.0 / r2c;
        const long long slot = a.slot_off[i];
        for (int r = lane; r < a.n; r += 32)
            a.slot_w[slot * a.n + r] = ok ? sm.A[r * a.stride + a.K] * inv_r2
                                          : __longlong_as_double(0x7ff8000000000000LL);
        if (lane == 0) {
            a.slot_lam[slot] = ok ? lam : __longlong_as_double(0x7ff8000000000000LL);
            atomicAdd(&a.ctr->n_fallback, 1ull);
            atomicAdd(&a.ctr->sum_cols, 1ull);
        }
        __syncwarp();
    }
}

// CSR: row i takes the weights of the column computed for it by its owner stencil (or its
// own fallback stencil), with the columns sorted ascending.
__global__ void __launch_bounds__(256) k_finalize(SolveArgs a, long long* __restrict__ row_ptr,
                                                  int* __restrict__ col, double* __restrict__ val,
                                                  double* __restrict__ lam_row,
                                                  unsigned char* __restrict__ is_center) {
    extern __shared__ int fin_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int n = a.n;
    int* cs = fin_smem + wib * n;
    for (int i = blockIdx.x * wpb + wib; i < a.N; i += gridDim.x * wpb) {
        const bool fb = a.fb_flag[i] != 0;
        const int s = fb ? i : a.owner[i];
        if (s == kNoOwner) {
            if (lane == 0) set_error(a.ctr, RBFFD_ECUDA);
            continue;
        }
        int t = 0;
        if (s != i) {
            const int L = a.ball_len[s];
            int found = -1;
            for (int u0 = 1; u0 < L; u0 += 32) {
                const int u = u0 + lane;
                const bool hit = u < L && a.nbr[(size_t)s * n + u] == i;
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
        for (int r = lane; r < n; r += 32) cs[r] = a.nbr[(size_t)s * n + r];
        __syncwarp();
        for (int r = lane; r < n; r += 32) {
            const int c = cs[r];
            int rank = 0;
            for (int u = 0; u < n; ++u) rank += cs[u] < c;
            col[(size_t)i * n + rank] = c;
            val[(size_t)i * n + rank] = a.slot_w[slot * n + r];
        }
        if (lane == 0) {
            if (fb) a.owner[i] = i;  // a fallback row names its own stencil
            row_ptr[i] = (long long)i * n;
            lam_row[i] = a.slot_lam[slot];
            is_center[i] = fb ? 2 : (s == i ? 1 : 0);
            if (i == a.N - 1) row_ptr[a.N] = (long long)a.N * n;
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

// ------------------------------------------------------------------ launchers
static int sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

template <int D>
static int traversal(const SolveArgs& a, const int* indeg, int wpb, cudaStream_t s, int* launches,
                     cudaEvent_t ev0, cudaEvent_t ev1) {
    int stride = 0;
    const size_t per_warp = solve_smem_per_warp(a.n, a.K, a.qcap, D, &stride);
    const int alpha_bytes = (a.M * D + 15) & ~15;
    const size_t smem = alpha_bytes + per_warp * wpb;
    if (RB_CUDA(cudaFuncSetAttribute(k_traversal<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem)))
        return RBFFD_EINVAL;
    int per_sm = 0;
    if (RB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traversal<D>, wpb * 32,
                                                              smem)) ||
        per_sm < 1)
        return RBFFD_EINVAL;
    const int tb = 256, nb = (a.N + tb - 1) / tb;
    k_traversal_init<<<nb, tb, 0, s>>>(a.N, indeg, a.state, a.pending, a.owner, a.queue,
                                       a.fb_flag);
    k_traversal_seed<<<nb, tb, 0, s>>>(a, indeg);
    *launches += 2;
    int grid = per_sm * sm_count();
    SolveArgs aa = a;
    size_t pw = per_warp;
    int ab = alpha_bytes;
    void* args[] = {&aa, &pw, &ab};
    if (ev0) cudaEventRecord(ev0, s);
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_traversal<D>, dim3(grid),
                                                dim3(wpb * 32), args, smem, s);
    if (ev1) cudaEventRecord(ev1, s);
    ++*launches;
    return RB_CUDA(e);
}

int launch_traversal(int D, const SolveArgs& a, const int* indeg, int wpb, cudaStream_t s,
                     int* launches, cudaEvent_t ev0, cudaEvent_t ev1) {
    return D == 2 ? traversal<2>(a, indeg, wpb, s, launches, ev0, ev1)
                  : traversal<3>(a, indeg, wpb, s, launches, ev0, ev1);
}

template <int D>
static int fallback(const SolveArgs& a, cudaStream_t s, int* launches) {
    const int tb = 256, nb = (a.N + tb - 1) / tb;
    k_fallback_collect<<<nb, tb, 0, s>>>(a);
    int stride = 0;
    const size_t per_warp = solve_smem_per_warp(a.n, a.K, a.qcap, D, &stride);
    const int alpha_bytes = (a.M * D + 15) & ~15;
    const int wpb = 2;
    const size_t smem = alpha_bytes + per_warp * wpb;
    if (RB_CUDA(cudaFuncSetAttribute(k_fallback_solve<D>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return RBFFD_EINVAL;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fallback_solve<D>, wpb * 32, smem);
    k_fallback_solve<D><<<max(per_sm, 1) * sm_count(), wpb * 32, smem, s>>>(a, per_warp, alpha_bytes);
    *launches += 2;
    return RB_LAUNCHED(__func__);
}

int launch_fallback(int D, const SolveArgs& a, cudaStream_t s, int* launches) {
    return D == 2 ? fallback<2>(a, s, launches) : fallback<3>(a, s, launches);
}

int launch_finalize(const SolveArgs& a, long long* row_ptr, int* col, double* val,
                    double* lam_row, unsigned char* is_center, cudaStream_t s, int* launches) {
    const int wpb = 8;
    const int blocks = (a.N + wpb - 1) / wpb;
    k_finalize<<<blocks, wpb * 32, wpb * a.n * sizeof(int), s>>>(a, row_ptr, col, val, lam_row,
                                                                is_center);
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
