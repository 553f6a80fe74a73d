// knn.cu -- stencil formation (§2, §4.1): exact k-nearest neighbours by (squared distance,
// index) on a uniform cell grid, the stencil width rho_k, the retention ball of radius
// (1 - delta) rho_k and the traversal dependencies (in-degree) of every node.
//
// Bit-exactness with a brute-force search: squared distances are formed without FMA in a
// fixed order, candidates are compared by (IEEE bits of d2, index), and the search ring
// stops only once n candidates lie strictly inside a radius that no point outside the
// searched cells can reach.
#include <cuda_runtime.h>

#include "rbffd_internal.cuh"

namespace rbffd {

// ------------------------------------------------------------------ exclusive scans
// Single-CTA exclusive scan, out[0..count] with out[count] = total.  The input is walked in
// tiles of 1024 x kScanCh elements: each tile is loaded and stored coalesced through shared
// memory, where thread t scans its kScanCh contiguous elements; the block-wide scan of the
// thread sums and the running total of earlier tiles give the offsets.  When count_dev is
// given the element count is min(count, *count_dev), read on the device (the number of grid
// cells in use is only known there).  Used for cell offsets and weight-slot offsets.
constexpr int kScanCh = 4;
constexpr int kScanTile = 1024 * kScanCh;
__device__ __forceinline__ int scan_pad(int e) { return e + (e >> 5); }  // fewer bank conflicts

template <typename TI, typename TO>
__global__ void __launch_bounds__(1024) k_scan(const TI* __restrict__ in, TO* __restrict__ out,
                                               int count, const int* __restrict__ count_dev) {
    __shared__ TO tile[kScanTile + kScanTile / 32];
    __shared__ TO warp_tot[32];
    if (count_dev) count = min(count, *count_dev);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    TO carry = 0;  // total of the earlier tiles (the same in every thread)
    for (int base = 0; base < count; base += kScanTile) {
#pragma unroll
        for (int k = 0; k < kScanCh; ++k) {
            const int e = k * 1024 + tid, g = base + e;
            tile[scan_pad(e)] = g < count ? (TO)in[g] : (TO)0;
        }
        __syncthreads();
        TO v[kScanCh], sum = 0;
#pragma unroll
        for (int k = 0; k < kScanCh; ++k) {
            v[k] = tile[scan_pad(tid * kScanCh + k)];
            sum += v[k];
        }
        TO incl = sum;  // inclusive warp scan of the thread sums
        for (int o = 1; o < 32; o <<= 1) {
            const TO t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            TO w = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const TO t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            warp_tot[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        TO run = carry + (wid > 0 ? warp_tot[wid - 1] : (TO)0) + (incl - sum);
#pragma unroll
        for (int k = 0; k < kScanCh; ++k) {
            tile[scan_pad(tid * kScanCh + k)] = run;
            run += v[k];
        }
        carry += warp_tot[31];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanCh; ++k) {
            const int e = k * 1024 + tid, g = base + e;
            if (g < count) out[g] = tile[scan_pad(e)];
        }
        __syncthreads();  // the next tile reuses tile[] and warp_tot[]
    }
    if (tid == 0) out[count] = carry;
}

int launch_scan_i32_to_i64(const int* in, long long* out, int count, cudaStream_t s,
                           int* launches) {
    k_scan<int, long long><<<1, 1024, 0, s>>>(in, out, count, nullptr);
    ++*launches;
    return RB_LAUNCHED(__func__);
}

// ------------------------------------------------------------------ grid build
// Order-preserving map of a finite FP64 value to an unsigned 64-bit key and back, so the
// bounding box is reduced with integer instructions and atomics (no FP64 min/max).
__device__ __forceinline__ unsigned long long ord_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double ord_val(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Cell size for about 2 nodes per cell and the first search ring, from the bounding box.
template <int D>
__device__ void set_grid_params(const double* L, const double* H, int N, int n, int ncell_max,
                                GridParams* gp) {
    double ext[3] = {0.0, 0.0, 0.0};
    double vol = 1.0, maxext = 0.0;
    for (int a = 0; a < D; ++a) {
        ext[a] = H[a] - L[a];
        maxext = fmax(maxext, ext[a]);
    }
    if (!(maxext > 0.0)) maxext = 1.0;
    for (int a = 0; a < D; ++a) vol *= fmax(ext[a], 1e-3 * maxext);
    const double ppc = 2.0;  // target nodes per cell
    double h = (D == 2) ? sqrt(vol * ppc / N) : cbrt(vol * ppc / N);
    if (!(h > 0.0)) h = maxext;
    int dims[3] = {1, 1, 1};
    long long nc = 1;
    for (int it = 0; it < 200; ++it) {
        nc = 1;
        for (int a = 0; a < D; ++a) {
            double c = floor(ext[a] / h) + 1.0;
            dims[a] = (int)fmin(c, 1048576.0);
            nc *= dims[a];
        }
        if (nc <= ncell_max) break;
        h *= 1.1;
    }
    for (int a = 0; a < D; ++a) gp->lo[a] = L[a];
    for (int a = D; a < 3; ++a) { gp->lo[a] = 0.0; dims[a] = 1; }
    gp->h = h;
    gp->inv_h = 1.0 / h;
    for (int a = 0; a < 3; ++a) gp->dims[a] = dims[a];
    gp->ncell = (int)nc;
    // ring whose ball holds about n nodes at the average density
    double per = (double)N / (double)nc;
    double w = (D == 2) ? 3.14159265358979 : 4.18879020478639;
    double r = (D == 2) ? sqrt(n / (per * w)) : cbrt(n / (per * w));
    gp->r0 = (int)fmax(1.0, ceil(r));
    // Coordinates rounded to FP32 are within 2^-24 |x| <= 2^-24 X (X = the largest coordinate
    // magnitude) of the node's, plus 2^-149 where they fall below the normal range; the FP32
    // difference of two of them rounds once more, by at most 2^-24 of its size (<= 2^-23 X).
    // So |fl32(fl32(a) - fl32(b))| <= |a - b| + 2^-22 X (1 + 2^-20) + 2^-148.
    double X = 0.0;
    for (int a = 0; a < D; ++a) X = fmax(X, fmax(fabs(L[a]), fabs(H[a])));
    gp->xerr = __double2float_ru(0x1p-22 * X * (1.0 + 0x1p-20) + 0x1p-148);
}

// Bounding box over all CTAs (integer keys, one set of atomics per CTA); the last CTA to
// finish derives the grid parameters.
template <int D>
__global__ void __launch_bounds__(256) k_grid_params(const double* __restrict__ X, int N, int n,
                                                     int ncell_max, BBoxAcc* acc,
                                                     GridParams* gp) {
    __shared__ unsigned long long s_lo[3][8], s_hi[3][8];
    __shared__ bool s_last;
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        for (int a = 0; a < D; ++a) {
            const unsigned long long k = ord_key(X[(size_t)i * D + a]);
            lo[a] = k < lo[a] ? k : lo[a];
            hi[a] = k > hi[a] ? k : hi[a];
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int a = 0; a < D; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo[a], o);
            const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi[a], o);
            lo[a] = l2 < lo[a] ? l2 : lo[a];
            hi[a] = h2 > hi[a] ? h2 : hi[a];
        }
        if (lane == 0) { s_lo[a][wid] = lo[a]; s_hi[a][wid] = hi[a]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < D; ++a) {
            unsigned long long l = s_lo[a][0], h = s_hi[a][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                l = s_lo[a][w] < l ? s_lo[a][w] : l;
                h = s_hi[a][w] > h ? s_hi[a][w] : h;
            }
            atomicMax(&acc->nlo[a], ~l);
            atomicMax(&acc->hi[a], h);
        }
        __threadfence();
        s_last = atomicAdd(&acc->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    double L[3], H[3];
    for (int a = 0; a < D; ++a) {
        L[a] = ord_val(~*((volatile unsigned long long*)&acc->nlo[a]));
        H[a] = ord_val(*((volatile unsigned long long*)&acc->hi[a]));
    }
    set_grid_params<D>(L, H, N, n, ncell_max, gp);
}

template <int D>
__device__ __forceinline__ int cell_coord(const GridParams& g, double x, int a) {
    double t = __dmul_rn(__dsub_rn(x, g.lo[a]), g.inv_h);
    int c = (int)t;  // x >= lo, so truncation is floor
    return min(max(c, 0), g.dims[a] - 1);
}

template <int D>
__device__ __forceinline__ int cell_index(const GridParams& g, const int* c) {
    int idx = c[0];
    if (D >= 2) idx += g.dims[0] * c[1];
    if (D == 3) idx += g.dims[0] * g.dims[1] * c[2];
    return idx;
}

template <int D>
__global__ void k_cell_count(const double* __restrict__ X, int N, const GridParams* __restrict__ gp,
                             int* __restrict__ cell_of, int* __restrict__ count) {
    const GridParams g = *gp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int c[3];
        for (int a = 0; a < D; ++a) c[a] = cell_coord<D>(g, X[(size_t)i * D + a], a);
        int id = cell_index<D>(g, c);
        cell_of[i] = id;
        atomicAdd(&count[id], 1);
    }
}

template <int D>
__global__ void k_cell_fill(const double* __restrict__ X, int N, const int* __restrict__ cell_of,
                            const int* __restrict__ cell_start, int* __restrict__ cursor,
                            int* __restrict__ sorted_idx, double* __restrict__ sorted_X,
                            float* __restrict__ sorted_Xf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int c = cell_of[i];
        int pos = cell_start[c] + atomicAdd(&cursor[c], 1);
        sorted_idx[pos] = i;
        for (int a = 0; a < D; ++a) {
            const double x = X[(size_t)i * D + a];
            sorted_X[(size_t)pos * D + a] = x;
            sorted_Xf[(size_t)pos * D + a] = __double2float_rn(x);
        }
    }
}

// ------------------------------------------------------------------ kNN
__device__ __forceinline__ bool key_less(unsigned long long ka, int ia, unsigned long long kb,
                                         int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Search box of ring r around the query's cell and the squared radius that no point outside
// the box can reach (+inf when the box covers the whole grid).  (The query's exact distance to
// the box faces is larger, but admitting more candidates only makes the sort dearer.)
template <int D>
__device__ __forceinline__ bool ring_box(const GridParams& g, const double* xq, const int* c0,
                                         int r, int* clo, int* chi, unsigned long long* bkey,
                                         float* thr) {
    (void)xq;
    bool all = true;
    for (int a = 0; a < D; ++a) {
        clo[a] = max(c0[a] - r, 0);
        chi[a] = min(c0[a] + r, g.dims[a] - 1);
        all = all && clo[a] == 0 && chi[a] == g.dims[a] - 1;
    }
    const double rb = (double)r * g.h;
    const double R2 = rb * rb * (1.0 - 1e-8);
    *bkey = dkey(all ? __longlong_as_double(0x7ff0000000000000LL)  // +inf
                     : R2);
    // FP32 screen threshold (screen_outside): above R2 by more than the screen's rounding
    *thr = all ? __int_as_float(0x7f800000) : __double2float_ru(R2 * (1.0 + 0x1p-19));
    return all;
}

// FP32 screen of a kNN candidate: true only if its squared distance to the query certainly
// exceeds the ring's guaranteed radius R2, so its exact FP64 distance is not needed (the
// candidate could not be collected).  Per axis t = max(0, |fl32(qf - pf)| - xerr) <= |dx| (1 +
// 2^-24) (see xerr), and the sum of the t^2 in FP32 (three roundings at most, FMA) is at most
// d^2 (1 + 2^-21); thr is R2 (1 + 2^-19) rounded up, so a screened-out candidate has d^2 > R2
// and its FP64 key is not below the ring's key either.  Coordinates outside the FP32 range
// give inf or NaN, which never screens out.
template <int D>
__device__ __forceinline__ bool screen_outside(const float* qf, const float* __restrict__ pf,
                                               float xerr, float thr) {
    float lb = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float t = fmaxf(fabsf(__fsub_rn(qf[a], pf[a])) - xerr, 0.0f);
        lb = __fmaf_rn(t, t, lb);
    }
    return lb > thr;
}

// First ring to search for a query: the radius that holds n nodes at the density of the
// 3^d cells around the query's cell, rounded up to whole cells (never below 1).  In dense
// clusters this keeps the box small; the search grows it when too few nodes lie inside.
template <int D>
__device__ __forceinline__ int first_ring(const GridParams& g, const int* c0, int n,
                                          const int* __restrict__ cell_start) {
    int lo[3], hi[3];
    for (int a = 0; a < D; ++a) {
        lo[a] = max(c0[a] - 1, 0);
        hi[a] = min(c0[a] + 1, g.dims[a] - 1);
    }
    int cnt = 0, cells = 0;
    const int nz = (D == 3) ? hi[2] - lo[2] + 1 : 1;
    for (int rz = 0; rz < nz; ++rz)
        for (int ry = lo[1]; ry <= hi[1]; ++ry) {
            int cc[3] = {lo[0], ry, (D == 3) ? lo[2] + rz : 0};
            const int row0 = cell_index<D>(g, cc);
            cnt += cell_start[row0 + (hi[0] - lo[0]) + 1] - cell_start[row0];
            cells += hi[0] - lo[0] + 1;
        }
    const float per = fmaxf((float)cnt / (float)cells, 0.05f);  // nodes per cell
    const float vol = (D == 2) ? 3.14159265f : 4.18879020f;
    const float rad = (D == 2) ? sqrtf((float)n / (per * vol)) : cbrtf((float)n / (per * vol));
    return max(1, (int)ceilf(rad));
}

// Streaming search (any number of candidates): the warp keeps the n best candidates seen so
// far as a sorted list in shared memory and merges batches of 32 into it (ranks by comparison
// counting, so the order is exact), growing the ring from r until n candidates lie inside the
// guaranteed radius.  Returns the buffer (0 or 1) that holds the list.
template <int D>
__device__ int knn_stream(const GridParams& g, const double* xq, const float* xqf, const int* c0,
                          int r, int n, const int* __restrict__ cell_start,
                          const int* __restrict__ sorted_idx, const double* __restrict__ sorted_X,
                          const float* __restrict__ sorted_Xf, unsigned long long* lk, int* li,
                          unsigned long long* bk, int* bi) {
    const int lane = threadIdx.x & 31;
    int cnt = 0, cur = 0;
    for (;;) {
        int clo[3], chi[3];
        unsigned long long bkey;
        float thr;
        const bool all = ring_box<D>(g, xq, c0, r, clo, chi, &bkey, &thr);
        cnt = 0;
        cur = 0;
        const int ny = chi[1] - clo[1] + 1;
        const int nz = (D == 3) ? chi[2] - clo[2] + 1 : 1;
        for (int rz = 0; rz < nz; ++rz)
            for (int ry = 0; ry < ny; ++ry) {
                int cc[3] = {clo[0], clo[1] + ry, (D == 3) ? clo[2] + rz : 0};
                const int row0 = cell_index<D>(g, cc);
                const int beg = cell_start[row0];
                const int end = cell_start[row0 + (chi[0] - clo[0]) + 1];
                for (int b0 = beg; b0 < end; b0 += 32) {
                    const int p = b0 + lane;
                    bool valid = p < end;
                    unsigned long long key = ~0ull;
                    int id = 0x7fffffff;
                    if (valid && screen_outside<D>(xqf, sorted_Xf + (size_t)p * D, g.xerr, thr))
                        valid = false;
                    if (valid) {
                        double xp[3];
                        for (int a = 0; a < D; ++a) xp[a] = sorted_X[(size_t)p * D + a];
                        key = dkey(sqdist_rn<D>(xq, xp));
                        id = sorted_idx[p];
                        valid = key < bkey;
                        if (valid && cnt == n) valid = key_less(key, id, lk[cur * n + n - 1], li[cur * n + n - 1]);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, valid);
                    if (bal == 0) continue;
                    int rb_ = 0;  // rank among the valid batch members
                    for (int s2 = 0; s2 < 32; ++s2) {
                        const unsigned long long ks = __shfl_sync(0xffffffffu, key, s2);
                        const int is = __shfl_sync(0xffffffffu, id, s2);
                        if (((bal >> s2) & 1u) && key_less(ks, is, key, id)) ++rb_;
                    }
                    int lo_ = 0, hi_ = cnt;  // position in the current list
                    while (lo_ < hi_) {
                        const int mid = (lo_ + hi_) >> 1;
                        if (key_less(lk[cur * n + mid], li[cur * n + mid], key, id)) lo_ = mid + 1;
                        else hi_ = mid;
                    }
                    bk[lane] = valid ? key : ~0ull;
                    bi[lane] = valid ? id : 0x7fffffff;
                    __syncwarp();
                    const int nxt = cur ^ 1;
                    for (int e = lane; e < cnt; e += 32) {
                        const unsigned long long ke = lk[cur * n + e];
                        const int ie = li[cur * n + e];
                        int before = 0;
                        for (int s2 = 0; s2 < 32; ++s2)
                            if (((bal >> s2) & 1u) && key_less(bk[s2], bi[s2], ke, ie)) ++before;
                        const int np = e + before;
                        if (np < n) { lk[nxt * n + np] = ke; li[nxt * n + np] = ie; }
                    }
                    if (valid) {
                        const int np = lo_ + rb_;
                        if (np < n) { lk[nxt * n + np] = key; li[nxt * n + np] = id; }
                    }
                    __syncwarp();
                    cnt = min(cnt + __popc(bal), n);
                    cur = nxt;
                }
            }
        if (cnt == n || all) break;
        ++r;
    }
    return cur;
}

// One warp per query node.  Usual case: every candidate of the search box that lies inside
// the guaranteed radius is collected into shared memory (growing the ring until there are n),
// and the warp sorts them by (IEEE bits of d2, index) with a bitonic network; the first n
// are the stencil.  Boxes with more such candidates than the buffer holds (256, or 512 for
// stencils of more than 64 nodes) take the streaming search instead.  Either way the order is
// exact.
__host__ __device__ __forceinline__ int knn_collect_cap(int n) { return n > 64 ? 512 : 256; }

__host__ __device__ __forceinline__ int knn_words(int n) {  // per-warp buffer entries
    return max(2 * n + 32, knn_collect_cap(n));
}

template <int D>
__global__ void __launch_bounds__(256) k_knn(const double* __restrict__ X, int N, int n,
                                             double omd2, const GridParams* __restrict__ gp,
                                             const int* __restrict__ cell_start,
                                             const int* __restrict__ sorted_idx,
                                             const double* __restrict__ sorted_X,
                                             const float* __restrict__ sorted_Xf,
                                             int* __restrict__ nbr, double* __restrict__ rho2,
                                             int* __restrict__ ball_len, int* __restrict__ indeg,
                                             const int* __restrict__ node_n, DevCounters* ctr) {
    extern __shared__ unsigned long long knn_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int W = knn_words(n);
    unsigned long long* wk = knn_smem + (size_t)wib * W;
    int* wi = reinterpret_cast<int*>(knn_smem + (size_t)wpb * W) + (size_t)wib * W;
    int* soff = reinterpret_cast<int*>(knn_smem + (size_t)wpb * W) + (size_t)wpb * W + wib * 128;
    int* sbeg = soff + 32;
    int* squeue = soff + 64;  // candidates that passed the FP32 screen, awaiting FP64 (< 64)
    const GridParams g = *gp;

    for (int q = blockIdx.x * wpb + wib; q < N; q += gridDim.x * wpb) {
        double xq[3];
        float xqf[3];
        int c0[3];
        for (int a = 0; a < D; ++a) {
            xq[a] = X[(size_t)q * D + a];
            xqf[a] = __double2float_rn(xq[a]);
            c0[a] = cell_coord<D>(g, xq[a], a);
        }
        const int kCollect = knn_collect_cap(n);
        // node q's own stencil size (per-node plans search only that many; row q of nbr is
        // padded with -1 beyond it)
        const int nq = node_n ? node_n[q] : n;
        int r = first_ring<D>(g, c0, nq, cell_start), cnt = 0;
        bool all = false;
        for (;;) {  // collect the candidates inside the guaranteed radius of ring r
            int clo[3], chi[3];
            unsigned long long bkey;
            float thr;
            all = ring_box<D>(g, xq, c0, r, clo, chi, &bkey, &thr);
            cnt = 0;
            const int ny = chi[1] - clo[1] + 1;
            const int nz = (D == 3) ? chi[2] - clo[2] + 1 : 1;
            const int nrows = ny * nz;
            // The box's cell rows (contiguous ranges of the cell-sorted nodes) are packed into
            // full batches of 32 candidates: an FP64 warp instruction costs the same with idle
            // lanes, and a row holds only a few nodes.  Lane l takes row g0 + l, the rows'
            // offsets are scanned, and each candidate finds its row by binary search.
            for (int g0 = 0; g0 < nrows && cnt <= kCollect; g0 += 32) {
                const int R = g0 + lane;
                int beg = 0, len = 0;
                if (R < nrows) {
                    const int rz = R / ny, ry = R - rz * ny;
                    int cc[3] = {clo[0], clo[1] + ry, (D == 3) ? clo[2] + rz : 0};
                    const int row0 = cell_index<D>(g, cc);
                    beg = cell_start[row0];
                    len = cell_start[row0 + (chi[0] - clo[0]) + 1] - beg;
                }
                int incl = len;
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                soff[lane] = incl - len;
                sbeg[lane] = beg;
                __syncwarp();
                // Each batch's candidates pass an FP32 screen first (screen_outside); those that
                // may lie inside the guaranteed radius queue up, and their exact FP64 distances
                // are formed a full warp at a time, so an FP64 instruction is issued only for
                // candidates that can be collected.
                int qn = 0;
                for (int b0 = 0; b0 < total && cnt <= kCollect; b0 += 32) {
                    const int e = b0 + lane;
                    bool pass = false;
                    int p = 0;
                    if (e < total) {
                        int lo = 0, hi = 31;  // the last row whose offset is <= e (non-empty)
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (soff[mid] <= e) lo = mid;
                            else hi = mid - 1;
                        }
                        p = sbeg[lo] + (e - soff[lo]);
                        pass = !screen_outside<D>(xqf, sorted_Xf + (size_t)p * D, g.xerr, thr);
                    }
                    const unsigned pb = __ballot_sync(0xffffffffu, pass);
                    if (pass) squeue[qn + __popc(pb & ((1u << lane) - 1u))] = p;
                    qn += __popc(pb);
                    __syncwarp();
                    const bool last = b0 + 32 >= total;
                    while (qn >= 32 || (last && qn > 0)) {
                        const int m = min(qn, 32);
                        unsigned long long key = ~0ull;
                        int id = 0;
                        if (lane < m) {
                            const int pp = squeue[lane];
                            double xp[3];
                            for (int a = 0; a < D; ++a) xp[a] = sorted_X[(size_t)pp * D + a];
                            key = dkey(sqdist_rn<D>(xq, xp));
                            id = sorted_idx[pp];
                        }
                        const bool in = lane < m && key < bkey;
                        const unsigned bal = __ballot_sync(0xffffffffu, in);
                        const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                        if (in && pos < kCollect) { wk[pos] = key; wi[pos] = id; }
                        cnt += __popc(bal);
                        __syncwarp();
                        const int rest = qn - m;  // (< 32)
                        const int moved = lane < rest ? squeue[m + lane] : 0;
                        __syncwarp();
                        if (lane < rest) squeue[lane] = moved;
                        __syncwarp();
                        qn = rest;
                    }
                }
                __syncwarp();  // soff/sbeg are rewritten by the next group
            }
            if (cnt > kCollect || cnt >= nq || all) break;
            ++r;
        }
        const unsigned long long* rk;
        const int* ri;
        if (cnt > kCollect) {  // too many candidates to sort: stream them
            __syncwarp();
            const int cur = knn_stream<D>(g, xq, xqf, c0, r, nq, cell_start, sorted_idx, sorted_X,
                                          sorted_Xf, wk, wi, wk + 2 * n, wi + 2 * n);
            rk = wk + cur * nq;
            ri = wi + cur * nq;
        } else {
            int P = 32;
            while (P < cnt) P <<= 1;
            for (int e = cnt + lane; e < P; e += 32) { wk[e] = ~0ull; wi[e] = 0x7fffffff; }
            __syncwarp();
            for (int k = 2; k <= P; k <<= 1)  // bitonic sort, ascending
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const int lj = 31 - __clz(j);
                    for (int t = lane; t < (P >> 1); t += 32) {
                        const int i = ((t >> lj) << (lj + 1)) | (t & (j - 1));
                        const int l = i + j;
                        const unsigned long long ki = wk[i], kl = wk[l];
                        const int ii = wi[i], il = wi[l];
                        const bool up = (i & k) == 0;
                        if (up ? key_less(kl, il, ki, ii) : key_less(ki, ii, kl, il)) {
                            wk[i] = kl; wi[i] = il;
                            wk[l] = ki; wi[l] = ii;
                        }
                    }
                    __syncwarp();
                }
            rk = wk;
            ri = wi;
        }
        // write the stencil (the nq nearest), its width and retention ball
        const double r2k = __longlong_as_double((long long)rk[nq - 1]);
        const double rball = __dmul_rn(omd2, r2k);
        int blen = 0;
        for (int t0 = 0; t0 < n; t0 += 32) {
            const int t = t0 + lane;
            bool inb = false;
            if (t < nq) {
                const int id = ri[t];
                const double dd = __longlong_as_double((long long)rk[t]);
                nbr[(size_t)q * n + t] = id;
                inb = dd <= rball;
                if (t >= 1 && dd == 0.0) set_error(ctr, RBFFD_EDUPLICATE);
            } else if (t < n) {
                nbr[(size_t)q * n + t] = -1;
            }
            blen += __popc(__ballot_sync(0xffffffffu, inb));
        }
        if (lane == 0) {
            if (ri[0] != q) set_error(ctr, RBFFD_EDUPLICATE);
            rho2[q] = r2k;
            ball_len[q] = blen;
            atomicMax(&ctr->max_ball, blen);
        }
        for (int t = 1 + lane; t < blen; t += 32) {
            const int i = ri[t];
            if (i > q) atomicAdd(&indeg[i], 1);
        }
        __syncwarp();
    }
}

// Retention balls and traversal in-degrees of another delta from a plan's stencils (§4.1):
// node q's closed ball of radius (1 - delta) rho_q is the prefix of its neighbour list with
// d^2 <= (1 - delta)^2 rho_q^2, d^2 formed exactly as k_knn forms it (sqdist_rn of the same
// coordinates, query first), so the balls equal the ones a new kNN pass would give.  One
// warp per node; indeg must be zero on entry.
template <int D>
__global__ void __launch_bounds__(256) k_balls(const double* __restrict__ X, int N, int n,
                                               double omd2, const int* __restrict__ nbr,
                                               const double* __restrict__ rho2,
                                               const int* __restrict__ node_n,
                                               int* __restrict__ ball_len, int* __restrict__ indeg,
                                               DevCounters* ctr) {
    const int lane = threadIdx.x & 31;
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= N) return;  // (whole warps)
    double xq[3];
    for (int a = 0; a < D; ++a) xq[a] = X[q * D + a];
    const int nq = node_n ? node_n[q] : n;
    const double rball = __dmul_rn(omd2, rho2[q]);
    const int* nb = nbr + q * n;
    int blen = 0;
    for (int t0 = 0; t0 < nq; t0 += 32) {
        const int t = t0 + lane;
        bool inb = false;
        if (t < nq) {
            const int id = nb[t];
            double xp[3];
            for (int a = 0; a < D; ++a) xp[a] = X[(size_t)id * D + a];
            inb = sqdist_rn<D>(xq, xp) <= rball;
        }
        blen += __popc(__ballot_sync(0xffffffffu, inb));
    }
    if (lane == 0) {
        ball_len[q] = blen;
        atomicMax(&ctr->max_ball, blen);
    }
    for (int t = 1 + lane; t < blen; t += 32) {
        const int i = nb[t];
        if (i > q) atomicAdd(&indeg[i], 1);
    }
}

// ------------------------------------------------------------------ launcher
// Every piece carved from the scratch buffer starts on a 256-byte boundary.
static size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

size_t grid_scratch_bytes(int N, int D, int ncell_max) {
    size_t b = round256(sizeof(GridParams)) + round256(sizeof(BBoxAcc));
    b += 3 * round256((size_t)(ncell_max + 1) * sizeof(int));  // count, start, cursor
    b += 2 * round256((size_t)N * sizeof(int));                // cell_of, sorted_idx
    b += round256((size_t)N * D * sizeof(double));             // sorted_X
    b += round256((size_t)N * D * sizeof(float));              // sorted_Xf (FP32 screen)
    return b;
}

template <int D>
static int grid_and_knn(const double* X, int N, int n, double omd2, void* scratch,
                        int ncell_max, int* nbr, double* rho2, int* ball_len, int* indeg,
                        const int* node_n, DevCounters* ctr, cudaStream_t s, int* launches) {
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += round256(bytes);
        return r;
    };
    GridParams* gp = reinterpret_cast<GridParams*>(take(sizeof(GridParams)));
    BBoxAcc* acc = reinterpret_cast<BBoxAcc*>(take(sizeof(BBoxAcc)));
    int* count = reinterpret_cast<int*>(take((size_t)(ncell_max + 1) * sizeof(int)));
    int* start = reinterpret_cast<int*>(take((size_t)(ncell_max + 1) * sizeof(int)));
    int* cursor = reinterpret_cast<int*>(take((size_t)(ncell_max + 1) * sizeof(int)));
    int* cell_of = reinterpret_cast<int*>(take((size_t)N * sizeof(int)));
    int* sorted_idx = reinterpret_cast<int*>(take((size_t)N * sizeof(int)));
    double* sorted_X = reinterpret_cast<double*>(take((size_t)N * D * sizeof(double)));
    float* sorted_Xf = reinterpret_cast<float*>(take((size_t)N * D * sizeof(float)));

    int rc;
    if ((rc = RB_CUDA(cudaMemsetAsync(acc, 0, sizeof(BBoxAcc), s))) ||
        (rc = RB_CUDA(cudaMemsetAsync(count, 0, (size_t)(ncell_max + 1) * sizeof(int), s))) ||
        (rc = RB_CUDA(cudaMemsetAsync(cursor, 0, (size_t)(ncell_max + 1) * sizeof(int), s))) ||
        (rc = RB_CUDA(cudaMemsetAsync(indeg, 0, (size_t)N * sizeof(int), s))))
        return rc;
    const int tb = 256;
    const int nb = (N + tb - 1) / tb;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_grid_params<D><<<nb < sms ? nb : sms, tb, 0, s>>>(X, N, n, ncell_max, acc, gp);
    k_cell_count<D><<<nb, tb, 0, s>>>(X, N, gp, cell_of, count);
    k_scan<int, int><<<1, 1024, 0, s>>>(count, start, ncell_max, &gp->ncell);
    k_cell_fill<D><<<nb, tb, 0, s>>>(X, N, cell_of, start, cursor, sorted_idx, sorted_X,
                                     sorted_Xf);
    const int wpb = 8;
    const int words = knn_words(n);
    size_t smem = (size_t)wpb * (words * (sizeof(unsigned long long) + sizeof(int)) + 128 * sizeof(int));
    if (smem > 48 * 1024 &&
        (rc = RB_CUDA(cudaFuncSetAttribute(k_knn<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem))))
        return rc;
    int blocks = (N + wpb - 1) / wpb;
    k_knn<D><<<blocks, wpb * 32, smem, s>>>(X, N, n, omd2, gp, start, sorted_idx, sorted_X,
                                            sorted_Xf, nbr, rho2, ball_len, indeg, node_n, ctr);
    *launches += 5;
    return RB_LAUNCHED(__func__);
}

int launch_grid_and_knn(int D, const double* X, int N, int n, double omd2, void* scratch,
                        size_t scratch_bytes, int ncell_max, int* nbr, double* rho2, int* ball_len,
                        int* indeg, const int* node_n, DevCounters* ctr, cudaStream_t s,
                        int* launches) {
    if (scratch_bytes < grid_scratch_bytes(N, D, ncell_max)) return RBFFD_EINVAL;
    if (D == 2)
        return grid_and_knn<2>(X, N, n, omd2, scratch, ncell_max, nbr, rho2, ball_len, indeg,
                               node_n, ctr, s, launches);
    return grid_and_knn<3>(X, N, n, omd2, scratch, ncell_max, nbr, rho2, ball_len, indeg, node_n,
                           ctr, s, launches);
}

int launch_balls(int D, const double* X, int N, int n, double omd2, const int* nbr,
                 const double* rho2, const int* node_n, int* ball_len, int* indeg,
                 DevCounters* ctr, cudaStream_t s, int* launches) {
    int rc = RB_CUDA(cudaMemsetAsync(indeg, 0, (size_t)N * sizeof(int), s));
    if (rc) return rc;
    const int tb = 256;
    const unsigned nb = (unsigned)(((size_t)N * 32 + tb - 1) / tb);
    if (D == 2) k_balls<2><<<nb, tb, 0, s>>>(X, N, n, omd2, nbr, rho2, node_n, ball_len, indeg, ctr);
    else k_balls<3><<<nb, tb, 0, s>>>(X, N, n, omd2, nbr, rho2, node_n, ball_len, indeg, ctr);
    ++*launches;
    return RB_LAUNCHED(__func__);
}

}  // namespace rbffd
