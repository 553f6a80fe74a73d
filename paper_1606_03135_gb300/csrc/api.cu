// api.cu -- the C ABI declared in include/rbffd.h: argument checks, device memory of a plan
// (stream-ordered allocations), the launch sequence and error reporting.  No call throws,
// traps, asserts or exits; every CUDA error becomes an RBFFD_* code.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "rbffd_internal.cuh"

using namespace rbffd;

struct rbffd_plan_s {
    int64_t N = 0;
    int d = 0, n = 0, ell = 0, m = 0, M = 0, K = 0;
    double delta = 1.0;
    rbffd_opts opts{};
    int device = 0;
    cudaStream_t last = nullptr;
    // stencils
    double* X = nullptr;
    int* nbr = nullptr;
    double* rho2 = nullptr;
    int* ball_len = nullptr;
    int* indeg = nullptr;
    long long* slot_off = nullptr;
    short* basis = nullptr;  // monomial recurrence + Laplacian tables of the degrees in use
    int basis_count = 0;
    int boff[kMaxEll + 1] = {};
    int Mof[kMaxEll + 1] = {};
    bool mixed = false;      // per-node n, ell, m (rbffd_plan_mixed)
    int* node_n = nullptr;
    unsigned char* ref_pos = nullptr;  // centroid reference of the Lebesgue test (or none)
    signed char* node_ell = nullptr;
    signed char* node_m = nullptr;
    // boundary nodes (rbffd_set_boundary)
    void* bc_block = nullptr;
    unsigned char* bc = nullptr;
    double* nrm = nullptr;
    long long n_boundary = 0;
    long long nnz = 0;
    DevCounters* ctr = nullptr;
    DevCounters h_ctr{};           // host copy of the device counters
    void* plan_block = nullptr;    // one allocation for the stencil arrays
    size_t plan_bytes = 0, asm_bytes = 0;
    void* asm_block = nullptr;     // one allocation for the traversal and CSR arrays
    int max_ball = 0;
    long long total_slots = 0;
    int qcap = 0, stride = 0;
    LaunchPlan lp;
    int refine_min_K = 0x7fffffff;  // systems with K >= this are refined
    long long rs_doubles = 0, rs_stride = 0;  // refinement scratch: size, per traversal CTA
    int rs_x0 = 0;                  // offset of the first solution within a slot
    double* rs = nullptr;
    // traversal and results
    bool have_asm = false, assembled = false;
    int* state = nullptr;
    int* pending = nullptr;
    int* owner = nullptr;
    int* queue = nullptr;
    unsigned char* fb_flag = nullptr;
    int* fb_list = nullptr;
    double* slot_w = nullptr;
    double* slot_lam = nullptr;
    unsigned char* slot_pass = nullptr;
    long long* row_ptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;
    double* lam_row = nullptr;
    unsigned char* is_center = nullptr;
    int* spec = nullptr;
    cudaEvent_t ev[8] = {};
    int launches = 0;
    bool counters_fresh = false;
};

namespace rbffd {
int cuda_status(cudaError_t e, const char* what, int line) {
    if (e == cudaSuccess) return RBFFD_OK;
    static const bool debug = getenv("RBFFD_DEBUG") != nullptr;
    if (debug) fprintf(stderr, "rbffd: %s (line %d): %s\n", what, line, cudaGetErrorString(e));
    cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? RBFFD_ENOMEM : RBFFD_ECUDA;
}
}  // namespace rbffd

namespace {

#define bad(e) RB_CUDA(e)

// One stream-ordered memory pool per device, owned by the library, that keeps freed blocks
// cached (release threshold = unlimited): repeated plans on a device reuse memory without
// handing it back to the CUDA runtime.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

int pool_for(int dev, cudaMemPool_t* out) {
    if (dev < 0 || dev >= kMaxDevices) return RBFFD_ECUDA;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        int rc = bad(cudaMemPoolCreate(&pool, &props));
        if (rc) return rc;
        uint64_t thr = ~0ull;
        if ((rc = bad(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr)))) {
            cudaMemPoolDestroy(pool);
            return rc;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return RBFFD_OK;
}

// Timing events are recycled per device: creating eight events per plan would cost host time
// while the GPU waits.  Events go back to the list only after their plan's stream is drained.
std::mutex g_ev_mu;
std::vector<cudaEvent_t> g_free_ev[kMaxDevices];

int event_acquire(int dev, cudaEvent_t* e) {
    if (dev < 0 || dev >= kMaxDevices) return RBFFD_ECUDA;
    {
        std::lock_guard<std::mutex> lock(g_ev_mu);
        if (!g_free_ev[dev].empty()) {
            *e = g_free_ev[dev].back();
            g_free_ev[dev].pop_back();
            return RBFFD_OK;
        }
    }
    return bad(cudaEventCreate(e));
}

void event_release(int dev, cudaEvent_t e) {
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lock(g_ev_mu);
        if (g_free_ev[dev].size() < 256) {
            g_free_ev[dev].push_back(e);
            return;
        }
    }
    cudaEventDestroy(e);
}

// Lays several arrays out in one allocation, each on a 256-byte boundary.
struct Carver {
    size_t bytes = 0;
    template <typename T>
    size_t add(size_t count) {
        const size_t off = bytes;
        bytes += (count * sizeof(T) + 255) & ~size_t(255);
        return off;
    }
};

int pool_alloc(void** p, size_t bytes, int dev, cudaStream_t s) {
    *p = nullptr;
    cudaMemPool_t pool;
    int rc = pool_for(dev, &pool);
    if (rc) return rc;
    return bad(cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, s));
}

template <typename T>
T* at(void* base, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

long long binom(int a, int b) {
    if (b < 0 || b > a) return 0;
    long long r = 1;
    for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

// exponents of the total-degree <= ell monomials in graded order: degree 0, 1, ..., ell;
// within a degree the first exponent descending, then the second
int monomial_table(int d, int ell, signed char* out) {
    int M = 0;
    for (int g = 0; g <= ell; ++g)
        for (int a = g; a >= 0; --a) {
            if (d == 2) {
                if (out) { out[2 * M] = (signed char)a; out[2 * M + 1] = (signed char)(g - a); }
                ++M;
            } else {
                for (int b = g - a; b >= 0; --b) {
                    if (out) {
                        out[3 * M] = (signed char)a;
                        out[3 * M + 1] = (signed char)b;
                        out[3 * M + 2] = (signed char)(g - a - b);
                    }
                    ++M;
                }
            }
        }
    return M;
}

// Tables that let the kernels build the monomial basis by recurrence: psi_l is
// psi_parent[l] times coordinate var[l]; the Laplacian of psi_l is the sum over axes a of
// lap_coef[l][a] * psi_lap_child[l][a] (child = exponent minus 2 e_a, coef = e_a (e_a - 1)).
// Layout: parent[M], var[M], lap_child[M][d], lap_coef[M][d] (int16).
int basis_tables(int d, int ell, short* out) {
    signed char ex[kMaxTerms * 3];
    const int M = monomial_table(d, ell, ex);
    auto index_of = [&](const int* e) {
        for (int l = 0; l < M; ++l) {
            bool same = true;
            for (int a = 0; a < d; ++a) same = same && ex[l * d + a] == e[a];
            if (same) return l;
        }
        return -1;
    };
    short* parent = out;
    short* var = out + M;
    short* lchild = out + 2 * M;
    short* lcoef = out + 2 * M + M * d;
    for (int l = 0; l < M; ++l) {
        int e[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) e[a] = ex[l * d + a];
        parent[l] = 0;
        var[l] = 0;
        for (int a = 0; a < d; ++a)
            if (e[a] > 0) {
                e[a] -= 1;
                parent[l] = (short)index_of(e);
                var[l] = (short)a;
                e[a] += 1;
                break;
            }
        for (int a = 0; a < d; ++a) {
            if (e[a] >= 2) {
                e[a] -= 2;
                lchild[l * d + a] = (short)index_of(e);
                lcoef[l * d + a] = (short)((e[a] + 2) * (e[a] + 1));
                e[a] += 2;
            } else {
                lchild[l * d + a] = -1;
                lcoef[l * d + a] = 0;
            }
        }
    }
    return M;
}

void free_assemble(rbffd_plan_s* p, cudaStream_t s) {
    if (p->asm_block) cudaFreeAsync(p->asm_block, s);
    p->asm_block = nullptr;
    p->have_asm = false;
    p->assembled = false;
}

void free_plan(rbffd_plan_s* p) {
    if (!p) return;
    cudaStream_t s = p->last;
    free_assemble(p, s);
    if (p->plan_block) cudaFreeAsync(p->plan_block, s);
    if (p->bc_block) cudaFreeAsync(p->bc_block, s);
    cudaStreamSynchronize(s);
    for (auto& e : p->ev)
        if (e) event_release(p->device, e);
    delete p;
}

// Copy the device counters of the last call to the host (waits for the plan's stream).
int refresh_counters(rbffd_plan_s* p) {
    int rc;  // always copied: a captured assembly may have been replayed since the last call
    long long nnz = (long long)p->N * p->n;
    if ((rc = bad(cudaMemcpyAsync(&p->h_ctr, p->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                                  p->last))))
        return rc;
    if (p->mixed && p->assembled &&
        (rc = bad(cudaMemcpyAsync(&nnz, p->row_ptr + p->N, sizeof(long long),
                                  cudaMemcpyDeviceToHost, p->last))))
        return rc;
    if ((rc = bad(cudaStreamSynchronize(p->last)))) return rc;
    p->nnz = nnz;
    p->counters_fresh = true;
    return RBFFD_OK;
}

// A named host range for profilers (nsys timelines, ncu --nvtx filters): the span of the call
// that enqueues a phase.  Without an attached tool the push and pop cost a few nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

int max_optin_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

}  // namespace

extern "C" {

const char* rbffd_strerror(int code) {
    switch (code) {
        case RBFFD_OK: return "ok";
        case RBFFD_EINVAL: return "invalid argument";
        case RBFFD_EDUPLICATE: return "two nodes coincide (singular stencil)";
        case RBFFD_ENOMEM: return "device allocation failed";
        case RBFFD_ESINGULAR: return "exactly zero pivot in a local system";
        case RBFFD_ETIMEOUT: return "a bounded device-side wait ran out";
        case RBFFD_ECUDA: return "CUDA runtime error";
        case RBFFD_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

}  // extern "C"

namespace {

// Shared by rbffd_plan (uniform n, ell, m: n_node == NULL), rbffd_plan_mixed (per-node
// host arrays; n is then the largest stencil size) and rbffd_plan_delta (like: the plan whose
// nodes and stencils the new one copies instead of running the kNN; nodes is then like->X).
int plan_impl(const double* nodes, int64_t N, int d, int n, int ell, int m,
              const int32_t* n_node, const int32_t* ell_node, const int32_t* m_node,
              double delta, const rbffd_opts* opts, void* stream, rbffd_plan_t* out,
              const rbffd_plan_s* like = nullptr) {
    if (!out) return RBFFD_EINVAL;
    *out = nullptr;
    if (!nodes || (d != 2 && d != 3) || n < 1 || n > kMaxStencil || N < n || N > 0x7ffffffeLL ||
        ell < 0 || ell > kMaxEll || m < 3 || m > 15 || (m % 2) == 0 || !(delta > 0.0) ||
        !(delta <= 1.0))
        return RBFFD_EINVAL;
    const bool mixed = n_node != nullptr;
    int ell_lo = ell, ell_hi = ell, K_max = n + (int)binom(ell + d, d);
    if ((int)binom(ell + d, d) > n) return RBFFD_EINVAL;
    if (mixed) {
        ell_lo = kMaxEll;
        ell_hi = 0;
        K_max = 0;
        for (int64_t k = 0; k < N; ++k) {
            const int nk = n_node[k], lk = ell_node[k], mk = m_node[k];
            if (nk < 1 || nk > n || lk < 0 || lk > kMaxEll || mk < 3 || mk > 15 || (mk % 2) == 0)
                return RBFFD_EINVAL;
            const int Mk = (int)binom(lk + d, d);
            if (Mk > nk) return RBFFD_EINVAL;
            ell_lo = lk < ell_lo ? lk : ell_lo;
            ell_hi = lk > ell_hi ? lk : ell_hi;
            K_max = nk + Mk > K_max ? nk + Mk : K_max;
        }
    }
    rbffd_opts o{RBFFD_STAB_SEQ, 0, 5000, 1, 0, RBFFD_FACTOR_LDLT, 0, 0, 0, RBFFD_LREF_CENTER,
                 RBFFD_REFINE_AUTO, 0};
    if (opts) o = *opts;
    if (o.stab_mode < 0 || o.stab_mode > 2 || o.fault_inject < 0 || o.fault_inject > 1 ||
        (o.factor != RBFFD_FACTOR_LDLT && o.factor != RBFFD_FACTOR_LU) || o.max_ctas < 0 ||
        (o.team != 0 && o.team != 32 && o.team != 64 && o.team != 96 && o.team != 128 &&
         o.team != 256 && o.team != 512) ||
        (o.factor == RBFFD_FACTOR_LU && o.team != 0 && o.team != 128 && o.team != 512) ||
        o.rhs_chunk < 0 || (o.factor == RBFFD_FACTOR_LU && o.rhs_chunk > 0) ||
        (o.lebesgue_ref != RBFFD_LREF_CENTER && o.lebesgue_ref != RBFFD_LREF_CENTROID) ||
        o.refine < RBFFD_REFINE_AUTO || o.refine > RBFFD_REFINE_NONE || o.elastic < 0)
        return RBFFD_EINVAL;
    if (o.timeout_ms <= 0) o.timeout_ms = 5000;

    rbffd_plan_s* p = new (std::nothrow) rbffd_plan_s();
    if (!p) return RBFFD_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->N = N; p->d = d; p->n = n; p->ell = ell; p->m = m; p->M = K_max - n; p->K = K_max;
    p->delta = delta; p->opts = o; p->last = s; p->mixed = mixed;
    cudaGetDevice(&p->device);
    int rc = RBFFD_OK, qmax = 1;  // qmax: columns of the largest retention ball
    void* scratch = nullptr;
    const int Ni = (int)N;
    const int ncell_max = 2 * Ni + 64;
    const size_t sbytes = grid_scratch_bytes(Ni, d, ncell_max);
    // basis tables of every degree in [ell_lo, ell_hi], one after the other
    short h_basis[(kMaxEll + 1) * kMaxTerms * 8];
    size_t basis_count = 0;
    for (int l = 0; l <= kMaxEll; ++l) {
        p->Mof[l] = (int)binom(l + d, d);
        p->boff[l] = 0;
    }
    for (int l = ell_lo; l <= ell_hi; ++l) {
        p->boff[l] = (int)basis_count;
        basis_tables(d, l, h_basis + basis_count);
        basis_count += (size_t)p->Mof[l] * (2 + 2 * d);
    }
    p->basis_count = (int)basis_count;
    for (auto& e : p->ev)
        if ((rc = event_acquire(p->device, &e)) != RBFFD_OK) goto fail;
    {
        Carver c;
        const size_t oX = c.add<double>((size_t)N * d), oN = c.add<int>((size_t)N * n),
                     oR = c.add<double>((size_t)N), oB = c.add<int>((size_t)N),
                     oI = c.add<int>((size_t)N), oS = c.add<long long>((size_t)N + 1),
                     oP = c.add<short>(basis_count), oC = c.add<DevCounters>(1),
                     oNn = c.add<int>(mixed ? (size_t)N : 0),
                     oNl = c.add<signed char>(mixed ? (size_t)N : 0),
                     oNm = c.add<signed char>(mixed ? (size_t)N : 0),
                     oRp = c.add<unsigned char>(
                         o.lebesgue_ref == RBFFD_LREF_CENTROID ? (size_t)N : 0);
        if ((rc = pool_alloc(&p->plan_block, c.bytes, p->device, s))) goto fail;
        p->plan_bytes = c.bytes;
        p->X = at<double>(p->plan_block, oX);
        p->nbr = at<int>(p->plan_block, oN);
        p->rho2 = at<double>(p->plan_block, oR);
        p->ball_len = at<int>(p->plan_block, oB);
        p->indeg = at<int>(p->plan_block, oI);
        p->slot_off = at<long long>(p->plan_block, oS);
        p->basis = at<short>(p->plan_block, oP);
        p->ctr = at<DevCounters>(p->plan_block, oC);
        if (o.lebesgue_ref == RBFFD_LREF_CENTROID) p->ref_pos = at<unsigned char>(p->plan_block, oRp);
        if (mixed) {
            p->node_n = at<int>(p->plan_block, oNn);
            p->node_ell = at<signed char>(p->plan_block, oNl);
            p->node_m = at<signed char>(p->plan_block, oNm);
        }
    }
    if (mixed) {  // per-node parameters to the device (small: staged through host vectors)
        signed char* tmp = new (std::nothrow) signed char[2 * (size_t)N];
        if (!tmp) { rc = RBFFD_ENOMEM; goto fail; }
        for (int64_t k = 0; k < N; ++k) { tmp[k] = (signed char)ell_node[k]; tmp[N + k] = (signed char)m_node[k]; }
        rc = bad(cudaMemcpyAsync(p->node_n, n_node, (size_t)N * sizeof(int), cudaMemcpyHostToDevice, s));
        if (!rc) rc = bad(cudaMemcpyAsync(p->node_ell, tmp, (size_t)N, cudaMemcpyHostToDevice, s));
        if (!rc) rc = bad(cudaMemcpyAsync(p->node_m, tmp + N, (size_t)N, cudaMemcpyHostToDevice, s));
        if (!rc) rc = bad(cudaStreamSynchronize(s));  // the staging buffer is freed next
        delete[] tmp;
        if (rc) goto fail;
    }
    if (!like && (rc = pool_alloc(&scratch, sbytes, p->device, s))) goto fail;
    if ((rc = bad(cudaMemcpyAsync(p->X, nodes, (size_t)N * d * sizeof(double),
                                  (o.nodes_on_host && !like) ? cudaMemcpyHostToDevice
                                                             : cudaMemcpyDeviceToDevice,
                                  s))))
        goto fail;
    if ((rc = bad(cudaMemcpyAsync(p->basis, h_basis, basis_count * sizeof(short),
                                  cudaMemcpyHostToDevice, s))) ||
        (rc = bad(cudaMemsetAsync(p->ctr, 0, sizeof(DevCounters), s))))
        goto fail;
    cudaEventRecord(p->ev[0], s);
    if (like) {  // the same nodes and stencil sizes: the same kNN; only the balls change
        if ((rc = bad(cudaMemcpyAsync(p->nbr, like->nbr, (size_t)N * n * sizeof(int),
                                      cudaMemcpyDeviceToDevice, s))) ||
            (rc = bad(cudaMemcpyAsync(p->rho2, like->rho2, (size_t)N * sizeof(double),
                                      cudaMemcpyDeviceToDevice, s))))
            goto fail;
        rc = launch_balls(d, p->X, Ni, n, (1.0 - delta) * (1.0 - delta), p->nbr, p->rho2,
                          p->node_n, p->ball_len, p->indeg, p->ctr, s, &p->launches);
    } else {
        rc = launch_grid_and_knn(d, p->X, Ni, n, (1.0 - delta) * (1.0 - delta), scratch, sbytes,
                                 ncell_max, p->nbr, p->rho2, p->ball_len, p->indeg, p->node_n,
                                 p->ctr, s, &p->launches);
    }
    if (rc) goto fail;
    rc = launch_scan_i32_to_i64(p->ball_len, p->slot_off, Ni, s, &p->launches);
    if (rc) goto fail;
    if (p->ref_pos) {
        rc = launch_centroid_ref(d, p->X, p->nbr, p->node_n, Ni, n, p->ref_pos, s, &p->launches);
        if (rc) goto fail;
    }
    cudaEventRecord(p->ev[1], s);
    if (scratch) cudaFreeAsync(scratch, s);
    scratch = nullptr;
    {
        long long slots = 0;  // pageable copies: each returns once the stream has reached it
        if ((rc = bad(cudaMemcpyAsync(&p->h_ctr, p->ctr, sizeof(DevCounters),
                                      cudaMemcpyDeviceToHost, s))) ||
            (rc = bad(cudaMemcpyAsync(&slots, p->slot_off + N, sizeof(long long),
                                      cudaMemcpyDeviceToHost, s))) ||
            (rc = bad(cudaStreamSynchronize(s))))
            goto fail;
        p->total_slots = slots;
    }
    if (p->h_ctr.status) { rc = p->h_ctr.status; goto fail; }
    p->max_ball = p->h_ctr.max_ball;
    {
        // device bytes the traversal and CSR arrays will take (same layout as rbffd_assemble)
        const size_t S = (size_t)p->total_slots, Nz = (size_t)N, nz = (size_t)n;
        Carver c;
        c.add<int>(Nz); c.add<int>(Nz); c.add<int>(Nz); c.add<int>(Nz);
        c.add<unsigned char>(Nz); c.add<int>(Nz); c.add<double>(S * nz); c.add<double>(S);
        c.add<unsigned char>(S); c.add<long long>(Nz + 1); c.add<int>(Nz * nz);
        c.add<double>(Nz * nz); c.add<double>(Nz); c.add<unsigned char>(Nz); c.add<int>(Nz);
        p->asm_bytes = c.bytes;
    }
    // right-hand-side columns carried through one factorization: every column of the largest
    // ball (LU always), or with LDL^T fewer, opts.rhs_chunk or as many as shared memory holds
    // (the rest are solved in chunks of that many)
    // columns of the largest ball, plus the Lebesgue reference node when it is not a member
    qmax = (p->max_ball < 1 ? 1 : (int)p->max_ball) + (o.lebesgue_ref == RBFFD_LREF_CENTROID);
    p->qcap = qmax;
    if (o.rhs_chunk > 0 && o.rhs_chunk < p->qcap) p->qcap = o.rhs_chunk;
    {
        const bool ldlt = o.factor == RBFFD_FACTOR_LDLT;
        const size_t avail = (size_t)max_optin_smem() - 64;
        int stride = 0;
        size_t per_cta = 0;
        for (;;) {
            per_cta = solve_smem_per_cta(n, p->K, p->qcap, qmax, d, ldlt, &stride) +
                      basis_smem_bytes((int)basis_count);
            if (per_cta <= avail || !ldlt || p->qcap == 1) break;
            --p->qcap;
        }
        p->stride = stride;
        if (per_cta > avail) { rc = RBFFD_EINVAL; goto fail; }
        // fallback classes: one per degree in use (per-node stencils) or one for all nodes
        if (!mixed) {
            p->lp.n_fb = 1;
            p->lp.fb[0].cls = -1;
            p->lp.fb[0].n = n;
            p->lp.fb[0].K = p->K;
        } else {
            int nmax_of[kMaxEll + 1] = {};
            for (int64_t k = 0; k < N; ++k)
                nmax_of[ell_node[k]] = n_node[k] > nmax_of[ell_node[k]] ? n_node[k] : nmax_of[ell_node[k]];
            for (int l = 0; l <= kMaxEll; ++l)
                if (nmax_of[l] > 0) {
                    FallbackClass& f = p->lp.fb[p->lp.n_fb++];
                    f.cls = l;
                    f.n = nmax_of[l];
                    f.K = nmax_of[l] + p->Mof[l];
                }
        }
        p->lp.force_nt = o.team;
        p->refine_min_K = (!ldlt || o.refine == RBFFD_REFINE_NONE) ? 0x7fffffff
                          : o.refine == RBFFD_REFINE_ALL           ? 0
                                                                   : RBFFD_REFINE_MIN_K;
        p->lp.refine_min_K = p->refine_min_K;
        rc = prepare_solve_kernels(d, o.factor == RBFFD_FACTOR_LDLT, n, p->K, p->qcap, qmax,
                                   (int)basis_count, &p->lp);
        if (rc) goto fail;
        // refinement scratch: one slot per CTA of every launch that refines (the traversal when
        // its largest system qualifies, the fallback classes that do), each the lower triangle
        // of the largest system plus its first solution of one chunk of columns
        if (p->K >= p->refine_min_K) {  // the largest over the traversal and fallback launches
            // per CTA: the full K x K matrix, then x0 and 4 partial sums per (unknown, column)
            auto sq32 = [](long long K) { return (K * K + 31) / 32 * 32; };
            const long long K = p->K;
            p->rs_x0 = (int)sq32(K);
            // (+ K qcap + qcap: the moved block of refine_kept_columns)
            p->rs_stride = (p->rs_x0 + 6 * K * p->qcap + p->qcap + 31) / 32 * 32;
            long long doubles = (long long)p->lp.grid * p->rs_stride;
            for (int c = 0; c < p->lp.n_fb; ++c) {
                FallbackClass& f = p->lp.fb[c];
                f.rs_x0 = (int)sq32(f.K);
                f.rs_stride = (f.rs_x0 + 5 * f.K + 31) / 32 * 32;
                if ((long long)f.grid * f.rs_stride > doubles) doubles = (long long)f.grid * f.rs_stride;
            }
            p->rs_doubles = doubles;
            p->asm_bytes += ((size_t)doubles * 8 + 255) & ~size_t(255);
        }
    }
    *out = p;
    return RBFFD_OK;
fail:
    if (scratch) cudaFreeAsync(scratch, s);
    free_plan(p);
    return rc;
}

}  // namespace

extern "C" {

int rbffd_plan(const double* nodes, int64_t N, int d, int n, int ell, int m, double delta,
               const rbffd_opts* opts, void* stream, rbffd_plan_t* out) {
    NvtxRange r("rbffd_plan");
    return plan_impl(nodes, N, d, n, ell, m, nullptr, nullptr, nullptr, delta, opts, stream, out);
}

int rbffd_plan_mixed(const double* nodes, int64_t N, int d, const int32_t* n_node,
                     const int32_t* ell_node, const int32_t* m_node, double delta,
                     const rbffd_opts* opts, void* stream, rbffd_plan_t* out) {
    NvtxRange r("rbffd_plan_mixed");
    if (!out) return RBFFD_EINVAL;
    *out = nullptr;
    if (!n_node || !ell_node || !m_node || N < 1) return RBFFD_EINVAL;
    int n_max = 0;
    for (int64_t k = 0; k < N; ++k) n_max = n_node[k] > n_max ? n_node[k] : n_max;
    return plan_impl(nodes, N, d, n_max, 0, 3, n_node, ell_node, m_node, delta, opts, stream,
                     out);
}

int rbffd_plan_delta(rbffd_plan_t base, double delta, const rbffd_opts* opts, void* stream,
                     rbffd_plan_t* out) {
    NvtxRange r("rbffd_plan_delta");
    if (!out) return RBFFD_EINVAL;
    *out = nullptr;
    if (!base) return RBFFD_EINVAL;
    if (!base->mixed)
        return plan_impl(base->X, base->N, base->d, base->n, base->ell, base->m, nullptr,
                         nullptr, nullptr, delta, opts, stream, out, base);
    // per-node parameters back from the base plan's device copies (host arrays for the checks
    // and the fallback classes, as rbffd_plan_mixed takes them)
    const size_t N = (size_t)base->N;
    std::vector<int32_t> nn(N), ll(N), mm(N);
    std::vector<signed char> t8(2 * N);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if ((rc = bad(cudaMemcpyAsync(nn.data(), base->node_n, N * sizeof(int), cudaMemcpyDeviceToHost, s))) ||
        (rc = bad(cudaMemcpyAsync(t8.data(), base->node_ell, N, cudaMemcpyDeviceToHost, s))) ||
        (rc = bad(cudaMemcpyAsync(t8.data() + N, base->node_m, N, cudaMemcpyDeviceToHost, s))) ||
        (rc = bad(cudaStreamSynchronize(s))))
        return rc;
    for (size_t k = 0; k < N; ++k) { ll[k] = t8[k]; mm[k] = t8[N + k]; }
    return plan_impl(base->X, base->N, base->d, base->n, 0, 3, nn.data(), ll.data(), mm.data(),
                     delta, opts, stream, out, base);
}

int rbffd_assemble(rbffd_plan_t p, void* stream, rbffd_csr* out) {
    NvtxRange r("rbffd_assemble");
    if (!p) return RBFFD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->last = s;
    const size_t N = (size_t)p->N, n = (size_t)p->n;
    int rc = RBFFD_OK;
    if (!p->have_asm) {
        Carver c;
        const size_t S = (size_t)p->total_slots;
        const size_t o_state = c.add<int>(N), o_pend = c.add<int>(N), o_own = c.add<int>(N),
                     o_q = c.add<int>(N), o_fbf = c.add<unsigned char>(N),
                     o_fbl = c.add<int>(N), o_sw = c.add<double>(S * n),
                     o_sl = c.add<double>(S), o_sp = c.add<unsigned char>(S),
                     o_rp = c.add<long long>(N + 1), o_col = c.add<int>(N * n),
                     o_val = c.add<double>(N * n), o_lam = c.add<double>(N),
                     o_isc = c.add<unsigned char>(N), o_spec = c.add<int>(N),
                     o_rs = c.add<double>((size_t)p->rs_doubles);
        if ((rc = pool_alloc(&p->asm_block, c.bytes, p->device, s))) return rc;
        void* b = p->asm_block;
        p->state = at<int>(b, o_state); p->pending = at<int>(b, o_pend);
        p->owner = at<int>(b, o_own); p->queue = at<int>(b, o_q);
        p->fb_flag = at<unsigned char>(b, o_fbf); p->fb_list = at<int>(b, o_fbl);
        p->slot_w = at<double>(b, o_sw); p->slot_lam = at<double>(b, o_sl);
        p->slot_pass = at<unsigned char>(b, o_sp); p->row_ptr = at<long long>(b, o_rp);
        p->col = at<int>(b, o_col); p->val = at<double>(b, o_val);
        p->lam_row = at<double>(b, o_lam); p->is_center = at<unsigned char>(b, o_isc);
        p->spec = at<int>(b, o_spec);
        p->rs = p->rs_doubles > 0 ? at<double>(b, o_rs) : nullptr;
        p->have_asm = true;
    }
    SolveArgs a{};
    a.X = p->X; a.nbr = p->nbr; a.rho2 = p->rho2; a.ball_len = p->ball_len;
    a.slot_off = p->slot_off; a.basis = p->basis; a.basis_count = p->basis_count;
    for (int l = 0; l <= kMaxEll; ++l) { a.boff[l] = p->boff[l]; a.Mof[l] = p->Mof[l]; }
    a.node_n = p->node_n; a.node_ell = p->node_ell; a.node_m = p->node_m;
    a.bc = p->n_boundary > 0 ? p->bc : nullptr;
    // speculation only pays where centers wait on each other (retention balls beyond the center)
    a.spec = (p->max_ball > 1 && p->opts.lebesgue_ref == RBFFD_LREF_CENTER) ? p->spec : nullptr;
    a.nrm = p->nrm;
    a.N = (int)p->N; a.n = p->n; a.M = p->M; a.K = p->K; a.m = p->m; a.ell = p->ell;
    a.qcap = p->qcap; a.stride = p->stride; a.mode = p->opts.stab_mode;
    a.qmax = (p->max_ball < 1 ? 1 : (int)p->max_ball) + (p->ref_pos ? 1 : 0);
    a.ref_pos = p->ref_pos;
    a.coef = (double)(p->m * (p->m + p->d - 2));
    a.timeout_ns = (unsigned long long)p->opts.timeout_ms * 1000000ull;
    a.state = p->state; a.pending = p->pending; a.owner = p->owner; a.queue = p->queue;
    a.fb_flag = p->fb_flag; a.fb_list = p->fb_list;
    a.slot_w = p->slot_w; a.slot_lam = p->slot_lam; a.slot_pass = p->slot_pass; a.ctr = p->ctr;
    a.no_seed = p->opts.fault_inject == 1;
    a.factor = p->opts.factor;
    a.max_ctas = p->opts.max_ctas;
    a.elastic = p->opts.elastic;
    a.rs = p->rs;
    a.fma_r2 = p->rs == nullptr ? 1 : 0;
    a.rs_stride = p->rs_stride;
    a.rs_x0 = p->rs_x0;
    a.refine_min_K = p->refine_min_K;
    a.refine_all = p->opts.refine == RBFFD_REFINE_ALL ? 1 : 0;

    if ((rc = bad(cudaMemsetAsync(p->ctr, 0, sizeof(DevCounters), s)))) return rc;
    {
        NvtxRange t("traversal");
        rc = launch_traversal(p->d, a, p->lp, p->indeg, s, &p->launches, p->ev[2], p->ev[3]);
    }
    if (rc) return rc;
    cudaEventRecord(p->ev[4], s);
    if (p->opts.stab_mode == RBFFD_STAB_FALLBACK || p->n_boundary > 0) {
        NvtxRange f("fallback and boundary rows");
        rc = launch_fallback(p->d, a, p->lp, s, &p->launches);
        if (rc) return rc;
    }
    cudaEventRecord(p->ev[5], s);
    rc = launch_finalize(a, p->row_ptr, p->col, p->val, p->lam_row, p->is_center, s,
                         &p->launches);
    if (rc) return rc;
    cudaEventRecord(p->ev[6], s);
    p->assembled = true;
    p->counters_fresh = false;
    if (p->opts.sync) {
        if ((rc = refresh_counters(p))) return rc;
    }
    if (out) {
        out->n_rows = p->N;
        out->nnz = p->opts.sync || !p->mixed ? (p->mixed ? p->nnz : p->N * p->n) : -1;
        out->row_ptr = reinterpret_cast<const int64_t*>(p->row_ptr);
        out->col = p->col;
        out->val = p->val;
    }
    return p->opts.sync ? p->h_ctr.status : RBFFD_OK;
}

int rbffd_set_boundary(rbffd_plan_t p, const uint8_t* bc, const double* normals) {
    if (!p || p->mixed) return RBFFD_EINVAL;
    cudaStream_t s = p->last;
    if (!bc) {
        p->n_boundary = 0;
        return RBFFD_OK;
    }
    const size_t N = (size_t)p->N, d = (size_t)p->d;
    long long nb = 0;
    bool neumann = false;
    for (size_t i = 0; i < N; ++i) {
        if (bc[i] > 2) return RBFFD_EINVAL;
        nb += bc[i] != 0;
        if (bc[i] == 2) {
            neumann = true;
            if (!normals) return RBFFD_EINVAL;
            for (size_t a = 0; a < d; ++a)
                if (!std::isfinite(normals[i * d + a])) return RBFFD_EINVAL;
        }
    }
    int rc;
    if (!p->bc_block) {
        Carver c;
        const size_t ob = c.add<unsigned char>(N), on = c.add<double>(N * d);
        if ((rc = pool_alloc(&p->bc_block, c.bytes, p->device, s))) return rc;
        p->bc = at<unsigned char>(p->bc_block, ob);
        p->nrm = at<double>(p->bc_block, on);
        p->plan_bytes += c.bytes;
    }
    if ((rc = bad(cudaMemcpyAsync(p->bc, bc, N, cudaMemcpyHostToDevice, s))) ||
        (neumann && (rc = bad(cudaMemcpyAsync(p->nrm, normals, N * d * sizeof(double),
                                                cudaMemcpyHostToDevice, s)))) ||
        (!neumann && (rc = bad(cudaMemsetAsync(p->nrm, 0, N * d * sizeof(double), s)))) ||
        (rc = bad(cudaStreamSynchronize(s))))
        return rc;
    p->n_boundary = nb;
    return RBFFD_OK;
}

int rbffd_timestep_matrix(rbffd_plan_t p, double c, double* val_out, void* stream) {
    if (!p || !val_out || !std::isfinite(c)) return RBFFD_EINVAL;
    if (!p->assembled) return RBFFD_ESTATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return launch_timestep((int)p->N, p->row_ptr, p->col, p->val,
                           p->n_boundary > 0 ? p->bc : nullptr, c, val_out, s, &p->launches);
}

int rbffd_apply(rbffd_plan_t p, const double* u, double* y, void* stream) {
    NvtxRange r("rbffd_apply");
    if (!p || !u || !y) return RBFFD_EINVAL;
    if (!p->assembled) return RBFFD_ESTATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return launch_spmv((int)p->N, p->n, p->row_ptr, p->col, p->val, u, y, s, &p->launches);
}

int rbffd_stats(rbffd_plan_t p, rbffd_stats_t* out) {
    if (!p || !out) return RBFFD_EINVAL;
    int rc = p->assembled ? refresh_counters(p) : bad(cudaStreamSynchronize(p->last));
    if (rc) return rc;
    memset(out, 0, sizeof(*out));
    const DevCounters& c = p->h_ctr;
    out->n_nodes = p->N;
    out->max_ball = p->max_ball;
    out->rhs_chunk = p->qcap;
    out->refine_min_K = p->refine_min_K;
    out->n = p->n; out->M = p->M; out->K = p->K; out->d = p->d;
    out->n_launches = p->launches;
    out->plan_bytes = (int64_t)p->plan_bytes;
    out->assemble_bytes = (int64_t)p->asm_bytes;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]) == cudaSuccess) out->ms_stencils = ms;
    if (p->assembled) {
        out->n_centers = (int64_t)c.n_centers;
        out->n_fallback = (int64_t)c.n_fallback;
        out->n_boundary = (int64_t)p->n_boundary;
        out->n_speculated = (int64_t)c.n_spec;
        out->n_spec_used = (int64_t)c.n_spec_used;
        out->n_rejected = (int64_t)c.n_rejected;
        out->sum_cols = (int64_t)c.sum_cols;
        out->n_singular = c.n_singular;
        out->status = c.status;
        // (1/3) K^3 (LDL^T) or (2/3) K^3 (LU) per factorization, 2 K^2 per owned row's solve
        const double c3 = p->opts.factor == RBFFD_FACTOR_LU ? 2.0 / 3.0 : 1.0 / 3.0;
        out->alg_flops = c3 * (double)c.sum_k3 + 2.0 * (double)c.sum_k2q;
        out->sum_k3 = (double)c.sum_k3;
        out->sum_k2_cols = (double)c.sum_k2c;
        out->flops_refine = 4.0 * (double)c.sum_k2r;
        out->nnz = p->nnz;
        if (cudaEventElapsedTime(&ms, p->ev[2], p->ev[3]) == cudaSuccess) out->ms_traversal = ms;
        if (cudaEventElapsedTime(&ms, p->ev[4], p->ev[5]) == cudaSuccess) out->ms_fallback = ms;
        if (cudaEventElapsedTime(&ms, p->ev[5], p->ev[6]) == cudaSuccess) out->ms_finalize = ms;
    }
    cudaGetLastError();
    return RBFFD_OK;
}

int rbffd_export(rbffd_plan_t p, int64_t* row_ptr, int32_t* col, double* val, int32_t* owner) {
    NvtxRange r("rbffd_export");
    if (!p) return RBFFD_EINVAL;
    if (!p->assembled) return RBFFD_ESTATE;
    cudaStream_t s = p->last;
    const size_t N = (size_t)p->N, n = (size_t)p->n;
    int rc = RBFFD_OK;
    if (row_ptr && (rc = bad(cudaMemcpyAsync(row_ptr, p->row_ptr, (N + 1) * 8, cudaMemcpyDeviceToHost, s)))) return rc;
    if ((rc = refresh_counters(p))) return rc;
    const size_t nnz = (size_t)p->nnz;
    (void)n;
    if (col && (rc = bad(cudaMemcpyAsync(col, p->col, nnz * 4, cudaMemcpyDeviceToHost, s)))) return rc;
    if (val && (rc = bad(cudaMemcpyAsync(val, p->val, nnz * 8, cudaMemcpyDeviceToHost, s)))) return rc;
    if (owner && (rc = bad(cudaMemcpyAsync(owner, p->owner, N * 4, cudaMemcpyDeviceToHost, s)))) return rc;
    return bad(cudaStreamSynchronize(s));
}

int rbffd_export_async(rbffd_plan_t p, int64_t* row_ptr, int32_t* col, double* val,
                       int32_t* owner, void* stream) {
    NvtxRange r("rbffd_export_async");
    if (!p) return RBFFD_EINVAL;
    if (!p->assembled) return RBFFD_ESTATE;
    if (p->mixed && !p->counters_fresh) return RBFFD_ESTATE;
    const size_t N = (size_t)p->N;
    const size_t nnz = p->mixed ? (size_t)p->nnz : N * (size_t)p->n;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool other = s != p->last;
    int rc = RBFFD_OK;
    if (other && (rc = bad(cudaStreamWaitEvent(s, p->ev[6], 0)))) return rc;  // the assembly
    if (row_ptr && (rc = bad(cudaMemcpyAsync(row_ptr, p->row_ptr, (N + 1) * 8, cudaMemcpyDeviceToHost, s)))) return rc;
    if (col && (rc = bad(cudaMemcpyAsync(col, p->col, nnz * 4, cudaMemcpyDeviceToHost, s)))) return rc;
    if (val && (rc = bad(cudaMemcpyAsync(val, p->val, nnz * 8, cudaMemcpyDeviceToHost, s)))) return rc;
    if (owner && (rc = bad(cudaMemcpyAsync(owner, p->owner, N * 4, cudaMemcpyDeviceToHost, s)))) return rc;
    if (other) {  // the plan's next work waits for the copies
        if ((rc = bad(cudaEventRecord(p->ev[7], s)))) return rc;
        if ((rc = bad(cudaStreamWaitEvent(p->last, p->ev[7], 0)))) return rc;
    }
    return RBFFD_OK;
}

int rbffd_export_stencils(rbffd_plan_t p, int32_t* nbr, double* rho2, int32_t* ball_len) {
    if (!p) return RBFFD_EINVAL;
    cudaStream_t s = p->last;
    const size_t N = (size_t)p->N, n = (size_t)p->n;
    int rc = RBFFD_OK;
    if (nbr && (rc = bad(cudaMemcpyAsync(nbr, p->nbr, N * n * 4, cudaMemcpyDeviceToHost, s)))) return rc;
    if (rho2 && (rc = bad(cudaMemcpyAsync(rho2, p->rho2, N * 8, cudaMemcpyDeviceToHost, s)))) return rc;
    if (ball_len && (rc = bad(cudaMemcpyAsync(ball_len, p->ball_len, N * 4, cudaMemcpyDeviceToHost, s)))) return rc;
    return bad(cudaStreamSynchronize(s));
}

int rbffd_export_lambda(rbffd_plan_t p, double* lam_row, uint8_t* is_center) {
    if (!p) return RBFFD_EINVAL;
    if (!p->assembled) return RBFFD_ESTATE;
    cudaStream_t s = p->last;
    const size_t N = (size_t)p->N;
    int rc = RBFFD_OK;
    if (lam_row && (rc = bad(cudaMemcpyAsync(lam_row, p->lam_row, N * 8, cudaMemcpyDeviceToHost, s)))) return rc;
    if (is_center && (rc = bad(cudaMemcpyAsync(is_center, p->is_center, N, cudaMemcpyDeviceToHost, s)))) return rc;
    return bad(cudaStreamSynchronize(s));
}

void rbffd_destroy(rbffd_plan_t p) { free_plan(p); }

}  // extern "C"
