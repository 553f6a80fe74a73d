// noalloc.cu -- rbffd_stencils_noalloc: the stencil kernels (cell grid, exact kNN, retention
// balls) run on a fixed file-scope device array instead of allocated scratch, for callers
// that cannot allocate device memory while they run.  Nothing here calls cudaMalloc,
// cudaFree or any allocating routine.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "rbffd_internal.cuh"

namespace rbffd {
namespace {

constexpr size_t r256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr int kMaxNodes = RBFFD_NOALLOC_MAX_NODES;
constexpr int kMaxCells = 2 * kMaxNodes + 64;  // the cell-grid bound rbffd_plan uses
// grid scratch for the largest case (3D) + in-degree counts + device status block
constexpr size_t kGridBytes = r256(sizeof(GridParams)) + r256(sizeof(BBoxAcc)) +
                              3 * r256((size_t)(kMaxCells + 1) * 4) +
                              2 * r256((size_t)kMaxNodes * 4) + r256((size_t)kMaxNodes * 3 * 8) +
                              r256((size_t)kMaxNodes * 3 * 4);
constexpr size_t kIndegBytes = r256((size_t)kMaxNodes * 4);
constexpr size_t kScratchBytes = kGridBytes + kIndegBytes + r256(sizeof(DevCounters));

// The working memory of every call, on every device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device;
// in host code the symbol itself is only a host-side stand-in).
int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    int rc = RB_CUDA(cudaGetDevice(&dev));
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices) return RBFFD_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        rc = RB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        if (rc) return rc;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return RBFFD_OK;
}

}  // namespace
}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_stencils_noalloc(const double* nodes, int64_t N, int d, int n,
                                      double delta, int32_t* nbr, double* rho2,
                                      int32_t* ball_len, void* stream) {
    if (!nodes || !nbr || !rho2 || !ball_len || (d != 2 && d != 3) || n < 1 ||
        n > kMaxStencil || N < n || N > kMaxNodes || !(delta > 0.0) || !(delta <= 1.0))
        return RBFFD_EINVAL;
    const int Ni = (int)N;
    const int ncell_max = 2 * Ni + 64;
    const size_t grid_bytes = grid_scratch_bytes(Ni, d, ncell_max);
    if (grid_bytes > kGridBytes) return RBFFD_EINVAL;
    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* indeg = reinterpret_cast<int*>(base + kGridBytes);
    DevCounters* ctr = reinterpret_cast<DevCounters*>(base + kGridBytes + kIndegBytes);
    // the array keeps the previous call's contents: reset the status block (the grid counts,
    // cursors and in-degrees are cleared inside the launch sequence)
    if ((rc = RB_CUDA(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s)))) return rc;
    int launches = 0;
    rc = launch_grid_and_knn(d, nodes, Ni, n, (1.0 - delta) * (1.0 - delta), base, grid_bytes,
                             ncell_max, nbr, rho2, ball_len, indeg, nullptr, ctr, s, &launches);
    if (rc) return rc;
    int status = 0;
    if ((rc = RB_CUDA(cudaMemcpyAsync(&status, &ctr->status, sizeof(int),
                                      cudaMemcpyDeviceToHost, s))))
        return rc;
    if ((rc = RB_CUDA(cudaStreamSynchronize(s)))) return rc;
    return status;
}
