// Field statistics for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// statistics: code running while another component owns the device memory
// budget (a memory pool with a hard cap, a framework that forbids allocations
// in its step loop), or code inside a region where an allocation would
// synchronise the device.  lbm_field_stats_noalloc gives them the FP64
// reductions of lbm_diagnostics without any allocation: the per-block partial
// sums live in the file-scope array below, which every GPU that loads this
// library holds until the process exits.
#include <cstring>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

// Partial sums of the two reduction passes: one row of DIAG_NSUM doubles per
// reduction block, at most LBM_NOALLOC_MAX_BLOCKS blocks (96 KiB in all).
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_BLOCKS;
static __device__ __align__(256) double g_stats_scratch[kMaxBlocks * lbm::DIAG_NSUM];

// Device address of g_stats_scratch per device ordinal, looked up once with
// that device current.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_stats_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_field_stats_noalloc(const double* phi, const double* c, const double* ux,
                                       const double* uy, int32_t nx, int32_t ny, int32_t walls_y,
                                       double beta, double c_max, double* result, void* stream) {
    if (!phi || !c || !ux || !uy || !result) return LBM_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || (walls_y != 0 && walls_y != 1) || !(c_max > 0.0))
        return LBM_ERR_INVALID_ARG;
    if ((int64_t)nx * (int64_t)ny > (int64_t)LBM_NOALLOC_MAX_CELLS) return LBM_ERR_INVALID_ARG;
    double* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    lbm::KParams p;
    std::memset(&p, 0, sizeof(p));
    p.nx = nx;
    p.ny = ny;
    p.walls = walls_y;
    p.beta = (float)beta;
    p.inv_cmax = (float)(1.0 / c_max);
    p.phi_a = 1.0f;  // the drop indicator of the shape moments: phases 1 and 0
    p.phi_b = 0.0f;
    const int nb = lbm::diag_blocks(p);
    if (nb > kMaxBlocks) return LBM_ERR_INVALID_ARG;
    lbm::launch_diag(p, phi, c, ux, uy, scratch, nb, result, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
