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
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

// Partial sums of the two reduction passes: one row of DIAG_NSUM doubles per
// reduction block, at most LBM_NOALLOC_MAX_BLOCKS blocks (96 KiB in all).
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_BLOCKS;
static __device__ __align__(256) double g_stats_scratch[kMaxBlocks * lbm::DIAG_NSUM];

// Device address of g_stats_scratch per CUDA context.  A context has its own
// copy of the module, and a context that is destroyed and created again
// (cudaDeviceReset, a context made by another component) gets a new ID, so
// the cache is keyed by context ID: an address is never used outside the
// context it was looked up in.  Without the driver's context calls the
// address is looked up on every call.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
constexpr int kCacheEntries = 64;
struct ScratchEntry {
    unsigned long long ctx_id;
    double* addr;
};
ScratchEntry g_cache[kCacheEntries];
int g_cache_used = 0, g_cache_next = 0;
std::mutex g_scratch_mutex;

template <class F>
F driver_fn(const char* name) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &ptr, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return reinterpret_cast<F>(ptr);
}

int lookup_scratch(double** out) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_stats_scratch);
    if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    *out = static_cast<double*>(ptr);
    return LBM_OK;
}

int scratch_for_current_context(double** out) {
    // the context the runtime launches into is the thread's current one; a
    // thread with none yet gets the device's primary context from the lookup
    static const CtxGetCurrentFn get_ctx = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_ctx || !get_id || get_ctx(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return lookup_scratch(out);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    for (int k = 0; k < g_cache_used; ++k)
        if (g_cache[k].ctx_id == id) {
            *out = g_cache[k].addr;
            return LBM_OK;
        }
    double* addr = nullptr;
    const int rc = lookup_scratch(&addr);
    if (rc != LBM_OK) return rc;
    ScratchEntry& en = g_cache[g_cache_used < kCacheEntries ? g_cache_used++ : g_cache_next];
    if (g_cache_used == kCacheEntries) g_cache_next = (g_cache_next + 1) % kCacheEntries;
    en = ScratchEntry{id, addr};
    *out = addr;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_field_stats_noalloc(const double* phi, const double* c, const double* ux,
                                       const double* uy, int32_t nx, int32_t ny, int32_t walls_y,
                                       double beta, double c_max, double phi_a, double phi_b,
                                       double* result, void* stream) {
    if (!phi || !c || !ux || !uy || !result) return LBM_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || (walls_y != 0 && walls_y != 1) || !(c_max > 0.0))
        return LBM_ERR_INVALID_ARG;
    if (!std::isfinite(phi_a) || !std::isfinite(phi_b) || (float)phi_a == (float)phi_b)
        return LBM_ERR_INVALID_ARG;
    if ((int64_t)nx * (int64_t)ny > (int64_t)LBM_NOALLOC_MAX_CELLS) return LBM_ERR_INVALID_ARG;
    double* scratch = nullptr;
    const int rc = scratch_for_current_context(&scratch);
    if (rc != LBM_OK) return rc;
    lbm::KParams p;
    std::memset(&p, 0, sizeof(p));
    p.nx = nx;
    p.ny = ny;
    p.walls = walls_y;
    p.beta = (float)beta;
    p.inv_cmax = (float)(1.0 / c_max);
    p.phi_a = (float)phi_a;  // the drop indicator of the shape moments
    p.phi_b = (float)phi_b;
    const int nb = lbm::diag_blocks(p);
    if (nb > kMaxBlocks) return LBM_ERR_INVALID_ARG;
    lbm::launch_diag(p, phi, c, ux, uy, scratch, nb, result, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
