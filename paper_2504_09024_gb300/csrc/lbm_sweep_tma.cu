// Fused step with bulk-tensor (TMA) staging, FP32 populations: the step
// kernels (single run and batched), tensor maps and launchers.  The sweep of
// one tile is in lbm_sweep_tile.cuh.
#include <cstdio>
#include <type_traits>

#include <cudaTypedefs.h>

#include "lbm_sweep_tile.cuh"

namespace lbm {

template <int BX, bool COUPLED>
__global__ void __launch_bounds__(2 * BX, tma_min_blocks<BX>()) k_sweep_tma(const __grid_constant__ CUtensorMap tmap,
                                                  KParams p, float* __restrict__ dst,
                                                  const float* __restrict__ F, int seg,
                                                  int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    const TmaSmem<BX, COUPLED, ST_F32> S(smem_raw);
    if (threadIdx.x == 0) {
        for (int k = 0; k <= TMA_STAGES; ++k) mbar_init(&S.bars[k], 1);  // [TMA_STAGES]: test hook
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t issued = 0;
    sweep_tile<BX, COUPLED, ST_F32>(&tmap, p, dst, F, seg, blockIdx.x, blockIdx.y, S, issued, err);
}

// Batched step: every block walks the flat tile list with a stride of the
// grid size; runs may differ in size and parameters.
template <int BX, bool COUPLED>
__global__ void __launch_bounds__(2 * BX, tma_min_blocks<BX>()) k_sweep_tma_batch(const RunDesc* __restrict__ runs,
                                                        const int4* __restrict__ items, int nitems,
                                                        int parity, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    const TmaSmem<BX, COUPLED, ST_F32> S(smem_raw);
    if (threadIdx.x == 0) {
        for (int k = 0; k <= TMA_STAGES; ++k) mbar_init(&S.bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    // the run's parameters are read from shared memory, not held in registers
    __shared__ KParams sp;
    uint32_t issued = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        const RunDesc* rd = runs + w.x;
        {
            const int* srcw = reinterpret_cast<const int*>(&rd->p);
            int* dstw = reinterpret_cast<int*>(&sp);
            for (int k = threadIdx.x; k < (int)(sizeof(KParams) / sizeof(int)); k += blockDim.x)
                dstw[k] = srcw[k];
        }
        __syncthreads();
        const int src = parity ^ rd->flip;
        const bool ok = sweep_tile<BX, COUPLED, ST_F32>(&rd->tmap[src], sp, rd->pop[1 - src],
                                                rd->fields, rd->seg, w.y, w.z, S, issued, err);
        if (!ok) break;
        __syncthreads();  // the next tile reuses the shared rings and parameters
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

template <int BX, bool COUPLED>
void set_attr() {
    cudaFuncSetAttribute(k_sweep_tma<BX, COUPLED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TmaLayout<BX, COUPLED, ST_F32>::bytes);
}

}  // namespace

bool tma_available() { return encode_fn() != nullptr; }

// Tensor map over one population buffer: dims {pitch, ny, planes}, box
// {bx + 4, 1, planes}.
bool make_tensor_map(CUtensorMap* map, float* alloc, const KParams& p, int nplanes, int bx) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)p.pitch, (cuuint64_t)p.ny, (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)p.pitch * sizeof(float),
                             (cuuint64_t)p.plane * sizeof(float)};
    cuuint32_t box[3] = {(cuuint32_t)(bx + 4), 1u, (cuuint32_t)nplanes};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, alloc, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

// Calls f with the block width as a compile-time constant (64, 128 or 192).
template <typename F>
auto with_bx(int bx, F&& f) {
    if (bx == 192) return f(std::integral_constant<int, 192>{});
    if (bx == 64) return f(std::integral_constant<int, 64>{});
    return f(std::integral_constant<int, 128>{});
}

bool bx_supported(int bx) { return bx == 64 || bx == 128 || bx == 192; }

template <int BX, bool COUPLED>
void set_attr_batch() {
    cudaFuncSetAttribute(k_sweep_tma_batch<BX, COUPLED>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TmaLayout<BX, COUPLED, ST_F32>::bytes);
}

}  // namespace

size_t tma_smem_bytes(int bx, bool coupled) {
    if (!bx_supported(bx)) return 0;
    return with_bx(bx, [&](auto B) -> size_t {
        return coupled ? TmaLayout<B(), true, ST_F32>::bytes : TmaLayout<B(), false, ST_F32>::bytes;
    });
}

cudaError_t configure_tma_smem() {
    for (int bx : {64, 128, 192})
        with_bx(bx, [](auto B) {
            set_attr<B(), true>();
            set_attr<B(), false>();
            set_attr_batch<B(), true>();
            set_attr_batch<B(), false>();
            return 0;
        });
    return cudaGetLastError();
}

int tma_batch_blocks_per_sm(int bx, bool coupled) {
    int n = 0;
    const size_t smem = tma_smem_bytes(bx, coupled);
    const cudaError_t e = with_bx(bx, [&](auto B) {
        return coupled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma_batch<B(), true>, 2 * B(), smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma_batch<B(), false>, 2 * B(), smem);
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

int tma_blocks_per_sm(int bx, bool coupled) {
    int n = 0;
    const size_t smem = tma_smem_bytes(bx, coupled);
    const cudaError_t e = with_bx(bx, [&](auto B) {
        return coupled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma<B(), true>, 2 * B(), smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma<B(), false>, 2 * B(), smem);
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

void launch_step_tma_batch(const RunDesc* runs, const int4* items, int nitems, int blocks,
                           int bx, bool coupled, int src, int* err, cudaStream_t st) {
    const size_t smem = tma_smem_bytes(bx, coupled);
    with_bx(bx, [&](auto B) {
        if (coupled)
            k_sweep_tma_batch<B(), true><<<blocks, 2 * B(), smem, st>>>(runs, items, nitems, src, err);
        else
            k_sweep_tma_batch<B(), false><<<blocks, 2 * B(), smem, st>>>(runs, items, nitems, src, err);
        return 0;
    });
}

void launch_step_tma(const KParams& p, const DevState& s, int src, const FusedShape& sh,
                     const CUtensorMap* maps, int* err, cudaStream_t st) {
    const int tx = sh.bx - 4;
    dim3 grid((p.nx + tx - 1) / tx, (p.ny + sh.seg - 1) / sh.seg);
    const size_t smem = tma_smem_bytes(sh.bx, p.coupled);
    float* dst = s.pop[1 - src];
    with_bx(sh.bx, [&](auto B) {
        if (p.coupled)
            k_sweep_tma<B(), true><<<grid, 2 * B(), smem, st>>>(maps[src], p, dst, s.fields, sh.seg, err);
        else
            k_sweep_tma<B(), false><<<grid, 2 * B(), smem, st>>>(maps[src], p, dst, s.fields, sh.seg, err);
        return 0;
    });
}

}  // namespace lbm
