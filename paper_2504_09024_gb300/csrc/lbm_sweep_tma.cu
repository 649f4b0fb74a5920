// Fused step with bulk-tensor (TMA) loads and stores, FP32 populations: the
// step kernels (single run, and the persistent kernel over the tiles of a
// batch of runs), tensor maps and launchers.  The sweep of one tile is in
// lbm_sweep2.cuh.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>

#include <cudaTypedefs.h>

#include "lbm_sweep2.cuh"

namespace lbm {

// Run parameters of the persistent batch kernel (the batch parameter bank).
__constant__ KParams c_batch_params[BATCH_PARAM_SLOTS];

// One time step of every run of a batch in one launch: each block walks the
// tiles of the table with a stride of the grid size.  Runs may differ in size
// and parameters; the entry of a tile is found by bisection over the table's
// first tiles.  A run's parameters come from the parameter bank, the
// addresses of its buffers and tensor maps from the table (a kernel
// parameter); the maps themselves are in global memory.
// Register budget of the persistent batch kernel.  A run's parameters come
// from the bank by an index known only at run time, so the compiler holds
// them in registers where the single-run kernel takes them as constant
// operands: the one-cell form needs 130-160 registers a thread instead of 80
// (held to 80 it spilled 200-300 bytes a thread and ran 1.6 times slower).
template <int BX, int CPT, bool COUPLED, int OUT>
constexpr int batch_min_blocks() {
    constexpr int threads = 2 * BX / CPT;
    constexpr int regs = CPT == 1 ? 128 : 168;
    constexpr int by_regs = 65536 / (regs * threads);
    return by_regs < 1 ? 1 : by_regs;
}

template <int BX, int CPT, bool COUPLED, int OUT>
__global__ void __launch_bounds__(2 * BX / CPT, (batch_min_blocks<BX, CPT, COUPLED, OUT>()))
    k_sweep2_batch(const __grid_constant__ BatchTable tab, int parity, int step_off,
                   int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the bulk-tensor copies need the carve-up on 128-byte boundaries
    if (smem_u32(smem_raw) & 127u) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    const SweepSmem<BX, CPT, COUPLED, ST_F32, OUT> S(smem_raw);
    if (threadIdx.x == 0) {
        // [STAGES]: the failure-path test hook
        for (int k = 0; k <= sw_stages(ST_F32, OUT); ++k) mbar_init(&S.bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t issued = 0;
    for (int it = blockIdx.x; it < tab.ntiles; it += gridDim.x) {
        int lo = 0, hi = tab.nentries;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tab.e[mid].first <= it) lo = mid;
            else hi = mid;
        }
        const BatchEntry& en = tab.e[lo];
        const KParams& p = c_batch_params[tab.slot0 + lo];
        const int local = it - en.first;
        const int sy = local / en.nsx, sx = local - sy * en.nsx;
        const int src = parity ^ en.flip;
        const bool ok = sweep_tile2<BX, CPT, COUPLED, ST_F32, OUT>(
            en.tmap[src], en.smap[1 - src], p, en.pop[1 - src], en.fields, en.seg, sx, sy, S,
            step_seed_at(p, step_off), issued, err);
        if (!ok) break;
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

// ---------------------------------------------------------------------------
// bulk-tensor sweep, FP32 storage: shapes, shared memory, launch
// ---------------------------------------------------------------------------

namespace {

// Calls f with (block width, cells per thread, store mode) as compile-time
// constants for the FP32 shapes: (64, 1), (128, 1), (192, 1), (128, 2),
// (192, 2), each with direct or staged stores.
template <typename F>
auto with_shape_f32(int bx, int cpt, int out, F&& f) {
    using std::integral_constant;
    auto go = [&](auto B, auto C) {
        return out == OUT_STAGED ? f(B, C, integral_constant<int, OUT_STAGED>{})
                                 : f(B, C, integral_constant<int, OUT_DIRECT>{});
    };
    if (cpt == 2)
        return bx == 192 ? go(integral_constant<int, 192>{}, integral_constant<int, 2>{})
                         : go(integral_constant<int, 128>{}, integral_constant<int, 2>{});
    if (bx == 192) return go(integral_constant<int, 192>{}, integral_constant<int, 1>{});
    if (bx == 64) return go(integral_constant<int, 64>{}, integral_constant<int, 1>{});
    return go(integral_constant<int, 128>{}, integral_constant<int, 1>{});
}

}  // namespace

bool sweep2_f32_shape_ok(int bx, int cpt) {
    return (cpt == 1 && (bx == 64 || bx == 128 || bx == 192)) ||
           (cpt == 2 && (bx == 128 || bx == 192));
}

size_t sweep2_f32_smem_bytes(int bx, int cpt, int out, bool coupled) {
    if (!sweep2_f32_shape_ok(bx, cpt)) return 0;
    return with_shape_f32(bx, cpt, out, [&](auto B, auto C, auto O) -> size_t {
        return coupled ? SweepLayout<B(), C(), true, ST_F32, O()>::bytes
                       : SweepLayout<B(), C(), false, ST_F32, O()>::bytes;
    });
}

cudaError_t configure_sweep2_f32_smem() {
    const int shapes[5][2] = {{64, 1}, {128, 1}, {192, 1}, {128, 2}, {192, 2}};
    for (const auto& sh : shapes)
        for (int out : {OUT_DIRECT, OUT_STAGED})
            with_shape_f32(sh[0], sh[1], out, [](auto B, auto C, auto O) {
                const int bt = (int)SweepLayout<B(), C(), true, ST_F32, O()>::bytes;
                const int bf = (int)SweepLayout<B(), C(), false, ST_F32, O()>::bytes;
                cudaFuncSetAttribute(k_sweep2<B(), C(), true, ST_F32, O()>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bt);
                cudaFuncSetAttribute(k_sweep2<B(), C(), false, ST_F32, O()>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bf);
                cudaFuncSetAttribute(k_sweep2_batch<B(), C(), true, O()>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bt);
                cudaFuncSetAttribute(k_sweep2_batch<B(), C(), false, O()>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bf);
                return 0;
            });
    return cudaGetLastError();
}

int sweep2_f32_blocks_per_sm(int bx, int cpt, int out, bool coupled) {
    int n = 0;
    const size_t smem = sweep2_f32_smem_bytes(bx, cpt, out, coupled);
    const cudaError_t e = with_shape_f32(bx, cpt, out, [&](auto B, auto C, auto O) {
        return coupled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_sweep2<B(), C(), true, ST_F32, O()>, 2 * B() / C(), smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_sweep2<B(), C(), false, ST_F32, O()>, 2 * B() / C(), smem);
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

void launch_sweep2_f32(const KParams& p, float* dst, const float* fields, const FusedShape& sh,
                       const CUtensorMap& load_map, const StoreMaps& store_maps, int* err,
                       cudaStream_t s) {
    const int tx = sh.bx - 4;
    dim3 grid((p.nx + tx - 1) / tx, (p.ny + sh.seg - 1) / sh.seg);
    const size_t smem = sweep2_f32_smem_bytes(sh.bx, sh.cpt, sh.out, p.coupled);
    with_shape_f32(sh.bx, sh.cpt, sh.out, [&](auto B, auto C, auto O) {
        if (p.coupled)
            k_sweep2<B(), C(), true, ST_F32, O()><<<grid, 2 * B() / C(), smem, s>>>(
                load_map, store_maps, p, dst, fields, sh.seg, err);
        else
            k_sweep2<B(), C(), false, ST_F32, O()><<<grid, 2 * B() / C(), smem, s>>>(
                load_map, store_maps, p, dst, fields, sh.seg, err);
        return 0;
    });
}

int sweep2_batch_blocks_per_sm(int bx, int cpt, int out, bool coupled) {
    int n = 0;
    const size_t smem = sweep2_f32_smem_bytes(bx, cpt, out, coupled);
    const cudaError_t e = with_shape_f32(bx, cpt, out, [&](auto B, auto C, auto O) {
        return coupled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_sweep2_batch<B(), C(), true, O()>, 2 * B() / C(), smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_sweep2_batch<B(), C(), false, O()>, 2 * B() / C(), smem);
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

void launch_sweep2_batch(const BatchTable& tab, int blocks, const FusedShape& sh, bool coupled,
                         int parity, int step_off, int* err, cudaStream_t st) {
    const size_t smem = sweep2_f32_smem_bytes(sh.bx, sh.cpt, sh.out, coupled);
    with_shape_f32(sh.bx, sh.cpt, sh.out, [&](auto B, auto C, auto O) {
        if (coupled)
            k_sweep2_batch<B(), C(), true, O()><<<blocks, 2 * B() / C(), smem, st>>>(
                tab, parity, step_off, err);
        else
            k_sweep2_batch<B(), C(), false, O()><<<blocks, 2 * B() / C(), smem, st>>>(
                tab, parity, step_off, err);
        return 0;
    });
}

// Parameter-bank slots in use, per device (host bookkeeping).
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_slot_mu;
unsigned char g_slot_used[kMaxDevices][BATCH_PARAM_SLOTS];
}  // namespace

int batch_params_alloc(int dev, int n) {
    if (dev < 0 || dev >= kMaxDevices || n < 1 || n > BATCH_PARAM_SLOTS) return -1;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int a = 0; a + n <= BATCH_PARAM_SLOTS; ++a) {
        int k = 0;
        while (k < n && !g_slot_used[dev][a + k]) ++k;
        if (k == n) {
            std::memset(&g_slot_used[dev][a], 1, (size_t)n);
            return a;
        }
        a += k;  // skip past the used slot
    }
    return -1;
}

void batch_params_free(int dev, int first, int n) {
    if (first < 0 || dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    std::memset(&g_slot_used[dev][first], 0, (size_t)n);
}

cudaError_t batch_params_upload(int first, const KParams* kp, int n, cudaStream_t st) {
    return cudaMemcpyToSymbolAsync(c_batch_params, kp, sizeof(KParams) * (size_t)n,
                                   sizeof(KParams) * (size_t)first, cudaMemcpyHostToDevice, st);
}

// Store maps over one buffer: dims {4 + nx rounded down to a multiple of 4
// (columns -4 .. that end), ny, planes}, boxes {bx - 4, 1, scalar planes} and
// {bx - 4, 1, flow planes}.  The column extent ends on a 16-byte boundary: a
// store box clipped elsewhere was seen to write past the extent (into the
// ghost columns), so the sweep stores the last nx mod 4 columns directly.
bool make_store_maps(StoreMaps* m, float* alloc, const KParams& p, int st, int bx) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const int nplanes = store_planes(st, p.coupled);
    const int ns = st == ST_F32 ? 18 : 10;
    const int nf = nplanes - ns;
    cuuint64_t dims[3] = {(cuuint64_t)(XGHOST + (p.nx & ~3)), (cuuint64_t)p.ny,
                          (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)p.pitch * sizeof(float),
                             (cuuint64_t)p.plane * sizeof(float)};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    auto encode = [&](CUtensorMap* map, int planes) {
        cuuint32_t box[3] = {(cuuint32_t)(bx - 4), 1u, (cuuint32_t)planes};
        return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, alloc, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
               CUDA_SUCCESS;
    };
    std::memset(m, 0, sizeof(StoreMaps));
    if (!encode(&m->s, ns)) return false;
    return nf == 0 || encode(&m->f, nf);
}

bool sweep2_shape_ok(int bx, int cpt, int st) {
    return st == ST_F32 ? sweep2_f32_shape_ok(bx, cpt) : sweep2_16_shape_ok(bx, cpt);
}

size_t sweep2_smem_bytes(int bx, int cpt, int out, bool coupled, int st) {
    return st == ST_F32 ? sweep2_f32_smem_bytes(bx, cpt, out, coupled)
                        : sweep2_16_smem_bytes(bx, cpt, out, coupled);
}

int sweep2_blocks_per_sm(int bx, int cpt, int out, bool coupled, int st) {
    return st == ST_F32 ? sweep2_f32_blocks_per_sm(bx, cpt, out, coupled)
                        : sweep2_16_blocks_per_sm(bx, cpt, out, coupled, st);
}

cudaError_t configure_sweep2_smem() {
    cudaError_t e = configure_sweep2_f32_smem();
    if (e != cudaSuccess) return e;
    return configure_sweep2_16_smem();
}

void launch_step_sweep2(const KParams& p, float* dst, const float* fields, const FusedShape& sh,
                        const CUtensorMap& load_map, const StoreMaps& store_maps, int st,
                        int* err, cudaStream_t s) {
    if (st == ST_F32)
        launch_sweep2_f32(p, dst, fields, sh, load_map, store_maps, err, s);
    else
        launch_sweep2_16(p, dst, fields, sh, load_map, store_maps, st, err, s);
}

}  // namespace lbm
