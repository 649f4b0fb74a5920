// Fused TMA step with 16-bit storage (FP16 or BF16 deviations, FP32
// collision arithmetic) and the conversions between the 16-bit state and the
// FP32 deviation-form state that initialisation and field output use.
//
// The word-plane layout is described in lbm_store16.cuh.  The per-cell
// arithmetic of the step is the FP32 step's (lbm_sweep_tile.cuh): only the
// pull (unpack, unscale) and the store (scale, round stochastically, pack)
// differ.  Whole-buffer packing (initialisation, set_populations) rounds to
// nearest.
#include <cudaTypedefs.h>
#include <type_traits>

#include "lbm_sweep_tile.cuh"

namespace lbm {

template <int BX, bool COUPLED, int ST>
__global__ void __launch_bounds__(2 * BX, tma_min_blocks<BX>()) k_sweep_tma16(
    const __grid_constant__ CUtensorMap tmap, KParams p, float* __restrict__ dst,
    const float* __restrict__ F, int seg, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    const TmaSmem<BX, COUPLED, ST> S(smem_raw);
    if (threadIdx.x == 0) {
        for (int k = 0; k <= TMA_STAGES; ++k) mbar_init(&S.bars[k], 1);  // [TMA_STAGES]: test hook
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t issued = 0;
    sweep_tile<BX, COUPLED, ST>(&tmap, p, dst, F, seg, blockIdx.x, blockIdx.y, S, issued, err);
}

// FP32 deviation-form buffer (27 or 18 float planes) -> 16-bit words (15 or
// 10 planes), element by element over whole planes (ghost columns included).
template <int ST>
__global__ void k_pack16(const float* __restrict__ src, float* __restrict__ dst, int64_t plane,
                         int coupled, float qs0, float qs1, float qs2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= plane) return;
    dst[e] = src[e];                              // S_f
    dst[P16_SH * plane + e] = src[9 * plane + e];  // S_h
#pragma unroll
    for (int q = 1; q < 9; ++q)
        dst[(P16_FH - 1 + q) * plane + e] =
            __uint_as_float(pack2<ST>(src[q * plane + e] * qs0, src[(9 + q) * plane + e] * qs1));
    if (coupled) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float a = src[(18 + 2 * k) * plane + e] * qs2;
            const float b = 2 * k + 1 < 9 ? src[(19 + 2 * k) * plane + e] * qs2 : 0.0f;
            dst[(P16_G + k) * plane + e] = __uint_as_float(pack2<ST>(a, b));
        }
    }
}

// 16-bit words -> FP32 deviation-form buffer (exact: every 16-bit value and
// every power-of-two unscaling is representable in FP32).
template <int ST>
__global__ void k_unpack16(const float* __restrict__ src, float* __restrict__ dst, int64_t plane,
                           int coupled, float qi0, float qi1, float qi2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= plane) return;
    dst[e] = src[e];
    dst[9 * plane + e] = src[P16_SH * plane + e];
#pragma unroll
    for (int q = 1; q < 9; ++q) {
        const float2 v = unpack2<ST>(__float_as_uint(src[(P16_FH - 1 + q) * plane + e]));
        dst[q * plane + e] = v.x * qi0;
        dst[(9 + q) * plane + e] = v.y * qi1;
    }
    if (coupled) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float2 v = unpack2<ST>(__float_as_uint(src[(P16_G + k) * plane + e]));
            dst[(18 + 2 * k) * plane + e] = v.x * qi2;
            if (2 * k + 1 < 9) dst[(19 + 2 * k) * plane + e] = v.y * qi2;
        }
    }
}

__global__ void k_step_advance(unsigned* ctr, unsigned n) { *ctr += n; }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

// Calls f with the block width (128 or 192) and the storage format as
// compile-time constants.
template <typename F>
auto with_bx_st(int bx, int st, F&& f) {
    if (bx == 192)
        return st == ST_F16 ? f(std::integral_constant<int, 192>{}, std::integral_constant<int, ST_F16>{})
                            : f(std::integral_constant<int, 192>{}, std::integral_constant<int, ST_BF16>{});
    return st == ST_F16 ? f(std::integral_constant<int, 128>{}, std::integral_constant<int, ST_F16>{})
                        : f(std::integral_constant<int, 128>{}, std::integral_constant<int, ST_BF16>{});
}

}  // namespace

size_t tma16_smem_bytes(int bx, bool coupled) {
    if (bx != 128 && bx != 192) return 0;
    // FP16 and BF16 words have the same layout
    return with_bx_st(bx, ST_F16, [&](auto B, auto) -> size_t {
        return coupled ? TmaLayout<B(), true, ST_F16>::bytes : TmaLayout<B(), false, ST_F16>::bytes;
    });
}

cudaError_t configure_tma16_smem() {
    for (int bx : {128, 192})
        for (int st : {ST_F16, ST_BF16})
            with_bx_st(bx, st, [&](auto B, auto S) {
                cudaFuncSetAttribute(k_sweep_tma16<B(), true, S()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tma16_smem_bytes(B(), true));
                cudaFuncSetAttribute(k_sweep_tma16<B(), false, S()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tma16_smem_bytes(B(), false));
                return 0;
            });
    return cudaGetLastError();
}

int tma16_blocks_per_sm(int bx, bool coupled, int st) {
    int n = 0;
    const size_t smem = tma16_smem_bytes(bx, coupled);
    const cudaError_t e = with_bx_st(bx, st, [&](auto B, auto S) {
        return coupled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma16<B(), true, S()>, 2 * B(), smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma16<B(), false, S()>, 2 * B(), smem);
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

void launch_step_tma16(const KParams& p, float* src16, float* dst16, const float* fields,
                       const FusedShape& sh, const CUtensorMap& map, int st, int* err,
                       cudaStream_t s) {
    const int tx = sh.bx - 4;
    dim3 grid((p.nx + tx - 1) / tx, (p.ny + sh.seg - 1) / sh.seg);
    const size_t smem = tma16_smem_bytes(sh.bx, p.coupled);
    (void)src16;
    with_bx_st(sh.bx, st, [&](auto B, auto S) {
        if (p.coupled)
            k_sweep_tma16<B(), true, S()><<<grid, 2 * B(), smem, s>>>(map, p, dst16, fields, sh.seg, err);
        else
            k_sweep_tma16<B(), false, S()><<<grid, 2 * B(), smem, s>>>(map, p, dst16, fields, sh.seg, err);
        return 0;
    });
}

void launch_step_advance(unsigned* ctr, unsigned n, cudaStream_t s) {
    k_step_advance<<<1, 1, 0, s>>>(ctr, n);
}

void launch_pack16(const KParams& p, const float* src32_alloc, float* dst16_alloc, int st,
                   cudaStream_t s) {
    const int64_t n = p.plane;
    const int blocks = (int)((n + 255) / 256);
    if (st == ST_F16)
        k_pack16<ST_F16><<<blocks, 256, 0, s>>>(src32_alloc, dst16_alloc, n, p.coupled, p.qs[0],
                                                p.qs[1], p.qs[2]);
    else
        k_pack16<ST_BF16><<<blocks, 256, 0, s>>>(src32_alloc, dst16_alloc, n, p.coupled, p.qs[0],
                                                 p.qs[1], p.qs[2]);
}

void launch_unpack16(const KParams& p, const float* src16_alloc, float* dst32_alloc, int st,
                     cudaStream_t s) {
    const int64_t n = p.plane;
    const int blocks = (int)((n + 255) / 256);
    if (st == ST_F16)
        k_unpack16<ST_F16><<<blocks, 256, 0, s>>>(src16_alloc, dst32_alloc, n, p.coupled,
                                                  p.qinv[0], p.qinv[1], p.qinv[2]);
    else
        k_unpack16<ST_BF16><<<blocks, 256, 0, s>>>(src16_alloc, dst32_alloc, n, p.coupled,
                                                   p.qinv[0], p.qinv[1], p.qinv[2]);
}

}  // namespace lbm
