// Fused TMA step with 16-bit storage (FP16 or BF16 deviations, FP32
// collision arithmetic) and the conversions between the 16-bit state and the
// FP32 deviation-form state that initialisation and field output use.
//
// The word-plane layout is described in lbm_store16.cuh.  The per-cell
// arithmetic of the step is the FP32 step's (lbm_sweep2.cuh): only the pull
// (unpack, unscale) and the store (scale, round stochastically, pack)
// differ.  Whole-buffer packing (initialisation, set_populations) rounds to
// nearest.
#include <cudaTypedefs.h>
#include <type_traits>

#include "lbm_sweep2.cuh"

namespace lbm {

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

__global__ void k_step_advance_many(unsigned* const* ctrs, int nctr, unsigned n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nctr) *ctrs[k] += n;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// bulk-tensor sweep, 16-bit storage: shapes (128 or 192 columns, 1 or 2 cells
// per thread), shared memory, launch
// ---------------------------------------------------------------------------

namespace {

template <typename F>
auto with_shape16(int bx, int cpt, int st, int out, F&& f) {
    using std::integral_constant;
    auto go2 = [&](auto B, auto C, auto S) {
        return out == OUT_DIRECT ? f(B, C, S, integral_constant<int, OUT_DIRECT>{})
                                 : f(B, C, S, integral_constant<int, OUT_STAGED>{});
    };
    auto go = [&](auto B, auto C) {
        return st == ST_F16 ? go2(B, C, integral_constant<int, ST_F16>{})
                            : go2(B, C, integral_constant<int, ST_BF16>{});
    };
    if (cpt == 2)
        return bx == 192 ? go(integral_constant<int, 192>{}, integral_constant<int, 2>{})
                         : go(integral_constant<int, 128>{}, integral_constant<int, 2>{});
    return bx == 192 ? go(integral_constant<int, 192>{}, integral_constant<int, 1>{})
                     : go(integral_constant<int, 128>{}, integral_constant<int, 1>{});
}

}  // namespace

bool sweep2_16_shape_ok(int bx, int cpt) { return (bx == 128 || bx == 192) && (cpt == 1 || cpt == 2); }

size_t sweep2_16_smem_bytes(int bx, int cpt, int out, bool coupled) {
    if (!sweep2_16_shape_ok(bx, cpt)) return 0;
    // FP16 and BF16 words have the same layout
    return with_shape16(bx, cpt, ST_F16, out, [&](auto B, auto C, auto, auto O) -> size_t {
        return coupled ? SweepLayout<B(), C(), true, ST_F16, O()>::bytes
                       : SweepLayout<B(), C(), false, ST_F16, O()>::bytes;
    });
}

cudaError_t configure_sweep2_16_smem() {
    for (int bx : {128, 192})
        for (int cpt : {1, 2})
            for (int st : {ST_F16, ST_BF16})
                for (int out : {OUT_DIRECT, OUT_STAGED})
                    with_shape16(bx, cpt, st, out, [&](auto B, auto C, auto S, auto O) {
                        cudaFuncSetAttribute(k_sweep2<B(), C(), true, S(), O()>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SweepLayout<B(), C(), true, S(), O()>::bytes);
                        cudaFuncSetAttribute(k_sweep2<B(), C(), false, S(), O()>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SweepLayout<B(), C(), false, S(), O()>::bytes);
                        return 0;
                    });
    return cudaGetLastError();
}

int sweep2_16_blocks_per_sm(int bx, int cpt, int out, bool coupled, int st) {
    int n = 0;
    const size_t smem = sweep2_16_smem_bytes(bx, cpt, out, coupled);
    const cudaError_t e = with_shape16(bx, cpt, st, out, [&](auto B, auto C, auto S, auto O) {
        return coupled ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_sweep2<B(), C(), true, S(), O()>, 2 * B() / C(), smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_sweep2<B(), C(), false, S(), O()>, 2 * B() / C(), smem);
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

void launch_sweep2_16(const KParams& p, float* dst, const float* fields, const FusedShape& sh,
                      const CUtensorMap& load_map, const StoreMaps& store_maps, int st, int* err,
                      cudaStream_t s) {
    const int tx = sh.bx - 4;
    dim3 grid((p.nx + tx - 1) / tx, (p.ny + sh.seg - 1) / sh.seg);
    const size_t smem = sweep2_16_smem_bytes(sh.bx, sh.cpt, sh.out, p.coupled);
    with_shape16(sh.bx, sh.cpt, st, sh.out, [&](auto B, auto C, auto S, auto O) {
        if (p.coupled)
            k_sweep2<B(), C(), true, S(), O()><<<grid, 2 * B() / C(), smem, s>>>(
                load_map, store_maps, p, dst, fields, sh.seg, err);
        else
            k_sweep2<B(), C(), false, S(), O()><<<grid, 2 * B() / C(), smem, s>>>(
                load_map, store_maps, p, dst, fields, sh.seg, err);
        return 0;
    });
}

void launch_step_advance(unsigned* ctr, unsigned n, cudaStream_t s) {
    k_step_advance<<<1, 1, 0, s>>>(ctr, n);
}

void launch_step_advance_many(unsigned* const* ctrs, int nctr, unsigned n, cudaStream_t s) {
    if (nctr > 0) k_step_advance_many<<<(nctr + 127) / 128, 128, 0, s>>>(ctrs, nctr, n);
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
