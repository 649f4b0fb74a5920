// 16-bit storage of the populations (FP16 or BF16 deviations, FP32 collision).
//
// Word-plane layout of one population buffer (32-bit words, pitched rows like
// the FP32 layout):
//   plane 0        S_f  phi's zeroth moment, fixed point (as in FP32 storage)
//   plane 1        S_h  c's zeroth moment, fixed point
//   planes 2..9    (d^f_q, d^h_q) for q = 1..8, one 16-bit pair per word
//   planes 10..14  (d^g_0, d^g_1), (d^g_2, d^g_3), ..., (d^g_8, 0)   coupled only
// where d^f_q = f~_q - w_q S_f and d^h_q likewise (the shift by the rest
// equilibrium), and d^g_q = g~_q - w_q P0 (the shift by the rest pressure),
// each multiplied by the lattice's power-of-two scale qs[l] before rounding
// (stochastically in the step, see pack2_sr).  f and h share a word per
// direction because their sources are the same neighbour: one shared-memory
// load feeds both pulls.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_device.cuh"

namespace lbm {

enum StoreKind { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

// word planes per cell: FP32 storage uses 9 float planes per lattice
__host__ __device__ constexpr int store_planes(int st, bool coupled) {
    return st == ST_F32 ? (coupled ? 27 : 18) : (coupled ? 15 : 10);
}

constexpr int P16_SH = 1;   // plane of S_h
constexpr int P16_FH = 2;   // first (d^f, d^h) plane (q = 1)
constexpr int P16_G = 10;   // first flow plane

template <int ST>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
    if constexpr (ST == ST_F16) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    } else {
        __nv_bfloat162 b;
        memcpy(&b, &w, 4);
        return __bfloat1622float2(b);
    }
}

// Round (a, b) to the 16-bit format (nearest, ties to even); a in the low half.
template <int ST>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    uint32_t w;
    if constexpr (ST == ST_F16) {
        const __half2 h = __floats2half2_rn(a, b);
        memcpy(&w, &h, 4);
    } else {
        const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        memcpy(&w, &v, 4);
    }
    return w;
}

// Stochastic rounding of the stored deviations.  Round-to-nearest makes the
// rounding error of a slowly varying deviation the same every step, and the
// zeroth moments integrate it; rounding up with probability equal to the
// dropped fraction makes it zero-mean.  The random bits come from the
// counter-based hash pcg_hash of (step, cell) (lbm_device.cuh), one hash per
// cell and warp group, spread over the words of the cell by word_bits.
// Random bits of word k of a cell from the cell's hash h: the product with a
// distinct odd constant per word is a bijection of the low bits (uniform if
// h is), which is all the rounding of one word needs.
__device__ __forceinline__ uint32_t word_bits(uint32_t h, int k) {
    return h * (0x9E3779B1u + 2u * (uint32_t)k * 0x632BE5ABu);
}

// (a, b) rounded stochastically to the 16-bit format, a in the low half:
// the sm_100-family conversion cvt.rs rounds away from zero with probability
// equal to the dropped fraction, drawing 16 random bits per value (the upper
// half of r for its first operand, which lands in the upper half of the word).
template <int ST>
__device__ __forceinline__ uint32_t pack2_sr(float a, float b, uint32_t r) {
    uint32_t w;
    if constexpr (ST == ST_BF16)
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(b), "f"(a), "r"(r));
    else
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(b), "f"(a), "r"(r));
    return w;
}

__device__ __forceinline__ uint32_t word_at(const float* p) { return __float_as_uint(*p); }

// Zeroth and first moments of f and h at one cell from staged 16-bit rows
// (same increments as pull_scalar_rows, for both scalar lattices at once).
// Rm, R0, Rp: plane 0 of rows j-1, j, j+1; PS: plane stride in words.
template <int ST>
__device__ __forceinline__ void pull_pair16(const float* __restrict__ Rm,
                                            const float* __restrict__ R0,
                                            const float* __restrict__ Rp, int PS, int cm, int c0,
                                            int cp, bool bot, bool top, const KParams& p,
                                            ScalarMoments& mf, ScalarMoments& mh) {
    const int Sf0 = __float_as_int(R0[c0]);
    const int Sh0 = __float_as_int(R0[P16_SH * PS + c0]);
    // The sums run on the scaled deviations and are unscaled once at the end
    // (the weights carry the scale instead): the scales are powers of two, so
    // moving them costs no accuracy, and it saves a multiply per value.
    float of[9], oh[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) {
        const float2 v = unpack2<ST>(word_at(R0 + (P16_FH - 1 + q) * PS + c0));
        of[q] = v.x;
        oh[q] = v.y;
    }
    const float wf1 = ((1.0f / 9.0f) * p.fx_inv[0]) * p.qs[0], wf5 = ((1.0f / 36.0f) * p.fx_inv[0]) * p.qs[0];
    const float wh1 = ((1.0f / 9.0f) * p.fx_inv[1]) * p.qs[1], wh5 = ((1.0f / 36.0f) * p.fx_inv[1]) * p.qs[1];
    float tf[9], th[9];
    auto pulled = [&](int q, const float* R, int col, bool diag) {
        const float2 v = unpack2<ST>(word_at(R + (P16_FH - 1 + q) * PS + col));
        tf[q] = (diag ? wf5 : wf1) * (float)(__float_as_int(R[col]) - Sf0) + v.x;
        th[q] = (diag ? wh5 : wh1) * (float)(__float_as_int(R[P16_SH * PS + col]) - Sh0) + v.y;
    };
    pulled(1, R0, cm, false);
    pulled(3, R0, cp, false);
    if (bot) {
        tf[2] = of[4]; th[2] = oh[4];
        tf[5] = of[7]; th[5] = oh[7];
        tf[6] = of[8]; th[6] = oh[8];
    } else {
        pulled(2, Rm, c0, false);
        pulled(5, Rm, cm, true);
        pulled(6, Rm, cp, true);
    }
    if (top) {
        tf[4] = of[2]; th[4] = oh[2];
        tf[7] = of[5]; th[7] = oh[5];
        tf[8] = of[6]; th[8] = oh[6];
    } else {
        pulled(4, Rp, c0, false);
        pulled(7, Rp, cp, true);
        pulled(8, Rp, cm, true);
    }
    auto moments = [](int S0, const float t[9], const float o[9], float qi, ScalarMoments& m) {
        m.s0 = S0;
        m.inc = ((((t[1] + t[3]) + (t[2] + t[4])) + ((t[5] + t[6]) + (t[7] + t[8]))) -
                 (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])))) * qi;
        m.jx = ((t[1] - t[3]) + (t[5] - t[6]) - (t[7] - t[8])) * qi;
        m.jy = ((t[2] - t[4]) + (t[5] + t[6]) - (t[7] + t[8])) * qi;
    };
    moments(Sf0, tf, of, p.qinv[0], mf);
    moments(Sh0, th, oh, p.qinv[1], mh);
}

// Post-streaming flow populations (shifted, unscaled) from staged 16-bit rows.
template <int ST>
__device__ __forceinline__ void pull9_16(const float* __restrict__ Rm,
                                         const float* __restrict__ R0,
                                         const float* __restrict__ Rp, int PS, int cm, int c0,
                                         int cp, bool bot, bool top, float qinv, float out[9]) {
    auto g_at = [&](const float* R, int q, int col) {
        const float2 v = unpack2<ST>(word_at(R + (P16_G + (q >> 1)) * PS + col));
        return ((q & 1) ? v.y : v.x) * qinv;
    };
    out[0] = g_at(R0, 0, c0);
    out[1] = g_at(R0, 1, cm);
    out[3] = g_at(R0, 3, cp);
    if (bot) {
        out[2] = g_at(R0, 4, c0);
        out[5] = g_at(R0, 7, c0);
        out[6] = g_at(R0, 8, c0);
    } else {
        out[2] = g_at(Rm, 2, c0);
        out[5] = g_at(Rm, 5, cm);
        out[6] = g_at(Rm, 6, cp);
    }
    if (top) {
        out[4] = g_at(R0, 2, c0);
        out[7] = g_at(R0, 5, c0);
        out[8] = g_at(R0, 6, c0);
    } else {
        out[4] = g_at(Rp, 4, c0);
        out[7] = g_at(Rp, 7, cp);
        out[8] = g_at(Rp, 8, cm);
    }
}

// Store n words of one cell (planes plane0 .. plane0+n-1) and their periodic
// ghost copies (gs: column offsets of the copies, 0 for none).
template <int N>
__device__ __forceinline__ void store_words(float* __restrict__ base, int64_t plane, int64_t idx,
                                            const int gs[2], int plane0, const uint32_t w[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k) base[(plane0 + k) * plane + idx] = __uint_as_float(w[k]);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        if (!gs[g]) continue;
#pragma unroll
        for (int k = 0; k < N; ++k) base[(plane0 + k) * plane + idx + gs[g]] = __uint_as_float(w[k]);
    }
}

}  // namespace lbm
