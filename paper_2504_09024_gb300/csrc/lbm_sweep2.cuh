// The row sweep of one tile of the fused bulk-tensor step, for every storage
// format (FP32 populations, FP16/BF16 deviations) and one or two cells per
// thread.
//
// A block owns a strip of columns and walks down a segment of rows, forming
// phi, c, sigma, P* one row ahead in shared-memory rings, the unit normal one
// row behind and colliding two (flow) and three (scalars) rows behind.  Raw
// rows arrive by one 3-D bulk-tensor load per row ({columns, 1 row, all
// planes}) issued by one thread into a ring of SW_STAGES rows, completing on
// an mbarrier; collided rows leave the same way: each warp group writes its
// row into a shared-memory staging area and one of its threads issues a
// bulk-tensor store of it.  Every population byte leaves HBM once per strip
// and is written once.  Periodic x needs no wrap logic: the boxes include the
// ghost columns that the writers maintain (the staged stores cover the own
// columns up to the last multiple of 4; the threads owning the columns beyond
// it and the four edge columns store those and the ghost copies directly).  Walls: rows beyond a wall are never loaded; their ring entries are
// mirror copies of rows already formed (row -1-k is row k, row ny+k is row
// ny-1-k).
//
// CPT = cells per thread: with CPT = 2 a thread owns two horizontally
// adjacent cells and computes both with the packed FP32 instructions of
// lbm_vec.cuh; block widths and CPT are chosen by the launch-shape autotuner.
#pragma once

#include <type_traits>

#include "lbm_cell.cuh"
#include "lbm_store16.cuh"
#include "lbm_tma.cuh"

namespace lbm {

// Collided rows leave either by direct stores from registers (OUT_DIRECT) or
// through a shared-memory staging area and one bulk-tensor store per row and
// warp group (OUT_STAGED).  The staging area costs shared memory that the
// ring of staged raw rows would otherwise use, so the ring is shorter there;
// the 16-bit rows are smaller, so their rings are longer.
// Staged raw rows in the ring: the three a row's pull reads, plus rows in
// flight ahead of them.
__host__ __device__ constexpr int sw_stages(int st, int out) {
    return out == OUT_DIRECT ? (st == 0 ? 4 : 6) : (st == 0 ? 3 : 5);
}
constexpr int SW_RING = 5;    // rows of phi, c, sigma, P* kept (and mirror copies)
constexpr int SW_NRING = 3;   // rows of n, |grad phi|
constexpr int SW_PAD = 2;     // ring rows carry two spare columns each side

// Ring slots: a mod M for any a; slot s advanced by m < M.
template <int M>
__device__ __forceinline__ int rmodm(int a) { return ((a % M) + M) % M; }
__device__ __forceinline__ int rmodm_rt(int a, int m) { return ((a % m) + m) % m; }
__device__ __forceinline__ int rmod5(int a) { return rmodm<SW_RING>(a); }
__device__ __forceinline__ int rmod3(int a) { return rmodm<SW_NRING>(a); }
__device__ __forceinline__ int ring_slot5(int s, int m) { return s + m >= SW_RING ? s + m - SW_RING : s + m; }
__device__ __forceinline__ int ring_slot3(int s, int m) { return s + m >= SW_NRING ? s + m - SW_NRING : s + m; }

// Cell type of CPT cells per thread.
template <int CPT> struct CellType;
template <> struct CellType<1> { using V = float; using VI = int; };
template <> struct CellType<2> { using V = f2; using VI = i2; };

template <int BX, int CPT, bool COUPLED, int ST, int OUT>
struct SweepLayout {
    static constexpr int STAGES = sw_stages(ST, OUT);
    static constexpr int NT = BX / CPT;                   // threads per warp group
    static constexpr int NL = store_planes(ST, COUPLED);  // word planes per staged row
    static constexpr int W = BX + 4;                      // staged columns x0-4 .. x0+BX-1
    static constexpr int SLOT = (NL * W + 31) / 32 * 32;  // floats per staged row (128-B multiple)
    static constexpr int TX = BX - 4;                     // own columns of a tile
    static constexpr int RW = BX + 2 * SW_PAD;            // floats per ring row
    static constexpr int NS = ST == ST_F32 ? 18 : 10;     // scalar-lattice word planes
    static constexpr int NF = COUPLED ? (ST == ST_F32 ? 9 : 5) : 0;  // flow-lattice word planes
    // staging of one scalar row and one flow row (staged stores only)
    static constexpr int OUT_S = OUT == OUT_STAGED ? (NS * TX + 31) / 32 * 32 : 0;
    static constexpr int OUT_F = OUT == OUT_STAGED ? (NF * TX + 31) / 32 * 32 : 0;
    static constexpr size_t floats = (size_t)STAGES * SLOT + OUT_S + OUT_F +
                                     (size_t)(4 * SW_RING + 3 * SW_NRING + 2 * 2) * RW;
    static constexpr size_t bytes = 128 /* barriers */ + sizeof(float) * floats;
    static_assert(BX % (32 * CPT) == 0, "whole warps per group");
    static_assert((TX * 4) % 16 == 0, "bulk-tensor boxes need 16-byte rows");
};

// Shared-memory carve-up of one block (barriers, staged rows, output
// staging, then the rings).
template <int BX, int CPT, bool COUPLED, int ST, int OUT>
struct SweepSmem {
    uint64_t* bars;
    float* raw;
    float *out_s, *out_f;
    int* s_phi;
    float *s_c, *s_sig, *s_dps, *s_nx, *s_ny, *s_gm, *s_ux, *s_uy;
    // smem_raw: the block's dynamic shared memory, declared 128-byte aligned.
    // The carve-up is pointer arithmetic on it (no round trip through an
    // integer), so the compiler keeps every access a shared-memory one.
    __device__ explicit SweepSmem(unsigned char* smem_raw) {
        using L = SweepLayout<BX, CPT, COUPLED, ST, OUT>;
        bars = reinterpret_cast<uint64_t*>(smem_raw);
        raw = reinterpret_cast<float*>(smem_raw + 128);
        out_s = raw + L::STAGES * L::SLOT;
        out_f = out_s + L::OUT_S;
        float* ring = out_f + L::OUT_F;
        // ring row s of an array starts at s * RW; column w of the window at + SW_PAD + w
        s_phi = reinterpret_cast<int*>(ring) + SW_PAD;  // [SW_RING][RW], fixed point
        s_c = ring + SW_RING * L::RW + SW_PAD;
        s_sig = s_c + SW_RING * L::RW;
        s_dps = s_sig + SW_RING * L::RW;
        s_nx = s_dps + SW_RING * L::RW;  // [SW_NRING][RW]
        s_ny = s_nx + SW_NRING * L::RW;
        s_gm = s_ny + SW_NRING * L::RW;
        s_ux = s_gm + SW_NRING * L::RW;  // [2][RW] velocity of the last flow-collided rows
        s_uy = s_ux + 2 * L::RW;
    }
};

// ---------------------------------------------------------------------------
// loads of CPT adjacent cells
// ---------------------------------------------------------------------------

// Values at columns c + DX .. c + DX + CPT - 1 of a row (c even for CPT = 2,
// the row 8-byte aligned): one 64-bit load when aligned, else two.
template <int CPT, int DX>
__device__ __forceinline__ typename CellType<CPT>::V ldv(const float* row, int c) {
    if constexpr (CPT == 1) {
        return row[c + DX];
    } else if constexpr ((DX & 1) == 0) {
        const float2 v = *reinterpret_cast<const float2*>(row + c + DX);
        return f2(v.x, v.y);
    } else {
        return f2(row[c + DX], row[c + DX + 1]);
    }
}
template <int CPT, int DX>
__device__ __forceinline__ typename CellType<CPT>::VI ldi(const float* row, int c) {
    if constexpr (CPT == 1) {
        return __float_as_int(row[c + DX]);
    } else if constexpr ((DX & 1) == 0) {
        const int2 v = *reinterpret_cast<const int2*>(row + c + DX);
        return i2{v.x, v.y};
    } else {
        return i2{__float_as_int(row[c + DX]), __float_as_int(row[c + DX + 1])};
    }
}
template <int CPT>
__device__ __forceinline__ void stv(float* row, int c, typename CellType<CPT>::V v) {
    if constexpr (CPT == 1) row[c] = v;
    else *reinterpret_cast<float2*>(row + c) = make_float2(v.x, v.y);
}
template <int CPT>
__device__ __forceinline__ void sti(int* row, int c, typename CellType<CPT>::VI v) {
    if constexpr (CPT == 1) row[c] = v;
    else *reinterpret_cast<int2*>(row + c) = make_int2(v.x, v.y);
}
template <int CPT>
__device__ __forceinline__ void stw(float* row, int c, const uint32_t* w) {
    if constexpr (CPT == 1) row[c] = __uint_as_float(w[0]);
    else *reinterpret_cast<uint2*>(row + c) = make_uint2(w[0], w[1]);
}

// The three stencil values (columns w-1, w, w+1) of each of the CPT cells
// starting at window column w0 of a ring row.
template <int CPT>
__device__ __forceinline__ void stencil3(const float* row, int w0, typename CellType<CPT>::V v[3]) {
    if constexpr (CPT == 1) {
        v[0] = row[w0 - 1];
        v[1] = row[w0];
        v[2] = row[w0 + 1];
    } else {
        const float2 a = *reinterpret_cast<const float2*>(row + w0 - 2);
        const float2 b = *reinterpret_cast<const float2*>(row + w0);
        const float2 c = *reinterpret_cast<const float2*>(row + w0 + 2);
        v[0] = f2(a.y, b.x);
        v[1] = f2(b.x, b.y);
        v[2] = f2(b.y, c.x);
    }
}
template <int CPT>
__device__ __forceinline__ void stencil3i(const int* row, int w0, typename CellType<CPT>::VI v[3]) {
    if constexpr (CPT == 1) {
        v[0] = row[w0 - 1];
        v[1] = row[w0];
        v[2] = row[w0 + 1];
    } else {
        const int2 a = *reinterpret_cast<const int2*>(row + w0 - 2);
        const int2 b = *reinterpret_cast<const int2*>(row + w0);
        const int2 c = *reinterpret_cast<const int2*>(row + w0 + 2);
        v[0] = i2{a.y, b.x};
        v[1] = i2{b.x, b.y};
        v[2] = i2{b.y, c.x};
    }
}

// ---------------------------------------------------------------------------
// pulls from the staged rows (Rm, R0, Rp: plane 0 of rows j-1, j, j+1; planes
// W floats apart; cells at staged columns cs .. cs + CPT - 1)
// ---------------------------------------------------------------------------

template <class V, class VI>
struct ScalarMomentsV {
    VI s0;    // S(x), fixed point
    V inc;    // zeroth moment = s0 * inv_scale + inc
    V jx, jy;
};

// Zeroth and first moments of an advection-diffusion lattice in deviation
// form (plane 0: S, planes 1..8: d_q; see pull_scalar_rows).
template <int CPT, int W>
__device__ __forceinline__ ScalarMomentsV<typename CellType<CPT>::V, typename CellType<CPT>::VI>
pull_scalar_v(const float* Rm, const float* R0, const float* Rp, int cs, bool bot, bool top,
              float inv) {
    using V = typename CellType<CPT>::V;
    using VI = typename CellType<CPT>::VI;
    const VI S0 = ldi<CPT, 0>(R0, cs);
    V o[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) o[q] = ldv<CPT, 0>(R0 + q * W, cs);
    const float w1 = (1.0f / 9.0f) * inv, w5 = (1.0f / 36.0f) * inv;
    V t[9];
    t[1] = vfma(w1, i2f(isub(ldi<CPT, -1>(R0, cs), S0)), ldv<CPT, -1>(R0 + 1 * W, cs));
    t[3] = vfma(w1, i2f(isub(ldi<CPT, 1>(R0, cs), S0)), ldv<CPT, 1>(R0 + 3 * W, cs));
    if (bot) {
        t[2] = o[4];
        t[5] = o[7];
        t[6] = o[8];
    } else {
        t[2] = vfma(w1, i2f(isub(ldi<CPT, 0>(Rm, cs), S0)), ldv<CPT, 0>(Rm + 2 * W, cs));
        t[5] = vfma(w5, i2f(isub(ldi<CPT, -1>(Rm, cs), S0)), ldv<CPT, -1>(Rm + 5 * W, cs));
        t[6] = vfma(w5, i2f(isub(ldi<CPT, 1>(Rm, cs), S0)), ldv<CPT, 1>(Rm + 6 * W, cs));
    }
    if (top) {
        t[4] = o[2];
        t[7] = o[5];
        t[8] = o[6];
    } else {
        t[4] = vfma(w1, i2f(isub(ldi<CPT, 0>(Rp, cs), S0)), ldv<CPT, 0>(Rp + 4 * W, cs));
        t[7] = vfma(w5, i2f(isub(ldi<CPT, 1>(Rp, cs), S0)), ldv<CPT, 1>(Rp + 7 * W, cs));
        t[8] = vfma(w5, i2f(isub(ldi<CPT, -1>(Rp, cs), S0)), ldv<CPT, -1>(Rp + 8 * W, cs));
    }
    ScalarMomentsV<V, VI> m;
    m.s0 = S0;
    const V d13 = t[1] - t[3], d56 = t[5] - t[6], d78 = t[7] - t[8];
    const V s56 = t[5] + t[6], s78 = t[7] + t[8];
    m.inc = (((t[1] + t[3]) + (t[2] + t[4])) + (s56 + s78)) -
            (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])));
    m.jx = (d13 + d56) - d78;
    m.jy = ((t[2] - t[4]) + s56) - s78;
    return m;
}

// Zeroth and first moments of f and h of one cell, f and h as the two lanes
// of the packed FP32 instructions (FP32 storage: f in planes 0..8, h in
// planes 9..17; the same increments as pull_scalar_v).
template <int W>
__device__ __forceinline__ ScalarMomentsV<f2, i2> pull_scalars_fh(const float* Rm, const float* R0,
                                                                  const float* Rp, int cs, bool bot,
                                                                  bool top, f2 inv) {
    auto S_at = [&](const float* R, int c) {
        return i2{__float_as_int(R[c]), __float_as_int(R[9 * W + c])};
    };
    auto d_at = [&](const float* R, int q, int c) { return f2(R[q * W + c], R[(9 + q) * W + c]); };
    const i2 S0 = S_at(R0, cs);
    f2 o[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) o[q] = d_at(R0, q, cs);
    const f2 w1 = (1.0f / 9.0f) * inv, w5 = (1.0f / 36.0f) * inv;
    f2 t[9];
    t[1] = vfma(w1, i2f(isub(S_at(R0, cs - 1), S0)), d_at(R0, 1, cs - 1));
    t[3] = vfma(w1, i2f(isub(S_at(R0, cs + 1), S0)), d_at(R0, 3, cs + 1));
    if (bot) {
        t[2] = o[4];
        t[5] = o[7];
        t[6] = o[8];
    } else {
        t[2] = vfma(w1, i2f(isub(S_at(Rm, cs), S0)), d_at(Rm, 2, cs));
        t[5] = vfma(w5, i2f(isub(S_at(Rm, cs - 1), S0)), d_at(Rm, 5, cs - 1));
        t[6] = vfma(w5, i2f(isub(S_at(Rm, cs + 1), S0)), d_at(Rm, 6, cs + 1));
    }
    if (top) {
        t[4] = o[2];
        t[7] = o[5];
        t[8] = o[6];
    } else {
        t[4] = vfma(w1, i2f(isub(S_at(Rp, cs), S0)), d_at(Rp, 4, cs));
        t[7] = vfma(w5, i2f(isub(S_at(Rp, cs + 1), S0)), d_at(Rp, 7, cs + 1));
        t[8] = vfma(w5, i2f(isub(S_at(Rp, cs - 1), S0)), d_at(Rp, 8, cs - 1));
    }
    ScalarMomentsV<f2, i2> m;
    m.s0 = S0;
    const f2 d13 = t[1] - t[3], d56 = t[5] - t[6], d78 = t[7] - t[8];
    const f2 s56 = t[5] + t[6], s78 = t[7] + t[8];
    m.inc = (((t[1] + t[3]) + (t[2] + t[4])) + (s56 + s78)) -
            (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])));
    m.jx = (d13 + d56) - d78;
    m.jy = ((t[2] - t[4]) + s56) - s78;
    return m;
}

// The same for 16-bit storage, where a word already holds (f, h) of a cell.
template <int ST, int W>
__device__ __forceinline__ ScalarMomentsV<f2, i2> pull_scalars_fh16(const float* Rm,
                                                                    const float* R0,
                                                                    const float* Rp, int cs,
                                                                    bool bot, bool top,
                                                                    const KParams& p) {
    auto S_at = [&](const float* R, int c) {
        return i2{__float_as_int(R[c]), __float_as_int(R[P16_SH * W + c])};
    };
    auto d_at = [&](const float* R, int q, int c) {
        return from_f2(unpack2<ST>(__float_as_uint(R[(P16_FH - 1 + q) * W + c])));
    };
    const i2 S0 = S_at(R0, cs);
    f2 o[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) o[q] = d_at(R0, q, cs);
    // sums on the scaled deviations, unscaled once at the end (the weights
    // carry the power-of-two scales)
    const f2 w1((1.0f / 9.0f) * p.fx_inv[0] * p.qs[0], (1.0f / 9.0f) * p.fx_inv[1] * p.qs[1]);
    const f2 w5((1.0f / 36.0f) * p.fx_inv[0] * p.qs[0], (1.0f / 36.0f) * p.fx_inv[1] * p.qs[1]);
    f2 t[9];
    t[1] = vfma(w1, i2f(isub(S_at(R0, cs - 1), S0)), d_at(R0, 1, cs - 1));
    t[3] = vfma(w1, i2f(isub(S_at(R0, cs + 1), S0)), d_at(R0, 3, cs + 1));
    if (bot) {
        t[2] = o[4];
        t[5] = o[7];
        t[6] = o[8];
    } else {
        t[2] = vfma(w1, i2f(isub(S_at(Rm, cs), S0)), d_at(Rm, 2, cs));
        t[5] = vfma(w5, i2f(isub(S_at(Rm, cs - 1), S0)), d_at(Rm, 5, cs - 1));
        t[6] = vfma(w5, i2f(isub(S_at(Rm, cs + 1), S0)), d_at(Rm, 6, cs + 1));
    }
    if (top) {
        t[4] = o[2];
        t[7] = o[5];
        t[8] = o[6];
    } else {
        t[4] = vfma(w1, i2f(isub(S_at(Rp, cs), S0)), d_at(Rp, 4, cs));
        t[7] = vfma(w5, i2f(isub(S_at(Rp, cs + 1), S0)), d_at(Rp, 7, cs + 1));
        t[8] = vfma(w5, i2f(isub(S_at(Rp, cs - 1), S0)), d_at(Rp, 8, cs - 1));
    }
    const f2 qi(p.qinv[0], p.qinv[1]);
    ScalarMomentsV<f2, i2> m;
    m.s0 = S0;
    m.inc = ((((t[1] + t[3]) + (t[2] + t[4])) + ((t[5] + t[6]) + (t[7] + t[8]))) -
             (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])))) * qi;
    m.jx = (((t[1] - t[3]) + (t[5] - t[6])) - (t[7] - t[8])) * qi;
    m.jy = (((t[2] - t[4]) + (t[5] + t[6])) - (t[7] + t[8])) * qi;
    return m;
}

// Post-streaming shifted flow populations (FP32 storage).
template <int CPT, int W>
__device__ __forceinline__ void pull_flow_v(const float* Rm, const float* R0, const float* Rp,
                                            int cs, bool bot, bool top,
                                            typename CellType<CPT>::V out[9]) {
    out[0] = ldv<CPT, 0>(R0, cs);
    out[1] = ldv<CPT, -1>(R0 + 1 * W, cs);
    out[3] = ldv<CPT, 1>(R0 + 3 * W, cs);
    if (bot) {
        out[2] = ldv<CPT, 0>(R0 + 4 * W, cs);
        out[5] = ldv<CPT, 0>(R0 + 7 * W, cs);
        out[6] = ldv<CPT, 0>(R0 + 8 * W, cs);
    } else {
        out[2] = ldv<CPT, 0>(Rm + 2 * W, cs);
        out[5] = ldv<CPT, -1>(Rm + 5 * W, cs);
        out[6] = ldv<CPT, 1>(Rm + 6 * W, cs);
    }
    if (top) {
        out[4] = ldv<CPT, 0>(R0 + 2 * W, cs);
        out[7] = ldv<CPT, 0>(R0 + 5 * W, cs);
        out[8] = ldv<CPT, 0>(R0 + 6 * W, cs);
    } else {
        out[4] = ldv<CPT, 0>(Rp + 4 * W, cs);
        out[7] = ldv<CPT, 1>(Rp + 7 * W, cs);
        out[8] = ldv<CPT, -1>(Rp + 8 * W, cs);
    }
}

// 16-bit storage: CPT words of one plane unpacked to (low halves, high halves).
template <int CPT, int ST, int DX>
__device__ __forceinline__ void ld16(const float* row, int c, typename CellType<CPT>::V& lo,
                                     typename CellType<CPT>::V& hi) {
    if constexpr (CPT == 1) {
        const float2 v = unpack2<ST>(__float_as_uint(row[c + DX]));
        lo = v.x;
        hi = v.y;
    } else {
        uint32_t wa, wb;
        if constexpr ((DX & 1) == 0) {
            const uint2 w = *reinterpret_cast<const uint2*>(row + c + DX);
            wa = w.x;
            wb = w.y;
        } else {
            wa = __float_as_uint(row[c + DX]);
            wb = __float_as_uint(row[c + DX + 1]);
        }
        const float2 a = unpack2<ST>(wa), b = unpack2<ST>(wb);
        lo = f2(a.x, b.x);
        hi = f2(a.y, b.y);
    }
}

// Zeroth and first moments of f and h from staged 16-bit rows (the same
// increments as pull_scalar_v; the sums run on the scaled deviations and are
// unscaled once at the end).
template <int CPT, int ST, int W>
__device__ __forceinline__ void pull_pair16_v(
    const float* Rm, const float* R0, const float* Rp, int cs, bool bot, bool top,
    const KParams& p,
    ScalarMomentsV<typename CellType<CPT>::V, typename CellType<CPT>::VI>& mf,
    ScalarMomentsV<typename CellType<CPT>::V, typename CellType<CPT>::VI>& mh) {
    using V = typename CellType<CPT>::V;
    using VI = typename CellType<CPT>::VI;
    const VI Sf0 = ldi<CPT, 0>(R0, cs);
    const VI Sh0 = ldi<CPT, 0>(R0 + P16_SH * W, cs);
    V of[9], oh[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) ld16<CPT, ST, 0>(R0 + (P16_FH - 1 + q) * W, cs, of[q], oh[q]);
    const float wf1 = ((1.0f / 9.0f) * p.fx_inv[0]) * p.qs[0], wf5 = ((1.0f / 36.0f) * p.fx_inv[0]) * p.qs[0];
    const float wh1 = ((1.0f / 9.0f) * p.fx_inv[1]) * p.qs[1], wh5 = ((1.0f / 36.0f) * p.fx_inv[1]) * p.qs[1];
    V tf[9], th[9];
    auto pulled = [&](auto dx, int q, const float* R, bool diag) {
        constexpr int DX = decltype(dx)::value;
        V vf, vh;
        ld16<CPT, ST, DX>(R + (P16_FH - 1 + q) * W, cs, vf, vh);
        tf[q] = vfma(diag ? wf5 : wf1, i2f(isub(ldi<CPT, DX>(R, cs), Sf0)), vf);
        th[q] = vfma(diag ? wh5 : wh1, i2f(isub(ldi<CPT, DX>(R + P16_SH * W, cs), Sh0)), vh);
    };
    using M1 = std::integral_constant<int, -1>;
    using Z0 = std::integral_constant<int, 0>;
    using P1 = std::integral_constant<int, 1>;
    pulled(M1{}, 1, R0, false);
    pulled(P1{}, 3, R0, false);
    if (bot) {
        tf[2] = of[4]; th[2] = oh[4];
        tf[5] = of[7]; th[5] = oh[7];
        tf[6] = of[8]; th[6] = oh[8];
    } else {
        pulled(Z0{}, 2, Rm, false);
        pulled(M1{}, 5, Rm, true);
        pulled(P1{}, 6, Rm, true);
    }
    if (top) {
        tf[4] = of[2]; th[4] = oh[2];
        tf[7] = of[5]; th[7] = oh[5];
        tf[8] = of[6]; th[8] = oh[6];
    } else {
        pulled(Z0{}, 4, Rp, false);
        pulled(P1{}, 7, Rp, true);
        pulled(M1{}, 8, Rp, true);
    }
    auto moments = [](VI S0, const V t[9], const V o[9], float qi,
                      ScalarMomentsV<V, VI>& m) {
        m.s0 = S0;
        m.inc = ((((t[1] + t[3]) + (t[2] + t[4])) + ((t[5] + t[6]) + (t[7] + t[8]))) -
                 (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])))) * qi;
        m.jx = (((t[1] - t[3]) + (t[5] - t[6])) - (t[7] - t[8])) * qi;
        m.jy = (((t[2] - t[4]) + (t[5] + t[6])) - (t[7] + t[8])) * qi;
    };
    moments(Sf0, tf, of, p.qinv[0], mf);
    moments(Sh0, th, oh, p.qinv[1], mh);
}

// Post-streaming flow populations (shifted, unscaled) from staged 16-bit rows.
template <int CPT, int ST, int W>
__device__ __forceinline__ void pull_flow16_v(const float* Rm, const float* R0, const float* Rp,
                                              int cs, bool bot, bool top, float qinv,
                                              typename CellType<CPT>::V out[9]) {
    using V = typename CellType<CPT>::V;
    auto g_at = [&](auto dx, const float* R, int q) {
        constexpr int DX = decltype(dx)::value;
        V lo, hi;
        ld16<CPT, ST, DX>(R + (P16_G + (q >> 1)) * W, cs, lo, hi);
        return ((q & 1) ? hi : lo) * qinv;
    };
    using M1 = std::integral_constant<int, -1>;
    using Z0 = std::integral_constant<int, 0>;
    using P1 = std::integral_constant<int, 1>;
    out[0] = g_at(Z0{}, R0, 0);
    out[1] = g_at(M1{}, R0, 1);
    out[3] = g_at(P1{}, R0, 3);
    if (bot) {
        out[2] = g_at(Z0{}, R0, 4);
        out[5] = g_at(Z0{}, R0, 7);
        out[6] = g_at(Z0{}, R0, 8);
    } else {
        out[2] = g_at(Z0{}, Rm, 2);
        out[5] = g_at(M1{}, Rm, 5);
        out[6] = g_at(P1{}, Rm, 6);
    }
    if (top) {
        out[4] = g_at(Z0{}, R0, 2);
        out[7] = g_at(Z0{}, R0, 5);
        out[8] = g_at(Z0{}, R0, 6);
    } else {
        out[4] = g_at(Z0{}, Rp, 4);
        out[7] = g_at(P1{}, Rp, 7);
        out[8] = g_at(M1{}, Rp, 8);
    }
}

// Per-tile facts about a thread's cells, for the stores: which cells are
// own columns (collided and stored), which of those lie beyond the last
// multiple of 4 (the bulk-tensor store maps end there, so that their clip
// falls on a 16-byte boundary; those cells are stored directly), and the
// column offsets of the periodic ghost copies of the four edge columns.
template <int CPT>
struct EdgeInfo {
    bool own[CPT], tail[CPT];
    int gs[CPT][2];
    bool all;    // every cell is an own column
    bool extra;  // some cell needs a ghost copy or a tail store
    __device__ EdgeInfo(const KParams& p, int col0, int x0, int xend, const int gi[CPT]) {
        const int nx4 = p.nx & ~3;
        all = true;
        extra = false;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int col = col0 + k;
            own[k] = col >= x0 && col < xend;
            tail[k] = own[k] && col >= nx4;
            gs[k][0] = own[k] ? ghost_right(p, gi[k]) : 0;
            gs[k][1] = own[k] ? ghost_left(p, gi[k]) : 0;
            all = all && own[k];
            extra = extra || tail[k] || gs[k][0] != 0 || gs[k][1] != 0;
        }
    }
};

// Plain stores of a staged cell that the bulk-tensor store does not cover
// (tail columns and ghost copies): NP word planes from staging plane 0 go to
// buffer planes plane0 + m of row j.
template <int NP, int CPT>
__device__ __forceinline__ void edge_stores(const KParams& p, float* __restrict__ dst,
                                            const float* out, int tx, int plane0, int j,
                                            const int gi[CPT], const EdgeInfo<CPT>& E) {
    if (!E.extra) return;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if (!(E.tail[k] || E.gs[k][0] || E.gs[k][1])) continue;
        float* d = dst + (int64_t)plane0 * p.plane + (int64_t)j * p.pitch + gi[k];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float v = out[m * tx + k];
            float* dm = d + (int64_t)m * p.plane;
            if (E.tail[k]) dm[0] = v;
            for (int e = 0; e < 2; ++e)
                if (E.gs[k][e]) dm[E.gs[k][e]] = v;
        }
    }
}

// Direct stores of one row's cells of a thread (OUT_DIRECT): NP word planes
// val(0 .. NP-1) to buffer planes plane0 + m of row j, and the ghost copies.
// Two cells go out as one 8-byte store.
__device__ __forceinline__ float as_float(int v) { return __int_as_float(v); }
__device__ __forceinline__ f2 as_float(i2 v) { return f2(__int_as_float(v.x), __int_as_float(v.y)); }
// The words of CPT cells (16-bit storage) as the value type of the stores.
template <int CPT>
__device__ __forceinline__ typename CellType<CPT>::V words_v(const uint32_t* w) {
    if constexpr (CPT == 1) return __uint_as_float(w[0]);
    else return f2(__uint_as_float(w[0]), __uint_as_float(w[1]));
}

template <int CPT, int NP, class G>
__device__ __forceinline__ void direct_stores(float* __restrict__ dst, const KParams& p,
                                              int plane0, int j, const int gi[CPT],
                                              const EdgeInfo<CPT>& E, G&& val) {
    if (!E.own[0]) return;
    float* row = dst + (int64_t)j * p.pitch + gi[0] + (int64_t)plane0 * p.plane;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const auto v = val(m);
        float* d = row + (int64_t)m * p.plane;
        if constexpr (CPT == 1) {
            *d = v;
        } else {
            if (E.all) *reinterpret_cast<float2*>(d) = make_float2(v.x, v.y);
            else *d = v.x;
        }
    }
    if (!E.extra) return;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if (!(E.gs[k][0] || E.gs[k][1])) continue;
        float* d = dst + (int64_t)plane0 * p.plane + (int64_t)j * p.pitch + gi[k];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float v = lane(val(m), k);
            for (int e = 0; e < 2; ++e)
                if (E.gs[k][e]) d[(int64_t)m * p.plane + E.gs[k][e]] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// the tile
// ---------------------------------------------------------------------------

// One tile: columns [bxi * (BX - 4), +BX - 4) and rows [byi * seg, +seg) of a
// run, swept by 2 BX / CPT threads: warps of group 0 own the scalar lattices
// f and h, warps of group 1 the flow lattice g, CPT adjacent columns per
// thread in each group.  `issued_base` counts the staged rows this block has
// issued before (it sets the barrier phases) and is advanced by this tile's
// rows.  Returns false if a staged row never landed (error flag set).
//
// Per swept row r:
//   A  both groups: moments of row r from the staged rows r-1, r, r+1
//      (group 0: phi, c, sigma(c); group 1: P*)
//   B  group 1: unit normal of row r-1
//   C  group 1: flow collision of row r-2 (forces, u, P), u into a ring;
//      group 0: f and h collisions of row r-3 with the u of that row.
// After C each group meets at its own barrier and its first thread issues the
// bulk-tensor store of the row it staged; that thread waits for the store to
// have read its staging area just before the next pass's barrier 1, so the
// read-out overlaps the next row's moments.
// `seed` is the hash of the step (step_seed).
template <int BX, int CPT, bool COUPLED, int ST, int OUT>
__device__ __forceinline__ bool sweep_tile2(const CUtensorMap* tmap, const StoreMaps* smap,
                                            const KParams& p, float* __restrict__ dst,
                                            const float* __restrict__ F, int seg, int bxi, int byi,
                                            const SweepSmem<BX, CPT, COUPLED, ST, OUT>& S,
                                            uint32_t seed, uint32_t& issued_base,
                                            int* __restrict__ err) {
    using L = SweepLayout<BX, CPT, COUPLED, ST, OUT>;
    constexpr int SW_STAGES = L::STAGES;
    using V = typename CellType<CPT>::V;
    using VI = typename CellType<CPT>::VI;
    using SM = ScalarMomentsV<V, VI>;
    constexpr int NL = L::NL, W = L::W, SLOT = L::SLOT, TX = L::TX, RW = L::RW, NT = L::NT;
    uint64_t* bars = S.bars;

    const int t = threadIdx.x % NT;
    const bool flow = threadIdx.x >= NT;  // warp-uniform group
    const int x0 = bxi * TX;
    const int xend = min(x0 + TX, p.nx);
    const int y0 = byi * seg;
    const int y1 = min(y0 + seg, p.ny);
    const int w0 = CPT * t;      // first window column of this thread (window column 0 is x0 - 2)
    const int cs = w0 + 2;       // its staged column (staged column 0 is x0 - 4)
    // The threads whose cells are all own columns (window columns 2 .. TX+1):
    // they collide and stage their cells; beyond xend (a ragged last tile)
    // the staged values fall outside the grid and the stores clip them.
    const bool worker = w0 >= 2 && w0 + CPT <= TX + 2;
    // grid column of each cell: the periodic image, in range also for the
    // lanes beyond a narrow grid (their results are not used)
    int gi[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) gi[k] = rmodm_rt(x0 - 2 + w0 + k, p.nx);
    const EdgeInfo<CPT> E(p, x0 - 2 + w0, x0, xend, gi);

    // rows swept: phi for y0-2 .. y1+1; beyond walls only mirror copies
    const int rs = p.walls ? max(y0 - 2, 0) : y0 - 2;
    const int re = p.walls ? min(y1 + 1, p.ny + 1) : y1 + 1;
    const int last_phys = p.walls ? min(re, p.ny - 1) : re;
    // staged raw rows: rs-1 .. last_phys+1, counter k = row - (rs - 1)
    const int nraw = last_phys - rs + 3;

    const uint32_t base_k = issued_base;
    auto issue = [&](int k) {  // thread 0: stage raw row rs - 1 + k
        if (k >= nraw) return;
        const int row = rs - 1 + k;
        const int y = p.walls ? row : wrap_i(row, p.ny);  // rows beyond walls read fill values
        const uint32_t slot = (base_k + k) % SW_STAGES;
        mbar_arrive_expect_tx(&bars[slot], (uint32_t)(NL * W * sizeof(float)));
        // padded x coordinate of column x0 - 4 is x0 (XGHOST == 4)
        tma_load_3d(S.raw + slot * SLOT, tmap, x0 - 4 + XGHOST, y, 0, &bars[slot]);
    };
    auto staged = [&](int row) { return S.raw + ((base_k + row - rs + 1) % SW_STAGES) * SLOT; };
    auto wait_row = [&](int row) -> bool {
        const uint32_t k = base_k + (row - rs + 1);
        return mbar_wait_bounded(&bars[k % SW_STAGES], (k / SW_STAGES) & 1u);
    };

    int issued = 0;  // staged rows issued so far (thread 0)
    if (threadIdx.x == 0) {
        fence_proxy_async();
        for (int k = 0; k < SW_STAGES; ++k) issue(k);
        issued = min(SW_STAGES, nraw);
    }

    bool failed = false;
    if (p.stall_test) {
        // failure-path test: wait on a barrier that no copy completes
        const bool ok = mbar_wait_bounded(&bars[SW_STAGES], 0, 4096);
        failed = !__syncthreads_and(ok);
    }
    constexpr int NB = 2 * NT;  // threads meeting at the phase barriers

    // The row loop of one warp group (each group runs its own copy, so each
    // holds only its own registers).  Named barrier 1 (both groups, once per
    // row) publishes the moments of row r; named barrier 2 (flow group)
    // publishes its normals to its own collisions; named barriers 3 (scalar
    // group) and 4 (flow group) publish each group's staged row to its store.
    auto rows = [&](auto group) -> bool {
        constexpr bool FLOW = decltype(group)::value;
        // the first thread of each group issues and awaits the group's stores
        const bool leader = threadIdx.x == (FLOW ? NT : 0);
        // values kept for the collisions, newest row first: group 0 keeps
        // f (jx, jy) and h (S, jx, jy) of rows r .. r-3, group 1 the nine
        // flow populations of rows r .. r-2
        V ks[4][4];
        VI kc[4];
        V kg[3][9];
        int s5 = rmod5(rs), s3 = rmod3(rs);
        for (int r = rs; r <= re + 1;
             ++r, s5 = s5 == SW_RING - 1 ? 0 : s5 + 1, s3 = s3 == SW_NRING - 1 ? 0 : s3 + 1) {
            const bool sweep = r <= re;  // the last pass only finishes the scalar collisions
            const bool phys = sweep && (!p.walls || r < p.ny);
            const int slot = s5;
            // ---------------- A: moments of row r ----------------
            if (phys) {
                bool ok = true;
                if (r == rs) ok = wait_row(r - 1) && wait_row(r);
                ok = ok && wait_row(r + 1);
                if (ok) {
                    const int jj = p.walls ? r : wrap_i(r, p.ny);
                    const bool bot = p.walls && jj == 0, top = p.walls && jj == p.ny - 1;
                    const float* Rm = staged(r - 1);
                    const float* R0 = staged(r);
                    const float* Rp = staged(r + 1);
                    if constexpr (!FLOW && CPT == 1) {
                        // one cell: f and h side by side in the packed lanes
                        ScalarMomentsV<f2, i2> m;
                        if constexpr (ST == ST_F32)
                            m = pull_scalars_fh<W>(Rm, R0, Rp, cs, bot, top,
                                                   f2(p.fx_inv[0], p.fx_inv[1]));
                        else
                            m = pull_scalars_fh16<ST, W>(Rm, R0, Rp, cs, bot, top, p);
                        const uint32_t b = moment_bits(seed, gi[0], jj, p.nx);
                        const int phi_fx = fx_add_sr(m.s0.x, m.inc.x, p.fx_scale[0], b);
                        const int c_fx = fx_add_sr(m.s0.y, m.inc.y, p.fx_scale[1], second_bits(b));
                        const float c = (float)c_fx * p.fx_inv[1];
                        S.s_phi[slot * RW + w0] = phi_fx;
                        S.s_c[slot * RW + w0] = c;
                        S.s_sig[slot * RW + w0] = sigma_of_c(p, c);
                        ks[0][0] = lane(m.jx, 0);
                        ks[0][1] = lane(m.jy, 0);
                        ks[0][2] = lane(m.jx, 1);
                        ks[0][3] = lane(m.jy, 1);
                        kc[0] = c_fx;
                    } else if constexpr (!FLOW) {
                        SM mf, mh;
                        if constexpr (ST == ST_F32) {
                            mf = pull_scalar_v<CPT, W>(Rm, R0, Rp, cs, bot, top, p.fx_inv[0]);
                            mh = pull_scalar_v<CPT, W>(Rm + 9 * W, R0 + 9 * W, Rp + 9 * W, cs, bot,
                                                       top, p.fx_inv[1]);
                        } else {
                            pull_pair16_v<CPT, ST, W>(Rm, R0, Rp, cs, bot, top, p, mf, mh);
                        }
                        // zeroth moments in fixed point, rounded without bias
                        VI phi_fx, c_fx;
#pragma unroll
                        for (int k = 0; k < CPT; ++k) {
                            const uint32_t b = moment_bits(seed, gi[k], jj, p.nx);
                            set_lane(phi_fx, k, fx_add_sr(lane(mf.s0, k), lane(mf.inc, k),
                                                          p.fx_scale[0], b));
                            set_lane(c_fx, k, fx_add_sr(lane(mh.s0, k), lane(mh.inc, k),
                                                        p.fx_scale[1], second_bits(b)));
                        }
                        const V c = i2f(c_fx) * p.fx_inv[1];
                        sti<CPT>(S.s_phi + slot * RW, w0, phi_fx);
                        stv<CPT>(S.s_c + slot * RW, w0, c);
                        stv<CPT>(S.s_sig + slot * RW, w0, sigma_of_c(p, c));
                        ks[0][0] = mf.jx;
                        ks[0][1] = mf.jy;
                        ks[0][2] = mh.jx;
                        ks[0][3] = mh.jy;
                        kc[0] = c_fx;
                    } else if (COUPLED) {
                        V a[9];
                        if constexpr (ST == ST_F32)
                            pull_flow_v<CPT, W>(Rm + 18 * W, R0 + 18 * W, Rp + 18 * W, cs, bot, top, a);
                        else
                            pull_flow16_v<CPT, ST, W>(Rm, R0, Rp, cs, bot, top, p.qinv[2], a);
                        stv<CPT>(S.s_dps + slot * RW, w0, sum9(a));
#pragma unroll
                        for (int q = 0; q < 9; ++q) kg[0][q] = a[q];
                    }
                    // mirror rows below the bottom wall, formed once rows 0 and 1 exist
                    if (p.walls && r == 1) {
                        for (int src = 0; src <= 1; ++src) {
                            const int g = -1 - src;
                            if (g < y0 - 2) continue;
                            const int gs = rmod5(g), ss = rmod5(src);
                            if constexpr (!FLOW) {
                                sti<CPT>(S.s_phi + gs * RW, w0, ldi<CPT, 0>(reinterpret_cast<const float*>(S.s_phi + ss * RW), w0));
                                stv<CPT>(S.s_c + gs * RW, w0, ldv<CPT, 0>(S.s_c + ss * RW, w0));
                                stv<CPT>(S.s_sig + gs * RW, w0, ldv<CPT, 0>(S.s_sig + ss * RW, w0));
                            } else {
                                stv<CPT>(S.s_dps + gs * RW, w0, ldv<CPT, 0>(S.s_dps + ss * RW, w0));
                            }
                        }
                    }
                }
                // the row this group staged in the previous pass has been read out
                if (leader) bulk_wait_read_all();
                // one barrier both publishes row r and agrees on a failed wait
                if (named_bar_or(!ok, NB)) return false;
                // the staged row r-1 is consumed: reuse its slot for row r-1+SW_STAGES
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    issue(r - rs + SW_STAGES);
                    issued = min(r - rs + SW_STAGES + 1, nraw);
                }
            } else {
                // mirror row above the top wall
                if (sweep) {
                    const int ss = rmod5(2 * p.ny - 1 - r);
                    if constexpr (!FLOW) {
                        sti<CPT>(S.s_phi + slot * RW, w0, ldi<CPT, 0>(reinterpret_cast<const float*>(S.s_phi + ss * RW), w0));
                        stv<CPT>(S.s_c + slot * RW, w0, ldv<CPT, 0>(S.s_c + ss * RW, w0));
                        stv<CPT>(S.s_sig + slot * RW, w0, ldv<CPT, 0>(S.s_sig + ss * RW, w0));
                    } else {
                        stv<CPT>(S.s_dps + slot * RW, w0, ldv<CPT, 0>(S.s_dps + ss * RW, w0));
                    }
                }
                if (leader) bulk_wait_read_all();
                named_bar_or(false, NB);
            }
            // ---------------- B: unit normal one row behind ----------------
            if (FLOW && sweep) {
                // normal of row rn from the phi ring slots of rows rn-1, rn, rn+1
                auto normal_row = [&](int sm1, int s0, int sp1, int ns) {
                    VI v[3][3];
                    stencil3i<CPT>(S.s_phi + sm1 * RW, w0, v[0]);
                    stencil3i<CPT>(S.s_phi + s0 * RW, w0, v[1]);
                    stencil3i<CPT>(S.s_phi + sp1 * RW, w0, v[2]);
                    V gx, gy, nx, ny, gm;
                    iso_grad_fx(v, p.fx_inv[0], gx, gy);
                    unit_normal(gx, gy, nx, ny, gm);
                    stv<CPT>(S.s_nx + ns * RW, w0, nx);
                    stv<CPT>(S.s_ny + ns * RW, w0, ny);
                    stv<CPT>(S.s_gm + ns * RW, w0, gm);
                };
                const int rn = r - 1;  // rows r-2, r-1, r
                if (rn >= y0 - 1 && rn <= y1 && !(p.walls && rn == -1))
                    normal_row(ring_slot5(s5, 3), ring_slot5(s5, 4), s5, ring_slot3(s3, 2));
                // with a bottom wall, n(-1) needs the mirror of row 1, available at r = 1
                if (p.walls && r == 1 && y0 == 0)
                    normal_row(rmod5(-2), rmod5(-1), rmod5(0), rmod3(-1));
            }
            // the flow group's own barrier: its collisions read the normals
            // its other warps just formed (group 0 does not wait here)
            if constexpr (FLOW) named_bar_sync<2>(NT);
            // ---------------- C: collisions ----------------
            if constexpr (FLOW) {
                // flow lattice of row r-2; its velocity goes to the ring for group 0
                const int jc = r - 2;
                if (COUPLED && worker && jc >= y0 && jc < y1) {
                    // rows jc - 1, jc, jc + 1 = r - 3, r - 2, r - 1
                    const int c0 = ring_slot5(s5, 3);
                    const int cr[3] = {ring_slot5(s5, 2), c0, ring_slot5(s5, 4)};
                    const int nr[3] = {s3, ring_slot3(s3, 1), ring_slot3(s3, 2)};
                    CellGeomT<V> g;
                    g.phi_fx = ldi<CPT, 0>(reinterpret_cast<const float*>(S.s_phi + c0 * RW), w0);
                    g.phi = i2f(g.phi_fx) * p.fx_inv[0];
                    g.c = ldv<CPT, 0>(S.s_c + c0 * RW, w0);
                    g.sig = ldv<CPT, 0>(S.s_sig + c0 * RW, w0);
                    g.dps = ldv<CPT, 0>(S.s_dps + c0 * RW, w0);
                    g.nx = ldv<CPT, 0>(S.s_nx + nr[1] * RW, w0);
                    g.ny = ldv<CPT, 0>(S.s_ny + nr[1] * RW, w0);
                    g.gm = ldv<CPT, 0>(S.s_gm + nr[1] * RW, w0);
                    V vx[3][3], vy[3][3], v[3][3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        stencil3<CPT>(S.s_nx + nr[d] * RW, w0, vx[d]);
                        stencil3<CPT>(S.s_ny + nr[d] * RW, w0, vy[d]);
                    }
                    g.kappa = iso_div(vx, vy);
#pragma unroll
                    for (int d = 0; d < 3; ++d) stencil3<CPT>(S.s_sig + cr[d] * RW, w0, v[d]);
                    iso_grad(v, g.sgx, g.sgy);
#pragma unroll
                    for (int d = 0; d < 3; ++d) stencil3<CPT>(S.s_dps + cr[d] * RW, w0, v[d]);
                    iso_grad(v, g.pgx, g.pgy);
                    if (!p.rho_uniform) {
                        VI vi[3][3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) stencil3i<CPT>(S.s_phi + cr[d] * RW, w0, vi[d]);
                        iso_grad_fx(vi, p.fx_inv[0], g.fgx, g.fgy);
                    } else {
                        g.fgx = g.fgy = vsplat<V>(0.0f);
                    }
                    V gg[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) gg[q] = kg[2][q];
                    // 16-bit storage: the collision leaves the populations scaled for packing
                    const CellOutT<V> o =
                        collide_flow_cell(p, g, jc, gg, true, ST == ST_F32 ? 1.0f : p.qs[2]);
                    stv<CPT>(S.s_ux + (jc & 1) * RW, w0, o.ux);
                    stv<CPT>(S.s_uy + (jc & 1) * RW, w0, o.uy);
                    // stage the row (tile column w0 - 2) and write the ghost copies,
                    // or store the cells directly
                    float* out = S.out_f + (w0 - 2);
                    if constexpr (OUT == OUT_DIRECT && ST == ST_F32) {
                        direct_stores<CPT, 9>(dst, p, L::NS, jc, gi, E,
                                              [&](int m) { return gg[m]; });
                    } else if constexpr (ST == ST_F32) {
#pragma unroll
                        for (int q = 0; q < 9; ++q) stv<CPT>(out + q * TX, 0, gg[q]);
                    } else {
                        uint32_t wv[5][CPT];
#pragma unroll
                        for (int k = 0; k < CPT; ++k) {
                            const uint32_t h = cell_bits(seed ^ 0x80000000u, gi[k], jc, p.nx);
#pragma unroll
                            for (int m = 0; m < 5; ++m)
                                wv[m][k] = pack2_sr<ST>(lane(gg[2 * m], k),
                                                        2 * m + 1 < 9 ? lane(gg[2 * m + 1], k) : 0.0f,
                                                        word_bits(h, 9 + m));
                        }
                        if constexpr (OUT == OUT_DIRECT) {
                            direct_stores<CPT, 5>(dst, p, L::NS, jc, gi, E,
                                                  [&](int m) { return words_v<CPT>(wv[m]); });
                        } else {
#pragma unroll
                            for (int m = 0; m < 5; ++m) stw<CPT>(out + m * TX, 0, wv[m]);
                        }
                    }
                    if constexpr (OUT == OUT_STAGED) {
                        fence_proxy_async();
                        edge_stores<L::NF, CPT>(p, dst, out, TX, L::NS, jc, gi, E);
                    }
                }
                // the group's staged row goes out while the next row's moments form
                if (OUT == OUT_STAGED && COUPLED && jc >= y0 && jc < y1 && x0 < (p.nx & ~3)) {
                    named_bar_sync<4>(NT);
                    if (leader) {
                        tma_store_3d(&smap->f, x0 + XGHOST, jc, L::NS, S.out_f);
                        bulk_commit();
                    }
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    kg[2][q] = kg[1][q];
                    kg[1][q] = kg[0][q];
                }
            } else {
                // scalar lattices of row r-3, one row behind the flow
                const int jc = r - 3;
                if (worker && jc >= y0 && jc < y1) {
                    const int c0 = ring_slot5(s5, 2), n0 = s3;  // row r - 3
                    const VI phi_fx = ldi<CPT, 0>(reinterpret_cast<const float*>(S.s_phi + c0 * RW), w0);
                    V ux, uy;
                    if (COUPLED) {
                        ux = ldv<CPT, 0>(S.s_ux + (jc & 1) * RW, w0);
                        uy = ldv<CPT, 0>(S.s_uy + (jc & 1) * RW, w0);
                    } else {
                        // prescribed velocity, cell by cell (a lane beyond a ragged
                        // edge reads its periodic image; its result is not stored)
#pragma unroll
                        for (int k = 0; k < CPT; ++k) {
                            const int64_t idx = (int64_t)jc * p.pitch + gi[k];
                            set_lane(ux, k, F[FP_UX * p.plane + idx]);
                            set_lane(uy, k, F[FP_UY * p.plane + idx]);
                        }
                    }
                    V df[9], dh[9];
                    if constexpr (CPT == 1)
                        collide_scalars_pair(p, phi_fx, i2f(phi_fx) * p.fx_inv[0],
                                             S.s_c[c0 * RW + w0], S.s_nx[n0 * RW + w0],
                                             S.s_ny[n0 * RW + w0], ux, uy,
                                             f2(ks[3][0], ks[3][2]), f2(ks[3][1], ks[3][3]), df,
                                             dh, ST == ST_F32 ? 1.0f : p.qs[0],
                                             ST == ST_F32 ? 1.0f : p.qs[1]);
                    else
                        collide_scalars_cell(p, phi_fx, i2f(phi_fx) * p.fx_inv[0],
                                             ldv<CPT, 0>(S.s_c + c0 * RW, w0),
                                             ldv<CPT, 0>(S.s_nx + n0 * RW, w0),
                                             ldv<CPT, 0>(S.s_ny + n0 * RW, w0), ux, uy, ks[3][0],
                                             ks[3][1], ks[3][2], ks[3][3], df, dh,
                                             ST == ST_F32 ? 1.0f : p.qs[0],
                                             ST == ST_F32 ? 1.0f : p.qs[1]);
                    float* out = S.out_s + (w0 - 2);
                    if constexpr (OUT == OUT_DIRECT && ST == ST_F32) {
                        const V s_f = as_float(phi_fx), s_h = as_float(kc[3]);
                        direct_stores<CPT, 18>(dst, p, 0, jc, gi, E, [&](int m) {
                            return m == 0 ? s_f : m == 9 ? s_h : m < 9 ? df[m] : dh[m - 9];
                        });
                    } else if constexpr (ST == ST_F32) {
                        sti<CPT>(reinterpret_cast<int*>(out), 0, phi_fx);
                        sti<CPT>(reinterpret_cast<int*>(out + 9 * TX), 0, kc[3]);
#pragma unroll
                        for (int q = 1; q < 9; ++q) {
                            stv<CPT>(out + q * TX, 0, df[q]);
                            stv<CPT>(out + (9 + q) * TX, 0, dh[q]);
                        }
                    } else {
                        uint32_t wv[8][CPT];
#pragma unroll
                        for (int k = 0; k < CPT; ++k) {
                            const uint32_t h = cell_bits(seed, gi[k], jc, p.nx);
#pragma unroll
                            for (int q = 1; q < 9; ++q)
                                wv[q - 1][k] = pack2_sr<ST>(lane(df[q], k), lane(dh[q], k),
                                                            word_bits(h, q));
                        }
                        if constexpr (OUT == OUT_DIRECT) {
                            const V s_f = as_float(phi_fx), s_h = as_float(kc[3]);
                            direct_stores<CPT, 10>(dst, p, 0, jc, gi, E, [&](int m) {
                                return m == 0 ? s_f : m == P16_SH ? s_h
                                                    : words_v<CPT>(wv[m >= P16_FH ? m - P16_FH : 0]);
                            });
                        } else {
                            sti<CPT>(reinterpret_cast<int*>(out), 0, phi_fx);
                            sti<CPT>(reinterpret_cast<int*>(out + P16_SH * TX), 0, kc[3]);
#pragma unroll
                            for (int q = 1; q < 9; ++q)
                                stw<CPT>(out + (P16_FH - 1 + q) * TX, 0, wv[q - 1]);
                        }
                    }
                    if constexpr (OUT == OUT_STAGED) {
                        fence_proxy_async();
                        edge_stores<L::NS, CPT>(p, dst, out, TX, 0, jc, gi, E);
                    }
                }
                if (OUT == OUT_STAGED && jc >= y0 && jc < y1 && x0 < (p.nx & ~3)) {
                    named_bar_sync<3>(NT);
                    if (leader) {
                        tma_store_3d(&smap->s, x0 + XGHOST, jc, 0, S.out_s);
                        bulk_commit();
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ks[3][q] = ks[2][q];
                    ks[2][q] = ks[1][q];
                    ks[1][q] = ks[0][q];
                }
                kc[3] = kc[2];
                kc[2] = kc[1];
                kc[1] = kc[0];
            }
        }
        return true;
    };
    if (!failed) failed = !(flow ? rows(std::true_type{}) : rows(std::false_type{}));
    if (failed) {
        // a staged row never landed: report, then let copies still in flight finish
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            for (int k = max(0, issued - SW_STAGES); k < issued; ++k) {
                const uint32_t kk = base_k + (uint32_t)k;
                mbar_wait_bounded(&bars[kk % SW_STAGES], (kk / SW_STAGES) & 1u);
            }
        }
        if (threadIdx.x == 0 || threadIdx.x == NT) bulk_wait_all();
        __syncthreads();
    } else {
        // the rows staged in the last passes are written before the block moves on
        if (threadIdx.x == 0 || threadIdx.x == NT) bulk_wait_all();
        __syncthreads();
    }
    issued_base = base_k + (uint32_t)nraw;
    return !failed;
}

// Registers a thread of the bulk-tensor sweep is given (launch bounds): the
// one-cell form runs 24 warps per SM at 80, the two-cell form keeps twice the
// values per thread.
template <int BX, int CPT, bool COUPLED, int ST, int OUT>
constexpr int sweep2_min_blocks() {
    constexpr int threads = 2 * BX / CPT;
    constexpr int regs = CPT == 1 ? 80 : 160;
    constexpr int by_regs = 65536 / (regs * threads);
    constexpr int by_smem = (228 * 1024) / (int)(SweepLayout<BX, CPT, COUPLED, ST, OUT>::bytes + 1024);
    constexpr int n = by_regs < by_smem ? by_regs : by_smem;
    return n < 1 ? 1 : n;
}

// One time step of one run (bulk-tensor loads; direct or staged stores; CPT
// cells per thread).
template <int BX, int CPT, bool COUPLED, int ST, int OUT>
__global__ void __launch_bounds__(2 * BX / CPT, (sweep2_min_blocks<BX, CPT, COUPLED, ST, OUT>()))
    k_sweep2(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ StoreMaps smap,
             KParams p, float* __restrict__ dst, const float* __restrict__ F, int seg,
             int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the bulk-tensor copies need the carve-up on 128-byte boundaries
    if (smem_u32(smem_raw) & 127u) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    const SweepSmem<BX, CPT, COUPLED, ST, OUT> S(smem_raw);
    if (threadIdx.x == 0) {
        // [STAGES]: the failure-path test hook
        for (int k = 0; k <= sw_stages(ST, OUT); ++k) mbar_init(&S.bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t issued = 0;
    sweep_tile2<BX, CPT, COUPLED, ST, OUT>(&tmap, &smap, p, dst, F, seg, blockIdx.x, blockIdx.y,
                                           S, step_seed(p), issued, err);
}

}  // namespace lbm
