// The row sweep of one tile of the fused TMA step, shared by the step
// kernels for every storage format (lbm_sweep_tma.cu: FP32 populations,
// lbm_sweep_tma16.cu: 16-bit deviations).
//
// A block owns a strip of columns and walks down a segment of rows, forming
// phi, c, sigma, P* one row ahead in shared-memory rings, the unit normal one
// row behind and colliding two (flow) and three (scalars) rows behind.  The
// raw rows are brought in by one 3-D TMA box per row ({columns, 1 row, all
// planes}) issued by one thread, TMA_STAGES - 3 rows ahead of use, and
// completing on an mbarrier.  Every pull then reads shared memory; every
// population byte leaves HBM once per strip.  Periodic x needs no wrap logic:
// the boxes include the ghost columns the writers maintain.  Walls: rows
// beyond a wall are never loaded; their ring entries are mirror copies of rows
// already formed (row -1-k is row k, row ny+k is ny-1-k).
#pragma once

#include <type_traits>

#include "lbm_cell.cuh"
#include "lbm_store16.cuh"
#include "lbm_tma.cuh"

namespace lbm {

namespace {

constexpr int TMA_STAGES = 4;  // staged raw rows: the three a row's pull reads, one ahead
constexpr int T_RING = 5;      // rows of phi, c, sigma, P* kept (and mirror copies)
constexpr int T_NRING = 3;     // rows of n, |grad phi|

template <int BX, bool COUPLED, int ST>
struct TmaLayout {
    static constexpr int NL = store_planes(ST, COUPLED);  // word planes per box
    static constexpr int W = BX + 4;                   // staged columns x0-4 .. x0+BX-1
    static constexpr int SLOT = (NL * W + 31) / 32 * 32;  // floats per staged row (128-B multiple)
    static constexpr size_t bytes =
        128 /* barriers */ + sizeof(float) * ((size_t)TMA_STAGES * SLOT + (size_t)T_RING * 4 * BX +
                                              (size_t)T_NRING * 3 * BX + (size_t)2 * 2 * BX) +
        128 /* alignment slack */;
};

__device__ __forceinline__ int rmod(int a, int m) { return ((a % m) + m) % m; }

// x mod m for 0 <= x < 2m
template <int M>
__device__ __forceinline__ int wrap_once(int x) { return x >= M ? x - M : x; }

}  // namespace

// Shared-memory carve-up of one block (the barriers come first).
template <int BX, bool COUPLED, int ST>
struct TmaSmem {
    uint64_t* bars;
    float* raw;
    int* s_phi;
    float *s_c, *s_sig, *s_dps, *s_nx, *s_ny, *s_gm, *s_ux, *s_uy;
    __device__ explicit TmaSmem(unsigned char* smem_raw) {
        using L = TmaLayout<BX, COUPLED, ST>;
        const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127;
        bars = reinterpret_cast<uint64_t*>(base);
        raw = reinterpret_cast<float*>(base + 128);
        s_phi = reinterpret_cast<int*>(raw + TMA_STAGES * L::SLOT);  // [T_RING][BX] fixed point
        s_c = reinterpret_cast<float*>(s_phi + T_RING * BX);
        s_sig = s_c + T_RING * BX;
        s_dps = s_sig + T_RING * BX;
        s_nx = s_dps + T_RING * BX;  // [T_NRING][BX]
        s_ny = s_nx + T_NRING * BX;
        s_gm = s_ny + T_NRING * BX;
        s_ux = s_gm + T_NRING * BX;  // [2][BX] velocity of the last flow-collided rows
        s_uy = s_ux + 2 * BX;
    }
};

// One tile: columns [bxi * (BX - 4), +BX - 4) and rows [byi * seg, +seg) of a
// run, swept by 2 BX threads: warps of group 0 own the scalar lattices f and
// h, warps of group 1 the flow lattice g, one column per thread in each group.
// `issued_base` counts the staged rows this block has issued before (it sets
// the barrier phases) and is advanced by this tile's rows.  Returns false if
// a staged row never landed (error flag set).
//
// Per swept row r:
//   A  both groups: moments of row r from the staged rows r-1, r, r+1
//      (group 0: phi, c, sigma(c); group 1: P*)
//   B  group 1: unit normal of row r-1
//   C  group 1: flow collision of row r-2 (forces, u, P), u into a ring;
//      group 0: f and h collisions of row r-3 with the u of that row.
// The pulled values a cell keeps for its collision wait in registers.
template <int BX, bool COUPLED, int ST>
__device__ __forceinline__ bool sweep_tile(const CUtensorMap* tmap, const KParams& p,
                                           float* __restrict__ dst, const float* __restrict__ F,
                                           int seg, int bxi, int byi,
                                           const TmaSmem<BX, COUPLED, ST>& S,
                                           uint32_t& issued_base, int* __restrict__ err) {
    using L = TmaLayout<BX, COUPLED, ST>;
    constexpr int NL = L::NL, W = L::W, SLOT = L::SLOT, TX = BX - 4;
    uint64_t* bars = S.bars;
    float* raw = S.raw;
    int* s_phi = S.s_phi;
    float* s_c = S.s_c;
    float* s_sig = S.s_sig;
    float* s_dps = S.s_dps;
    float* s_nx = S.s_nx;
    float* s_ny = S.s_ny;
    float* s_gm = S.s_gm;
    float* s_ux = S.s_ux;
    float* s_uy = S.s_uy;

    const int t = threadIdx.x % BX;
    const bool flow = threadIdx.x >= BX;  // warp-uniform group
    const int x0 = bxi * TX;
    const int xend = min(x0 + TX, p.nx);
    const int y0 = byi * seg;
    const int y1 = min(y0 + seg, p.ny);
    const int col = x0 - 2 + t;
    // Column roles: 3 the tile's own columns (collided and stored), 2 the
    // halo columns whose sigma, P* and normals the stencils of the own columns
    // read, 1 the outer halo columns whose phi the normals of role 2 read, 0
    // columns beyond the grid in a ragged last tile.  The moments (A) are
    // formed in every column; the normals (B) for roles 1-3; the collisions
    // and stores (C) for role 3 only.
    int role = 0;
    if (col >= x0 && col < xend) role = 3;
    else if (col == x0 - 1 || col == xend) role = 2;
    else if (col == x0 - 2 || col == xend + 1) role = 1;
    const int i = wrap_i(col, p.nx);
    // ghost copies of column i, fixed per tile (FP32 stores; the 16-bit stores
    // form them per call, which measured faster there)
    const int gsT[2] = {ghost_right(p, i), ghost_left(p, i)};
    const int cs = t + 2;  // this column's index in a staged row (staged column 0 is x0 - 4)

    // rows swept: phi for y0-2 .. y1+1; beyond walls only mirror copies
    const int rs = p.walls ? max(y0 - 2, 0) : y0 - 2;
    const int re = p.walls ? min(y1 + 1, p.ny + 1) : y1 + 1;
    const int last_phys = p.walls ? min(re, p.ny - 1) : re;
    // staged raw rows: rs-1 .. last_phys+1, counter k = row - (rs - 1)
    const int nraw = last_phys - rs + 3;

    const uint32_t base_k = issued_base;
    // per-step salt of the stochastic rounding (16-bit storage)
    uint32_t step_seed = 0;
    if constexpr (ST != ST_F32) step_seed = pcg_hash(__ldg(p.step_ctr) + (uint32_t)p.step_off);
    auto issue = [&](int k) {  // thread 0: stage raw row rs - 1 + k
        if (k >= nraw) return;
        const int row = rs - 1 + k;
        const int y = p.walls ? row : wrap_i(row, p.ny);  // rows beyond walls read fill values
        const uint32_t slot = (base_k + k) % TMA_STAGES;
        mbar_arrive_expect_tx(&bars[slot], (uint32_t)(NL * W * sizeof(float)));
        // padded x coordinate of column x0 - 4 is x0 (XGHOST == 4)
        tma_load_3d(raw + slot * SLOT, tmap, x0 - 4 + XGHOST, y, 0, &bars[slot]);
    };
    auto staged = [&](int row) { return raw + ((base_k + row - rs + 1) % TMA_STAGES) * SLOT; };
    auto wait_row = [&](int row) -> bool {
        const uint32_t k = base_k + (row - rs + 1);
        return mbar_wait_bounded(&bars[k % TMA_STAGES], (k / TMA_STAGES) & 1u);
    };

    int issued = 0;  // staged rows issued so far (thread 0)
    if (threadIdx.x == 0) {
        fence_proxy_async();
        for (int k = 0; k < TMA_STAGES; ++k) issue(k);
        issued = min(TMA_STAGES, nraw);
    }

    bool failed = false;
    if (p.stall_test) {
        // failure-path test: wait on a barrier that no copy completes
        const bool ok = mbar_wait_bounded(&bars[TMA_STAGES], 0, 4096);
        failed = !__syncthreads_and(ok);
    }
    constexpr int NT = 2 * BX;  // threads meeting at the phase barriers

    // The row loop of one warp group (each group runs its own copy, so each
    // holds only its own registers).  Named barrier 1 (both groups, once per
    // row) publishes the moments of row r; named barrier 2 (flow group only)
    // publishes its normals to its own collisions.
    auto rows = [&](auto group) -> bool {
        constexpr bool FLOW = decltype(group)::value;
        // values kept for the collisions, newest row first: group 0 keeps
        // f (jx, jy) and h (S, jx, jy) of rows r .. r-3, group 1 the nine
        // flow populations of rows r .. r-2
        float ks[4][5];
        float kg[3][9];
        // ring slots of row r, advanced with the loop (rows r-k sit at
        // wrap_once(s5 + T_RING - k) and wrap_once(s3 + T_NRING - k))
        int s5 = rmod(rs, T_RING), s3 = rmod(rs, T_NRING);
        for (int r = rs; r <= re + 1;
             ++r, s5 = wrap_once<T_RING>(s5 + 1), s3 = wrap_once<T_NRING>(s3 + 1)) {
            const bool sweep = r <= re;  // the last pass only finishes the scalar collisions
            const bool phys = sweep && (!p.walls || r < p.ny);
            const int slot = s5;
            // ---------------- A: moments of row r ----------------
            if (phys) {
                bool ok = true;
                if (r == rs) ok = wait_row(r - 1) && wait_row(r);
                ok = ok && wait_row(r + 1);
                // Every thread forms the moments of its column, including the halo
                // columns whose results nobody reads and, in a ragged last tile,
                // columns beyond the grid (their staged values are padding or
                // fill): per-thread tests here cost more than the idle lanes save.
                if (ok) {
                    const int jj = p.walls ? r : wrap_i(r, p.ny);
                    const bool bot = p.walls && jj == 0, top = p.walls && jj == p.ny - 1;
                    const float* Rm = staged(r - 1);
                    const float* R0 = staged(r);
                    const float* Rp = staged(r + 1);
                    if constexpr (!FLOW) {
                        ScalarMoments m, mh;
                        if constexpr (ST == ST_F32) {
                            m = pull_scalar_rows(Rm, R0, Rp, W, cs - 1, cs, cs + 1, bot, top,
                                                 p.fx_inv[0]);
                        } else {
                            pull_pair16<ST>(Rm, R0, Rp, W, cs - 1, cs, cs + 1, bot, top, p, m, mh);
                        }
                        s_phi[slot * BX + t] = fx_add(m.s0, m.inc, p.fx_scale[0]);
                        ks[0][0] = m.jx;
                        ks[0][1] = m.jy;
                        {  // h: c and sigma(c)
                            if constexpr (ST == ST_F32)
                                m = pull_scalar_rows(Rm + 9 * W, R0 + 9 * W, Rp + 9 * W, W, cs - 1,
                                                     cs, cs + 1, bot, top, p.fx_inv[1]);
                            else
                                m = mh;
                            const int c_fx = fx_add(m.s0, m.inc, p.fx_scale[1]);
                            const float c = (float)c_fx * p.fx_inv[1];
                            s_c[slot * BX + t] = c;
                            s_sig[slot * BX + t] = sigma_of_c(p, c);
                            ks[0][2] = __int_as_float(c_fx);
                            ks[0][3] = m.jx;
                            ks[0][4] = m.jy;
                        }
                    } else if (COUPLED) {
                        float a[9];
                        if constexpr (ST == ST_F32)
                            pull9_rows(Rm + 18 * W, R0 + 18 * W, Rp + 18 * W, W, cs - 1, cs, cs + 1,
                                       bot, top, a);
                        else
                            pull9_16<ST>(Rm, R0, Rp, W, cs - 1, cs, cs + 1, bot, top, p.qinv[2], a);
                        s_dps[slot * BX + t] = sum9(a);
                        // every pulled row enters the ring: rows and columns that do not
                        // collide never read it, and an unconditional write lets the pull
                        // land in the ring's registers directly
#pragma unroll
                        for (int q = 0; q < 9; ++q) kg[0][q] = a[q];
                    }
                    // mirror rows below the bottom wall, formed once rows 0 and 1 exist
                    if (p.walls && r == 1) {
                        for (int src = 0; src <= 1; ++src) {
                            const int g = -1 - src;
                            if (g < y0 - 2) continue;
                            const int gs = rmod(g, T_RING), ss = rmod(src, T_RING);
                            if constexpr (!FLOW) {
                                s_phi[gs * BX + t] = s_phi[ss * BX + t];
                                if (role >= 2) {
                                    s_c[gs * BX + t] = s_c[ss * BX + t];
                                    s_sig[gs * BX + t] = s_sig[ss * BX + t];
                                }
                            } else if (role >= 2) {
                                s_dps[gs * BX + t] = s_dps[ss * BX + t];
                            }
                        }
                    }
                }
                // one barrier both publishes row r and agrees on a failed wait
                if (named_bar_or(!ok, NT)) return false;
                // the staged row r-1 is consumed: reuse its slot for row r-1+TMA_STAGES
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    issue(r - rs + TMA_STAGES);
                    issued = min(r - rs + TMA_STAGES + 1, nraw);
                }
            } else {
                // mirror row above the top wall
                if (sweep && role > 0) {
                    const int ss = rmod(2 * p.ny - 1 - r, T_RING);
                    if constexpr (!FLOW) {
                        s_phi[slot * BX + t] = s_phi[ss * BX + t];
                        if (role >= 2) {
                            s_c[slot * BX + t] = s_c[ss * BX + t];
                            s_sig[slot * BX + t] = s_sig[ss * BX + t];
                        }
                    } else if (role >= 2) {
                        s_dps[slot * BX + t] = s_dps[ss * BX + t];
                    }
                }
                named_bar_or(false, NT);
            }
            // ---------------- B: unit normal one row behind ----------------
            if (FLOW && sweep && role > 0) {
                // normal of row rn from the phi ring slots of rows rn-1, rn, rn+1
                auto normal_row = [&](int sm1, int s0, int sp1, int ns) {
                    int v[3][3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        v[0][e] = s_phi[sm1 * BX + t - 1 + e];
                        v[1][e] = s_phi[s0 * BX + t - 1 + e];
                        v[2][e] = s_phi[sp1 * BX + t - 1 + e];
                    }
                    float gx, gy, nx, ny, gm;
                    iso_grad_fx(v, p.fx_inv[0], gx, gy);
                    unit_normal(gx, gy, nx, ny, gm);
                    s_nx[ns * BX + t] = nx;
                    s_ny[ns * BX + t] = ny;
                    s_gm[ns * BX + t] = gm;
                };
                const int rn = r - 1;  // rows r-2, r-1, r
                if (rn >= y0 - 1 && rn <= y1 && !(p.walls && rn == -1))
                    normal_row(wrap_once<T_RING>(s5 + 3), wrap_once<T_RING>(s5 + 4), s5,
                               wrap_once<T_NRING>(s3 + 2));
                // with a bottom wall, n(-1) needs the mirror of row 1, available at r = 1
                if (p.walls && r == 1 && y0 == 0)
                    normal_row(rmod(-2, T_RING), rmod(-1, T_RING), rmod(0, T_RING), rmod(-1, T_NRING));
            }
            // the flow group's own barrier: its collisions read the normals
            // its other warps just formed (group 0 does not wait here)
            if constexpr (FLOW) named_bar_sync<2>(BX);
            // ---------------- C: collisions ----------------
            if constexpr (FLOW) {
                // flow lattice of row r-2; its velocity goes to the ring for group 0
                const int jc = r - 2;
                if (COUPLED && role == 3 && jc >= y0 && jc < y1) {
                    // rows jc - 1, jc, jc + 1 = r - 3, r - 2, r - 1
                    const int c0 = wrap_once<T_RING>(s5 + 3);
                    const int cr[3] = {wrap_once<T_RING>(s5 + 2), c0, wrap_once<T_RING>(s5 + 4)};
                    const int nr[3] = {s3, wrap_once<T_NRING>(s3 + 1), wrap_once<T_NRING>(s3 + 2)};
                    CellGeom g;
                    g.phi_fx = s_phi[c0 * BX + t];
                    g.phi = (float)g.phi_fx * p.fx_inv[0];
                    g.c = s_c[c0 * BX + t];
                    g.sig = s_sig[c0 * BX + t];
                    g.dps = s_dps[c0 * BX + t];
                    g.nx = s_nx[nr[1] * BX + t];
                    g.ny = s_ny[nr[1] * BX + t];
                    g.gm = s_gm[nr[1] * BX + t];
                    float vx[3][3], vy[3][3], v[3][3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            vx[d][e] = s_nx[nr[d] * BX + t - 1 + e];
                            vy[d][e] = s_ny[nr[d] * BX + t - 1 + e];
                        }
                    g.kappa = iso_div(vx, vy);
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int e = 0; e < 3; ++e) v[d][e] = s_sig[cr[d] * BX + t - 1 + e];
                    iso_grad(v, g.sgx, g.sgy);
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int e = 0; e < 3; ++e) v[d][e] = s_dps[cr[d] * BX + t - 1 + e];
                    iso_grad(v, g.pgx, g.pgy);
                    if (!p.rho_uniform) {
                        int vi[3][3];
#pragma unroll
                        for (int d = 0; d < 3; ++d)
#pragma unroll
                            for (int e = 0; e < 3; ++e) vi[d][e] = s_phi[cr[d] * BX + t - 1 + e];
                        iso_grad_fx(vi, p.fx_inv[0], g.fgx, g.fgy);
                    } else {
                        g.fgx = g.fgy = 0.0f;
                    }
                    float gg[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) gg[q] = kg[2][q];
                    // 16-bit storage: the collision leaves the populations scaled for packing
                    const CellOut o =
                        collide_flow_cell(p, g, jc, gg, true, ST == ST_F32 ? 1.0f : p.qs[2]);
                    s_ux[(jc & 1) * BX + t] = o.ux;
                    s_uy[(jc & 1) * BX + t] = o.uy;
                    const int64_t idx = (int64_t)jc * p.pitch + i;
                    if constexpr (ST == ST_F32) {
                        uint32_t w[9];
#pragma unroll
                        for (int q = 0; q < 9; ++q) w[q] = __float_as_uint(gg[q]);
                        store_words<9>(dst, p.plane, idx, gsT, 18, w);
                    } else {
                        const uint32_t seed = pcg_hash(step_seed ^ (uint32_t)(jc * p.nx + i) ^ 0x80000000u);
                        uint32_t w[5];
#pragma unroll
                        for (int k = 0; k < 5; ++k)
                            w[k] = pack2_sr<ST>(gg[2 * k], 2 * k + 1 < 9 ? gg[2 * k + 1] : 0.0f,
                                                word_bits(seed, 9 + k));
                        const int gs[2] = {ghost_right(p, i), ghost_left(p, i)};
                        store_words<5>(dst, p.plane, idx, gs, P16_G, w);
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
                if (role == 3 && jc >= y0 && jc < y1) {
                    const int c0 = wrap_once<T_RING>(s5 + 2), n0 = s3;  // row r - 3
                    const int phi_fx = s_phi[c0 * BX + t];
                    const int64_t idx = (int64_t)jc * p.pitch + i;
                    float ux, uy;
                    if (COUPLED) {
                        ux = s_ux[(jc & 1) * BX + t];
                        uy = s_uy[(jc & 1) * BX + t];
                    } else {
                        ux = F[FP_UX * p.plane + idx];
                        uy = F[FP_UY * p.plane + idx];
                    }
                    float df[9], dh[9];
                    collide_scalars_cell(p, phi_fx, (float)phi_fx * p.fx_inv[0], s_c[c0 * BX + t],
                                         s_nx[n0 * BX + t], s_ny[n0 * BX + t], ux, uy, ks[3][0],
                                         ks[3][1], ks[3][3], ks[3][4], df, dh,
                                         ST == ST_F32 ? 1.0f : p.qs[0],
                                         ST == ST_F32 ? 1.0f : p.qs[1]);
                    if constexpr (ST == ST_F32) {
                        uint32_t w[9];
                        w[0] = (uint32_t)phi_fx;
#pragma unroll
                        for (int q = 1; q < 9; ++q) w[q] = __float_as_uint(df[q]);
                        store_words<9>(dst, p.plane, idx, gsT, 0, w);
                        w[0] = __float_as_uint(ks[3][2]);
#pragma unroll
                        for (int q = 1; q < 9; ++q) w[q] = __float_as_uint(dh[q]);
                        store_words<9>(dst, p.plane, idx, gsT, 9, w);
                    } else {
                        const uint32_t seed = pcg_hash(step_seed ^ (uint32_t)(jc * p.nx + i));
                        uint32_t w[10];
                        w[0] = (uint32_t)phi_fx;
                        w[1] = __float_as_uint(ks[3][2]);
#pragma unroll
                        for (int q = 1; q < 9; ++q) w[1 + q] = pack2_sr<ST>(df[q], dh[q], word_bits(seed, q));
                        const int gs[2] = {ghost_right(p, i), ghost_left(p, i)};
                        store_words<10>(dst, p.plane, idx, gs, 0, w);
                    }
                }
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    ks[3][q] = ks[2][q];
                    ks[2][q] = ks[1][q];
                    ks[1][q] = ks[0][q];
                }
            }
        }
        return true;
    };
    if (!failed) failed = !(flow ? rows(std::true_type{}) : rows(std::false_type{}));
    if (failed) {
        // a staged row never landed: report, then let copies still in flight finish
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            for (int k = max(0, issued - TMA_STAGES); k < issued; ++k) {
                const uint32_t kk = base_k + (uint32_t)k;
                mbar_wait_bounded(&bars[kk % TMA_STAGES], (kk / TMA_STAGES) & 1u);
            }
        }
        __syncthreads();
    }
    issued_base = base_k + (uint32_t)nraw;
    return !failed;
}

// Resident blocks per SM the register budget is set for: 768 threads (24
// warps) per SM at 80 registers, which the coupled kernel's shared memory
// also allows (three blocks at BX = 128, two at BX = 192).
template <int BX>
constexpr int tma_min_blocks() { return 384 / BX; }

}  // namespace lbm
