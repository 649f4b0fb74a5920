// Per-cell pieces of the coupled step shared by every step kernel: equilibria,
// field-plane stencil loads, the three collisions of one cell (Sec. 3, App. C,
// App. D) and the state stores that keep the periodic ghost columns.
#pragma once

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------

template <class V>
__device__ __forceinline__ V sum9(const V a[9]) {
    return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])) + a[8];
}

template <class V>
__device__ __forceinline__ V lerp_phase(const KParams& p, V phi, float va, float vb) {
    return vb + ((va - vb) * p.inv_dphi) * (phi - p.phi_b);
}

template <class V>
__device__ __forceinline__ V rate_from_coeff(V coeff) {
    return vmap(coeff, [](float c) { return 1.0f / (c * 3.0f + 0.5f); });
}

template <class V>
__device__ __forceinline__ V vdiv(V a, V b) {
    V q;
#pragma unroll
    for (int k = 0; k < Lanes<V>::n; ++k) set_lane(q, k, lane(a, k) / lane(b, k));
    return q;
}

// Deviation-form equilibrium of the flow lattice without source: shifted
// populations g^eq - w P0 for pressure deviation dP = P - P0.
__device__ __forceinline__ void eq_flow_shifted(float a[9], float dP, float rho, float ux,
                                                float uy) {
    const float ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const float R = rho * CS2, RmP = R - dP;
    float k[9];
    k[0] = dP;
    k[1] = ux * RmP;
    k[2] = uy * RmP;
    k[3] = -R * ux2 + dP * (CS2 + ux2);
    k[4] = -R * uy2 + dP * (CS2 + uy2);
    k[5] = -RmP * uxy;
    k[6] = RmP * (ux2 + CS2) * uy;
    k[7] = RmP * (uy2 + CS2) * ux;
    k[8] = -R * (ux2 * uy2 + CS2 * (ux2 + uy2)) + dP * (ux2 + CS2) * (uy2 + CS2);
    float r[9];
    central_to_raw(k, ux, uy, r);
    raw_to_pops(r, a);
}

__device__ __forceinline__ void eq_scalar(float a[9], float s, float qx, float qy, float ux,
                                          float uy) {
    float k[9] = {s, qx, qy, CS2 * s, CS2 * s, 0.0f, 0.0f, 0.0f, CS2 * CS2 * s};
    float r[9];
    central_to_raw(k, ux, uy, r);
    raw_to_pops(r, a);
}

// 3x3 neighbourhood of a field plane on the extended (periodic / mirrored)
// grid; ysign = -1 flips the sign of mirrored ghost rows (y component of n).
__device__ __forceinline__ void load3x3(const float* __restrict__ F, const KParams& p, int i, int j,
                                        float v[3][3], bool odd_under_mirror = false) {
    const int im = wrap_i(i - 1, p.nx), ip = wrap_i(i + 1, p.nx);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int jj = j + dy;
        const int64_t r = (int64_t)ext_row(jj, p.ny, p.walls) * p.pitch;
        const float s = odd_under_mirror ? mirror_sign(jj, p.ny, p.walls) : 1.0f;
        v[dy + 1][0] = s * F[r + im];
        v[dy + 1][1] = s * F[r + i];
        v[dy + 1][2] = s * F[r + ip];
    }
}

__device__ __forceinline__ void load3x3_fx(const float* __restrict__ F, const KParams& p, int i,
                                           int j, int v[3][3]) {
    const int im = wrap_i(i - 1, p.nx), ip = wrap_i(i + 1, p.nx);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int64_t r = (int64_t)ext_row(j + dy, p.ny, p.walls) * p.pitch;
        v[dy + 1][0] = __float_as_int(F[r + im]);
        v[dy + 1][1] = __float_as_int(F[r + i]);
        v[dy + 1][2] = __float_as_int(F[r + ip]);
    }
}

// Local values and stencil results one cell's (or two cells') collisions need.
template <class V, class VI = typename Lanes<V>::I>
struct CellGeomT {
    VI phi_fx;               // phi in fixed point (exact interface factors)
    V phi, c, sig, dps;      // zeroth moments, sigma(c), P* - P0
    V nx, ny, gm;            // unit normal, |grad phi|
    V kappa;                 // div n
    V sgx, sgy;              // grad sigma
    V pgx, pgy;              // grad (P* - P0)
    V fgx, fgy;              // grad phi (for grad rho)
};
using CellGeom = CellGeomT<float>;

template <class V>
struct CellOutT {
    V ux, uy, dP;
};
using CellOut = CellOutT<float>;

// Flow part of one cell's collisions (App. D): forces, velocity, pressure
// and, with do_collide, the flow populations gg collided in place.
// out_scale: power-of-two factor on the output populations (16-bit storage).
template <class V>
__device__ __forceinline__ CellOutT<V> collide_flow_cell(const KParams& p, const CellGeomT<V>& g,
                                                         int j, V gg[9], bool do_collide,
                                                         float out_scale = 1.0f) {
    CellOutT<V> o;
    // surface-tension force, Eq. (Fs)
    const V g2n = p.N_sigma * (g.gm * g.gm);
    const V nds = g.nx * g.sgx + g.ny * g.sgy;
    const V sk = g.sig * g.kappa;
    const V Fsx = g2n * ((g.sgx - g.nx * nds) - sk * g.nx);
    const V Fsy = g2n * ((g.sgy - g.ny * nds) - sk * g.ny);
    const V Ftx = Fsx + p.fext_x, Fty = Fsy + p.fext_y;
    const V rho = p.rho_uniform ? vsplat<V>(p.rho_a) : lerp_phase(p, g.phi, p.rho_a, p.rho_b);
    const V jx = ((gg[1] - gg[3]) + (gg[5] - gg[6])) - (gg[7] - gg[8]);
    const V jy = ((gg[2] - gg[4]) + (gg[5] + gg[6])) - (gg[7] + gg[8]);
    // cs2 rho u = sum e g + cs2 F_t / 2  (App. D), with the same rounded
    // rho cs2 as the equilibrium.
    const V R = rho * CS2;
    if (p.rho_uniform) {
        // one density: multiply by the reciprocal of the same rounded rho cs2
        const float iR = 1.0f / (p.rho_a * CS2);
        o.ux = vfma(0.5f * CS2, Ftx, jx) * iR;
        o.uy = vfma(0.5f * CS2, Fty, jy) * iR;
    } else {
        o.ux = vdiv(vfma(0.5f * CS2, Ftx, jx), R);
        o.uy = vdiv(vfma(0.5f * CS2, Fty, jy), R);
    }
    // F_p = -grad psi with psi = P* - rho cs2
    V Fpx = -g.pgx, Fpy = -g.pgy;
    if (!p.rho_uniform) {
        const float drho = CS2 * (p.rho_a - p.rho_b) * p.inv_dphi;
        Fpx = vfma(drho, g.fgx, Fpx);
        Fpy = vfma(drho, g.fgy, Fpy);
    }
    const V G = Fpx * o.ux + Fpy * o.uy;
    o.dP = vfma(0.5f, G, g.dps);  // P = sum g + sigma_00 / 2
    if (do_collide) {
        FlowMacroT<V> m;
        m.ux = o.ux;
        m.uy = o.uy;
        m.rho = rho;
        m.dPs = g.dps;
        m.dP = o.dP;
        m.Ftx = Ftx;
        m.Fty = Fty;
        m.Fpx = Fpx;
        m.Fpy = Fpy;
        m.w_nu = p.nu_uniform ? vsplat<V>(p.w_nu) : rate_from_coeff(lerp_phase(p, g.phi, p.nu_a, p.nu_b));
        collide_flow(gg, m, p.w_zeta, out_scale);
        wall_correct_flow(gg, p, j, rho, out_scale);
    }
    return o;
}

// Scalar part of one cell's collisions: f (Sec. 3, App. C) and h (Sec. 2.2)
// given the velocity; f and h enter as their first moments (the zeroth
// moments are phi and c) and leave in deviation form df, dh (q = 1..8).
template <class V, class VI>
__device__ __forceinline__ void collide_scalars_cell(const KParams& p, VI phi_fx, V phi, V c, V nx,
                                                     V ny, V ux, V uy, V fjx, V fjy, V hjx, V hjy,
                                                     V df[9], V dh[9], float sf = 1.0f,
                                                     float sh = 1.0f) {
    // Eq. (theta) and the theta_c of Eq. (ISS)
    V theta, theta_c;
    interface_coeffs(p, phi_fx, c, theta, theta_c);
    const V mt = p.M_phi * theta, dt = p.D_s * theta_c;
    collide_scalar_dev(phi, fjx, fjy, mt * nx, mt * ny, p.w_kappa, ux, uy, df, sf);
    collide_scalar_dev(c, hjx, hjy, dt * nx, dt * ny, p.w_chi, ux, uy, dh, sh);
}

// The same two collisions of one cell with f and h as the two lanes of the
// packed FP32 instructions (they share the velocity and the whole sequence of
// operations); df[q] and dh[q] as above.
__device__ __forceinline__ void collide_scalars_pair(const KParams& p, int phi_fx, float phi,
                                                     float c, float nx, float ny, float ux,
                                                     float uy, f2 fj_x, f2 fj_y, float df[9],
                                                     float dh[9], float sf = 1.0f,
                                                     float sh = 1.0f) {
    float theta, theta_c;
    interface_coeffs(p, phi_fx, c, theta, theta_c);
    const f2 coef(p.M_phi * theta, p.D_s * theta_c);
    f2 d[9];
    collide_scalar_dev(f2(phi, c), fj_x, fj_y, coef * nx, coef * ny, f2(p.w_kappa, p.w_chi),
                       f2(ux), f2(uy), d, f2(sf, sh));
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        df[q] = d[q].x;
        dh[q] = d[q].y;
    }
}

// The three collisions of one cell at row j.  f and h enter as their first
// moments (the zeroth moments are g.phi and g.c) and leave as deviation-form
// outputs df, dh (q = 1..8); the flow populations gg are collided in place.
template <bool COUPLED>
__device__ __forceinline__ CellOut collide_cell(const KParams& p, const CellGeom& g, int j,
                                                float ux_fixed, float uy_fixed, float fjx,
                                                float fjy, float hjx, float hjy, float gg[9],
                                                float df[9], float dh[9], bool do_collide) {
    CellOut o;
    if (COUPLED) {
        o = collide_flow_cell(p, g, j, gg, do_collide);
    } else {
        o.ux = ux_fixed;
        o.uy = uy_fixed;
        o.dP = 0.0f;
    }
    if (do_collide)
        collide_scalars_cell(p, g.phi_fx, g.phi, g.c, g.nx, g.ny, o.ux, o.uy, fjx, fjy, hjx, hjy,
                             df, dh);
    return o;
}

// Offsets of the periodic ghost copies of column i: columns below XGHOST are
// mirrored to the right ghosts (i + nx), columns from nx - XGHOST to the left
// ghosts (i - nx); on grids narrower than 2 XGHOST a column has both.
__device__ __forceinline__ int ghost_right(const KParams& p, int i) { return i < XGHOST ? p.nx : 0; }
__device__ __forceinline__ int ghost_left(const KParams& p, int i) {
    return i >= p.nx - XGHOST ? -p.nx : 0;
}

// Store a deviation-form lattice: plane 0 <- S (fixed point), planes 1..8 <- d;
// edge columns also refresh their ghost copies.
__device__ __forceinline__ void store_dev(float* __restrict__ base, const KParams& p, int64_t idx,
                                          int i, int s_fx, const float d[9]) {
    const int gs[2] = {ghost_right(p, i), ghost_left(p, i)};
    base[idx] = __int_as_float(s_fx);
#pragma unroll
    for (int q = 1; q < 9; ++q) base[q * p.plane + idx] = d[q];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!gs[k]) continue;
        base[idx + gs[k]] = __int_as_float(s_fx);
#pragma unroll
        for (int q = 1; q < 9; ++q) base[q * p.plane + idx + gs[k]] = d[q];
    }
}

__device__ __forceinline__ void store9(float* __restrict__ base, const KParams& p, int64_t idx,
                                       int i, const float a[9]) {
    const int gs[2] = {ghost_right(p, i), ghost_left(p, i)};
#pragma unroll
    for (int q = 0; q < 9; ++q) base[q * p.plane + idx] = a[q];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!gs[k]) continue;
#pragma unroll
        for (int q = 0; q < 9; ++q) base[q * p.plane + idx + gs[k]] = a[q];
    }
}

// Plain store for scratch buffers (no ghost copy).
__device__ __forceinline__ void store9_plain(float* __restrict__ base, const KParams& p,
                                             int64_t idx, const float a[9]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) base[q * p.plane + idx] = a[q];
}

}  // namespace lbm
