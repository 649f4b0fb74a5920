// sm_103a kernels of the coupled central-moment LBM step (arXiv 2504.09024).
//
//  * k_fused_sweep  -- the hot path: one launch per time step.  Each block owns
//    a strip of columns (plus a 2-column halo) and sweeps down a segment of
//    rows.  Per row it pulls the three lattices, forms phi, c, sigma(c) and
//    P* into shared-memory row rings, computes the unit normal one row behind,
//    and collides two rows behind with the curvature, Marangoni and pressure
//    stencils read from the rings.  Populations are read once per cell (plus
//    the halo columns and the segment ends) and written once.
//  * k_fields / k_normals / k_collide -- the same step as a three-kernel chain
//    with the fields materialised in global memory; used as a cross-check, for
//    the macroscopic outputs and for initialisation.
//  * initialisation, population import/export and FP64 reductions.
#include <cmath>

#include "lbm_cell.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// three-kernel chain
// ---------------------------------------------------------------------------

template <bool COUPLED>
__global__ void k_fields(KParams p, const float* __restrict__ src, float* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    const uint32_t bits = moment_bits(step_seed(p), i, j, p.nx);
    ScalarMoments m = pull_scalar(src, p, 0, i, j);
    F[FP_PHI * p.plane + idx] = __int_as_float(fx_add_sr(m.s0, m.inc, p.fx_scale[0], bits));
    m = pull_scalar(src + 9 * p.plane, p, 1, i, j);
    const int c_fx = fx_add_sr(m.s0, m.inc, p.fx_scale[1], second_bits(bits));
    F[FP_C * p.plane + idx] = __int_as_float(c_fx);
    F[FP_SIG * p.plane + idx] = sigma_of_c(p, (float)c_fx * p.fx_inv[1]);
    if (COUPLED) {
        float a[9];
        pull9(src + 18 * p.plane, p, i, j, a);
        F[FP_DPS * p.plane + idx] = sum9(a);
    }
}

__global__ void k_normals(KParams p, float* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    int v[3][3];
    load3x3_fx(F + FP_PHI * p.plane, p, i, j, v);
    float gx, gy, nx, ny, gm;
    iso_grad_fx(v, p.fx_inv[0], gx, gy);
    unit_normal(gx, gy, nx, ny, gm);
    F[FP_NX * p.plane + idx] = nx;
    F[FP_NY * p.plane + idx] = ny;
    F[FP_GM * p.plane + idx] = gm;
}

template <bool COUPLED>
__device__ __forceinline__ CellGeom gather_geom(const KParams& p, const float* __restrict__ F, int i,
                                                int j) {
    const int64_t idx = (int64_t)j * p.pitch + i;
    CellGeom g;
    g.phi_fx = __float_as_int(F[FP_PHI * p.plane + idx]);
    g.phi = (float)g.phi_fx * p.fx_inv[0];
    g.c = (float)__float_as_int(F[FP_C * p.plane + idx]) * p.fx_inv[1];
    g.nx = F[FP_NX * p.plane + idx];
    g.ny = F[FP_NY * p.plane + idx];
    g.gm = F[FP_GM * p.plane + idx];
    g.sig = F[FP_SIG * p.plane + idx];
    if (COUPLED) {
        g.dps = F[FP_DPS * p.plane + idx];
        float vx[3][3], vy[3][3], v[3][3];
        load3x3(F + FP_NX * p.plane, p, i, j, vx);
        load3x3(F + FP_NY * p.plane, p, i, j, vy, true);
        g.kappa = iso_div(vx, vy);
        load3x3(F + FP_SIG * p.plane, p, i, j, v);
        iso_grad(v, g.sgx, g.sgy);
        load3x3(F + FP_DPS * p.plane, p, i, j, v);
        iso_grad(v, g.pgx, g.pgy);
        if (!p.rho_uniform) {
            int vi[3][3];
            load3x3_fx(F + FP_PHI * p.plane, p, i, j, vi);
            iso_grad_fx(vi, p.fx_inv[0], g.fgx, g.fgy);
        } else {
            g.fgx = g.fgy = 0.0f;
        }
    } else {
        g.dps = 0.0f;
        g.kappa = g.sgx = g.sgy = g.pgx = g.pgy = g.fgx = g.fgy = 0.0f;
    }
    return g;
}

template <bool COUPLED>
__global__ void k_collide(KParams p, const float* __restrict__ src, float* __restrict__ dst,
                          const float* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    CellGeom g = gather_geom<COUPLED>(p, F, i, j);
    const ScalarMoments mf = pull_scalar(src, p, 0, i, j);
    const ScalarMoments mh = pull_scalar(src + 9 * p.plane, p, 1, i, j);
    const uint32_t bits = moment_bits(step_seed(p), i, j, p.nx);
    const int f_fx = fx_add_sr(mf.s0, mf.inc, p.fx_scale[0], bits);
    const int h_fx = fx_add_sr(mh.s0, mh.inc, p.fx_scale[1], second_bits(bits));
    float gg[9], df[9], dh[9];
    float ufx = 0.0f, ufy = 0.0f;
    if (COUPLED) {
        pull9(src + 18 * p.plane, p, i, j, gg);
    } else {
        ufx = F[FP_UX * p.plane + idx];
        ufy = F[FP_UY * p.plane + idx];
    }
    collide_cell<COUPLED>(p, g, j, ufx, ufy, mf.jx, mf.jy, mh.jx, mh.jy, gg, df, dh, true);
    store_dev(dst, p, idx, i, f_fx, df);
    store_dev(dst + 9 * p.plane, p, idx, i, h_fx, dh);
    if (COUPLED) store9(dst + 18 * p.plane, p, idx, i, gg);
}

template <bool COUPLED>
__global__ void k_macro_out(KParams p, const float* __restrict__ src, const float* __restrict__ F,
                            double* __restrict__ ophi, double* __restrict__ oc,
                            double* __restrict__ oux, double* __restrict__ ouy,
                            double* __restrict__ oP) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    const int64_t o = (int64_t)j * p.nx + i;
    CellGeom g = gather_geom<COUPLED>(p, F, i, j);
    float gg[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    float ufx = 0.0f, ufy = 0.0f;
    if (COUPLED) {
        pull9(src + 18 * p.plane, p, i, j, gg);
    } else {
        ufx = F[FP_UX * p.plane + idx];
        ufy = F[FP_UY * p.plane + idx];
    }
    CellOut r = collide_cell<COUPLED>(p, g, j, ufx, ufy, 0.0f, 0.0f, 0.0f, 0.0f, gg, nullptr,
                                      nullptr, false);
    if (ophi) ophi[o] = fx_to_double(g.phi_fx, p.fx_scale[0]);
    if (oc) oc[o] = fx_to_double(__float_as_int(F[FP_C * p.plane + idx]), p.fx_scale[1]);
    if (oux) oux[o] = r.ux;
    if (ouy) ouy[o] = r.uy;
    if (oP) oP[o] = COUPLED ? (double)p.P0 + (double)r.dP : 0.0;
}

// ---------------------------------------------------------------------------
// fused sweep kernel
// ---------------------------------------------------------------------------

constexpr int RING = 5;    // rows kept of phi, c, sigma, P* (current row and four behind)
constexpr int NRING = 3;   // rows kept of n and |grad phi|
constexpr int PRING = 3;   // rows of interior cells waiting for their collision
constexpr int PSLOT = 15;  // per waiting cell: f (jx, jy), h (S, jx, jy), g (9 populations)

size_t fused_smem_bytes(int bx) {
    return sizeof(float) * (size_t)bx * (4 * RING + 3 * NRING + PSLOT * PRING);
}

// Block = bx threads = bx - 4 interior columns plus two halo columns each side.
// Rows [y0, y1) are collided; rows y0-2 .. y1+1 are streamed for phi and rows
// y0-1 .. y1 for c, sigma and P* (ghost rows beyond walls hold the mirrored
// values, so the stencils there reproduce the mirrored extended field).
template <bool COUPLED>
__global__ void __launch_bounds__(128) k_fused_sweep(KParams p, const float* __restrict__ src,
                                                     float* __restrict__ dst,
                                                     const float* __restrict__ F, int seg) {
    extern __shared__ float sm[];
    const int bx = blockDim.x;
    const int t = threadIdx.x;
    int* s_phi = reinterpret_cast<int*>(sm);  // [RING][bx] phi, fixed point
    float* s_c = sm + RING * bx;
    float* s_sig = s_c + RING * bx;
    float* s_dps = s_sig + RING * bx;
    float* s_nx = s_dps + RING * bx;         // [NRING][bx]
    float* s_ny = s_nx + NRING * bx;
    float* s_gm = s_ny + NRING * bx;
    float* s_pop = s_gm + NRING * bx;        // [PRING][PSLOT][bx]

    const int tx = bx - 4;
    const int x0 = blockIdx.x * tx;
    const int xend = min(x0 + tx, p.nx);
    const int y0 = blockIdx.y * seg;
    const int y1 = min(y0 + seg, p.ny);
    const int col = x0 - 2 + t;
    // role: 3 interior, 2 first halo column, 1 second halo column, 0 idle
    int role = 0;
    if (col >= x0 && col < xend) role = 3;
    else if (col == x0 - 1 || col == xend) role = 2;
    else if (col == x0 - 2 || col == xend + 1) role = 1;
    const int i = wrap_i(col, p.nx);
    const uint32_t seed = step_seed(p);

    for (int r = y0 - 2; r <= y1 + 1; ++r) {
        // A: stream row r and form its moments
        const int slot = (r + 2 * RING) % RING;
        if (role > 0) {
            const int jj = ext_row(r, p.ny, p.walls);
            const bool keep = role == 3 && r >= y0 && r < y1;
            float* pp = s_pop + ((r + 3 * PRING) % PRING) * PSLOT * bx;
            const uint32_t bits = moment_bits(seed, i, jj, p.nx);
            ScalarMoments m = pull_scalar(src, p, 0, i, jj);
            s_phi[slot * bx + t] = fx_add_sr(m.s0, m.inc, p.fx_scale[0], bits);
            if (keep) {
                pp[0 * bx + t] = m.jx;
                pp[1 * bx + t] = m.jy;
            }
            if (role >= 2 && r >= y0 - 1 && r <= y1) {
                m = pull_scalar(src + 9 * p.plane, p, 1, i, jj);
                const int c_fx = fx_add_sr(m.s0, m.inc, p.fx_scale[1], second_bits(bits));
                const float c = (float)c_fx * p.fx_inv[1];
                s_c[slot * bx + t] = c;
                s_sig[slot * bx + t] = sigma_of_c(p, c);
                if (keep) {
                    pp[2 * bx + t] = __int_as_float(c_fx);
                    pp[3 * bx + t] = m.jx;
                    pp[4 * bx + t] = m.jy;
                }
                if (COUPLED) {
                    float a[9];
                    pull9(src + 18 * p.plane, p, i, jj, a);
                    s_dps[slot * bx + t] = sum9(a);
                    if (keep) {
#pragma unroll
                        for (int q = 0; q < 9; ++q) pp[(6 + q) * bx + t] = a[q];
                    }
                }
            }
        }
        __syncthreads();
        // B: normal at row r-1 (needs phi rows r-2 .. r)
        const int rn = r - 1;
        if (role >= 2 && rn >= y0 - 1 && rn <= y1) {
            const int sm1 = (rn - 1 + 2 * RING) % RING, s0 = (rn + 2 * RING) % RING,
                      sp1 = (rn + 1 + 2 * RING) % RING;
            int v[3][3];
            v[0][0] = s_phi[sm1 * bx + t - 1]; v[0][1] = s_phi[sm1 * bx + t]; v[0][2] = s_phi[sm1 * bx + t + 1];
            v[1][0] = s_phi[s0 * bx + t - 1];  v[1][1] = s_phi[s0 * bx + t];  v[1][2] = s_phi[s0 * bx + t + 1];
            v[2][0] = s_phi[sp1 * bx + t - 1]; v[2][1] = s_phi[sp1 * bx + t]; v[2][2] = s_phi[sp1 * bx + t + 1];
            float gx, gy, nx, ny, gm;
            iso_grad_fx(v, p.fx_inv[0], gx, gy);
            unit_normal(gx, gy, nx, ny, gm);
            const int ns = (rn + 3 * NRING) % NRING;
            s_nx[ns * bx + t] = nx;
            s_ny[ns * bx + t] = ny;
            s_gm[ns * bx + t] = gm;
        }
        __syncthreads();
        // C: collide row r-2
        const int jc = r - 2;
        if (role == 3 && jc >= y0 && jc < y1) {
            const int cm1 = (jc - 1 + 2 * RING) % RING, c0 = (jc + 2 * RING) % RING,
                      cp1 = (jc + 1 + 2 * RING) % RING;
            const int nm1 = (jc - 1 + 3 * NRING) % NRING, n0 = (jc + 3 * NRING) % NRING,
                      np1 = (jc + 1 + 3 * NRING) % NRING;
            CellGeom g;
            g.phi_fx = s_phi[c0 * bx + t];
            g.phi = (float)g.phi_fx * p.fx_inv[0];
            g.c = s_c[c0 * bx + t];
            g.sig = s_sig[c0 * bx + t];
            g.nx = s_nx[n0 * bx + t];
            g.ny = s_ny[n0 * bx + t];
            g.gm = s_gm[n0 * bx + t];
            if (COUPLED) {
                g.dps = s_dps[c0 * bx + t];
                float vx[3][3], vy[3][3], v[3][3];
                const int nr[3] = {nm1, n0, np1};
                const int cr[3] = {cm1, c0, cp1};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        vx[d][e] = s_nx[nr[d] * bx + t - 1 + e];
                        vy[d][e] = s_ny[nr[d] * bx + t - 1 + e];
                    }
                }
                g.kappa = iso_div(vx, vy);
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int e = 0; e < 3; ++e) v[d][e] = s_sig[cr[d] * bx + t - 1 + e];
                iso_grad(v, g.sgx, g.sgy);
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int e = 0; e < 3; ++e) v[d][e] = s_dps[cr[d] * bx + t - 1 + e];
                iso_grad(v, g.pgx, g.pgy);
                if (!p.rho_uniform) {
                    int vi[3][3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int e = 0; e < 3; ++e) vi[d][e] = s_phi[cr[d] * bx + t - 1 + e];
                    iso_grad_fx(vi, p.fx_inv[0], g.fgx, g.fgy);
                } else {
                    g.fgx = g.fgy = 0.0f;
                }
            } else {
                g.dps = 0.0f;
                g.kappa = g.sgx = g.sgy = g.pgx = g.pgy = g.fgx = g.fgy = 0.0f;
            }
            const float* pp = s_pop + ((jc + 3 * PRING) % PRING) * PSLOT * bx;
            const float fjx = pp[0 * bx + t], fjy = pp[1 * bx + t];
            const int h_fx = __float_as_int(pp[2 * bx + t]);
            const float hjx = pp[3 * bx + t], hjy = pp[4 * bx + t];
            float gg[9], df[9], dh[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) gg[q] = COUPLED ? pp[(6 + q) * bx + t] : 0.0f;
            const int64_t idx = (int64_t)jc * p.pitch + i;
            float ufx = 0.0f, ufy = 0.0f;
            if (!COUPLED) {
                ufx = F[FP_UX * p.plane + idx];
                ufy = F[FP_UY * p.plane + idx];
            }
            collide_cell<COUPLED>(p, g, jc, ufx, ufy, fjx, fjy, hjx, hjy, gg, df, dh, true);
            store_dev(dst, p, idx, i, g.phi_fx, df);
            store_dev(dst + 9 * p.plane, p, idx, i, h_fx, dh);
            if (COUPLED) store9(dst + 18 * p.plane, p, idx, i, gg);
        }
    }
}

// ---------------------------------------------------------------------------
// initialisation and population import / export
// ---------------------------------------------------------------------------

__global__ void k_init_fields(KParams p, const double* __restrict__ phi,
                              const double* __restrict__ c, const double* __restrict__ ux,
                              const double* __restrict__ uy, const double* __restrict__ P,
                              float* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    const int64_t o = (int64_t)j * p.nx + i;
    const float fphi = (float)phi[o];
    const float fc = (float)c[o];
    F[FP_PHI * p.plane + idx] = __int_as_float(fx_from_double(phi[o], p.fx_scale[0]));
    F[FP_C * p.plane + idx] = __int_as_float(fx_from_double(c[o], p.fx_scale[1]));
    F[FP_SIG * p.plane + idx] = sigma_of_c(p, fc);
    F[FP_UX * p.plane + idx] = (float)ux[o];
    F[FP_UY * p.plane + idx] = (float)uy[o];
    // default pressure: uniform, the rest pressure P0 = cs2 (rho_a + rho_b) / 2
    // (with equal densities, rho cs2 everywhere)
    const double Pv = P ? P[o] : (double)p.P0;
    F[FP_DPS * p.plane + idx] = (float)(Pv - (double)p.P0);
}

// Equilibrium post-streaming populations into `pre` (dense-pitched [nlat*9]).
template <bool COUPLED>
__global__ void k_init_pre(KParams p, const float* __restrict__ F, float* __restrict__ pre) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    const int phi_fx = __float_as_int(F[FP_PHI * p.plane + idx]);
    const float phi = (float)phi_fx * p.fx_inv[0];
    const float c = (float)__float_as_int(F[FP_C * p.plane + idx]) * p.fx_inv[1];
    const float nx = F[FP_NX * p.plane + idx];
    const float ny = F[FP_NY * p.plane + idx];
    const float ux = F[FP_UX * p.plane + idx];
    const float uy = F[FP_UY * p.plane + idx];
    float theta, theta_c;
    interface_coeffs(p, phi_fx, c, theta, theta_c);
    float a[9];
    eq_scalar(a, phi, p.M_phi * theta * nx, p.M_phi * theta * ny, ux, uy);
    store9_plain(pre, p, idx, a);
    eq_scalar(a, c, p.D_s * theta_c * nx, p.D_s * theta_c * ny, ux, uy);
    store9_plain(pre + 9 * p.plane, p, idx, a);
    if (COUPLED) {
        const float rho = p.rho_uniform ? p.rho_a : lerp_phase(p, phi, p.rho_a, p.rho_b);
        eq_flow_shifted(a, F[FP_DPS * p.plane + idx], rho, ux, uy);
        store9_plain(pre + 18 * p.plane, p, idx, a);
    }
}

// Stored (post-collision, pull-ready) form from post-streaming populations:
// slot q at y is read by the pull of cell y + e_q, or, when y + e_q lies
// beyond a wall, by the bounce-back of direction opp(q) at y.  The two
// advection-diffusion lattices are then written in deviation form
// (S = sum of the slots, d_q = slot_q - w_q S); the flow lattice as is.
__global__ void k_unstream(KParams p, int nlat, const float* __restrict__ pre,
                           float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    for (int l = 0; l < nlat; ++l) {
        const float* pl = pre + (int64_t)l * 9 * p.plane;
        float* dl = dst + (int64_t)l * 9 * p.plane;
        float u[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int ti = wrap_i(i + ex(q), p.nx);
            const int tj = j + ey(q);
            if (p.walls && (tj < 0 || tj >= p.ny)) {
                u[q] = pl[opp(q) * p.plane + idx];
            } else {
                u[q] = pl[q * p.plane + (int64_t)wrap_i(tj, p.ny) * p.pitch + ti];
            }
        }
        if (l < 2) {
            double S = 0.0;
#pragma unroll
            for (int q = 0; q < 9; ++q) S += (double)u[q];
            const int S_fx = fx_from_double(S, p.fx_scale[l]);
            const double Sr = fx_to_double(S_fx, p.fx_scale[l]);
            float d[9];
#pragma unroll
            for (int q = 1; q < 9; ++q) d[q] = (float)((double)u[q] - (double)wq(q) * Sr);
            store_dev(dl, p, idx, i, S_fx, d);
        } else {
            store9(dl, p, idx, i, u);
        }
    }
}

// Post-streaming populations of the stored state, into a pitched float buffer.
__global__ void k_pull_pre(KParams p, int nlat, const float* __restrict__ src,
                           float* __restrict__ pre) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    for (int l = 0; l < nlat; ++l) {
        float a[9];
        if (l < 2)
            pull9_dev<float>(src + (int64_t)l * 9 * p.plane, p, l, i, j, a);
        else
            pull9(src + (int64_t)l * 9 * p.plane, p, i, j, a);
        store9_plain(pre + (int64_t)l * 9 * p.plane, p, idx, a);
    }
}

// Post-streaming populations as float64 dense [nlat*9][ny][nx], unshifted.
__global__ void k_export_pops(KParams p, int nlat, const float* __restrict__ src,
                              double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t n = (int64_t)p.nx * p.ny;
    const int64_t o = (int64_t)j * p.nx + i;
    for (int l = 0; l < nlat; ++l) {
        double a[9];
        if (l < 2) {
            pull9_dev<double>(src + (int64_t)l * 9 * p.plane, p, l, i, j, a);
        } else {
            float b[9];
            pull9(src + (int64_t)l * 9 * p.plane, p, i, j, b);
#pragma unroll
            for (int q = 0; q < 9; ++q) a[q] = (double)b[q] + (double)wq(q) * (double)p.P0;
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) out[(l * 9 + q) * n + o] = a[q];
    }
}

// One lattice of float64 dense post-streaming populations into the pitched
// float pre-form (flow lattice shifted by w P0).
__global__ void k_f64_to_pre(KParams p, int lat, const double* __restrict__ in,
                             float* __restrict__ pre) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int64_t idx = (int64_t)j * p.pitch + i;
    const int64_t n = (int64_t)p.nx * p.ny;
    const int64_t o = (int64_t)j * p.nx + i;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double v = in[q * n + o];
        if (lat == 2) v -= (double)wq(q) * (double)p.P0;
        pre[(lat * 9 + q) * p.plane + idx] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// FP64 reductions (fixed order: per-block partials, one finishing block)
// ---------------------------------------------------------------------------

constexpr int DIAG_THREADS = 256;
constexpr double TWO_PI = 6.283185307179586476925286766559;

__device__ __forceinline__ bool finite_cell(double a, double b, double c, double d) {
    return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
}

template <int NS>
__device__ void block_sum(double (&v)[NS], double* partial_out) {
    __shared__ double red[NS][DIAG_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) {
            double s = 0.0;
            for (int q = 0; q < DIAG_THREADS / 32; ++q) s += red[k][q];
            partial_out[k] = s;
        }
    }
}

// Drop indicator: (phi - phi_b) / (phi_a - phi_b) clipped to [0, 1].  The
// shape moments (centroid, Ixx, Iyy, Ixy; D = (L - B) / (L + B) of Sec. 4.3)
// belong to the drop region: the clip keeps the small over- and undershoot of
// phi away from the interface, which its distance would weigh heavily, out.
__device__ __forceinline__ double drop_indicator(const KParams& p, double phi) {
    const double w = (phi - (double)p.phi_b) / ((double)p.phi_a - (double)p.phi_b);
    return fmin(fmax(w, 0.0), 1.0);
}

// Pass 1 sums: phi, c, w cos/sin(2 pi x / nx), w cos/sin(2 pi y / ny), w y,
// nonfinite count, sigma<0 count, max |u| (as max), w (w: drop indicator).
constexpr int DIAG_SW = 10;  // slot of sum w; after pass 1, block 0's slot holds the total
__global__ void k_diag1(KParams p, const double* __restrict__ phi, const double* __restrict__ c,
                        const double* __restrict__ ux, const double* __restrict__ uy,
                        double* __restrict__ partial) {
    double v[DIAG_NSUM];
    for (int k = 0; k < DIAG_NSUM; ++k) v[k] = 0.0;
    double umax = 0.0;
    const int64_t n = (int64_t)p.nx * p.ny;
    for (int64_t o = (int64_t)blockIdx.x * DIAG_THREADS + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * DIAG_THREADS) {
        const int i = (int)(o % p.nx), j = (int)(o / p.nx);
        const double f = phi[o], cc = c[o], a = ux[o], b = uy[o];
        if (!finite_cell(f, cc, a, b)) {
            v[7] += 1.0;
            continue;
        }
        const double ax = TWO_PI * (i + 0.5) / p.nx, ay = TWO_PI * (j + 0.5) / p.ny;
        const double w = drop_indicator(p, f);
        v[0] += f;
        v[1] += cc;
        v[2] += w * cos(ax);
        v[3] += w * sin(ax);
        v[4] += w * cos(ay);
        v[5] += w * sin(ay);
        v[6] += w * (j + 0.5);
        v[DIAG_SW] += w;
        const double arg = 1.0 - cc * (double)p.inv_cmax;
        if (p.beta != 0.0f && (arg <= 0.0 || 1.0 + (double)p.beta * log(arg) < 0.0)) v[8] += 1.0;
        umax = fmax(umax, sqrt(a * a + b * b));
    }
    for (int o = 16; o > 0; o >>= 1) umax = fmax(umax, __shfl_down_sync(0xffffffffu, umax, o));
    __shared__ double smax[DIAG_THREADS / 32];
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = umax;
    block_sum<DIAG_NSUM>(v, partial + (int64_t)blockIdx.x * DIAG_NSUM);
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int q = 0; q < DIAG_THREADS / 32; ++q) m = fmax(m, smax[q]);
        partial[(int64_t)blockIdx.x * DIAG_NSUM + 9] = m;
    }
}

// result layout: [0] sum_phi [1] sum_c [2] xc [3] yc [4] nonfinite [5] sigma_neg [6] umax
//                [7] Ixx [8] Iyy [9] Ixy [10] L [11] B [12] D
// Sums over the nb partial rows (slot 9 by max instead when MAX9) by one
// block of DIAG_FINISH threads: thread t adds rows t, t + DIAG_FINISH, ... in
// order, then a fixed tree over the threads, so the result does not depend
// on scheduling.  Thread 0 receives the totals in s.
constexpr int DIAG_FINISH = 256;
template <int NK, bool MAX9>
__device__ __forceinline__ void finish_sums(const double* __restrict__ partial, int nb,
                                            double s[NK]) {
    __shared__ double red[NK][DIAG_FINISH];
    for (int k = 0; k < NK; ++k) s[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += DIAG_FINISH)
        for (int k = 0; k < NK; ++k) {
            const double v = partial[(int64_t)b * DIAG_NSUM + k];
            s[k] = (MAX9 && k == 9) ? fmax(s[k], v) : s[k] + v;
        }
    for (int k = 0; k < NK; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = DIAG_FINISH / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < NK; ++k)
                red[k][threadIdx.x] = (MAX9 && k == 9)
                                          ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + w])
                                          : red[k][threadIdx.x] + red[k][threadIdx.x + w];
        __syncthreads();
    }
    for (int k = 0; k < NK; ++k) s[k] = red[k][0];
}

__global__ void __launch_bounds__(DIAG_FINISH) k_diag_finish1(KParams p, double* __restrict__ partial,
                                                              int nb, double* __restrict__ res) {
    double s[DIAG_NSUM];
    finish_sums<DIAG_NSUM, true>(partial, nb, s);
    if (threadIdx.x != 0) return;
    const double m = s[9];
    res[0] = s[0];
    res[1] = s[1];
    double xc = 0.5 * p.nx, yc = 0.5 * p.ny;
    if (s[DIAG_SW] != 0.0) {
        double ax = atan2(s[3], s[2]);
        if (ax < 0) ax += TWO_PI;
        xc = ax * p.nx / TWO_PI;
        if (p.walls) {
            yc = s[6] / s[DIAG_SW];
        } else {
            double ay = atan2(s[5], s[4]);
            if (ay < 0) ay += TWO_PI;
            yc = ay * p.ny / TWO_PI;
        }
    }
    res[2] = xc;
    res[3] = yc;
    res[4] = s[7];
    res[5] = s[8];
    res[6] = m;
    // the normalisation of pass 2 (the result array has no free slot)
    partial[DIAG_SW] = s[DIAG_SW];
}

__device__ __forceinline__ double min_image(double d, int n, bool periodic) {
    if (!periodic) return d;
    while (d >= 0.5 * n) d -= n;
    while (d < -0.5 * n) d += n;
    return d;
}

__global__ void k_diag2(KParams p, const double* __restrict__ phi, const double* __restrict__ c,
                        const double* __restrict__ ux, const double* __restrict__ uy,
                        const double* __restrict__ res, double* __restrict__ partial) {
    double v[3] = {0.0, 0.0, 0.0};
    const double xc = res[2], yc = res[3];
    const int64_t n = (int64_t)p.nx * p.ny;
    for (int64_t o = (int64_t)blockIdx.x * DIAG_THREADS + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * DIAG_THREADS) {
        const int i = (int)(o % p.nx), j = (int)(o / p.nx);
        const double f = phi[o];
        if (!finite_cell(f, c[o], ux[o], uy[o])) continue;
        const double dx = min_image(i + 0.5 - xc, p.nx, true);
        const double dy = min_image(j + 0.5 - yc, p.ny, !p.walls);
        const double w = drop_indicator(p, f);
        v[0] += w * dx * dx;
        v[1] += w * dy * dy;
        v[2] += w * dx * dy;
    }
    block_sum<3>(v, partial + (int64_t)blockIdx.x * DIAG_NSUM);
}

__global__ void __launch_bounds__(DIAG_FINISH) k_diag_finish2(const double* __restrict__ partial,
                                                              int nb, double* __restrict__ res) {
    double I[3];
    finish_sums<3, false>(partial, nb, I);
    if (threadIdx.x != 0) return;
    const double s0 = partial[DIAG_SW];  // sum of the drop indicator (pass 1)
    if (s0 != 0.0)
        for (int k = 0; k < 3; ++k) I[k] /= s0;
    const double tr = I[0] + I[1], det = I[0] * I[1] - I[2] * I[2];
    const double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
    const double l1 = 0.5 * tr + disc, l2 = fmax(0.5 * tr - disc, 0.0);
    const double L = 4.0 * sqrt(l1), B = 4.0 * sqrt(l2);
    res[7] = I[0];
    res[8] = I[1];
    res[9] = I[2];
    res[10] = L;
    res[11] = B;
    res[12] = (L + B) > 0.0 ? (L - B) / (L + B) : 0.0;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static dim3 row_grid(const KParams& p, int bx) { return dim3((p.nx + bx - 1) / bx, p.ny); }

void launch_fields(const KParams& p, const DevState& s, int src, cudaStream_t st) {
    const int bx = 128;
    if (p.coupled)
        k_fields<true><<<row_grid(p, bx), bx, 0, st>>>(p, s.pop[src], s.fields);
    else
        k_fields<false><<<row_grid(p, bx), bx, 0, st>>>(p, s.pop[src], s.fields);
    k_normals<<<row_grid(p, bx), bx, 0, st>>>(p, s.fields);
}

void launch_step_split(const KParams& p, const DevState& s, int src, cudaStream_t st) {
    launch_fields(p, s, src, st);
    const int bx = 128;
    if (p.coupled)
        k_collide<true><<<row_grid(p, bx), bx, 0, st>>>(p, s.pop[src], s.pop[1 - src], s.fields);
    else
        k_collide<false><<<row_grid(p, bx), bx, 0, st>>>(p, s.pop[src], s.pop[1 - src], s.fields);
}

void launch_step_fused(const KParams& p, const DevState& s, int src, const FusedShape& sh,
                       cudaStream_t st) {
    const int tx = sh.bx - 4;
    dim3 grid((p.nx + tx - 1) / tx, (p.ny + sh.seg - 1) / sh.seg);
    const size_t smem = fused_smem_bytes(sh.bx);
    if (p.coupled)
        k_fused_sweep<true><<<grid, sh.bx, smem, st>>>(p, s.pop[src], s.pop[1 - src], s.fields,
                                                      sh.seg);
    else
        k_fused_sweep<false><<<grid, sh.bx, smem, st>>>(p, s.pop[src], s.pop[1 - src], s.fields,
                                                       sh.seg);
}

cudaError_t configure_fused_smem() {
    const int maxb = (int)fused_smem_bytes(128);
    cudaError_t e = cudaFuncSetAttribute(k_fused_sweep<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fused_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                maxb);
}

void launch_macro_out(const KParams& p, const DevState& s, int src, double* phi, double* c,
                      double* ux, double* uy, double* P, cudaStream_t st) {
    const int bx = 128;
    if (p.coupled)
        k_macro_out<true><<<row_grid(p, bx), bx, 0, st>>>(p, s.pop[src], s.fields, phi, c, ux, uy, P);
    else
        k_macro_out<false><<<row_grid(p, bx), bx, 0, st>>>(p, s.pop[src], s.fields, phi, c, ux, uy, P);
}

void launch_init(const KParams& p, const DevState& s, int dst, const double* phi,
                 const double* c, const double* ux, const double* uy, const double* P,
                 cudaStream_t st) {
    const int bx = 128;
    k_init_fields<<<row_grid(p, bx), bx, 0, st>>>(p, phi, c, ux, uy, P, s.fields);
    k_normals<<<row_grid(p, bx), bx, 0, st>>>(p, s.fields);
    float* tmp = s.pop[1 - dst];
    if (p.coupled)
        k_init_pre<true><<<row_grid(p, bx), bx, 0, st>>>(p, s.fields, tmp);
    else
        k_init_pre<false><<<row_grid(p, bx), bx, 0, st>>>(p, s.fields, tmp);
    k_unstream<<<row_grid(p, bx), bx, 0, st>>>(p, s.nlat, tmp, s.pop[dst]);
}

void launch_get_pops(const KParams& p, const DevState& s, int src, double* out, cudaStream_t st) {
    const int bx = 128;
    k_export_pops<<<row_grid(p, bx), bx, 0, st>>>(p, s.nlat, s.pop[src], out);
}

void launch_set_pops(const KParams& p, const DevState& s, int dst, const double* f,
                     const double* h, const double* g, cudaStream_t st) {
    const int bx = 128;
    float* tmp = s.pop[1 - dst];
    k_pull_pre<<<row_grid(p, bx), bx, 0, st>>>(p, s.nlat, s.pop[dst], tmp);
    const double* in[3] = {f, h, g};
    for (int l = 0; l < s.nlat; ++l)
        if (in[l]) k_f64_to_pre<<<row_grid(p, bx), bx, 0, st>>>(p, l, in[l], tmp);
    k_unstream<<<row_grid(p, bx), bx, 0, st>>>(p, s.nlat, tmp, s.pop[dst]);
}

int diag_blocks(const KParams& p) {
    const int64_t n = (int64_t)p.nx * p.ny;
    int64_t b = (n + DIAG_THREADS * 8 - 1) / (DIAG_THREADS * 8);
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

void launch_diag(const KParams& p, const double* phi, const double* c, const double* ux,
                 const double* uy, double* partial, int nb, double* result, cudaStream_t st) {
    k_diag1<<<nb, DIAG_THREADS, 0, st>>>(p, phi, c, ux, uy, partial);
    k_diag_finish1<<<1, DIAG_FINISH, 0, st>>>(p, partial, nb, result);
    k_diag2<<<nb, DIAG_THREADS, 0, st>>>(p, phi, c, ux, uy, result, partial);
    k_diag_finish2<<<1, DIAG_FINISH, 0, st>>>(partial, nb, result);
}

// ---------------------------------------------------------------------------
// 4-connected components of {phi > level}: labels by minimum-index
// propagation with pointer jumping (the label of a cell is the smallest cell
// index reachable inside the set), then a count of the roots.
// ---------------------------------------------------------------------------

__global__ void k_label_init(const KParams p, const float* __restrict__ F, float level,
                             int* __restrict__ label) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)p.nx * p.ny) return;
    const int i = (int)(k % p.nx), j = (int)(k / p.nx);
    // the phi plane holds the fixed-point zeroth moment
    const int phi_fx = __float_as_int(F[FP_PHI * p.plane + (int64_t)j * p.pitch + i]);
    label[k] = (phi_fx != FX_INVALID && (float)phi_fx * p.fx_inv[0] > level) ? (int)k : -1;
}

__global__ void k_label_step(const KParams p, int* __restrict__ label, int* __restrict__ changed) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)p.nx * p.ny) return;
    const int own = label[k];
    if (own < 0) return;
    const int i = (int)(k % p.nx), j = (int)(k / p.nx);
    int m = own;
    const int nb[4][2] = {{wrap_i(i - 1, p.nx), j}, {wrap_i(i + 1, p.nx), j}, {i, j - 1}, {i, j + 1}};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        int jj = nb[d][1];
        if (jj < 0 || jj >= p.ny) {
            if (p.walls) continue;  // no neighbour across a wall
            jj = wrap_i(jj, p.ny);
        }
        const int v = label[(int64_t)jj * p.nx + nb[d][0]];
        if (v >= 0 && v < m) m = v;
    }
    m = min(m, label[m]);  // pointer jumping
    if (m < own) {
        atomicMin(&label[k], m);
        *changed = 1;
    }
}

__global__ void k_label_roots(const KParams p, const int* __restrict__ label, int* __restrict__ count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)p.nx * p.ny) return;
    if (label[k] == (int)k) atomicAdd(count, 1);
}

void launch_label_init(const KParams& p, const float* fields, float level, int* label,
                       cudaStream_t st) {
    const int64_t n = (int64_t)p.nx * p.ny;
    k_label_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, fields, level, label);
}

void launch_label_step(const KParams& p, int* label, int* changed, cudaStream_t st) {
    const int64_t n = (int64_t)p.nx * p.ny;
    k_label_step<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, label, changed);
}

void launch_label_roots(const KParams& p, const int* label, int* count, cudaStream_t st) {
    const int64_t n = (int64_t)p.nx * p.ny;
    k_label_roots<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, label, count);
}

}  // namespace lbm
