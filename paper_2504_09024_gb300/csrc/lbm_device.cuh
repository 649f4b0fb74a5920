// Device-side building blocks of the coupled central-moment LBM step
// (Schupbach & Premnath, arXiv 2504.09024): pull streaming with half-way
// bounce-back, isotropic stencils, the surface-tension force of Eq. (Fs) with
// the Langmuir isotherm of Eq. (EOS), and the three central-moment collisions
// (Sec. 3 Eq. LBE; App. C Eq. LBE_CACE; App. D Eq. centralmomentLBE2fluidflow)
// written out algebraically for FP32 registers.
//
// Storage: post-collision state, SoA planes [lattice][q][ny][pitch], read by a
// pull.  Both advection-diffusion lattices (f, h) are kept in deviation form:
// plane 0 holds the post-collision zeroth moment S (= phi or c) as a 32-bit
// fixed-point integer (resolution 2^-29 for values of order one) and planes
// 1..8 hold FP32 deviations d_q = a~_q - w_q S (the rest deviation is
// -sum d_q).  Fixed point keeps the slow interface dynamics: an FP32 S would
// drop increments below half an ulp every step, and S near phi_a = 1 would
// lose the phi_a - phi that the sharpening flux depends on.  Differences of S
// between neighbours are exact integer subtractions.  The flow lattice is
// stored as g - w_q P0 (P0 = cs2 * reference density) so that FP32 keeps the
// O(u) information of g; every flow-lattice quantity below is a deviation from
// the rest state P0 w.
#pragma once

#include <type_traits>

#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_vec.cuh"

namespace lbm {

constexpr float CS2 = 1.0f / 3.0f;
constexpr float EPS_N = 1e-12f;  // |grad phi| below which n = 0

// D2Q9 in the order of the paper's P matrix (App. A).
__host__ __device__ constexpr int ex(int q) {
    return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int q) {
    return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int q) {
    return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4 + 1) : ((q - 5 + 2) % 4 + 5));
}
__host__ __device__ constexpr float wq(int q) {
    return q == 0 ? 4.0f / 9.0f : (q <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}

// Kernel parameters (float copies of lbm_params plus derived rates).
// Row layout: [XGHOST ghost columns | nx columns | XGHOST ghost columns | pad],
// pitch a multiple of 32 floats.  Kernels receive pointers to column 0; the
// ghost columns -XGHOST..-1 and nx..nx+XGHOST-1 mirror the periodic images and
// let bulk-tensor loads read whole rows without wrapping.
constexpr int XGHOST = 4;

struct KParams {
    int nx, ny, pitch, walls;
    int coupled;
    int nu_uniform, rho_uniform;
    int64_t plane;          // pitch * ny
    float u_wall;
    float W, phi_a, phi_b, phi_m, inv_dphi;
    float M_phi, D_s;
    float w_kappa, w_chi, w_zeta, w_nu;  // w_nu valid when nu_uniform
    float nu_a, nu_b, rho_a, rho_b, rho_ref;
    float sigma_o, beta, inv_cmax;
    float N_sigma;
    float fext_x, fext_y;
    float P0;               // rest pressure of the shifted flow storage
    float four_over_W, eight_over_W;
    // fixed-point zeroth moments: value = S * fx_inv[l] (l = 0: phi, 1: c)
    float fx_scale[2], fx_inv[2];
    int phi_a_fx, phi_b_fx, phi_m_fx;  // phi_a, phi_b, phi_m in phi fixed point
    // 16-bit storage: deviations are stored times qs[l] (powers of two;
    // l = 0: f, 1: h, 2: g), qinv[l] = 1 / qs[l]
    float qs[3], qinv[3];
    // 16-bit storage: step counter for the stochastic rounding (device word
    // holding the step of the launch with step_off 0; see lbm_store16.cuh)
    const unsigned* step_ctr;
    int step_off;
    int stall_test;         // test hook: wait on a barrier nothing completes (bounded)
};

// ---------------------------------------------------------------------------
// index helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int wrap_i(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Row of the extended field: periodic, or mirrored about the wall planes
// (row -1-k is row k, row ny+k is row ny-1-k); valid for -2 <= j <= ny+1.
__device__ __forceinline__ int ext_row(int j, int ny, int walls) {
    if (!walls) return wrap_i(j, ny);
    if (j < 0) return -1 - j;
    if (j >= ny) return 2 * ny - 1 - j;
    return j;
}
// +1 for rows inside or periodic images, -1 for mirrored ghost rows (the
// y component of the normal field changes sign under the mirror).
__device__ __forceinline__ float mirror_sign(int j, int ny, int walls) {
    return (walls && (j < 0 || j >= ny)) ? -1.0f : 1.0f;
}

// ---------------------------------------------------------------------------
// streaming (pull) with half-way bounce-back
// ---------------------------------------------------------------------------

// Gather the 9 post-streaming populations of one cell of a lattice: a_q(x) =
// a~_q(x - e_q).  Rm, R0, Rp point at plane 0 of rows j-1, j, j+1; planes are
// PS elements apart; cm, c0, cp are the columns x-1, x, x+1.  A source beyond
// a wall (bot: j is the bottom row, top: the top row) is replaced by the
// cell's own opposite slot, which the writer has already bounce-back
// corrected.
__device__ __forceinline__ void pull9_rows(const float* __restrict__ Rm,
                                           const float* __restrict__ R0,
                                           const float* __restrict__ Rp, int64_t PS, int cm,
                                           int c0, int cp, bool bot, bool top, float out[9]) {
    out[0] = R0[c0];
    out[1] = R0[1 * PS + cm];
    out[3] = R0[3 * PS + cp];
    if (bot) {
        out[2] = R0[4 * PS + c0];
        out[5] = R0[7 * PS + c0];
        out[6] = R0[8 * PS + c0];
    } else {
        out[2] = Rm[2 * PS + c0];
        out[5] = Rm[5 * PS + cm];
        out[6] = Rm[6 * PS + cp];
    }
    if (top) {
        out[4] = R0[2 * PS + c0];
        out[7] = R0[5 * PS + c0];
        out[8] = R0[6 * PS + c0];
    } else {
        out[4] = Rp[4 * PS + c0];
        out[7] = Rp[7 * PS + cp];
        out[8] = Rp[8 * PS + cm];
    }
}

__device__ __forceinline__ void pull9(const float* __restrict__ base, const KParams& p, int i, int j,
                                      float out[9]) {
    const bool bot = p.walls && j == 0, top = p.walls && j == p.ny - 1;
    const float* R0 = base + (int64_t)j * p.pitch;
    const float* Rm = base + (int64_t)wrap_i(j - 1, p.ny) * p.pitch;
    const float* Rp = base + (int64_t)wrap_i(j + 1, p.ny) * p.pitch;
    pull9_rows(Rm, R0, Rp, p.plane, wrap_i(i - 1, p.nx), i, wrap_i(i + 1, p.nx), bot, top, out);
}

// Zeroth and first moments of the post-streaming populations of a lattice in
// deviation form (plane 0: S, planes 1..8: d_q):
//   a_q(x) = w_q S(x - e_q) + d_q(x - e_q)           (q >= 1, pulled)
//   a_0(x) = w_0 S(x) - sum_{q>=1} d_q(x)            (rest, own cell)
// so that  sum_q a_q(x) = S(x) + inc  with the small increment
//   inc = sum_{q>=1} [w_q (S(x-e_q) - S(x)) + d_q(x-e_q)] - sum_{q>=1} d_q(x)
// and  sum_q e_q a_q(x) = sum_{q>=1} e_q [w_q (S(x-e_q) - S(x)) + d_q(x-e_q)].
// A source beyond a wall is the cell's own opposite slot (bounce-back).
struct ScalarMoments {
    int s0;      // S(x), fixed point
    float inc;   // zeroth moment = s0 * inv_scale + inc
    float jx, jy;
};

__device__ __forceinline__ int fx_load(const float* p) { return __float_as_int(*p); }

// Invalid fixed-point value (the analogue of NaN): produced by non-finite or
// out-of-range increments and kept by every later addition.
constexpr int FX_INVALID = INT_MIN;
constexpr int FX_RANGE = 1 << 30;  // |value| beyond this (twice the bounds) is invalid

// Fixed-point value after adding a float increment.
// An invalid s0 needs no test of its own: INT_MIN plus an increment below
// 1e9 < 2^30 in magnitude lands outside [-FX_RANGE, FX_RANGE] (the sum is
// formed in unsigned arithmetic, so it wraps instead of overflowing).
__device__ __forceinline__ int fx_add(int s0, float inc, float scale) {
    const float v = inc * scale;
    if (!(fabsf(v) < 1.0e9f)) return FX_INVALID;
    const unsigned r = (unsigned)s0 + (unsigned)__float2int_rn(v);
    return r + (unsigned)FX_RANGE > 2u * (unsigned)FX_RANGE ? FX_INVALID : (int)r;
}

// Counter-based hash for the stochastic roundings: the PCG hash of Jarzynski
// and Olano, "Hash Functions for GPU Rendering", JCGT 9(3), 2020 (the output
// permutation of the PCG generator, O'Neill 2014, applied to one LCG step of
// the input).
__device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    const uint32_t state = v * 747796405u + 2891336453u;
    const uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

// Seed of one step's roundings: the step about to be taken is the device
// counter plus the launch's offset within its graph.
__device__ __forceinline__ uint32_t step_seed_at(const KParams& p, int step_off) {
    return pcg_hash((p.step_ctr ? __ldg(p.step_ctr) : 0u) + (uint32_t)step_off);
}
__device__ __forceinline__ uint32_t step_seed(const KParams& p) { return step_seed_at(p, p.step_off); }

// Random bits of cell (i, j) in one step: the PCG hash of the step's hash
// offset by a Weyl sequence over the cells (the golden-ratio increment).  The
// hash makes the bits of neighbouring cells independent: the Weyl sequence
// alone, or a product of it with a constant, advances by a fixed fraction
// per cell, and where that fraction is small (0.0026 per cell for one
// constant tried) neighbouring cells round alike, their rounding errors no
// longer cancel in the totals, and the total of c wandered about a hundred
// times further than with independent bits (FP32 emulation and GB300 runs).
__device__ __forceinline__ uint32_t cell_bits(uint32_t seed, int i, int j, int nx) {
    return pcg_hash(seed + 0x9E3779B9u * (uint32_t)(j * nx + i));
}

// Random bits of cell (i, j) for the rounding of phi's zeroth moment; the
// rounding of c's takes second_bits of them.
__device__ __forceinline__ uint32_t moment_bits(uint32_t seed, int i, int j, int nx) {
    return cell_bits(seed ^ 0x5bd1e995u, i, j, nx);
}

// Fixed-point value after adding a float increment, rounded stochastically:
// up with probability equal to the dropped fraction, drawn from the high 24
// bits of r.  Rounding to nearest drops every increment below half a unit,
// and in the tails of the interface profiles, where the increments are tiny
// and of one sign step after step, that bias moves the totals of phi and c;
// the zero-mean rounding keeps them (to the random walk of the roundings).
// The increment is split exactly into its floor and its fraction (v - floor(v)
// is exact in FP32), and the fraction is compared with the random number:
// adding the random number to v in FP32 instead would round the sum to the
// float grid of v, which biases the result upwards by about a quarter of
// that grid's spacing (0.07 units at |v| ~ 3e6 units).
__device__ __forceinline__ int fx_add_sr(int s0, float inc, float scale, uint32_t r) {
    const float v = inc * scale;
    if (!(fabsf(v) < 1.0e9f)) return FX_INVALID;
    const float fl = floorf(v);
    const float q = (v - fl) * 16777216.0f;  // the fraction in units of 2^-24
    const unsigned up = (float)(r >> 8) < q ? 1u : 0u;
    const unsigned sum = (unsigned)s0 + (unsigned)(int)fl + up;
    return sum + (unsigned)FX_RANGE > 2u * (unsigned)FX_RANGE ? FX_INVALID : (int)sum;
}
__device__ __forceinline__ i2 fx_add_sr(i2 s0, f2 inc, float scale, uint32_t ra, uint32_t rb) {
    return i2{fx_add_sr(s0.x, inc.x, scale, ra), fx_add_sr(s0.y, inc.y, scale, rb)};
}
// The bits of c's rounding from the same cell draw: its product with an odd
// constant (a bijection of 32-bit words, so uniform where the draw is).
__device__ __forceinline__ uint32_t second_bits(uint32_t b) { return b * 0x2C1B3C6Du; }

// Float value of a fixed-point number (NaN for the invalid marker).
__device__ __forceinline__ double fx_to_double(int s, float scale) {
    return s == FX_INVALID ? __longlong_as_double(0x7ff8000000000000ll) : (double)s / (double)scale;
}

__device__ __forceinline__ int fx_from_double(double v, float scale) {
    const double x = v * (double)scale;
    return (isfinite(x) && fabs(x) <= (double)FX_RANGE) ? __double2int_rn(x) : FX_INVALID;
}

__device__ __forceinline__ ScalarMoments pull_scalar_rows(const float* __restrict__ Rm,
                                                          const float* __restrict__ R0,
                                                          const float* __restrict__ Rp,
                                                          int64_t PS, int cm, int c0, int cp,
                                                          bool bot, bool top, float inv) {
    const int S0 = fx_load(R0 + c0);
    float o[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) o[q] = R0[q * PS + c0];
    const float w1 = (1.0f / 9.0f) * inv, w5 = (1.0f / 36.0f) * inv;
    float t[9];
    t[1] = w1 * (float)(fx_load(R0 + cm) - S0) + R0[1 * PS + cm];
    t[3] = w1 * (float)(fx_load(R0 + cp) - S0) + R0[3 * PS + cp];
    if (bot) {
        t[2] = o[4];
        t[5] = o[7];
        t[6] = o[8];
    } else {
        t[2] = w1 * (float)(fx_load(Rm + c0) - S0) + Rm[2 * PS + c0];
        t[5] = w5 * (float)(fx_load(Rm + cm) - S0) + Rm[5 * PS + cm];
        t[6] = w5 * (float)(fx_load(Rm + cp) - S0) + Rm[6 * PS + cp];
    }
    if (top) {
        t[4] = o[2];
        t[7] = o[5];
        t[8] = o[6];
    } else {
        t[4] = w1 * (float)(fx_load(Rp + c0) - S0) + Rp[4 * PS + c0];
        t[7] = w5 * (float)(fx_load(Rp + cp) - S0) + Rp[7 * PS + cp];
        t[8] = w5 * (float)(fx_load(Rp + cm) - S0) + Rp[8 * PS + cm];
    }
    ScalarMoments m;
    m.s0 = S0;
    m.inc = (((t[1] + t[3]) + (t[2] + t[4])) + ((t[5] + t[6]) + (t[7] + t[8]))) -
            (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])));
    m.jx = (t[1] - t[3]) + (t[5] - t[6]) - (t[7] - t[8]);
    m.jy = (t[2] - t[4]) + (t[5] + t[6]) - (t[7] + t[8]);
    return m;
}

__device__ __forceinline__ ScalarMoments pull_scalar(const float* __restrict__ base,
                                                     const KParams& p, int l, int i, int j) {
    const bool bot = p.walls && j == 0, top = p.walls && j == p.ny - 1;
    const float* R0 = base + (int64_t)j * p.pitch;
    const float* Rm = base + (int64_t)wrap_i(j - 1, p.ny) * p.pitch;
    const float* Rp = base + (int64_t)wrap_i(j + 1, p.ny) * p.pitch;
    return pull_scalar_rows(Rm, R0, Rp, p.plane, wrap_i(i - 1, p.nx), i, wrap_i(i + 1, p.nx), bot,
                            top, p.fx_inv[l]);
}

// Plain post-streaming populations of a lattice in deviation form (for export
// and re-import), in precision R.
template <typename R>
__device__ __forceinline__ void pull9_dev(const float* __restrict__ base, const KParams& p, int l,
                                          int i, int j, R out[9]) {
    const int64_t P = p.plane;
    const int im = wrap_i(i - 1, p.nx), ip = wrap_i(i + 1, p.nx);
    const int64_t r0 = (int64_t)j * p.pitch;
    const bool bot = p.walls && j == 0, top = p.walls && j == p.ny - 1;
    const R inv = (R)1 / (R)p.fx_scale[l];
    const R S0 = (R)fx_to_double(fx_load(base + r0 + i), p.fx_scale[l]);
    R o[9];
    R osum = 0;
#pragma unroll
    for (int q = 1; q < 9; ++q) {
        o[q] = (R)base[q * P + r0 + i];
        osum += o[q];
    }
    const R w0 = (R)4 / (R)9, w1 = (R)1 / (R)9, w5 = (R)1 / (R)36;
    out[0] = w0 * S0 - osum;
    out[1] = w1 * (R)fx_load(base + r0 + im) * inv + (R)base[1 * P + r0 + im];
    out[3] = w1 * (R)fx_load(base + r0 + ip) * inv + (R)base[3 * P + r0 + ip];
    if (bot) {
        out[2] = w1 * S0 + o[4];
        out[5] = w5 * S0 + o[7];
        out[6] = w5 * S0 + o[8];
    } else {
        const int64_t rm = (int64_t)wrap_i(j - 1, p.ny) * p.pitch;
        out[2] = w1 * (R)fx_load(base + rm + i) * inv + (R)base[2 * P + rm + i];
        out[5] = w5 * (R)fx_load(base + rm + im) * inv + (R)base[5 * P + rm + im];
        out[6] = w5 * (R)fx_load(base + rm + ip) * inv + (R)base[6 * P + rm + ip];
    }
    if (top) {
        out[4] = w1 * S0 + o[2];
        out[7] = w5 * S0 + o[5];
        out[8] = w5 * S0 + o[6];
    } else {
        const int64_t rp = (int64_t)wrap_i(j + 1, p.ny) * p.pitch;
        out[4] = w1 * (R)fx_load(base + rp + i) * inv + (R)base[4 * P + rp + i];
        out[7] = w5 * (R)fx_load(base + rp + ip) * inv + (R)base[7 * P + rp + ip];
        out[8] = w5 * (R)fx_load(base + rp + im) * inv + (R)base[8 * P + rp + im];
    }
}

// Isotropic gradient of a fixed-point field from exact integer differences.
template <class V, class VI>
__device__ __forceinline__ void iso_grad_fx(const VI v[3][3], float inv, V& gx, V& gy) {
    gx = ((1.0f / 3.0f) * i2f(isub(v[1][2], v[1][0])) +
          (1.0f / 12.0f) * (i2f(isub(v[2][2], v[2][0])) + i2f(isub(v[0][2], v[0][0])))) * inv;
    gy = ((1.0f / 3.0f) * i2f(isub(v[2][1], v[0][1])) +
          (1.0f / 12.0f) * (i2f(isub(v[2][2], v[0][2])) + i2f(isub(v[2][0], v[0][0])))) * inv;
}

// theta (Eq. theta) and theta_c (Eq. ISS) from the fixed-point phi: the
// factors phi_a - phi, phi - phi_b and phi_m - phi are exact integer
// differences before the conversion to float.
template <class V, class VI>
__device__ __forceinline__ void interface_coeffs(const KParams& p, VI phi_fx, V c, V& theta,
                                                 V& theta_c) {
    const float inv = p.fx_inv[0];
    const V A = i2f(isub(p.phi_a_fx, phi_fx)) * inv;
    const V B = i2f(isub(phi_fx, p.phi_b_fx)) * inv;
    const V M = i2f(isub(p.phi_m_fx, phi_fx)) * inv;
    theta = (p.four_over_W * p.inv_dphi) * (A * B);
    theta_c = (p.eight_over_W * p.inv_dphi) * (c * M);
}

// ---------------------------------------------------------------------------
// stencils on 3x3 neighbourhoods v[dy+1][dx+1]
// ---------------------------------------------------------------------------

// Isotropic gradient (1/cs2) sum_q w_q e_q A(x + e_q).
template <class V>
__device__ __forceinline__ void iso_grad(const V v[3][3], V& gx, V& gy) {
    gx = (1.0f / 3.0f) * (v[1][2] - v[1][0]) +
         (1.0f / 12.0f) * ((v[2][2] - v[2][0]) + (v[0][2] - v[0][0]));
    gy = (1.0f / 3.0f) * (v[2][1] - v[0][1]) +
         (1.0f / 12.0f) * ((v[2][2] + v[2][0]) - (v[0][2] + v[0][0]));
}

// Isotropic divergence of a vector field given on the 3x3 neighbourhood.
template <class V>
__device__ __forceinline__ V iso_div(const V vx[3][3], const V vy[3][3]) {
    const V dxx = (1.0f / 3.0f) * (vx[1][2] - vx[1][0]) +
                  (1.0f / 12.0f) * ((vx[2][2] - vx[2][0]) + (vx[0][2] - vx[0][0]));
    const V dyy = (1.0f / 3.0f) * (vy[2][1] - vy[0][1]) +
                  (1.0f / 12.0f) * ((vy[2][2] + vy[2][0]) - (vy[0][2] + vy[0][0]));
    return dxx + dyy;
}

template <class V>
__device__ __forceinline__ void unit_normal(V gx, V gy, V& nx, V& ny, V& mag) {
    // branch-free: below the threshold the normal and the magnitude are 0
    const V g2 = gx * gx + gy * gy;
    const V inv = vmap(g2, [](float v) { return v > EPS_N * EPS_N ? rsqrtf(v) : 0.0f; });
    nx = gx * inv;
    ny = gy * inv;
    mag = g2 * inv;
}

// Langmuir isotherm, Eq. (EOS).  beta = 0 (clean interface) gives sigma_o
// whatever c is: 0 * log(<= 0) would be NaN once a passive surfactant reaches
// c_max, so the product is selected away rather than formed.
template <class V>
__device__ __forceinline__ V sigma_of_c(const KParams& p, V c) {
    if (p.beta == 0.0f) return vsplat<V>(p.sigma_o);
    const V t = vmap(1.0f - c * p.inv_cmax, [](float v) { return __logf(v); });
    return p.sigma_o + (p.sigma_o * p.beta) * t;
}

// ---------------------------------------------------------------------------
// collisions
// ---------------------------------------------------------------------------

// P^-1 applied to raw moments r = (00,10,01,20,02,11,21,12,22) (App. A),
// times s (a power of two: the 16-bit storage scale, folded into the factors
// 1/2 and 1/4 at no cost and without rounding; 1 for FP32 storage).
template <class V, class SC = float>
__device__ __forceinline__ void raw_to_pops(const V r[9], V out[9], SC s = 1.0f) {
    // factored: the eight pair sums and differences are shared by two outputs each
    const V a = r[3] - r[8], b = r[1] - r[7], c = r[4] - r[8], d = r[2] - r[6];
    const V e = r[8] + r[5], f = r[6] + r[7], g = r[8] - r[5], h = r[6] - r[7];
    const SC h2 = 0.5f * s, h4 = 0.25f * s;
    out[0] = ((r[0] - r[3]) - c) * s;
    out[1] = h2 * (a + b);
    out[2] = h2 * (c + d);
    out[3] = h2 * (a - b);
    out[4] = h2 * (c - d);
    out[5] = h4 * (e + f);
    out[6] = h4 * (g + h);
    out[7] = h4 * (e - f);
    out[8] = h4 * (g - h);
}

// F^-1(u) applied to central moments k (binomial expansion of ((e-u)+u)^m).
template <class V>
__device__ __forceinline__ void central_to_raw(const V k[9], V ux, V uy, V r[9]) {
    const V ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    r[0] = k[0];
    r[1] = ux * k[0] + k[1];
    r[2] = uy * k[0] + k[2];
    r[3] = ux2 * k[0] + 2.0f * ux * k[1] + k[3];
    r[4] = uy2 * k[0] + 2.0f * uy * k[2] + k[4];
    r[5] = uxy * k[0] + uy * k[1] + ux * k[2] + k[5];
    r[6] = ux2 * uy * k[0] + 2.0f * uxy * k[1] + ux2 * k[2] + uy * k[3] + 2.0f * ux * k[5] + k[6];
    r[7] = ux * uy2 * k[0] + uy2 * k[1] + 2.0f * uxy * k[2] + ux * k[4] + 2.0f * uy * k[5] + k[7];
    r[8] = ux2 * uy2 * k[0] + 2.0f * ux * uy2 * k[1] + 2.0f * ux2 * uy * k[2] + uy2 * k[3] +
           ux2 * k[4] + 4.0f * uxy * k[5] + 2.0f * uy * k[6] + 2.0f * ux * k[7] + k[8];
}

// The same transform as central_to_raw, applied as two one-dimensional shifts
// (F^-1(u) is the tensor product of the x and y binomial shifts): per order-2
// triple (c0, c1, c2) -> (c0, c1 + u c0, c2 + u (c1 + (c1 + u c0))).
__device__ __forceinline__ void central_to_raw_sep(const float k[9], float ux, float uy,
                                                   float r[9]) {
    // x shift of the rows b = 0, 1, 2 (k indices: 00 0, 10 1, 20 3 | 01 2, 11 5, 21 6 | 02 4, 12 7, 22 8)
    const float m10 = k[1] + ux * k[0], m20 = k[3] + ux * (k[1] + m10);
    const float m11 = k[5] + ux * k[2], m21 = k[6] + ux * (k[5] + m11);
    const float m12 = k[7] + ux * k[4], m22 = k[8] + ux * (k[7] + m12);
    // y shift of the columns a = 0, 1, 2
    r[0] = k[0];
    r[2] = k[2] + uy * k[0];
    r[4] = k[4] + uy * (k[2] + r[2]);
    r[1] = m10;
    r[5] = m11 + uy * m10;
    r[7] = m12 + uy * (m11 + r[5]);
    r[3] = m20;
    r[6] = m21 + uy * m20;
    r[8] = m22 + uy * (m21 + r[6]);
}

// Advection-diffusion collision returning deviation-form output:
// d_q = a~_q - w_q s for q = 1..8 (a~ = P^-1 F^-1(u) k), where all central
// moments are set to their equilibria (s, q, cs2 s, cs2 s, 0, 0, 0, cs4 s)
// except the first-order ones, which relax at rate w (f with s = phi,
// q = M_phi theta n; h with s = c, q = D_s theta_c n).  The raw moments of
// the deviation are s (raw moments of the equilibrium shape at u minus those
// at rest) plus the raw moments of F^-1(u) (0, k10~, k01~, 0, ...), so no
// O(s) term is formed.
template <class V, class W, class SC = float>
__device__ __forceinline__ void collide_scalar_dev(V s, V jx, V jy, V qx, V qy, W w, V ux, V uy,
                                                   V d[9], SC out_scale = 1.0f) {
    const V k10 = jx - ux * s, k01 = jy - uy * s;
    const V a = vfma(w, qx - k10, k10);
    const V b = vfma(w, qy - k01, k01);
    const V ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const V su = s * ux, sv = s * uy;
    V R[9];
    R[0] = vsplat<V>(0.0f);
    R[1] = su + a;
    R[2] = sv + b;
    R[3] = vfma(su, ux, 2.0f * (ux * a));
    R[4] = vfma(sv, uy, 2.0f * (uy * b));
    R[5] = vfma(su, uy, vfma(uy, a, ux * b));
    R[6] = vfma(sv, ux2 + CS2, uxy * (2.0f * a) + ux2 * b);
    R[7] = vfma(su, uy2 + CS2, uy2 * a + uxy * (2.0f * b));
    R[8] = vfma(s, ux2 * uy2 + CS2 * (ux2 + uy2), 2.0f * (uxy * (uy * a + ux * b)));
    raw_to_pops(R, d, out_scale);
}

// Advection-diffusion collision on full populations (initialisation and the
// cross-check kernels): all central moments to equilibrium except the first
// order, which relaxes at rate w.  In/out: pre-/post-collision populations.
__device__ __forceinline__ void collide_scalar(float a[9], float s, float qx, float qy, float w,
                                               float ux, float uy) {
    const float jx = (a[1] - a[3]) + (a[5] - a[6]) - (a[7] - a[8]);
    const float jy = (a[2] - a[4]) + (a[5] + a[6]) - (a[7] + a[8]);
    const float k10 = jx - ux * s, k01 = jy - uy * s;  // central first moments
    float k[9];
    k[0] = s;
    k[1] = k10 + w * (qx - k10);
    k[2] = k01 + w * (qy - k01);
    k[3] = CS2 * s;
    k[4] = CS2 * s;
    k[5] = 0.0f;
    k[6] = 0.0f;
    k[7] = 0.0f;
    k[8] = CS2 * CS2 * s;
    float r[9];
    central_to_raw(k, ux, uy, r);
    raw_to_pops(r, a);
}

// Macroscopic inputs of the flow collision at one cell (or two).
template <class V>
struct FlowMacroT {
    V ux, uy;      // velocity
    V rho;         // density
    V dP;          // P - P0 (after the half-source correction)
    V dPs;         // sum of shifted g = P* - P0
    V Ftx, Fty;    // total force F_s + F_ext
    V Fpx, Fpy;    // pressure force -grad psi
    V w_nu;        // shear relaxation rate
};
using FlowMacro = FlowMacroT<float>;

// Flow lattice, Eq. (centralmomentLBE2fluidflow), on shifted populations
// a = g - w P0.  Central moments of the shift are P0 W(u) with W(u) the
// central moments of the weights about u; they cancel in eq - moments, so the
// collision runs on deviations: d_eta^eq = rho cs2 (M(u) - W(u)) + dP W(u).
// out_scale: power-of-two factor applied to the output populations (16-bit
// storage scale; 1 for FP32 storage).
// One cell.  The order of the operations is part of the result: in a steady
// shear the stored populations carry the momentum with the same rounding
// every step, and the velocity profile integrates that error.  This order
// leaves 2.4e-6 relative velocity error after 5000 steps of the 2048 x 1024
// drop against the FP64 oracle; a reassociated form of the same expressions
// (products grouped differently, FMAs placed elsewhere) left 1.3e-5.
__device__ __forceinline__ void collide_flow_cell_scalar(float a[9], const FlowMacroT<float>& m,
                                                         float w_zeta, float out_scale) {
    const float ux = m.ux, uy = m.uy;
    const float ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    // raw moments of the shifted populations that relax at non-unit rates
    const float jx = (a[1] - a[3]) + (a[5] - a[6]) - (a[7] - a[8]);
    const float jy = (a[2] - a[4]) + (a[5] + a[6]) - (a[7] + a[8]);
    const float corner = (a[5] + a[6]) + (a[7] + a[8]);
    const float r20 = (a[1] + a[3]) + corner;
    const float r02 = (a[2] + a[4]) + corner;
    const float r11 = (a[5] - a[6]) + (a[7] - a[8]);
    const float s0 = m.dPs;
    // pre-collision central moments (deviation form)
    const float e20 = r20 - 2.0f * ux * jx + ux2 * s0;
    const float e02 = r02 - 2.0f * uy * jy + uy2 * s0;
    const float e11 = r11 - uy * jx - ux * jy + uxy * s0;
    // equilibria (deviation form); first order -psi u (the sign reading of App. D)
    const float R = m.rho * CS2, dP = m.dP;
    const float RmP = R - dP;
    const float q20 = -R * ux2 + dP * (CS2 + ux2);
    const float q02 = -R * uy2 + dP * (CS2 + uy2);
    const float q11 = -RmP * uxy;
    // source central moments (App. D)
    const float G = m.Fpx * ux + m.Fpy * uy;
    const float s10 = CS2 * m.Ftx - ux * G;
    const float s01 = CS2 * m.Fty - uy * G;
    const float s20 = 2.0f * CS2 * m.Fpx * ux + (ux2 + CS2) * G;
    const float s02 = 2.0f * CS2 * m.Fpy * uy + (uy2 + CS2) * G;
    const float s11 = CS2 * (m.Fpx * uy + m.Fpy * ux) + uxy * G;
    // relax in the combined basis (B): 2s at w_zeta, 2d and 11 at w_nu, rest at 1
    const float wn = m.w_nu;
    const float h2s = e20 + e02, h2d = e20 - e02;
    const float t2s = h2s + w_zeta * ((q20 + q02) - h2s) + (1.0f - 0.5f * w_zeta) * (s20 + s02);
    const float t2d = h2d + wn * ((q20 - q02) - h2d) + (1.0f - 0.5f * wn) * (s20 - s02);
    float k[9];
    k[0] = dP + 0.5f * G;
    k[1] = ux * RmP + 0.5f * s10;
    k[2] = uy * RmP + 0.5f * s01;
    k[3] = 0.5f * (t2s + t2d);
    k[4] = 0.5f * (t2s - t2d);
    k[5] = e11 + wn * (q11 - e11) + (1.0f - 0.5f * wn) * s11;
    k[6] = RmP * (ux2 + CS2) * uy;
    k[7] = RmP * (uy2 + CS2) * ux;
    k[8] = -R * (ux2 * uy2 + CS2 * (ux2 + uy2)) + dP * (ux2 + CS2) * (uy2 + CS2);
    float r[9];
    central_to_raw_sep(k, ux, uy, r);
    // The raw first moments of the post-collision state are exactly
    // rho cs2 u + cs2 F_t / 2 = j + cs2 F_t (j: pre-collision momentum, with
    // rho cs2 u = j + cs2 F_t / 2).  Formed from j they carry the momentum
    // forward without passing through the rounded u: re-forming it from u
    // every step adds the rounding of u to the momentum, and for a slowly
    // varying flow that rounding repeats step after step and accumulates.
    // Explicit FMAs: every kernel that inlines this rounds it the same way.
    r[1] = __fmaf_rn(CS2, m.Ftx, jx);
    r[2] = __fmaf_rn(CS2, m.Fty, jy);
    raw_to_pops(r, a, out_scale);
}

// The same collision for one or two cells: two cells are collided lane by
// lane with the one-cell code, so that every cell's result is the same bits
// whatever the cells per thread.
template <class V>
__device__ __forceinline__ void collide_flow(V a[9], const FlowMacroT<V>& m, float w_zeta,
                                             float out_scale = 1.0f) {
    if constexpr (std::is_same<V, float>::value) {
        collide_flow_cell_scalar(a, m, w_zeta, out_scale);
    } else {
#pragma unroll
        for (int k = 0; k < Lanes<V>::n; ++k) {
            float ak[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) ak[q] = lane(a[q], k);
            FlowMacroT<float> mk;
            mk.ux = lane(m.ux, k);
            mk.uy = lane(m.uy, k);
            mk.rho = lane(m.rho, k);
            mk.dP = lane(m.dP, k);
            mk.dPs = lane(m.dPs, k);
            mk.Ftx = lane(m.Ftx, k);
            mk.Fty = lane(m.Fty, k);
            mk.Fpx = lane(m.Fpx, k);
            mk.Fpy = lane(m.Fpy, k);
            mk.w_nu = lane(m.w_nu, k);
            collide_flow_cell_scalar(ak, mk, w_zeta, out_scale);
#pragma unroll
            for (int q = 0; q < 9; ++q) set_lane(a[q], k, ak[q]);
        }
    }
}

// Moving-wall term added when a flow population is written into a slot that
// is only read back by the bounce-back of the same cell (App. D set-up,
// half-way bounce-back): slot q at the bottom row (e_qy = -1) feeds direction
// opp(q) with u_w = (-u_wall, 0); at the top row (e_qy = +1) u_w = (+u_wall, 0).
template <class V>
__device__ __forceinline__ void wall_correct_flow(V a[9], const KParams& p, int j, V rho,
                                                  float out_scale = 1.0f) {
    if (!p.walls) return;
    if (j == 0) {
        // 2 w_opp rho (e_opp . u_w), u_w = -u_wall: opp(4)=2 (0), opp(7)=5 (+1), opp(8)=6 (-1)
        const V t = (2.0f * (1.0f / 36.0f) * (-p.u_wall) * out_scale) * rho;
        a[7] += t;   // e_5x = +1
        a[8] -= t;   // e_6x = -1
    }
    if (j == p.ny - 1) {
        const V t = (2.0f * (1.0f / 36.0f) * (p.u_wall) * out_scale) * rho;
        a[5] -= t;   // opp(5) = 7, e_7x = -1
        a[6] += t;   // opp(6) = 8, e_8x = +1
    }
}

}  // namespace lbm
