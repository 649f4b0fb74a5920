// D3Q27 form of the phase-field (f, App. C) and interface-bound surfactant
// (h, Sec. 3) central-moment lattices under a prescribed velocity: one
// z-marching kernel per time step behind the C ABI of include/lbm3.h.
//
// Collision in closed form.  Both lattices relax every central moment but
// the three first-order ones to its Maxwellian equilibrium (rate 1).  With
// the tensor-product moment basis |e_x^m e_y^n e_z^p> the post-collision
// central moments are
//     s mu(m) mu(n) mu(p) + k'_x [100] + k'_y [010] + k'_z [001],
//     mu = (1, 0, cs^2),  k'_i = k_i + w (K theta n_i - k_i),  k_i = j_i - u_i s,
// and P^-1 F^-1(u) is the Kronecker product of its one-dimensional factors,
// so the outgoing population of velocity (a, b, c) is
//     s Ax[a] Ay[b] Az[c] + k'_x Bx[a] Cy[b] Cz[c] + (k'_y By[b] Cz[c] + k'_z Cy[b] Bz[c]) Cx[a]
// with, per axis of velocity u (e = 0, +1, -1):
//     A = central (1, 0, cs^2) -> (1 - cs^2 - u^2, (cs^2 + u^2 + u)/2, (cs^2 + u^2 - u)/2)
//     B = central (0, 1, 0)    -> (-2u, u + 1/2, u - 1/2)
//     C = central (1, 0, 0)    -> (1 - u^2, (u^2 + u)/2, (u^2 - u)/2).
// A collision therefore needs only s = sum a and j = sum e a of the incoming
// populations: the pull loads are summed as they arrive.
//
// Storage in fixed point.  Populations are int32 in units of 2^-28 (range
// +-8), plane by plane: word (z, q, y, x) of a lattice is at
// ((z * 27 + q) * ny + y) * nx + x, so every offset inside a plane's 27
// populations fits 32 bits (27 nx ny < 2^31) and only the plane base is 64-bit.  The pull sums are exact integer sums; the collision runs in FP32 on
// those moments, its 26 moving outputs are rounded to the grid, and the rest
// population takes the integer remainder s - sum(others), so every collision
// conserves sum f and sum h exactly.  (With FP32 storage every cell of a
// uniform region makes the same rounding error in every step and the region's
// phi drifts coherently; in integers a uniform region is an exact fixed
// point.)  A cell whose zeroth moment leaves (-4, 4) stores FX_BAD in all its
// populations; the reductions count them.
//
// Step kernel.  A block owns a 30 x (ROWS - 2) column tile with a one-cell
// halo (one warp per row of 32 columns) and marches through seg_z planes.
// At plane k it pulls the f populations of plane k + 1 for every tile and
// halo cell (phi into a four-plane shared ring, the first moments of the
// tile cells kept in registers for the next plane) and the h populations of
// plane k for the tile cells, waits at one barrier, then updates the tile
// cells of plane k: gradient of phi from the ring, normal, theta, theta_c,
// both collisions, 54 coalesced stores.  With four ring slots the slot
// written at plane k + 1 is one no thread still reads, and the one written at
// plane k + 2 was last read before the barrier of plane k + 1, so one barrier
// per plane suffices.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "lbm3.h"

namespace {

constexpr int Q27 = 27;
constexpr int TILE_W = 32;   // columns of a tile row, halo included
constexpr int TILE_IN = 30;  // columns a block updates
constexpr float FX_ONE = 268435456.0f;        // 2^28 units per unit value
constexpr float FX_INV = 1.0f / 268435456.0f;
constexpr double FX_ONE_D = 268435456.0;
constexpr double FX_INV_D = 1.0 / 268435456.0;
constexpr int FX_BAD = (-2147483647 - 1);       // invalid population marker
constexpr float S_MAX = 4.0f;                   // valid |zeroth moment|
constexpr int SUM_BLOCKS = 1024;
constexpr int SUM_THREADS = 256;

struct Nvtx {
    explicit Nvtx(const char* name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
};

struct K3Params {
    int nx, ny, nz, seg_z;
    long long N, nxny;
    float w_kappa, w_chi, M_phi, D_s;
    float c4W, c8W, phi_a, phi_b, phim, inv_dphi;
    float u[3];
    float fac[3][3][3];  // uniform u: [axis][A, B, C][e = 0, +1, -1] factors
    const float* uf;     // per-cell velocity [3][N], or null for the uniform u
};

__host__ __device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// One-dimensional factors of P^-1 F^-1(u) (index 0: e = 0, 1: e = +1, 2: e = -1).
template <class T>
__device__ __forceinline__ void axis_factors(T u, T* A, T* B, T* C) {
    const T u2 = u * u;
    const T t = T(1) / T(3) + u2;
    A[0] = T(1) - t;
    A[1] = T(0.5) * (t + u);
    A[2] = T(0.5) * (t - u);
    B[0] = T(-2) * u;
    B[1] = u + T(0.5);
    B[2] = u - T(0.5);
    C[0] = T(1) - u2;
    C[1] = T(0.5) * (u2 + u);
    C[2] = T(0.5) * (u2 - u);
}

// Outgoing populations of one collision; out(q, value) receives each.
template <class T, class Out>
__device__ __forceinline__ void emit27(const T (&Ax)[3], const T (&Bx)[3], const T (&Cx)[3],
                                       const T (&Ay)[3], const T (&By)[3], const T (&Cy)[3],
                                       const T (&Az)[3], const T (&Bz)[3], const T (&Cz)[3],
                                       T s, T kx, T ky, T kz, Out out) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T P = s * (Ay[b] * Az[c]);
            const T X = kx * (Cy[b] * Cz[c]);
            const T R = ky * (By[b] * Cz[c]) + kz * (Cy[b] * Bz[c]);
#pragma unroll
            for (int a = 0; a < 3; ++a) out(a + 3 * b + 9 * c, P * Ax[a] + X * Bx[a] + R * Cx[a]);
        }
    }
}

// Zeroth and first raw moments of the 27 populations pulled into a cell:
// population (a, b, c) comes from (x - e_a, y - e_b, z - e_c).  Exact integer
// sums (two's complement wrap-around is harmless: the true sums are in range).
struct Moments {
    uint32_t s, jx, jy, jz;
};

__device__ __forceinline__ Moments pull_moments(const int* __restrict__ base, long long pstride, int nxny,
                                                const int (&zs)[3], const int (&ys)[3], const int (&xs)[3]) {
    Moments m{0u, 0u, 0u, 0u};
    const int x1 = nxny + xs[1], x2 = 2 * nxny + xs[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int* q0 = base + zs[c] * pstride + 9 * c * nxny;  // population (0, 0, c) of the plane
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int* row = q0 + ys[b];
            q0 += 3 * nxny;
            const uint32_t v0 = (uint32_t)__ldg(row + xs[0]);
            const uint32_t v1 = (uint32_t)__ldg(row + x1);
            const uint32_t v2 = (uint32_t)__ldg(row + x2);
            const uint32_t sx = v0 + v1 + v2;
            m.s += sx;
            m.jx += v1 - v2;
            if (b == 1) m.jy += sx;
            if (b == 2) m.jy -= sx;
            if (c == 1) m.jz += sx;
            if (c == 2) m.jz -= sx;
        }
    }
    return m;
}

__device__ __forceinline__ float fx_to_f(uint32_t v) { return (float)(int)v * FX_INV; }

// Round the 26 moving outputs to the grid and give the rest population the
// remainder of the exact zeroth moment s_fx (or FX_BAD everywhere).
__device__ __forceinline__ void store_collision(int* __restrict__ o, int nxny, bool ok, uint32_t s_fx,
                                                const float (&Ax)[3], const float (&Bx)[3], const float (&Cx)[3],
                                                const float (&Ay)[3], const float (&By)[3], const float (&Cy)[3],
                                                const float (&Az)[3], const float (&Bz)[3], const float (&Cz)[3],
                                                float s, const float (&k)[3]) {
    uint32_t moved = 0u;
    emit27(Ax, Bx, Cx, Ay, By, Cy, Az, Bz, Cz, s, k[0], k[1], k[2], [&](int q, float v) {
        if (q == 0) return;
        const int iv = ok ? __float2int_rn(v * FX_ONE) : FX_BAD;
        moved += (uint32_t)iv;
        o[q * nxny] = iv;
    });
    o[0] = ok ? (int)(s_fx - moved) : FX_BAD;
}

// Resident blocks per SM the register budget is sized for: 96 registers a
// thread at 10 and 18 rows, 80 at 6 rows (four blocks of six warps; the
// uniform-velocity variant spills 40 bytes there and is still the fastest
// shape measured).
template <int ROWS>
constexpr int k3_min_blocks() { return ROWS == 6 ? 4 : ROWS == 10 ? 2 : 1; }

template <int ROWS, bool UFIELD>
__global__ void __launch_bounds__(ROWS * 32, k3_min_blocks<ROWS>()) k3_step(const K3Params p, const int* __restrict__ fa,
                                                     const int* __restrict__ ha, int* __restrict__ fb,
                                                     int* __restrict__ hb) {
    __shared__ float ring[4][ROWS][TILE_W];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int gx = blockIdx.x * TILE_IN + tx - 1;
    const int gy = blockIdx.y * (ROWS - 2) + ty - 1;
    const bool inner = tx >= 1 && tx <= TILE_IN && ty >= 1 && ty <= ROWS - 2 && gx < p.nx && gy < p.ny;
    const int x = wrapi(gx, p.nx), y = wrapi(gy, p.ny);
    // source column / row of the velocity component e = 0, +1, -1
    const int xs[3] = {x, wrapi(gx - 1, p.nx), wrapi(gx + 1, p.nx)};
    const int ys[3] = {y * p.nx, wrapi(gy - 1, p.ny) * p.nx, wrapi(gy + 1, p.ny) * p.nx};
    const long long N = p.N;
    const int nxny = (int)p.nxny;
    const long long pstride = 27LL * nxny;  // words of one plane's 27 populations
    const int z0 = blockIdx.z * p.seg_z;
    const int z1 = min(p.nz, z0 + p.seg_z);

    // source plane of the velocity component e = 0, +1, -1
    auto planes = [&](int z, int (&zs)[3]) {
        zs[0] = z;
        zs[1] = wrapi(z - 1, p.nz);
        zs[2] = wrapi(z + 1, p.nz);
    };

    int sm = 0, sc = 1, sp = 2, sf = 3;  // ring slots of planes k - 1, k, k + 1 (sf: free)
    int zs[3];
    planes(wrapi(z0 - 1, p.nz), zs);
    ring[sm][ty][tx] = fx_to_f(pull_moments(fa, pstride, nxny, zs, ys, xs).s);
    planes(z0, zs);
    Moments cur = pull_moments(fa, pstride, nxny, zs, ys, xs);
    ring[sc][ty][tx] = fx_to_f(cur.s);

    const float w1[3] = {1.0f / 6.0f, 2.0f / 3.0f, 1.0f / 6.0f};  // offsets -1, 0, +1

    int zc[3];  // planes of the current k (for the h pull)
    planes(z0, zc);
    for (int k = z0; k < z1; ++k) {
        planes(wrapi(k + 1, p.nz), zs);
        const Moments nxt = pull_moments(fa, pstride, nxny, zs, ys, xs);
        ring[sp][ty][tx] = fx_to_f(nxt.s);
        Moments hm{0u, 0u, 0u, 0u};
        if (inner) hm = pull_moments(ha, pstride, nxny, zc, ys, xs);
        __syncthreads();
        if (inner) {
            // gradient d_i phi = (1/cs2) sum_a w_a e_ai phi(x + e_a), accumulated
            // value by value from the ring (weights (1/2) w1 w1 on the two
            // transverse offsets)
            float gxv = 0.f, gyv = 0.f, gzv = 0.f;
#pragma unroll
            for (int dz = 0; dz < 3; ++dz) {
                const float(*plane)[TILE_W] = ring[dz == 0 ? sm : dz == 1 ? sc : sp];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        if (dx == 1 && dy == 1 && dz == 1) continue;
                        const float v = plane[ty + dy - 1][tx + dx - 1];
                        if (dx != 1) gxv += (dx == 2 ? w1[dy] * w1[dz] : -w1[dy] * w1[dz]) * v;
                        if (dy != 1) gyv += (dy == 2 ? w1[dx] * w1[dz] : -w1[dx] * w1[dz]) * v;
                        if (dz != 1) gzv += (dz == 2 ? w1[dx] * w1[dy] : -w1[dx] * w1[dy]) * v;
                    }
            }
            gxv *= 0.5f;
            gyv *= 0.5f;
            gzv *= 0.5f;
            const float g2 = gxv * gxv + gyv * gyv + gzv * gzv;
            const float inv = g2 > 1e-24f ? rsqrtf(g2) : 0.f;
            const float n3[3] = {gxv * inv, gyv * inv, gzv * inv};

            const int co = ys[0] + x;                       // offset inside the plane
            const long long cell = (long long)k * nxny + co;  // cell index (velocity field)
            // velocity factors: from the parameters (uniform u) or per cell
            float u3[3] = {p.u[0], p.u[1], p.u[2]};
            float F[3][3][3];
            if constexpr (UFIELD) {
                u3[0] = p.uf[cell];
                u3[1] = p.uf[N + cell];
                u3[2] = p.uf[2 * N + cell];
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) axis_factors(u3[ax], F[ax][0], F[ax][1], F[ax][2]);
            }
            const float(*Fx)[3][3] = UFIELD ? F : p.fac;
            const float(&Ax)[3] = Fx[0][0], (&Bx)[3] = Fx[0][1], (&Cx)[3] = Fx[0][2];
            const float(&Ay)[3] = Fx[1][0], (&By)[3] = Fx[1][1], (&Cy)[3] = Fx[1][2];
            const float(&Az)[3] = Fx[2][0], (&Bz)[3] = Fx[2][1], (&Cz)[3] = Fx[2][2];
            // theta (Eq. theta) and theta_c (Eq. ISS)
            const float phi = fx_to_f(cur.s), c = fx_to_f(hm.s);
            const float theta = p.c4W * (p.phi_a - phi) * (phi - p.phi_b) * p.inv_dphi;
            const float thetac = p.c8W * c * (p.phim - phi) * p.inv_dphi;
            const float qf = p.M_phi * theta, qh = p.D_s * thetac;
            // first-order central moments k = j - u s, relaxed towards K theta n
            const float jf[3] = {fx_to_f(cur.jx), fx_to_f(cur.jy), fx_to_f(cur.jz)};
            const float jh[3] = {fx_to_f(hm.jx), fx_to_f(hm.jy), fx_to_f(hm.jz)};
            float kf[3], kh[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float a = jf[i] - u3[i] * phi;
                kf[i] = a + p.w_kappa * (qf * n3[i] - a);
                const float b = jh[i] - u3[i] * c;
                kh[i] = b + p.w_chi * (qh * n3[i] - b);
            }
            const bool ok = fabsf(phi) < S_MAX && fabsf(c) < S_MAX;
            store_collision(fb + k * pstride + co, nxny, ok, cur.s, Ax, Bx, Cx, Ay, By, Cy, Az, Bz, Cz, phi, kf);
            store_collision(hb + k * pstride + co, nxny, ok, hm.s, Ax, Bx, Cx, Ay, By, Cy, Az, Bz, Cz, c, kh);
        }
        const int t = sm;
        sm = sc;
        sc = sp;
        sp = sf;
        sf = t;
        cur = nxt;
#pragma unroll
        for (int i = 0; i < 3; ++i) zc[i] = zs[i];
    }
}

// Discrete equilibria of the given fields, written where the pull of the
// first step reads them: the pull gives cell x population a from x - e_a of
// buffer A, so population a of cell x is stored at x - e_a and the state (the
// pulled populations) is the equilibrium at every cell.  FP64 arithmetic,
// FP32 storage.
__global__ void k3_init(const K3Params p, const double* __restrict__ phi, const double* __restrict__ c,
                        const double* __restrict__ ux, const double* __restrict__ uy,
                        const double* __restrict__ uz, double W, double phi_a, double phi_b,
                        double M_phi, double D_s, int* __restrict__ fa, int* __restrict__ ha,
                        float* __restrict__ uf) {
    const long long N = p.N;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < N;
         cell += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(cell % p.nx);
        const int y = (int)((cell / p.nx) % p.ny);
        const int z = (int)(cell / p.nxny);
        const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
        double g[3] = {0.0, 0.0, 0.0};
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const double v = phi[((long long)wrapi(z + dz, p.nz) * p.ny + wrapi(y + dy, p.ny)) * p.nx +
                                         wrapi(x + dx, p.nx)];
                    const double w = 3.0 * w1[dx + 1] * w1[dy + 1] * w1[dz + 1];
                    g[0] += w * dx * v;
                    g[1] += w * dy * v;
                    g[2] += w * dz * v;
                }
        const double m = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        double n[3];
        for (int i = 0; i < 3; ++i) n[i] = m > 1e-12 ? g[i] / m : 0.0;
        const double ph = phi[cell], cc = c[cell];
        const double dphi = phi_a - phi_b;
        const double theta = (4.0 / W) * (phi_a - ph) * (ph - phi_b) / dphi;
        const double thetac = (8.0 * cc / W) * (0.5 * (phi_a + phi_b) - ph) / dphi;
        double u[3] = {p.u[0], p.u[1], p.u[2]};
        if (ux) {
            u[0] = ux[cell];
            u[1] = uy[cell];
            u[2] = uz[cell];
            uf[cell] = (float)u[0];
            uf[N + cell] = (float)u[1];
            uf[2 * N + cell] = (float)u[2];
        }
        double Ax[3], Bx[3], Cx[3], Ay[3], By[3], Cy[3], Az[3], Bz[3], Cz[3];
        axis_factors(u[0], Ax, Bx, Cx);
        axis_factors(u[1], Ay, By, Cy);
        axis_factors(u[2], Az, Bz, Cz);
        // destination of population (a, b, c): the cell x - e
        const int xd[3] = {x, wrapi(x - 1, p.nx), wrapi(x + 1, p.nx)};
        const int yd[3] = {y, wrapi(y - 1, p.ny), wrapi(y + 1, p.ny)};
        const int zd[3] = {z, wrapi(z - 1, p.nz), wrapi(z + 1, p.nz)};
        auto dest = [&](int q) {
            const int a = q % 3, b = (q / 3) % 3, cq = q / 9;
            return ((long long)zd[cq] * Q27 + q) * p.nxny + (long long)yd[b] * p.nx + xd[a];
        };
        const double qf = M_phi * theta, qh = D_s * thetac;
        // non-finite or out-of-range values become FX_BAD
        const bool ok = fabs(ph) < (double)S_MAX && fabs(cc) < (double)S_MAX;
        auto fx = [&](double v) { return ok && fabs(v) < 8.0 ? (int)__double2ll_rn(v * FX_ONE_D) : FX_BAD; };
        emit27(Ax, Bx, Cx, Ay, By, Cy, Az, Bz, Cz, ph, qf * n[0], qf * n[1], qf * n[2],
               [&](int q, double v) { fa[dest(q)] = fx(v); });
        emit27(Ax, Bx, Cx, Ay, By, Cy, Az, Bz, Cz, cc, qh * n[0], qh * n[1], qh * n[2],
               [&](int q, double v) { ha[dest(q)] = fx(v); });
    }
}

// State of cell x: population a is buffer A's value at x - e_a (plane-major
// word index, see the storage note at the top).
__device__ __forceinline__ long long pull_src(const K3Params& p, long long cell, int q) {
    const int x = (int)(cell % p.nx);
    const int y = (int)((cell / p.nx) % p.ny);
    const int z = (int)(cell / p.nxny);
    const int E[3] = {0, 1, -1};
    const int a = q % 3, b = (q / 3) % 3, c = q / 9;
    return ((long long)wrapi(z - E[c], p.nz) * Q27 + q) * p.nxny + (long long)wrapi(y - E[b], p.ny) * p.nx +
           wrapi(x - E[a], p.nx);
}

// phi = sum f and c = sum h of the state: exact integer sums, then FP64
// (NaN where a pulled population is FX_BAD).
__global__ void k3_fields(const K3Params p, const int* __restrict__ fa, const int* __restrict__ ha,
                          double* __restrict__ phi, double* __restrict__ c) {
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < p.N;
         cell += (long long)gridDim.x * blockDim.x) {
        long long sf = 0, sh = 0;
        bool bf = false, bh = false;
        for (int q = 0; q < Q27; ++q) {
            const long long src = pull_src(p, cell, q);
            const int a = fa[src], b = ha[src];
            bf |= a == FX_BAD;
            bh |= b == FX_BAD;
            sf += a;
            sh += b;
        }
        if (phi) phi[cell] = bf ? nan("") : (double)sf * FX_INV_D;
        if (c) c[cell] = bh ? nan("") : (double)sh * FX_INV_D;
    }
}

// The state's populations as float64 [27][N] (NaN for FX_BAD).
__global__ void k3_pops(const K3Params p, const int* __restrict__ fa, const int* __restrict__ ha,
                        double* __restrict__ f, double* __restrict__ h) {
    const long long total = Q27 * p.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / p.N);
        const long long src = pull_src(p, i % p.N, q);
        const int a = fa[src], b = ha[src];
        if (f) f[i] = a == FX_BAD ? nan("") : (double)a * FX_INV_D;
        if (h) h[i] = b == FX_BAD ? nan("") : (double)b * FX_INV_D;
    }
}

// Totals: sum f, sum h (exact, in integer units) and the FX_BAD count over the
// whole buffer (the pull is a permutation, so the state's totals are the
// buffer's).  Fixed grid and reduction order.
__global__ void __launch_bounds__(SUM_THREADS) k3_sum1(long long total, const int* __restrict__ fa,
                                                       const int* __restrict__ ha,
                                                       long long* __restrict__ partial) {
    long long sf = 0, sh = 0, bad = 0;
    for (long long i = blockIdx.x * (long long)SUM_THREADS + threadIdx.x; i < total;
         i += (long long)SUM_BLOCKS * SUM_THREADS) {
        const int a = fa[i], b = ha[i];
        if (a != FX_BAD) sf += a; else bad += 1;
        if (b != FX_BAD) sh += b; else bad += 1;
    }
    __shared__ long long red[3][SUM_THREADS];
    red[0][threadIdx.x] = sf;
    red[1][threadIdx.x] = sh;
    red[2][threadIdx.x] = bad;
    __syncthreads();
    for (int w = SUM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) partial[3 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(SUM_THREADS) k3_sum2(const long long* __restrict__ partial,
                                                       double* __restrict__ out) {
    __shared__ long long red[3][SUM_THREADS];
    long long acc[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < SUM_BLOCKS; b += SUM_THREADS)
        for (int k = 0; k < 3; ++k) acc[k] += partial[3 * b + k];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = SUM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = threadIdx.x < 2 ? (double)red[threadIdx.x][0] * FX_INV_D
                                                            : (double)red[threadIdx.x][0];
}

}  // namespace

struct lbm3_ctx {
    lbm3_params p;
    K3Params kp;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int* buf[2] = {nullptr, nullptr};    // each: f [nz][27][ny][nx] then h, fixed point
    float* uf = nullptr;                 // [3][N] prescribed velocity (velocity_field = 1)
    long long* partial = nullptr;        // 3 x SUM_BLOCKS partial sums
    double* result = nullptr;            // 3 totals
    int cur = 0;
    int rows = 10, seg_z = 64;
    int64_t step = 0;
    int pending_error = LBM_OK;
};

namespace {

int fail(lbm3_ctx* ctx, cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    if (ctx) ctx->pending_error = LBM_ERR_CUDA;
    return e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
}

double rate_of(double coeff) { return 1.0 / (coeff * 3.0 + 0.5); }

int* fbuf(lbm3_ctx* ctx, int which) { return ctx->buf[which]; }
int* hbuf(lbm3_ctx* ctx, int which) { return ctx->buf[which] + (size_t)Q27 * ctx->kp.N; }

int grid_1d(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

int launch_step(lbm3_ctx* ctx) {
    const K3Params& kp = ctx->kp;
    K3Params p = kp;
    p.seg_z = ctx->seg_z;
    const int rows = ctx->rows;
    dim3 grid((kp.nx + TILE_IN - 1) / TILE_IN, (kp.ny + rows - 3) / (rows - 2),
              (kp.nz + ctx->seg_z - 1) / ctx->seg_z);
    const int src = ctx->cur, dst = 1 - ctx->cur;
    const bool field = kp.uf != nullptr;
    auto go = [&](auto kern, int threads) {
        kern<<<grid, threads, 0, ctx->stream>>>(p, fbuf(ctx, src), hbuf(ctx, src), fbuf(ctx, dst), hbuf(ctx, dst));
    };
    switch (rows) {
        case 6:
            field ? go(k3_step<6, true>, 6 * 32) : go(k3_step<6, false>, 6 * 32);
            break;
        case 10:
            field ? go(k3_step<10, true>, 10 * 32) : go(k3_step<10, false>, 10 * 32);
            break;
        case 18:
            field ? go(k3_step<18, true>, 18 * 32) : go(k3_step<18, false>, 18 * 32);
            break;
        default:
            return LBM_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, e);
    ctx->cur = dst;
    ctx->step += 1;
    return LBM_OK;
}

bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int lbm3_params_default(lbm3_params* p) {
    if (!p) return LBM_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->W = 4.0;
    p->phi_a = 1.0;
    p->phi_b = 0.0;
    p->M_phi = 0.1;
    p->D_s = 0.1;
    return LBM_OK;
}

int lbm3_create(const lbm3_params* p, void* stream, lbm3_ctx** out) {
    if (!p || !out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBM_ERR_INVALID_ARG;
    if ((long long)p->nx * p->ny * p->nz > LBM3_MAX_CELLS) return LBM_ERR_INVALID_ARG;
    if (27LL * p->nx * p->ny > 2147483647LL) return LBM_ERR_INVALID_ARG;  // 32-bit in-plane offsets
    if (p->velocity_field != 0 && p->velocity_field != 1) return LBM_ERR_INVALID_ARG;
    const double vals[8] = {p->W, p->phi_a, p->phi_b, p->M_phi, p->D_s, p->u[0], p->u[1], p->u[2]};
    if (!finite_all(vals, 8) || !(p->W > 0.0) || p->phi_a == p->phi_b) return LBM_ERR_INVALID_ARG;
    if (std::fabs(p->phi_a) > 2.0 || std::fabs(p->phi_b) > 2.0) return LBM_ERR_INVALID_ARG;
    if (std::fabs(p->u[0]) >= 0.5 || std::fabs(p->u[1]) >= 0.5 || std::fabs(p->u[2]) >= 0.5)
        return LBM_ERR_INVALID_ARG;
    if (!(p->M_phi > 0.0) || !(p->D_s > 0.0)) return LBM_ERR_RATE;
    lbm3_ctx* ctx = new (std::nothrow) lbm3_ctx();
    if (!ctx) return LBM_ERR_NOMEM;
    ctx->p = *p;
    K3Params& kp = ctx->kp;
    kp.nx = p->nx;
    kp.ny = p->ny;
    kp.nz = p->nz;
    kp.nxny = (long long)p->nx * p->ny;
    kp.N = kp.nxny * p->nz;
    kp.seg_z = ctx->seg_z;
    kp.w_kappa = (float)rate_of(p->M_phi);
    kp.w_chi = (float)rate_of(p->D_s);
    kp.M_phi = (float)p->M_phi;
    kp.D_s = (float)p->D_s;
    kp.c4W = (float)(4.0 / p->W);
    kp.c8W = (float)(8.0 / p->W);
    kp.phi_a = (float)p->phi_a;
    kp.phi_b = (float)p->phi_b;
    kp.phim = (float)(0.5 * (p->phi_a + p->phi_b));
    kp.inv_dphi = (float)(1.0 / (p->phi_a - p->phi_b));
    for (int i = 0; i < 3; ++i) {
        kp.u[i] = (float)p->u[i];
        // the one-dimensional factors A, B, C of P^-1 F^-1(u) (see axis_factors)
        const double u = p->u[i], u2 = u * u, t = 1.0 / 3.0 + u2;
        const double f[3][3] = {{1.0 - t, 0.5 * (t + u), 0.5 * (t - u)},
                                {-2.0 * u, u + 0.5, u - 0.5},
                                {1.0 - u2, 0.5 * (u2 + u), 0.5 * (u2 - u)}};
        for (int k = 0; k < 3; ++k)
            for (int e = 0; e < 3; ++e) kp.fac[i][k][e] = (float)f[k][e];
    }
    kp.uf = nullptr;
    ctx->seg_z = p->nz < 64 ? p->nz : 64;
    cudaError_t e = cudaSuccess;
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        ctx->own_stream = e == cudaSuccess;
    }
    const size_t pop_bytes = sizeof(int) * 2 * Q27 * (size_t)kp.N;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&ctx->buf[i], pop_bytes);
    if (e == cudaSuccess && p->velocity_field) e = cudaMalloc(&ctx->uf, sizeof(float) * 3 * (size_t)kp.N);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->partial, sizeof(long long) * 3 * SUM_BLOCKS);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->result, sizeof(double) * 3);
    // defined contents before the first init (the autotuner may step them)
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMemsetAsync(ctx->buf[i], 0, pop_bytes, ctx->stream);
    if (e == cudaSuccess && ctx->uf) e = cudaMemsetAsync(ctx->uf, 0, sizeof(float) * 3 * (size_t)kp.N, ctx->stream);
    if (e != cudaSuccess) {
        const int rc = fail(nullptr, e);
        lbm3_destroy(ctx);
        cudaGetLastError();
        return rc;
    }
    kp.uf = ctx->uf;
    *out = ctx;
    return LBM_OK;
}

void lbm3_destroy(lbm3_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (int i = 0; i < 2; ++i) cudaFree(ctx->buf[i]);
    cudaFree(ctx->uf);
    cudaFree(ctx->partial);
    cudaFree(ctx->result);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int lbm3_init_fields_device(lbm3_ctx* ctx, const double* phi, const double* c, const double* ux,
                            const double* uy, const double* uz) {
    if (!ctx || !phi || !c) return LBM_ERR_INVALID_ARG;
    const bool field = ctx->p.velocity_field != 0;
    if (field && (!ux || !uy || !uz)) return LBM_ERR_INVALID_ARG;
    Nvtx r("lbm3_init_fields");
    const lbm3_params& p = ctx->p;
    ctx->cur = 0;
    k3_init<<<grid_1d(ctx->kp.N, 256), 256, 0, ctx->stream>>>(
        ctx->kp, phi, c, field ? ux : nullptr, field ? uy : nullptr, field ? uz : nullptr, p.W, p.phi_a,
        p.phi_b, p.M_phi, p.D_s, fbuf(ctx, 0), hbuf(ctx, 0), ctx->uf);
    ctx->step = 0;
    return fail(ctx, cudaGetLastError());
}

int lbm3_init_fields(lbm3_ctx* ctx, const double* phi, const double* c, const double* ux,
                     const double* uy, const double* uz) {
    if (!ctx || !phi || !c) return LBM_ERR_INVALID_ARG;
    const bool field = ctx->p.velocity_field != 0;
    if (field && (!ux || !uy || !uz)) return LBM_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)ctx->kp.N;
    const int nin = field ? 5 : 2;
    const double* host[5] = {phi, c, ux, uy, uz};
    double* dev = nullptr;
    cudaError_t e = cudaMallocAsync(&dev, bytes * nin, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);
    for (int i = 0; i < nin && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(dev + i * (size_t)ctx->kp.N, host[i], bytes, cudaMemcpyHostToDevice, ctx->stream);
    int rc = e == cudaSuccess ? LBM_OK : fail(ctx, e);
    if (rc == LBM_OK) {
        const size_t n = ctx->kp.N;
        rc = lbm3_init_fields_device(ctx, dev, dev + n, field ? dev + 2 * n : nullptr,
                                     field ? dev + 3 * n : nullptr, field ? dev + 4 * n : nullptr);
    }
    cudaFreeAsync(dev, ctx->stream);
    const int sync = lbm3_synchronize(ctx);
    return rc != LBM_OK ? rc : sync;
}

int lbm3_step(lbm3_ctx* ctx, int64_t nsteps) {
    if (!ctx || nsteps < 0) return LBM_ERR_INVALID_ARG;
    Nvtx r("lbm3_step");
    for (int64_t s = 0; s < nsteps; ++s) {
        const int rc = launch_step(ctx);
        if (rc != LBM_OK) return rc;
    }
    return LBM_OK;
}

int lbm3_get_fields_device(lbm3_ctx* ctx, double* phi, double* c) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (!phi && !c) return LBM_OK;
    k3_fields<<<grid_1d(ctx->kp.N, 256), 256, 0, ctx->stream>>>(ctx->kp, fbuf(ctx, ctx->cur),
                                                                 hbuf(ctx, ctx->cur), phi, c);
    return fail(ctx, cudaGetLastError());
}

int lbm3_get_fields(lbm3_ctx* ctx, double* phi, double* c) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (!phi && !c) return LBM_OK;
    const size_t n = ctx->kp.N, bytes = sizeof(double) * n;
    double* dev = nullptr;
    cudaError_t e = cudaMallocAsync(&dev, 2 * bytes, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);
    int rc = lbm3_get_fields_device(ctx, dev, dev + n);
    if (rc == LBM_OK && phi) rc = fail(ctx, cudaMemcpyAsync(phi, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (rc == LBM_OK && c) rc = fail(ctx, cudaMemcpyAsync(c, dev + n, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    cudaFreeAsync(dev, ctx->stream);
    const int sync = lbm3_synchronize(ctx);
    return rc != LBM_OK ? rc : sync;
}

int lbm3_get_populations_device(lbm3_ctx* ctx, double* f, double* h) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (!f && !h) return LBM_OK;
    const long long n = (long long)Q27 * ctx->kp.N;
    k3_pops<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(ctx->kp, fbuf(ctx, ctx->cur), hbuf(ctx, ctx->cur), f, h);
    return fail(ctx, cudaGetLastError());
}

int lbm3_get_populations(lbm3_ctx* ctx, double* f, double* h) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (!f && !h) return LBM_OK;
    const size_t n = (size_t)Q27 * ctx->kp.N, bytes = sizeof(double) * n;
    double* dev = nullptr;
    cudaError_t e = cudaMallocAsync(&dev, 2 * bytes, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);
    int rc = lbm3_get_populations_device(ctx, dev, dev + n);
    if (rc == LBM_OK && f) rc = fail(ctx, cudaMemcpyAsync(f, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (rc == LBM_OK && h) rc = fail(ctx, cudaMemcpyAsync(h, dev + n, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    cudaFreeAsync(dev, ctx->stream);
    const int sync = lbm3_synchronize(ctx);
    return rc != LBM_OK ? rc : sync;
}

int lbm3_sums(lbm3_ctx* ctx, double out[3]) {
    if (!ctx || !out) return LBM_ERR_INVALID_ARG;
    const long long total = Q27 * ctx->kp.N;
    k3_sum1<<<SUM_BLOCKS, SUM_THREADS, 0, ctx->stream>>>(total, fbuf(ctx, ctx->cur), hbuf(ctx, ctx->cur),
                                                         ctx->partial);
    k3_sum2<<<1, SUM_THREADS, 0, ctx->stream>>>(ctx->partial, ctx->result);
    int rc = fail(ctx, cudaGetLastError());
    if (rc == LBM_OK)
        rc = fail(ctx, cudaMemcpyAsync(out, ctx->result, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                       ctx->stream));
    const int sync = lbm3_synchronize(ctx);
    return rc != LBM_OK ? rc : sync;
}

int lbm3_velocities(int32_t out[81]) {
    if (!out) return LBM_ERR_INVALID_ARG;
    const int E[3] = {0, 1, -1};
    for (int q = 0; q < Q27; ++q) {
        out[3 * q + 0] = E[q % 3];
        out[3 * q + 1] = E[(q / 3) % 3];
        out[3 * q + 2] = E[q / 9];
    }
    return LBM_OK;
}

int lbm3_synchronize(lbm3_ctx* ctx) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, e);
    const int pend = ctx->pending_error;
    ctx->pending_error = LBM_OK;
    return pend;
}

int64_t lbm3_get_step(const lbm3_ctx* ctx) { return ctx ? ctx->step : -1; }

int lbm3_set_launch_shape(lbm3_ctx* ctx, int32_t rows, int32_t seg_z) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (rows != 0 && rows != 6 && rows != 10 && rows != 18) return LBM_ERR_INVALID_ARG;
    if (seg_z < 0) return LBM_ERR_INVALID_ARG;
    if (rows) ctx->rows = rows;
    if (seg_z) ctx->seg_z = seg_z < ctx->kp.nz ? seg_z : ctx->kp.nz;
    return LBM_OK;
}

int lbm3_get_launch_shape(const lbm3_ctx* ctx, int32_t* rows, int32_t* seg_z) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (rows) *rows = ctx->rows;
    if (seg_z) *seg_z = ctx->seg_z;
    return LBM_OK;
}

int lbm3_autotune(lbm3_ctx* ctx, int32_t steps, int32_t* rows_out, int32_t* seg_out, double* ms_out) {
    if (!ctx || steps < 1) return LBM_ERR_INVALID_ARG;
    Nvtx r("lbm3_autotune");
    const int nz = ctx->kp.nz;
    const int row_c[3] = {6, 10, 18};
    std::vector<int> segs;
    for (int s : {4, 8, 16, 32, 64, nz}) {
        const int v = s < nz ? s : nz;
        bool seen = false;
        for (int t : segs) seen = seen || t == v;
        if (!seen) segs.push_back(v);
    }
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return fail(ctx, cudaGetLastError());
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(ctx, cudaGetLastError());
    }
    double best = -1.0;
    int best_rows = ctx->rows, best_seg = ctx->seg_z;
    int rc = LBM_OK;
    for (int rows : row_c) {
        for (int seg : segs) {
            ctx->rows = rows;
            ctx->seg_z = seg;
            rc = launch_step(ctx);  // warm-up
            if (rc != LBM_OK) break;
            cudaEventRecord(ev[0], ctx->stream);
            for (int s = 0; s < steps && rc == LBM_OK; ++s) rc = launch_step(ctx);
            cudaEventRecord(ev[1], ctx->stream);
            if (rc != LBM_OK) break;
            cudaError_t e = cudaEventSynchronize(ev[1]);
            if (e != cudaSuccess) {
                rc = fail(ctx, e);
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            const double per = ms / steps;
            if (best < 0.0 || per < best) {
                best = per;
                best_rows = rows;
                best_seg = seg;
            }
        }
        if (rc != LBM_OK) break;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    ctx->rows = best_rows;
    ctx->seg_z = best_seg;
    if (rc != LBM_OK) return rc;
    if (rows_out) *rows_out = best_rows;
    if (seg_out) *seg_out = best_seg;
    if (ms_out) *ms_out = best;
    return lbm3_synchronize(ctx);
}

}  // extern "C"
