// C ABI of liblbm.so (declared in include/lbm.h): context management,
// parameter validation, host <-> device staging, CUDA-graph replay of long
// step loops, diagnostics and checkpoints.  All arithmetic of the method runs
// in the kernels of lbm_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

// NVTX range over a host call (header-only NVTX: free when no profiler is
// attached), for timelines of steps, graph replays, diagnostics and tuning.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

namespace lbm {
cudaError_t configure_fused_smem();
}

namespace {

constexpr int GRAPH_STEPS = 32;  // steps per captured graph (even: parity preserved)
// A single run replays any step count from captured graphs of 32, 16, 8, 4, 2
// and 1 steps (largest first), so short and long step counts take the same
// launch path; each chunk size has one graph per buffer parity.
constexpr int GRAPH_CHUNKS = 6;
constexpr int BATCH_SIDE_STREAMS = 16;  // concurrent run chains in a batch's graph

}  // namespace

struct lbm_ctx {
    lbm_params prm;
    lbm::KParams kp;
    lbm::DevState ds;           // kernel view: pointers to column 0 of each row
    float* pop_alloc[2] = {nullptr, nullptr};
    float* fields_alloc = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    int cur = 0;
    int64_t step = 0;
    int kernel = LBM_KERNEL_FUSED;
    lbm::FusedShape shape{128, 32};
    double* stage = nullptr;
    size_t stage_bytes = 0;
    double* dpartial = nullptr;
    double* dresult = nullptr;
    int diag_nb = 0;
    cudaGraphExec_t graph[GRAPH_CHUNKS][2] = {};  // [log2(32 / steps)][parity]
    CUtensorMap tmaps[2];   // bulk-tensor load maps over the two population buffers
    lbm::StoreMaps smaps[2];  // bulk-tensor store maps over the same buffers
    // 16-bit storage: the state lives in pop16 (word planes, lbm_store16.cuh);
    // the FP32 buffers stage initialisation and field output
    int st = lbm::ST_F32;
    float* pop16_alloc[2] = {nullptr, nullptr};
    unsigned* dstep = nullptr;  // step counter of the stochastic roundings
    int* derr = nullptr;    // device flag: a bounded wait expired
    int pending_error = LBM_OK;
};

namespace {

int cuda_fail(lbm_ctx* ctx, cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    if (ctx) ctx->pending_error = LBM_ERR_CUDA;
    return LBM_ERR_CUDA;
}

int check_launch(lbm_ctx* ctx) { return cuda_fail(ctx, cudaGetLastError()); }

void drop_graphs(lbm_ctx* ctx) {
    for (int c = 0; c < GRAPH_CHUNKS; ++c)
        for (int k = 0; k < 2; ++k)
            if (ctx->graph[c][k]) {
                cudaGraphExecDestroy(ctx->graph[c][k]);
                ctx->graph[c][k] = nullptr;
            }
}

int ensure_stage(lbm_ctx* ctx, size_t bytes) {
    if (ctx->stage_bytes >= bytes) return LBM_OK;
    if (ctx->stage) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
    }
    if (cudaMalloc(&ctx->stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_NOMEM;
    }
    ctx->stage_bytes = bytes;
    return LBM_OK;
}

int64_t cells(const lbm_ctx* ctx) { return (int64_t)ctx->prm.nx * ctx->prm.ny; }

int validate(const lbm_params* p) {
    if (!p) return LBM_ERR_INVALID_ARG;
    if (p->nx < 4 || p->ny < 4) return LBM_ERR_INVALID_ARG;
    if ((int64_t)p->nx * p->ny > (int64_t)1 << 31) return LBM_ERR_INVALID_ARG;
    if (p->walls_y != 0 && p->walls_y != 1) return LBM_ERR_INVALID_ARG;
    if (p->mode != LBM_COUPLED && p->mode != LBM_FIXED_U) return LBM_ERR_INVALID_ARG;
    if (p->kernel < LBM_KERNEL_AUTO || p->kernel > LBM_KERNEL_TMA) return LBM_ERR_INVALID_ARG;
    if (p->reserved != 0) return LBM_ERR_INVALID_ARG;
    if (p->dtype != LBM_F32 && p->dtype != LBM_F16S && p->dtype != LBM_BF16S)
        return LBM_ERR_INVALID_ARG;
    // 16-bit storage runs on the TMA sweep only
    if (p->dtype != LBM_F32 && p->kernel != LBM_KERNEL_AUTO && p->kernel != LBM_KERNEL_TMA)
        return LBM_ERR_UNSUPPORTED;
    if (!(p->W > 0.0) || p->phi_a == p->phi_b || !(p->c_max > 0.0)) return LBM_ERR_INVALID_ARG;
    if (!(p->M_phi > 0.0) || !(p->D_s > 0.0)) return LBM_ERR_RATE;
    if (p->mode == LBM_COUPLED) {
        if (!(p->nu_a > 0.0) || !(p->nu_b > 0.0) || !(p->zeta > 0.0)) return LBM_ERR_RATE;
        if (!(p->rho_a > 0.0) || !(p->rho_b > 0.0)) return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

lbm::KParams make_kparams(const lbm_params& p) {
    lbm::KParams k{};
    k.nx = p.nx;
    k.ny = p.ny;
    k.pitch = (p.nx + 2 * lbm::XGHOST + 31) / 32 * 32;
    k.walls = p.walls_y;
    k.coupled = p.mode == LBM_COUPLED;
    k.plane = (int64_t)k.pitch * p.ny;
    k.u_wall = (float)p.u_wall;
    k.W = (float)p.W;
    k.phi_a = (float)p.phi_a;
    k.phi_b = (float)p.phi_b;
    k.phi_m = (float)(0.5 * (p.phi_a + p.phi_b));
    k.inv_dphi = (float)(1.0 / (p.phi_a - p.phi_b));
    k.M_phi = (float)p.M_phi;
    k.D_s = (float)p.D_s;
    // D = cs2 (1/w - 1/2) for each transport coefficient
    k.w_kappa = (float)(1.0 / (3.0 * p.M_phi + 0.5));
    k.w_chi = (float)(1.0 / (3.0 * p.D_s + 0.5));
    k.w_zeta = (float)(1.0 / (3.0 * p.zeta + 0.5));
    k.nu_uniform = p.nu_a == p.nu_b;
    k.w_nu = (float)(1.0 / (3.0 * p.nu_a + 0.5));
    k.nu_a = (float)p.nu_a;
    k.nu_b = (float)p.nu_b;
    k.rho_uniform = p.rho_a == p.rho_b;
    k.rho_a = (float)p.rho_a;
    k.rho_b = (float)p.rho_b;
    k.rho_ref = (float)(0.5 * (p.rho_a + p.rho_b));
    k.sigma_o = (float)p.sigma_o;
    k.beta = (float)p.beta;
    k.inv_cmax = (float)(1.0 / p.c_max);
    const double dphi = p.phi_a - p.phi_b;
    k.N_sigma = p.sigma_literal ? 1.0f : (float)(1.5 * p.W / (dphi * dphi));
    k.fext_x = (float)p.fext_x;
    k.fext_y = (float)p.fext_y;
    k.P0 = (float)(0.5 * (p.rho_a + p.rho_b) / 3.0);
    k.four_over_W = (float)(4.0 / p.W);
    k.eight_over_W = (float)(8.0 / p.W);
    // fixed-point zeroth moments: 2^29 units per 2^e, with 2^e >= the largest
    // bound, so values within twice the bounds differ by less than 2^31
    const double bounds[2] = {std::fmax(std::fabs(p.phi_a), std::fabs(p.phi_b)), p.c_max};
    for (int l = 0; l < 2; ++l) {
        const int e = bounds[l] > 1.0 ? (int)std::ceil(std::log2(bounds[l])) : 0;
        const double scale = std::ldexp(1.0, 29 - e);
        k.fx_scale[l] = (float)scale;
        k.fx_inv[l] = (float)(1.0 / scale);
    }
    k.phi_a_fx = (int)std::llround(p.phi_a * k.fx_scale[0]);
    k.phi_b_fx = (int)std::llround(p.phi_b * k.fx_scale[0]);
    k.phi_m_fx = (int)std::llround(0.5 * (p.phi_a + p.phi_b) * k.fx_scale[0]);
    // 16-bit deviations: per-lattice power-of-two scales that bring the
    // expected largest deviation (a third of the largest first moment:
    // |u| + flux of the interface terms) near 1; FP16 only (BF16 has the FP32
    // exponent range).  k <= 14 keeps |d| up to 4 below FP16's 65504.
    const double U = std::fabs(p.u_wall);
    const double dphi_abs = std::fabs(p.phi_a - p.phi_b);
    const double mag[3] = {(U + p.M_phi / p.W) * dphi_abs / 3.0,
                           p.c_max * (U + 4.0 * p.D_s / p.W) / 3.0,
                           (U + 1e-6) / 3.0};
    for (int l = 0; l < 3; ++l) {
        int e = 0;
        if (p.dtype == LBM_F16S) {
            const double m = std::fmax(mag[l], std::ldexp(1.0, -14));
            e = (int)std::floor(std::log2(1.0 / m));
            e = e < 0 ? 0 : (e > 14 ? 14 : e);
        }
        k.qs[l] = (float)std::ldexp(1.0, e);
        k.qinv[l] = (float)std::ldexp(1.0, -e);
    }
    return k;
}

// One time step from buffer src; step_off is the launch's offset within a
// captured graph (the step counter of the stochastic roundings).
void launch_one_step(lbm_ctx* ctx, int src, cudaStream_t st, int step_off = 0) {
    lbm::KParams kp = ctx->kp;
    kp.step_off = step_off;
    if (ctx->kernel == LBM_KERNEL_TMA) {
        float* dst = ctx->st == lbm::ST_F32 ? ctx->ds.pop[1 - src]
                                            : ctx->pop16_alloc[1 - src] + lbm::XGHOST;
        lbm::launch_step_sweep2(kp, dst, ctx->ds.fields, ctx->shape, ctx->tmaps[src],
                                ctx->smaps[1 - src], ctx->st, ctx->derr, st);
    } else if (ctx->kernel == LBM_KERNEL_SPLIT) {
        lbm::launch_step_split(kp, ctx->ds, src, st);
    } else {
        lbm::launch_step_fused(kp, ctx->ds, src, ctx->shape, st);
    }
}

int build_tensor_maps(lbm_ctx* ctx) {
    if (ctx->kernel != LBM_KERNEL_TMA) return LBM_OK;
    const int nplanes = lbm::store_planes(ctx->st, ctx->kp.coupled);
    for (int b = 0; b < 2; ++b) {
        float* base = ctx->st == lbm::ST_F32 ? ctx->pop_alloc[b] : ctx->pop16_alloc[b];
        if (!lbm::make_tensor_map(&ctx->tmaps[b], base, ctx->kp, nplanes, ctx->shape.bx) ||
            !lbm::make_store_maps(&ctx->smaps[b], base, ctx->kp, ctx->st, ctx->shape.bx))
            return LBM_ERR_UNSUPPORTED;
    }
    return LBM_OK;
}

// Launch shape of a single run (the caller has checked it).
int set_shape(lbm_ctx* ctx, const lbm::FusedShape& sh) {
    ctx->shape = sh;
    drop_graphs(ctx);
    return build_tensor_maps(ctx);
}

// The device step counter of the stochastic rounding follows ctx->step
// (asynchronous on the context stream; no-op for FP32 storage).
void sync_step_ctr(lbm_ctx* ctx) {
    if (!ctx->dstep) return;
    static_assert(sizeof(unsigned) == 4, "32-bit counter");
    const unsigned v = (unsigned)ctx->step;
    cudaMemcpyAsync(ctx->dstep, &v, sizeof(unsigned), cudaMemcpyHostToDevice, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
}

// Words of one state buffer (the current storage format).
size_t state_words(const lbm_ctx* ctx) {
    return (size_t)lbm::store_planes(ctx->st, ctx->kp.coupled) * (size_t)ctx->kp.plane;
}

float* state_alloc(lbm_ctx* ctx, int b) {
    return ctx->st == lbm::ST_F32 ? ctx->pop_alloc[b] : ctx->pop16_alloc[b];
}

// The current state in FP32 deviation form, in buffer `b` of the FP32 pair
// (16-bit storage: expanded into FP32 buffer 0).  Returns the FP32 buffer index.
int fp32_view(lbm_ctx* ctx) {
    if (ctx->st == lbm::ST_F32) return ctx->cur;
    lbm::launch_unpack16(ctx->kp, ctx->pop16_alloc[ctx->cur], ctx->pop_alloc[0], ctx->st,
                         ctx->stream);
    return 0;
}

// Graph of GRAPH_STEPS >> chunk steps starting from buffer `parity`.
int build_graph(lbm_ctx* ctx, int parity, int chunk) {
    const int n = GRAPH_STEPS >> chunk;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    int src = parity;
    for (int s = 0; s < n; ++s) {
        launch_one_step(ctx, src, ctx->cap_stream, s);
        src ^= 1;
    }
    if (ctx->dstep) lbm::launch_step_advance(ctx->dstep, n, ctx->cap_stream);
    e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    e = cudaGraphInstantiate(&ctx->graph[chunk][parity], g, 0);
    cudaGraphDestroy(g);
    return cuda_fail(ctx, e);
}

}  // namespace

extern "C" {

int lbm_params_default(lbm_params* p) {
    if (!p) return LBM_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->mode = LBM_COUPLED;
    p->dtype = LBM_F32;
    p->kernel = LBM_KERNEL_AUTO;
    p->W = 4.0;
    p->phi_a = 1.0;
    p->phi_b = 0.0;
    p->M_phi = 0.1;
    p->D_s = 0.1;
    p->nu_a = p->nu_b = 0.1;
    p->zeta = 1.0 / 6.0;
    p->rho_a = p->rho_b = 1.0;
    p->c_max = 1.0;
    return LBM_OK;
}

int lbm_debug_stall_next_step(lbm_ctx* ctx) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (ctx->kernel != LBM_KERNEL_TMA) return LBM_ERR_UNSUPPORTED;
    ctx->kp.stall_test = 1;
    drop_graphs(ctx);
    return LBM_OK;
}

const char* lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_ERR_INVALID_ARG: return "invalid argument";
        case LBM_ERR_RATE: return "transport coefficient gives a relaxation rate outside (0, 2)";
        case LBM_ERR_SIGMA_NEG: return "Langmuir surface tension negative for the given concentration";
        case LBM_ERR_CUDA: return "CUDA runtime error";
        case LBM_ERR_NONFINITE: return "non-finite values in the state";
        case LBM_ERR_TIMEOUT: return "bounded device wait expired";
        case LBM_ERR_UNSUPPORTED: return "unsupported option";
        case LBM_ERR_IO: return "file input/output error";
        case LBM_ERR_NOMEM: return "allocation failed";
        default: return "unknown error";
    }
}

int lbm_create(const lbm_params* p, void* stream, lbm_ctx** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    int v = validate(p);
    if (v != LBM_OK) return v;
    lbm_ctx* ctx = new (std::nothrow) lbm_ctx();
    if (!ctx) return LBM_ERR_NOMEM;
    ctx->prm = *p;
    ctx->kp = make_kparams(*p);
    ctx->kernel = p->kernel == LBM_KERNEL_AUTO ? (lbm::tma_available() ? LBM_KERNEL_TMA
                                                                       : LBM_KERNEL_FUSED)
                                               : p->kernel;
    ctx->st = p->dtype == LBM_F16S ? lbm::ST_F16 : (p->dtype == LBM_BF16S ? lbm::ST_BF16 : lbm::ST_F32);
    // 16-bit rows leave through the staging area (staged bulk-tensor stores)
    ctx->shape.out = ctx->st == lbm::ST_F32 ? lbm::OUT_DIRECT : lbm::OUT_STAGED;
    if (ctx->kernel == LBM_KERNEL_TMA && !lbm::tma_available()) {
        delete ctx;
        return LBM_ERR_UNSUPPORTED;
    }
    cudaGetDevice(&ctx->device);
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return LBM_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        lbm_destroy(ctx);
        return LBM_ERR_CUDA;
    }
    if (lbm::configure_fused_smem() != cudaSuccess || lbm::configure_sweep2_smem() != cudaSuccess) {
        cudaGetLastError();
        lbm_destroy(ctx);
        return LBM_ERR_CUDA;
    }
    ctx->ds.nlat = ctx->kp.coupled ? 3 : 2;
    const size_t pop_bytes = sizeof(float) * (size_t)ctx->ds.nlat * 9 * (size_t)ctx->kp.plane;
    const size_t fld_bytes = sizeof(float) * (size_t)lbm::FP_COUNT * (size_t)ctx->kp.plane;
    ctx->diag_nb = lbm::diag_blocks(ctx->kp);
    if (cudaMalloc(&ctx->pop_alloc[0], pop_bytes) != cudaSuccess ||
        cudaMalloc(&ctx->pop_alloc[1], pop_bytes) != cudaSuccess ||
        cudaMalloc(&ctx->fields_alloc, fld_bytes) != cudaSuccess ||
        cudaMalloc(&ctx->dpartial, sizeof(double) * lbm::DIAG_NSUM * ctx->diag_nb) != cudaSuccess ||
        cudaMalloc(&ctx->dresult, sizeof(double) * 16) != cudaSuccess ||
        cudaMalloc(&ctx->derr, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->dstep, sizeof(unsigned)) != cudaSuccess ||
        (ctx->st != lbm::ST_F32 &&
         (cudaMalloc(&ctx->pop16_alloc[0], sizeof(float) * state_words(ctx)) != cudaSuccess ||
          cudaMalloc(&ctx->pop16_alloc[1], sizeof(float) * state_words(ctx)) != cudaSuccess))) {
        cudaGetLastError();
        lbm_destroy(ctx);
        return LBM_ERR_NOMEM;
    }
    for (int b = 0; b < 2 && ctx->st != lbm::ST_F32; ++b)
        cudaMemsetAsync(ctx->pop16_alloc[b], 0, sizeof(float) * state_words(ctx), ctx->stream);
    ctx->kp.step_ctr = ctx->dstep;
    if (ctx->dstep) cudaMemsetAsync(ctx->dstep, 0, sizeof(unsigned), ctx->stream);
    // a defined state before initialisation
    for (int b = 0; b < 2; ++b) ctx->ds.pop[b] = ctx->pop_alloc[b] + lbm::XGHOST;
    ctx->ds.fields = ctx->fields_alloc + lbm::XGHOST;
    cudaMemsetAsync(ctx->pop_alloc[0], 0, pop_bytes, ctx->stream);
    cudaMemsetAsync(ctx->pop_alloc[1], 0, pop_bytes, ctx->stream);
    cudaMemsetAsync(ctx->fields_alloc, 0, fld_bytes, ctx->stream);
    cudaMemsetAsync(ctx->derr, 0, sizeof(int), ctx->stream);
    if (build_tensor_maps(ctx) != LBM_OK) {
        lbm_destroy(ctx);
        return LBM_ERR_UNSUPPORTED;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        lbm_destroy(ctx);
        return LBM_ERR_CUDA;
    }
    *out = ctx;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    cudaFree(ctx->pop_alloc[0]);
    cudaFree(ctx->pop_alloc[1]);
    cudaFree(ctx->fields_alloc);
    cudaFree(ctx->stage);
    cudaFree(ctx->dpartial);
    cudaFree(ctx->dresult);
    cudaFree(ctx->derr);
    cudaFree(ctx->pop16_alloc[0]);
    cudaFree(ctx->pop16_alloc[1]);
    cudaFree(ctx->dstep);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int lbm_init_fields_device(lbm_ctx* ctx, const double* phi, const double* c, const double* ux,
                           const double* uy, const double* P) {
    if (!ctx || !phi || !c || !ux || !uy) return LBM_ERR_INVALID_ARG;
    lbm::launch_init(ctx->kp, ctx->ds, 0, phi, c, ux, uy, P, ctx->stream);
    if (ctx->st != lbm::ST_F32)
        lbm::launch_pack16(ctx->kp, ctx->pop_alloc[0], ctx->pop16_alloc[0], ctx->st, ctx->stream);
    ctx->cur = 0;
    ctx->step = 0;
    sync_step_ctr(ctx);
    return check_launch(ctx);
}

int lbm_init_fields(lbm_ctx* ctx, const double* phi, const double* c, const double* ux,
                    const double* uy, const double* P) {
    if (!ctx || !phi || !c || !ux || !uy) return LBM_ERR_INVALID_ARG;
    const int64_t n = cells(ctx);
    // the isotherm must stay positive over the given concentrations (Eq. EOS)
    double cmax_in = -1e300;
    for (int64_t k = 0; k < n; ++k) cmax_in = c[k] > cmax_in ? c[k] : cmax_in;
    if (ctx->prm.mode == LBM_COUPLED && ctx->prm.beta != 0.0) {
        const double arg = 1.0 - cmax_in / ctx->prm.c_max;
        if (!(arg > 0.0) || 1.0 + ctx->prm.beta * std::log(arg) < 0.0) return LBM_ERR_SIGMA_NEG;
    }
    int rc = ensure_stage(ctx, sizeof(double) * 5 * (size_t)n);
    if (rc != LBM_OK) return rc;
    const double* src[5] = {phi, c, ux, uy, P};
    for (int k = 0; k < 5; ++k)
        if (src[k] && cudaMemcpyAsync(ctx->stage + k * n, src[k], sizeof(double) * n,
                                      cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
            return cuda_fail(ctx, cudaGetLastError());
    rc = lbm_init_fields_device(ctx, ctx->stage, ctx->stage + n, ctx->stage + 2 * n,
                                ctx->stage + 3 * n, P ? ctx->stage + 4 * n : nullptr);
    if (rc != LBM_OK) return rc;
    return lbm_synchronize(ctx);
}

int lbm_step(lbm_ctx* ctx, int64_t nsteps) {
    if (!ctx || nsteps < 0) return LBM_ERR_INVALID_ARG;
    NvtxRange range("lbm_step");
    while (nsteps > 0) {
        if (!ctx->kp.stall_test) {
            int chunk = 0;
            while ((GRAPH_STEPS >> chunk) > nsteps) ++chunk;
            const int n = GRAPH_STEPS >> chunk;
            if (!ctx->graph[chunk][ctx->cur]) {
                int rc = build_graph(ctx, ctx->cur, chunk);
                if (rc != LBM_OK) return rc;
            }
            {
                NvtxRange replay("graph replay");
                if (cudaGraphLaunch(ctx->graph[chunk][ctx->cur], ctx->stream) != cudaSuccess)
                    return cuda_fail(ctx, cudaGetLastError());
            }
            ctx->cur ^= n & 1;
            ctx->step += n;
            nsteps -= n;
        } else {
            launch_one_step(ctx, ctx->cur, ctx->stream);
            if (ctx->dstep) lbm::launch_step_advance(ctx->dstep, 1, ctx->stream);
            ctx->cur ^= 1;
            ctx->step += 1;
            nsteps -= 1;
            if (ctx->kp.stall_test) {  // one-shot test hook
                ctx->kp.stall_test = 0;
                drop_graphs(ctx);
            }
        }
    }
    return check_launch(ctx);
}

int lbm_get_fields_device(lbm_ctx* ctx, double* phi, double* c, double* ux, double* uy,
                          double* P) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    const int b = fp32_view(ctx);
    lbm::launch_fields(ctx->kp, ctx->ds, b, ctx->stream);
    lbm::launch_macro_out(ctx->kp, ctx->ds, b, phi, c, ux, uy, P, ctx->stream);
    return check_launch(ctx);
}

int lbm_get_fields(lbm_ctx* ctx, double* phi, double* c, double* ux, double* uy, double* P) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    const int64_t n = cells(ctx);
    int rc = ensure_stage(ctx, sizeof(double) * 5 * (size_t)n);
    if (rc != LBM_OK) return rc;
    double* d[5] = {ctx->stage, ctx->stage + n, ctx->stage + 2 * n, ctx->stage + 3 * n,
                    ctx->stage + 4 * n};
    double* h[5] = {phi, c, ux, uy, P};
    rc = lbm_get_fields_device(ctx, h[0] ? d[0] : nullptr, h[1] ? d[1] : nullptr,
                               h[2] ? d[2] : nullptr, h[3] ? d[3] : nullptr,
                               h[4] ? d[4] : nullptr);
    if (rc != LBM_OK) return rc;
    for (int k = 0; k < 5; ++k)
        if (h[k] && cudaMemcpyAsync(h[k], d[k], sizeof(double) * n, cudaMemcpyDeviceToHost,
                                    ctx->stream) != cudaSuccess)
            return cuda_fail(ctx, cudaGetLastError());
    return lbm_synchronize(ctx);
}

int lbm_get_populations(lbm_ctx* ctx, double* f, double* h, double* g) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    const int64_t n = cells(ctx);
    const int nl = ctx->ds.nlat;
    int rc = ensure_stage(ctx, sizeof(double) * 9 * nl * (size_t)n);
    if (rc != LBM_OK) return rc;
    lbm::launch_get_pops(ctx->kp, ctx->ds, fp32_view(ctx), ctx->stage, ctx->stream);
    rc = check_launch(ctx);
    if (rc != LBM_OK) return rc;
    double* out[3] = {f, h, g};
    for (int l = 0; l < nl; ++l)
        if (out[l] && cudaMemcpyAsync(out[l], ctx->stage + (size_t)l * 9 * n,
                                      sizeof(double) * 9 * n, cudaMemcpyDeviceToHost,
                                      ctx->stream) != cudaSuccess)
            return cuda_fail(ctx, cudaGetLastError());
    return lbm_synchronize(ctx);
}

int lbm_set_populations(lbm_ctx* ctx, const double* f, const double* h, const double* g) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    const int64_t n = cells(ctx);
    const int nl = ctx->ds.nlat;
    int rc = ensure_stage(ctx, sizeof(double) * 9 * nl * (size_t)n);
    if (rc != LBM_OK) return rc;
    const double* in[3] = {f, h, g};
    const double* dev[3] = {nullptr, nullptr, nullptr};
    for (int l = 0; l < nl; ++l) {
        if (!in[l]) continue;
        if (cudaMemcpyAsync(ctx->stage + (size_t)l * 9 * n, in[l], sizeof(double) * 9 * n,
                            cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
            return cuda_fail(ctx, cudaGetLastError());
        dev[l] = ctx->stage + (size_t)l * 9 * n;
    }
    const int b = fp32_view(ctx);
    lbm::launch_set_pops(ctx->kp, ctx->ds, b, dev[0], dev[1], dev[2], ctx->stream);
    if (ctx->st != lbm::ST_F32)
        lbm::launch_pack16(ctx->kp, ctx->pop_alloc[0], ctx->pop16_alloc[ctx->cur], ctx->st,
                           ctx->stream);
    rc = check_launch(ctx);
    if (rc != LBM_OK) return rc;
    return lbm_synchronize(ctx);
}

int lbm_diagnostics(lbm_ctx* ctx, lbm_diag* out) {
    if (!ctx || !out) return LBM_ERR_INVALID_ARG;
    NvtxRange range("lbm_diagnostics");
    const int64_t n = cells(ctx);
    int rc = ensure_stage(ctx, sizeof(double) * 5 * (size_t)n);
    if (rc != LBM_OK) return rc;
    double* d = ctx->stage;
    rc = lbm_get_fields_device(ctx, d, d + n, d + 2 * n, d + 3 * n, nullptr);
    if (rc != LBM_OK) return rc;
    lbm::launch_diag(ctx->kp, d, d + n, d + 2 * n, d + 3 * n, ctx->dpartial, ctx->diag_nb,
                     ctx->dresult, ctx->stream);
    rc = check_launch(ctx);
    if (rc != LBM_OK) return rc;
    double res[16];
    if (cudaMemcpyAsync(res, ctx->dresult, sizeof(double) * 13, cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError());
    rc = lbm_synchronize(ctx);
    if (rc != LBM_OK) return rc;
    std::memset(out, 0, sizeof(*out));
    out->step = ctx->step;
    out->sum_phi = res[0];
    out->sum_c = res[1];
    out->xc = res[2];
    out->yc = res[3];
    out->nonfinite = (int64_t)res[4];
    out->sigma_neg = (int64_t)res[5];
    out->umax = res[6];
    out->L = res[10];
    out->B = res[11];
    out->D = res[12];
    out->status = out->nonfinite > 0 ? LBM_ERR_NONFINITE : LBM_OK;
    return LBM_OK;
}

int lbm_count_components(lbm_ctx* ctx, double level, int32_t* count) {
    if (!ctx || !count) return LBM_ERR_INVALID_ARG;
    const int64_t n = cells(ctx);
    // labels and flags live in the staging buffer (int32 per cell, then 2 ints)
    int rc = ensure_stage(ctx, sizeof(int) * (size_t)(n + 2) + sizeof(double));
    if (rc != LBM_OK) return rc;
    int* label = reinterpret_cast<int*>(ctx->stage);
    int* flag = label + n;  // [0]: changed, [1]: root count
    const int b = fp32_view(ctx);
    lbm::launch_fields(ctx->kp, ctx->ds, b, ctx->stream);
    lbm::launch_label_init(ctx->kp, ctx->ds.fields, (float)level, label, ctx->stream);
    // each sweep moves every label at least one cell and halves pointer
    // chains, so n sweeps always suffice
    for (int64_t it = 0; it < n + 1; ++it) {
        int changed = 0;
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream);
        if (e == cudaSuccess) {
            lbm::launch_label_step(ctx->kp, label, flag, ctx->stream);
            e = cudaMemcpyAsync(&changed, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
        if (!changed) break;
    }
    int roots = 0;
    cudaError_t e = cudaMemsetAsync(flag + 1, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) {
        lbm::launch_label_roots(ctx->kp, label, flag + 1, ctx->stream);
        e = cudaMemcpyAsync(&roots, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    *count = roots;
    return lbm_synchronize(ctx);
}

int lbm_synchronize(lbm_ctx* ctx) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    int timed_out = 0;
    e = cudaMemcpy(&timed_out, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    if (timed_out) {
        // 1: a bounded wait expired; 2: a kernel found its shared memory misaligned
        cudaMemset(ctx->derr, 0, sizeof(int));
        ctx->pending_error = LBM_OK;
        return timed_out == 1 ? LBM_ERR_TIMEOUT : LBM_ERR_CUDA;
    }
    int pend = ctx->pending_error;
    ctx->pending_error = LBM_OK;
    return pend;
}

int64_t lbm_get_step(const lbm_ctx* ctx) { return ctx ? ctx->step : -1; }

int lbm_kernel_in_use(const lbm_ctx* ctx) { return ctx ? ctx->kernel : LBM_ERR_INVALID_ARG; }

int lbm_launches_per_step(const lbm_ctx* ctx) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    return ctx->kernel == LBM_KERNEL_SPLIT ? 3 : 1;
}

int lbm_set_launch_shape(lbm_ctx* ctx, int32_t tile_x, int32_t seg_y) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (ctx->kernel == LBM_KERNEL_SPLIT) return LBM_ERR_UNSUPPORTED;
    if (tile_x < 0 || (tile_x != 0 && (tile_x % 32 != 0 || tile_x < 64 || tile_x > 512)))
        return LBM_ERR_INVALID_ARG;
    if (seg_y != 0 && seg_y < 4) return LBM_ERR_INVALID_ARG;
    const bool tma = ctx->kernel == LBM_KERNEL_TMA;
    const bool ok_bx = tile_x == 0 || (tma ? lbm::sweep2_shape_ok(tile_x, ctx->shape.cpt, ctx->st)
                                           : tile_x == 128);
    if (!ok_bx) return LBM_ERR_UNSUPPORTED;
    if (tile_x) ctx->shape.bx = tile_x;
    if (seg_y) ctx->shape.seg = seg_y;
    drop_graphs(ctx);
    return build_tensor_maps(ctx);
}

int lbm_get_launch_shape(const lbm_ctx* ctx, int32_t* tile_x, int32_t* seg_y) {
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (tile_x) *tile_x = ctx->shape.bx;
    if (seg_y) *seg_y = ctx->shape.seg;
    return LBM_OK;
}

int lbm_set_cells_per_thread(lbm_ctx* ctx, int32_t cells) {
    if (!ctx || cells < 1 || cells > 2) return LBM_ERR_INVALID_ARG;
    if (ctx->kernel != LBM_KERNEL_TMA) return cells == 1 ? LBM_OK : LBM_ERR_UNSUPPORTED;
    if (!lbm::sweep2_shape_ok(ctx->shape.bx, cells, ctx->st)) return LBM_ERR_UNSUPPORTED;
    ctx->shape.cpt = cells;
    drop_graphs(ctx);
    return LBM_OK;
}

int32_t lbm_get_cells_per_thread(const lbm_ctx* ctx) {
    return ctx ? ctx->shape.cpt : LBM_ERR_INVALID_ARG;
}

int lbm_set_store_mode(lbm_ctx* ctx, int32_t mode) {
    if (!ctx || (mode != LBM_STORE_DIRECT && mode != LBM_STORE_STAGED)) return LBM_ERR_INVALID_ARG;
    if (ctx->kernel != LBM_KERNEL_TMA) return mode == LBM_STORE_DIRECT ? LBM_OK : LBM_ERR_UNSUPPORTED;
    ctx->shape.out = mode;
    drop_graphs(ctx);
    return LBM_OK;
}

int32_t lbm_get_store_mode(const lbm_ctx* ctx) {
    return ctx ? ctx->shape.out : LBM_ERR_INVALID_ARG;
}

// Checkpoint file: magic, ABI version, parameters, step, buffer sizes, then
// the raw current population buffer and (fixed-velocity mode) the velocity.
static const char kMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '2'};

int lbm_save_state(lbm_ctx* ctx, const char* path) {
    if (!ctx || !path) return LBM_ERR_INVALID_ARG;
    int rc = lbm_synchronize(ctx);
    if (rc != LBM_OK) return rc;
    const size_t pop_n = state_words(ctx);
    const size_t vel_n = ctx->kp.coupled ? 0 : 2 * (size_t)ctx->kp.plane;
    float* host = (float*)std::malloc(sizeof(float) * (pop_n + vel_n));
    if (!host) return LBM_ERR_NOMEM;
    cudaError_t e = cudaMemcpy(host, state_alloc(ctx, ctx->cur), sizeof(float) * pop_n,
                               cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && vel_n)
        e = cudaMemcpy(host + pop_n, ctx->fields_alloc + lbm::FP_UX * ctx->kp.plane,
                       sizeof(float) * vel_n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        std::free(host);
        return cuda_fail(ctx, e);
    }
    FILE* fp = std::fopen(path, "wb");
    if (!fp) {
        std::free(host);
        return LBM_ERR_IO;
    }
    int32_t ver = LBM_ABI_VERSION;
    uint64_t np = pop_n, nv = vel_n;
    bool ok = std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(&ver, 4, 1, fp) == 1 &&
              std::fwrite(&ctx->prm, sizeof(lbm_params), 1, fp) == 1 &&
              std::fwrite(&ctx->step, 8, 1, fp) == 1 &&
              std::fwrite(&np, 8, 1, fp) == 1 &&
              std::fwrite(&nv, 8, 1, fp) == 1 &&
              std::fwrite(host, sizeof(float), pop_n + vel_n, fp) == pop_n + vel_n;
    ok = (std::fclose(fp) == 0) && ok;
    std::free(host);
    return ok ? LBM_OK : LBM_ERR_IO;
}

int lbm_load_state(lbm_ctx* ctx, const char* path) {
    if (!ctx || !path) return LBM_ERR_INVALID_ARG;
    int rc = lbm_synchronize(ctx);
    if (rc != LBM_OK) return rc;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return LBM_ERR_IO;
    char magic[8];
    int32_t ver = 0;
    lbm_params prm;
    int64_t step = 0;
    uint64_t np = 0, nv = 0;
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&ver, 4, 1, fp) == 1 && ver == LBM_ABI_VERSION &&
              std::fread(&prm, sizeof(lbm_params), 1, fp) == 1 &&
              std::fread(&step, 8, 1, fp) == 1 &&
              std::fread(&np, 8, 1, fp) == 1 &&
              std::fread(&nv, 8, 1, fp) == 1;
    if (!ok) {
        std::fclose(fp);
        return LBM_ERR_IO;
    }
    const size_t pop_n = state_words(ctx);
    const size_t vel_n = ctx->kp.coupled ? 0 : 2 * (size_t)ctx->kp.plane;
    lbm_params mine = ctx->prm, theirs = prm;
    mine.kernel = theirs.kernel = 0;  // the kernel variant does not change the state
    if (std::memcmp(&mine, &theirs, sizeof(lbm_params)) != 0 || np != pop_n || nv != vel_n) {
        std::fclose(fp);
        return LBM_ERR_INVALID_ARG;
    }
    float* host = (float*)std::malloc(sizeof(float) * (pop_n + vel_n));
    if (!host) {
        std::fclose(fp);
        return LBM_ERR_NOMEM;
    }
    ok = std::fread(host, sizeof(float), pop_n + vel_n, fp) == pop_n + vel_n;
    std::fclose(fp);
    if (!ok) {
        std::free(host);
        return LBM_ERR_IO;
    }
    cudaError_t e = cudaMemcpy(state_alloc(ctx, ctx->cur), host, sizeof(float) * pop_n,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess && vel_n)
        e = cudaMemcpy(ctx->fields_alloc + lbm::FP_UX * ctx->kp.plane, host + pop_n,
                       sizeof(float) * vel_n, cudaMemcpyHostToDevice);
    std::free(host);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    ctx->step = step;
    sync_step_ctr(ctx);
    return lbm_synchronize(ctx);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many runs advanced together, in one of two forms.
//  * persistent: every step is one launch of the persistent batch kernel over
//    the tiles of all runs (one launch per table of BATCH_TABLE_RUNS runs);
//    all runs share the block width, cells per thread and rows per tile.
//  * chains: every run is stepped by its own single-run launches, each run
//    with its own launch shape, the runs' chains spread over side streams.
// Either form is replayed from captured graphs of 32, 16, 8, 4, 2 and 1
// steps.  Both run the same tile sweep, so a batched step gives the same bits
// as stepping each run's context on its own with the same launch shape.
// ---------------------------------------------------------------------------

struct lbm_batch {
    int nruns = 0;
    lbm_ctx** runs = nullptr;       // sub-contexts (own their buffers; share the stream)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    bool coupled = true;
    int form = LBM_BATCH_PERSISTENT;
    lbm::FusedShape shape{192, 32, 1};  // shape of the persistent form
    // persistent form: tables of run parameters and tilings, grids
    int ntab = 0;
    lbm::BatchTable* htab = nullptr;    // [ntab]
    int* tab_blocks = nullptr;          // [ntab] grid sizes
    int nitems = 0;                     // tiles of a step
    lbm::RunDesc* hdesc = nullptr;      // host copy of the run table
    lbm::RunDesc* ddesc = nullptr;
    int slot0 = -1;                     // the runs' first parameter-bank slot (-1: none)
    int dev = 0;                        // the device the batch was created on
    unsigned** dctrs = nullptr;         // the runs' step counters (device array)
    lbm::KParams* hkp = nullptr;        // the runs' parameters the graphs were built with
    int* derr = nullptr;
    int parity = 0;
    bool desc_valid = false;
    cudaGraphExec_t graph[GRAPH_CHUNKS][2] = {};
    int pending_error = LBM_OK;
    // chains form: side streams for the per-run chains, fork/join events
    int nside = 0;
    cudaStream_t side[BATCH_SIDE_STREAMS] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[BATCH_SIDE_STREAMS] = {};
};

namespace {

void batch_drop_graphs(lbm_batch* b) {
    for (int c = 0; c < GRAPH_CHUNKS; ++c)
        for (int k = 0; k < 2; ++k)
            if (b->graph[c][k]) {
                cudaGraphExecDestroy(b->graph[c][k]);
                b->graph[c][k] = nullptr;
            }
}

int batch_fail(lbm_batch* b, cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    cudaGetLastError();
    b->pending_error = LBM_ERR_CUDA;
    return LBM_ERR_CUDA;
}

// Tensor maps, parameter tables, tilings and grids of the persistent form
// for its current launch shape; run tables to the device.
int batch_build_tiles(lbm_batch* b) {
    batch_drop_graphs(b);
    const int bx = b->shape.bx, tx = bx - 4;
    const int nl = b->coupled ? 3 : 2;
    int64_t total = 0;
    for (int r = 0; r < b->nruns; ++r) {
        const lbm_ctx* c = b->runs[r];
        total += (int64_t)((c->kp.nx + tx - 1) / tx) * ((c->kp.ny + b->shape.seg - 1) / b->shape.seg);
    }
    if (total > (int64_t)1 << 30) return LBM_ERR_INVALID_ARG;
    const int per_sm = lbm::sweep2_batch_blocks_per_sm(bx, b->shape.cpt, b->shape.out, b->coupled);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int r = 0; r < b->nruns; ++r) {
        lbm_ctx* c = b->runs[r];
        lbm::RunDesc& d = b->hdesc[r];
        for (int k = 0; k < 2; ++k) {
            if (!lbm::make_tensor_map(&d.tmap[k], c->pop_alloc[k], c->kp, nl * 9, bx) ||
                !lbm::make_store_maps(&d.smap[k], c->pop_alloc[k], c->kp, lbm::ST_F32, bx))
                return LBM_ERR_UNSUPPORTED;
            d.pop[k] = c->ds.pop[k];
        }
        d.fields = c->ds.fields;
        d.seg = b->shape.seg;
        d.flip = c->cur ^ b->parity;
        b->hkp[r] = c->kp;
    }
    // table t: runs t * BATCH_TABLE_RUNS + e, tiles run after run
    for (int t = 0; t < b->ntab; ++t) {
        lbm::BatchTable& tab = b->htab[t];
        const int r0 = t * lbm::BATCH_TABLE_RUNS;
        const int r1 = std::min(b->nruns, r0 + lbm::BATCH_TABLE_RUNS);
        int first = 0;
        for (int r = r0; r < r1; ++r) {
            const lbm_ctx* c = b->runs[r];
            const lbm::RunDesc& d = b->hdesc[r];
            lbm::BatchEntry& en = tab.e[r - r0];
            const int nsx = (c->kp.nx + tx - 1) / tx, nsy = (c->kp.ny + b->shape.seg - 1) / b->shape.seg;
            for (int k = 0; k < 2; ++k) {
                en.tmap[k] = &b->ddesc[r].tmap[k];
                en.smap[k] = &b->ddesc[r].smap[k];
                en.pop[k] = d.pop[k];
            }
            en.fields = d.fields;
            en.first = first;
            en.nsx = nsx;
            en.seg = d.seg;
            en.flip = d.flip;
            first += nsx * nsy;
        }
        tab.nentries = r1 - r0;
        tab.ntiles = first;
        tab.slot0 = b->slot0 + r0;
        b->tab_blocks[t] = std::min(first, per_sm * (nsm > 0 ? nsm : 1));
    }
    cudaError_t e = cudaMemcpy(b->ddesc, b->hdesc, sizeof(lbm::RunDesc) * b->nruns,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b->slot0 >= 0)
        e = lbm::batch_params_upload(b->slot0, b->hkp, b->nruns, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e);
    b->nitems = (int)total;
    b->desc_valid = true;
    return LBM_OK;
}

// Re-upload the run table if a run was stepped, re-initialised or reloaded
// on its own since the last batched step (its buffer parity or parameters
// may differ from the table's).
int batch_sync_desc(lbm_batch* b) {
    bool dirty = !b->desc_valid;
    for (int r = 0; r < b->nruns && !dirty; ++r) {
        const lbm_ctx* c = b->runs[r];
        dirty = b->hdesc[r].flip != (c->cur ^ b->parity) ||
                std::memcmp(&b->hkp[r], &c->kp, sizeof(lbm::KParams)) != 0;
    }
    if (!dirty) return LBM_OK;
    batch_drop_graphs(b);  // the graphs' launches carry the old parities and parameters
    for (int r = 0; r < b->nruns; ++r) {
        b->hdesc[r].flip = b->runs[r]->cur ^ b->parity;
        b->hkp[r] = b->runs[r]->kp;
        b->htab[r / lbm::BATCH_TABLE_RUNS].e[r % lbm::BATCH_TABLE_RUNS].flip = b->hdesc[r].flip;
    }
    cudaError_t e = cudaMemcpyAsync(b->ddesc, b->hdesc, sizeof(lbm::RunDesc) * b->nruns,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && b->slot0 >= 0)
        e = lbm::batch_params_upload(b->slot0, b->hkp, b->nruns, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    b->desc_valid = true;
    return batch_fail(b, e);
}

// n steps of the persistent form from batch parity `parity` on stream st
// (step_off: offset of the first step within its graph).
void batch_persistent_steps(lbm_batch* b, int parity, int n, cudaStream_t st) {
    for (int s = 0; s < n; ++s)
        for (int t = 0; t < b->ntab; ++t) {
            lbm::BatchTable& tab = b->htab[t];
            lbm::launch_sweep2_batch(tab, b->tab_blocks[t], b->shape, b->coupled,
                                     parity ^ (s & 1), s, b->derr, st);
        }
    lbm::launch_step_advance_many(b->dctrs, b->nruns, (unsigned)n, st);
}

// n steps of the chains form: run r's chain starts from its buffer
// parity ^ flip[r].  Runs go to the side streams largest first, each to the
// stream with the fewest cells so far, so the chains end together.
cudaError_t batch_chain_steps(lbm_batch* b, int parity, int n, cudaStream_t st) {
    cudaError_t e = cudaEventRecord(b->fork_ev, st);
    for (int k = 0; k < b->nside && e == cudaSuccess; ++k)
        e = cudaStreamWaitEvent(b->side[k], b->fork_ev, 0);
    int64_t load[BATCH_SIDE_STREAMS] = {};
    bool* done = (bool*)std::calloc((size_t)b->nruns, sizeof(bool));
    if (!done && e == cudaSuccess) e = cudaErrorMemoryAllocation;
    for (int a = 0; a < b->nruns && e == cudaSuccess; ++a) {
        int r = -1;
        int64_t best = -1;
        for (int q = 0; q < b->nruns; ++q) {
            const int64_t cells = (int64_t)b->runs[q]->kp.nx * b->runs[q]->kp.ny;
            if (!done[q] && cells > best) {
                best = cells;
                r = q;
            }
        }
        done[r] = true;
        int k = 0;
        for (int q = 1; q < b->nside; ++q)
            if (load[q] < load[k]) k = q;
        load[k] += best;
        lbm_ctx* c = b->runs[r];
        int src = parity ^ b->hdesc[r].flip;
        for (int s = 0; s < n; ++s) {
            lbm::KParams kp = c->kp;
            kp.step_off = s;
            float* dst = c->ds.pop[1 - src];
            lbm::launch_step_sweep2(kp, dst, c->ds.fields, c->shape, c->tmaps[src],
                                    c->smaps[1 - src], lbm::ST_F32, b->derr, b->side[k]);
            src ^= 1;
        }
        lbm::launch_step_advance(c->dstep, (unsigned)n, b->side[k]);
        e = cudaGetLastError();
    }
    std::free(done);
    for (int k = 0; k < b->nside && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join_ev[k], b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join_ev[k], 0);
    }
    return e;
}

// Graph of GRAPH_STEPS >> chunk steps of the batch's form from batch parity `parity`.
int batch_build_graph(lbm_batch* b, int parity, int chunk) {
    const int n = GRAPH_STEPS >> chunk;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, e);
    if (b->form == LBM_BATCH_PERSISTENT) {
        batch_persistent_steps(b, parity, n, b->cap_stream);
        e = cudaGetLastError();
    } else {
        e = batch_chain_steps(b, parity, n, b->cap_stream);
    }
    const cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &g);
    if (e == cudaSuccess) e = ee;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return batch_fail(b, e);
    }
    e = cudaGraphInstantiate(&b->graph[chunk][parity], g, 0);
    cudaGraphDestroy(g);
    return batch_fail(b, e);
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params* params, int32_t nruns, void* stream, lbm_batch** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || nruns < 1) return LBM_ERR_INVALID_ARG;
    for (int r = 0; r < nruns; ++r) {
        const int v = validate(&params[r]);
        if (v != LBM_OK) return v;
        if (params[r].mode != params[0].mode) return LBM_ERR_INVALID_ARG;
        if (params[r].kernel != LBM_KERNEL_AUTO && params[r].kernel != LBM_KERNEL_TMA)
            return LBM_ERR_UNSUPPORTED;
        if (params[r].dtype != LBM_F32) return LBM_ERR_UNSUPPORTED;  // batches store FP32
    }
    if (!lbm::tma_available()) return LBM_ERR_UNSUPPORTED;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_NOMEM;
    b->coupled = params[0].mode == LBM_COUPLED;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return LBM_ERR_CUDA;
        }
        b->own_stream = true;
    }
    b->ntab = (nruns + lbm::BATCH_TABLE_RUNS - 1) / lbm::BATCH_TABLE_RUNS;
    b->runs = (lbm_ctx**)std::calloc((size_t)nruns, sizeof(lbm_ctx*));
    b->hdesc = (lbm::RunDesc*)std::calloc((size_t)nruns, sizeof(lbm::RunDesc));
    b->hkp = (lbm::KParams*)std::calloc((size_t)nruns, sizeof(lbm::KParams));
    b->htab = (lbm::BatchTable*)std::calloc((size_t)b->ntab, sizeof(lbm::BatchTable));
    b->tab_blocks = (int*)std::calloc((size_t)b->ntab, sizeof(int));
    if (!b->runs || !b->hdesc || !b->hkp || !b->htab || !b->tab_blocks) {
        lbm_batch_destroy(b);
        return LBM_ERR_NOMEM;
    }
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
        lbm_batch_destroy(b);
        return LBM_ERR_CUDA;
    }
    for (int k = 0; k < std::min<int>(nruns, BATCH_SIDE_STREAMS); ++k) {
        if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming) != cudaSuccess) {
            lbm_batch_destroy(b);
            return LBM_ERR_CUDA;
        }
        b->nside = k + 1;
    }
    for (int r = 0; r < nruns; ++r) {
        lbm_params pr = params[r];
        pr.kernel = LBM_KERNEL_TMA;
        const int rc = lbm_create(&pr, b->stream, &b->runs[r]);
        if (rc != LBM_OK) {
            lbm_batch_destroy(b);
            return rc;
        }
        b->nruns = r + 1;
    }
    unsigned** hctrs = (unsigned**)std::malloc(sizeof(unsigned*) * (size_t)nruns);
    if (!hctrs) {
        lbm_batch_destroy(b);
        return LBM_ERR_NOMEM;
    }
    for (int r = 0; r < nruns; ++r) hctrs[r] = b->runs[r]->dstep;
    // parameter-bank slots of the persistent form; without them the batch
    // runs in the chains form only
    if (cudaGetDevice(&b->dev) != cudaSuccess) cudaGetLastError();
    b->slot0 = lbm::batch_params_alloc(b->dev, nruns);
    if (b->slot0 < 0) b->form = LBM_BATCH_CHAINS;
    cudaError_t e = cudaMalloc(&b->ddesc, sizeof(lbm::RunDesc) * (size_t)nruns);
    if (e == cudaSuccess) e = cudaMalloc(&b->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->dctrs, sizeof(unsigned*) * (size_t)nruns);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dctrs, hctrs, sizeof(unsigned*) * (size_t)nruns, cudaMemcpyHostToDevice);
    std::free(hctrs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lbm_batch_destroy(b);
        return LBM_ERR_NOMEM;
    }
    cudaMemset(b->derr, 0, sizeof(int));
    // the runs' own shapes (chains form) follow the persistent shape until tuned
    for (int r = 0; r < nruns; ++r) {
        const int rc = set_shape(b->runs[r], b->shape);
        if (rc != LBM_OK) {
            lbm_batch_destroy(b);
            return rc;
        }
    }
    const int rc = batch_build_tiles(b);
    if (rc != LBM_OK) {
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    if (b->slot0 >= 0) lbm::batch_params_free(b->dev, b->slot0, b->nruns);
    for (int r = 0; r < b->nruns; ++r) lbm_destroy(b->runs[r]);
    std::free(b->runs);
    std::free(b->hdesc);
    std::free(b->hkp);
    std::free(b->htab);
    std::free(b->tab_blocks);
    cudaFree(b->ddesc);
    cudaFree(b->dctrs);
    cudaFree(b->derr);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int k = 0; k < BATCH_SIDE_STREAMS; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int32_t lbm_batch_size(const lbm_batch* b) { return b ? b->nruns : LBM_ERR_INVALID_ARG; }

lbm_ctx* lbm_batch_run(lbm_batch* b, int32_t run) {
    if (!b || run < 0 || run >= b->nruns) return nullptr;
    return b->runs[run];
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_INVALID_ARG;
    NvtxRange range("lbm_batch_step");
    int rc = batch_sync_desc(b);
    if (rc != LBM_OK) return rc;
    bool stall = false;
    for (int r = 0; r < b->nruns; ++r) stall = stall || b->runs[r]->kp.stall_test;
    int64_t left = nsteps;
    while (left > 0) {
        if (stall) {
            // the test hook: one uncaptured step with the stall flags, then clear them
            const cudaError_t e = b->form == LBM_BATCH_PERSISTENT
                                      ? (batch_persistent_steps(b, b->parity, 1, b->stream),
                                         cudaGetLastError())
                                      : batch_chain_steps(b, b->parity, 1, b->stream);
            if (e != cudaSuccess) return batch_fail(b, e);
            b->parity ^= 1;
            left -= 1;
            for (int r = 0; r < b->nruns; ++r) {
                b->runs[r]->kp.stall_test = 0;
                b->hkp[r].stall_test = 0;
                drop_graphs(b->runs[r]);
            }
            // (stream-ordered after the step that read the flags)
            if (b->slot0 >= 0) {
                const cudaError_t e2 =
                    lbm::batch_params_upload(b->slot0, b->hkp, b->nruns, b->stream);
                if (e2 != cudaSuccess) return batch_fail(b, e2);
            }
            stall = false;
            continue;
        }
        int chunk = 0;
        while ((GRAPH_STEPS >> chunk) > left) ++chunk;
        const int n = GRAPH_STEPS >> chunk;
        if (!b->graph[chunk][b->parity]) {
            rc = batch_build_graph(b, b->parity, chunk);
            if (rc != LBM_OK) return rc;
        }
        if (cudaGraphLaunch(b->graph[chunk][b->parity], b->stream) != cudaSuccess)
            return batch_fail(b, cudaGetLastError());
        b->parity ^= n & 1;
        left -= n;
    }
    // every run advanced by nsteps: its current buffer follows the batch parity
    for (int r = 0; r < b->nruns; ++r) {
        lbm_ctx* c = b->runs[r];
        c->cur = b->parity ^ b->hdesc[r].flip;
        c->step += nsteps;
    }
    return batch_fail(b, cudaGetLastError());
}

int lbm_batch_synchronize(lbm_batch* b) {
    if (!b) return LBM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e);
    int timed_out = 0;
    e = cudaMemcpy(&timed_out, b->derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return batch_fail(b, e);
    if (timed_out) {
        cudaMemset(b->derr, 0, sizeof(int));
        b->pending_error = LBM_OK;
        return timed_out == 1 ? LBM_ERR_TIMEOUT : LBM_ERR_CUDA;
    }
    const int pend = b->pending_error;
    b->pending_error = LBM_OK;
    return pend;
}

int lbm_batch_set_form(lbm_batch* b, int32_t form) {
    if (!b || (form != LBM_BATCH_CHAINS && form != LBM_BATCH_PERSISTENT))
        return LBM_ERR_INVALID_ARG;
    if (form == LBM_BATCH_PERSISTENT && b->slot0 < 0) return LBM_ERR_UNSUPPORTED;
    const int rc = lbm_batch_synchronize(b);
    if (rc != LBM_OK) return rc;
    b->form = form;
    batch_drop_graphs(b);
    return LBM_OK;
}

int32_t lbm_batch_get_form(const lbm_batch* b) { return b ? b->form : LBM_ERR_INVALID_ARG; }

int lbm_batch_set_launch_shape(lbm_batch* b, int32_t tile_x, int32_t seg_y) {
    if (!b) return LBM_ERR_INVALID_ARG;
    if (tile_x != 0 && !lbm::sweep2_shape_ok(tile_x, b->shape.cpt, lbm::ST_F32))
        return LBM_ERR_UNSUPPORTED;
    if (seg_y != 0 && seg_y < 4) return LBM_ERR_INVALID_ARG;
    const int rc = lbm_batch_synchronize(b);
    if (rc != LBM_OK) return rc;
    if (tile_x) b->shape.bx = tile_x;
    if (seg_y) b->shape.seg = seg_y;
    for (int r = 0; r < b->nruns; ++r) {
        const int rr = set_shape(b->runs[r], b->shape);
        if (rr != LBM_OK) return rr;
    }
    return batch_build_tiles(b);
}

int lbm_batch_set_store_mode(lbm_batch* b, int32_t mode) {
    if (!b || (mode != LBM_STORE_DIRECT && mode != LBM_STORE_STAGED)) return LBM_ERR_INVALID_ARG;
    const int rc = lbm_batch_synchronize(b);
    if (rc != LBM_OK) return rc;
    b->shape.out = mode;
    for (int r = 0; r < b->nruns; ++r) {
        const int rr = set_shape(b->runs[r], b->shape);
        if (rr != LBM_OK) return rr;
    }
    return batch_build_tiles(b);
}

int lbm_batch_set_cells_per_thread(lbm_batch* b, int32_t cells) {
    if (!b || cells < 1 || cells > 2) return LBM_ERR_INVALID_ARG;
    if (!lbm::sweep2_shape_ok(b->shape.bx, cells, lbm::ST_F32)) return LBM_ERR_UNSUPPORTED;
    const int rc = lbm_batch_synchronize(b);
    if (rc != LBM_OK) return rc;
    b->shape.cpt = cells;
    for (int r = 0; r < b->nruns; ++r) {
        const int rr = set_shape(b->runs[r], b->shape);
        if (rr != LBM_OK) return rr;
    }
    return batch_build_tiles(b);
}

int lbm_batch_get_launch_shape(const lbm_batch* b, int32_t* tile_x, int32_t* seg_y,
                               int32_t* blocks, int32_t* tiles) {
    if (!b) return LBM_ERR_INVALID_ARG;
    if (tile_x) *tile_x = b->shape.bx;
    if (seg_y) *seg_y = b->shape.seg;
    int nb = 0;
    for (int t = 0; t < b->ntab; ++t) nb += b->tab_blocks[t];
    if (blocks) *blocks = nb;
    if (tiles) *tiles = b->nitems;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch-shape autotuner: times candidate (block width, rows per block) pairs
// on the live state, then puts the state back as it was.
// ---------------------------------------------------------------------------

namespace {

int sm_count() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

// Rows per block worth trying for a grid of nx x ny: a fixed ladder plus the
// values that fill one or two waves of resident blocks.
int seg_candidates(int nx, int ny, int bx, int per_sm, int* out, int cap) {
    int n = 0;
    auto add = [&](int seg) {
        if (seg < 4) seg = 4;
        if (seg > ny && ny >= 4) seg = ny;
        for (int k = 0; k < n; ++k)
            if (out[k] == seg) return;
        if (n < cap) out[n++] = seg;
    };
    const int ladder[] = {8, 16, 32, 64, 128};
    for (int v : ladder) add(v);
    const int strips = (nx + bx - 5) / (bx - 4);
    const int slots = per_sm * sm_count();
    for (int w = 1; w <= 2; ++w) {
        const int nseg = (w * slots) / strips;
        if (nseg >= 1) add((ny + nseg - 1) / nseg);
    }
    return n;
}

}  // namespace

extern "C" {

int lbm_autotune(lbm_ctx* ctx, int32_t steps, int32_t* tile_x, int32_t* seg_y,
                 double* ms_per_step) {
    NvtxRange range("lbm_autotune");
    if (!ctx || steps < 1) return LBM_ERR_INVALID_ARG;
    if (ctx->kernel == LBM_KERNEL_SPLIT) return LBM_ERR_UNSUPPORTED;
    int rc = lbm_synchronize(ctx);
    if (rc != LBM_OK) return rc;
    const size_t pop_bytes = sizeof(float) * state_words(ctx);
    float* snap = nullptr;
    if (cudaMalloc(&snap, pop_bytes) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_NOMEM;
    }
    const int cur0 = ctx->cur;
    const int64_t step0 = ctx->step;
    const lbm::FusedShape shape0 = ctx->shape;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMemcpy(snap, state_alloc(ctx, cur0), pop_bytes, cudaMemcpyDeviceToDevice);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    double best = 1e300;
    lbm::FusedShape best_shape = shape0;
    // (block width, cells per thread, store mode) candidates of the kernel in use
    int cand[10][3] = {{128, 1, 0}};
    int ncand = 1;
    if (ctx->kernel == LBM_KERNEL_TMA) {
        const int all[5][2] = {{128, 1}, {192, 1}, {64, 1}, {128, 2}, {192, 2}};
        ncand = 0;
        for (int out = 0; out < 2; ++out)
            for (const auto& c : all)
                if (lbm::sweep2_shape_ok(c[0], c[1], ctx->st)) {
                    cand[ncand][0] = c[0];
                    cand[ncand][1] = c[1];
                    cand[ncand][2] = out;
                    ++ncand;
                }
    }
    for (int a = 0; a < ncand && ce == cudaSuccess && rc == LBM_OK; ++a) {
        const int bx = cand[a][0], cpt = cand[a][1], out = cand[a][2];
        const int per_sm = ctx->kernel != LBM_KERNEL_TMA
                               ? 2
                               : lbm::sweep2_blocks_per_sm(bx, cpt, out, ctx->kp.coupled, ctx->st);
        int segs[8];
        const int ns = seg_candidates(ctx->kp.nx, ctx->kp.ny, bx, per_sm, segs, 8);
        for (int k = 0; k < ns && rc == LBM_OK; ++k) {
            rc = set_shape(ctx, lbm::FusedShape{bx, segs[k], cpt, out});
            if (rc != LBM_OK) break;
            // twice the timed count first: captures the graphs the timed
            // steps replay, from either buffer parity
            rc = lbm_step(ctx, 2 * (int64_t)steps);
            if (rc == LBM_OK) rc = cuda_fail(ctx, cudaEventRecord(e0, ctx->stream));
            if (rc == LBM_OK) rc = lbm_step(ctx, steps);
            if (rc == LBM_OK) rc = cuda_fail(ctx, cudaEventRecord(e1, ctx->stream));
            if (rc == LBM_OK) rc = lbm_synchronize(ctx);
            float ms = 0.0f;
            if (rc == LBM_OK) rc = cuda_fail(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (rc == LBM_OK && ms / steps < best) {
                best = ms / steps;
                best_shape = lbm::FusedShape{bx, segs[k], cpt, out};
            }
            // put the state back before the next candidate
            ce = cudaMemcpy(state_alloc(ctx, cur0), snap, pop_bytes, cudaMemcpyDeviceToDevice);
            ctx->cur = cur0;
            ctx->step = step0;
            sync_step_ctr(ctx);
            if (ce != cudaSuccess) break;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(snap);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce);
    const int rc2 = set_shape(ctx, best_shape);
    if (rc != LBM_OK) return rc;
    if (rc2 != LBM_OK) return rc2;
    if (tile_x) *tile_x = best_shape.bx;
    if (seg_y) *seg_y = best_shape.seg;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int32_t steps, int32_t* tile_x, int32_t* seg_y,
                       double* ms_per_step) {
    NvtxRange range("lbm_batch_autotune");
    if (!b || steps < 1) return LBM_ERR_INVALID_ARG;
    const int tsteps = (steps + GRAPH_STEPS - 1) / GRAPH_STEPS * GRAPH_STEPS;
    int rc = lbm_batch_synchronize(b);
    if (rc != LBM_OK) return rc;
    float** snap = (float**)std::calloc((size_t)b->nruns, sizeof(float*));
    int* cur0 = (int*)std::calloc((size_t)b->nruns, sizeof(int));
    int64_t* step0 = (int64_t*)std::calloc((size_t)b->nruns, sizeof(int64_t));
    lbm::FusedShape* run_shape = (lbm::FusedShape*)std::calloc((size_t)b->nruns, sizeof(lbm::FusedShape));
    lbm::FusedShape* best_runs = (lbm::FusedShape*)std::calloc((size_t)b->nruns, sizeof(lbm::FusedShape));
    if (!snap || !cur0 || !step0 || !run_shape || !best_runs) {
        std::free(snap);
        std::free(cur0);
        std::free(step0);
        std::free(run_shape);
        std::free(best_runs);
        return LBM_ERR_NOMEM;
    }
    cudaError_t ce = cudaSuccess;
    auto bytes_of = [&](int r) {
        const lbm_ctx* c = b->runs[r];
        return sizeof(float) * (size_t)c->ds.nlat * 9 * (size_t)c->kp.plane;
    };
    for (int r = 0; r < b->nruns && ce == cudaSuccess; ++r) {
        cur0[r] = b->runs[r]->cur;
        step0[r] = b->runs[r]->step;
        ce = cudaMalloc(&snap[r], bytes_of(r));
        if (ce == cudaSuccess)
            ce = cudaMemcpy(snap[r], b->runs[r]->pop_alloc[cur0[r]], bytes_of(r),
                            cudaMemcpyDeviceToDevice);
    }
    auto restore = [&]() {
        for (int r = 0; r < b->nruns && ce == cudaSuccess; ++r) {
            lbm_ctx* c = b->runs[r];
            ce = cudaMemcpy(c->pop_alloc[cur0[r]], snap[r], bytes_of(r), cudaMemcpyDeviceToDevice);
            c->cur = cur0[r];
            c->step = step0[r];
            sync_step_ctr(c);
        }
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    // time the current form and shape: one graph of warm-up, then tsteps
    auto time_it = [&](double& ms_step) -> int {
        int r2 = lbm_batch_step(b, GRAPH_STEPS);
        if (r2 == LBM_OK) r2 = batch_fail(b, cudaEventRecord(e0, b->stream));
        if (r2 == LBM_OK) r2 = lbm_batch_step(b, tsteps);
        if (r2 == LBM_OK) r2 = batch_fail(b, cudaEventRecord(e1, b->stream));
        if (r2 == LBM_OK) r2 = lbm_batch_synchronize(b);
        float ms = 0.0f;
        if (r2 == LBM_OK) r2 = batch_fail(b, cudaEventElapsedTime(&ms, e0, e1));
        ms_step = ms / tsteps;
        restore();
        return r2;
    };
    const int form0 = b->form;
    const lbm::FusedShape shape0 = b->shape;
    lbm::FusedShape best_shape = shape0;
    int best_form = form0;
    double best = 1e300;
    // persistent form (when the batch holds parameter-bank slots)
    b->form = LBM_BATCH_PERSISTENT;
    // block widths, cells per thread and store modes, each with a range of
    // tile heights (the tile count against the grid decides the last wave)
    const int ncand = b->slot0 >= 0 ? 6 : 0;
    const int cand[6][3] = {{64, 1, 0}, {128, 1, 0}, {192, 1, 0}, {64, 1, 1}, {128, 1, 1}, {128, 2, 1}};
    const int segs[7] = {24, 32, 40, 48, 56, 64, 80};
    for (int a = 0; a < ncand && ce == cudaSuccess && rc == LBM_OK; ++a) {
        for (int k = 0; k < 7 && ce == cudaSuccess && rc == LBM_OK; ++k) {
            b->shape = lbm::FusedShape{cand[a][0], segs[k], cand[a][1], cand[a][2]};
            rc = batch_build_tiles(b);
            double ms = 0.0;
            if (rc == LBM_OK) rc = time_it(ms);
            if (rc == LBM_OK && ms < best) {
                best = ms;
                best_form = LBM_BATCH_PERSISTENT;
                best_shape = b->shape;
            }
        }
    }
    // chains form: every grid size tuned on its first run (the shape shared
    // by the runs of that size), then a few shapes common to all runs (with
    // the runs' chains side by side, wider tiles can win over the shapes a
    // run picks when it has the GPU to itself)
    auto time_chains = [&]() {
        for (int r = 0; r < b->nruns && rc == LBM_OK; ++r) rc = set_shape(b->runs[r], run_shape[r]);
        b->form = LBM_BATCH_CHAINS;
        batch_drop_graphs(b);
        double ms = 0.0;
        if (rc == LBM_OK) rc = time_it(ms);
        if (rc == LBM_OK && ms < best) {
            best = ms;
            best_form = LBM_BATCH_CHAINS;
            std::memcpy(best_runs, run_shape, sizeof(lbm::FusedShape) * (size_t)b->nruns);
        }
    };
    if (ce == cudaSuccess && rc == LBM_OK) {
        for (int r = 0; r < b->nruns && rc == LBM_OK; ++r) {
            lbm_ctx* c = b->runs[r];
            int src_run = -1;
            for (int q = 0; q < r && src_run < 0; ++q)
                if (b->runs[q]->kp.nx == c->kp.nx && b->runs[q]->kp.ny == c->kp.ny) src_run = q;
            if (src_run >= 0) {
                run_shape[r] = run_shape[src_run];
            } else {
                int tx = 0, sy = 0;
                rc = lbm_autotune(c, 32, &tx, &sy, nullptr);
                run_shape[r] = c->shape;
            }
        }
        if (rc == LBM_OK) time_chains();
        const lbm::FusedShape common[3] = {{192, 38, 1, 0}, {128, 32, 1, 0}, {192, 38, 2, 0}};
        for (int a = 0; a < 3 && ce == cudaSuccess && rc == LBM_OK; ++a) {
            for (int r = 0; r < b->nruns; ++r) run_shape[r] = common[a];
            time_chains();
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int r = 0; r < b->nruns; ++r) cudaFree(snap[r]);
    std::free(snap);
    std::free(cur0);
    std::free(step0);
    std::free(run_shape);
    if (ce != cudaSuccess || rc != LBM_OK) {
        std::free(best_runs);
        return ce != cudaSuccess ? batch_fail(b, ce) : rc;
    }
    // keep the winner: the persistent shape always; the runs' own shapes
    // are the winning chains shapes if the chains form won, else follow the
    // persistent shape
    b->form = best_form;
    b->shape = best_shape;
    for (int r = 0; r < b->nruns && rc == LBM_OK; ++r)
        rc = set_shape(b->runs[r], best_form == LBM_BATCH_CHAINS ? best_runs[r] : best_shape);
    std::free(best_runs);
    if (rc == LBM_OK) rc = batch_build_tiles(b);
    if (rc != LBM_OK) return rc;
    if (tile_x) *tile_x = best_shape.bx;
    if (seg_y) *seg_y = best_shape.seg;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

}  // extern "C"
