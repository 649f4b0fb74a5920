// C ABI of liblbm.so (declared in include/lbm.h): context management,
// parameter validation, host <-> device staging, CUDA-graph replay of long
// step loops, diagnostics and checkpoints.  All arithmetic of the method runs
// in the kernels of lbm_kernels.cu.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {
cudaError_t configure_fused_smem();
}

namespace {

constexpr int GRAPH_STEPS = 32;  // steps per captured graph (even: parity preserved)

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
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    CUtensorMap tmaps[2];   // bulk-tensor maps over the two population buffers
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
    for (int k = 0; k < 2; ++k)
        if (ctx->graph[k]) {
            cudaGraphExecDestroy(ctx->graph[k]);
            ctx->graph[k] = nullptr;
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
    if (p->dtype != LBM_F32) {
        if (p->dtype == LBM_F16S || p->dtype == LBM_BF16S) return LBM_ERR_UNSUPPORTED;
        return LBM_ERR_INVALID_ARG;
    }
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
    return k;
}

void launch_one_step(lbm_ctx* ctx, int src, cudaStream_t st) {
    if (ctx->kernel == LBM_KERNEL_SPLIT)
        lbm::launch_step_split(ctx->kp, ctx->ds, src, st);
    else if (ctx->kernel == LBM_KERNEL_TMA)
        lbm::launch_step_tma(ctx->kp, ctx->ds, src, ctx->shape, ctx->tmaps, ctx->derr, st);
    else
        lbm::launch_step_fused(ctx->kp, ctx->ds, src, ctx->shape, st);
}

int build_tensor_maps(lbm_ctx* ctx) {
    if (ctx->kernel != LBM_KERNEL_TMA) return LBM_OK;
    const int nplanes = ctx->ds.nlat * 9;
    for (int b = 0; b < 2; ++b)
        if (!lbm::make_tensor_map(&ctx->tmaps[b], ctx->pop_alloc[b], ctx->kp, nplanes,
                                  ctx->shape.bx))
            return LBM_ERR_UNSUPPORTED;
    return LBM_OK;
}

int build_graph(lbm_ctx* ctx, int parity) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    int src = parity;
    for (int s = 0; s < GRAPH_STEPS; ++s) {
        launch_one_step(ctx, src, ctx->cap_stream);
        src ^= 1;
    }
    e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    e = cudaGraphInstantiate(&ctx->graph[parity], g, 0);
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
    if (lbm::configure_fused_smem() != cudaSuccess || lbm::configure_tma_smem() != cudaSuccess) {
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
        cudaMalloc(&ctx->derr, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        lbm_destroy(ctx);
        return LBM_ERR_NOMEM;
    }
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
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int lbm_init_fields_device(lbm_ctx* ctx, const double* phi, const double* c, const double* ux,
                           const double* uy, const double* P) {
    if (!ctx || !phi || !c || !ux || !uy) return LBM_ERR_INVALID_ARG;
    lbm::launch_init(ctx->kp, ctx->ds, 0, phi, c, ux, uy, P, ctx->stream);
    ctx->cur = 0;
    ctx->step = 0;
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
    while (nsteps > 0) {
        if (nsteps >= GRAPH_STEPS && !ctx->kp.stall_test) {
            if (!ctx->graph[ctx->cur]) {
                int rc = build_graph(ctx, ctx->cur);
                if (rc != LBM_OK) return rc;
            }
            if (cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError());
            ctx->step += GRAPH_STEPS;
            nsteps -= GRAPH_STEPS;
        } else {
            launch_one_step(ctx, ctx->cur, ctx->stream);
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
    lbm::launch_fields(ctx->kp, ctx->ds, ctx->cur, ctx->stream);
    lbm::launch_macro_out(ctx->kp, ctx->ds, ctx->cur, phi, c, ux, uy, P, ctx->stream);
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
    lbm::launch_get_pops(ctx->kp, ctx->ds, ctx->cur, ctx->stage, ctx->stream);
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
    lbm::launch_set_pops(ctx->kp, ctx->ds, ctx->cur, dev[0], dev[1], dev[2], ctx->stream);
    rc = check_launch(ctx);
    if (rc != LBM_OK) return rc;
    return lbm_synchronize(ctx);
}

int lbm_diagnostics(lbm_ctx* ctx, lbm_diag* out) {
    if (!ctx || !out) return LBM_ERR_INVALID_ARG;
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
        cudaMemset(ctx->derr, 0, sizeof(int));
        ctx->pending_error = LBM_OK;
        return LBM_ERR_TIMEOUT;
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
    const bool ok_bx = tile_x == 0 || tile_x == 128 || (tile_x == 64 && ctx->kernel == LBM_KERNEL_TMA);
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

// Checkpoint file: magic, ABI version, parameters, step, buffer sizes, then
// the raw current population buffer and (fixed-velocity mode) the velocity.
static const char kMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '2'};

int lbm_save_state(lbm_ctx* ctx, const char* path) {
    if (!ctx || !path) return LBM_ERR_INVALID_ARG;
    int rc = lbm_synchronize(ctx);
    if (rc != LBM_OK) return rc;
    const size_t pop_n = (size_t)ctx->ds.nlat * 9 * (size_t)ctx->kp.plane;
    const size_t vel_n = ctx->kp.coupled ? 0 : 2 * (size_t)ctx->kp.plane;
    float* host = (float*)std::malloc(sizeof(float) * (pop_n + vel_n));
    if (!host) return LBM_ERR_NOMEM;
    cudaError_t e = cudaMemcpy(host, ctx->pop_alloc[ctx->cur], sizeof(float) * pop_n,
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
    const size_t pop_n = (size_t)ctx->ds.nlat * 9 * (size_t)ctx->kp.plane;
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
    cudaError_t e = cudaMemcpy(ctx->pop_alloc[ctx->cur], host, sizeof(float) * pop_n,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess && vel_n)
        e = cudaMemcpy(ctx->fields_alloc + lbm::FP_UX * ctx->kp.plane, host + pop_n,
                       sizeof(float) * vel_n, cudaMemcpyHostToDevice);
    std::free(host);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    ctx->step = step;
    return LBM_OK;
}

}  // extern "C"
