// Host-side declarations shared by the C-ABI layer and the kernel launchers.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_store16.cuh"

namespace lbm {

// Field scratch planes (float, pitched like the populations).
enum FieldPlane {
    FP_PHI = 0, FP_C, FP_DPS, FP_SIG, FP_NX, FP_NY, FP_GM, FP_UX, FP_UY, FP_COUNT
};

struct DevState {
    float* pop[2];          // ping-pong population buffers [nlat*9][ny][pitch]
    float* fields;          // FP_COUNT planes
    int nlat;               // 2 (fixed velocity) or 3 (coupled)
};

// Fused-kernel launch shape.
struct FusedShape {
    int bx;    // threads per block = interior columns + 4
    int seg;   // rows per block
};

// One run of a batch, as the batched step kernel sees it.
struct alignas(128) RunDesc {
    CUtensorMap tmap[2];    // bulk-tensor maps over the run's two population buffers
    KParams p;
    float* pop[2];
    float* fields;
    int seg;                // rows per tile
    int flip;               // the run reads buffer (parity ^ flip) at batch parity `parity`
};

// Launchers (all asynchronous on `st`).
void launch_step_split(const KParams& p, const DevState& s, int src, cudaStream_t st);
void launch_step_fused(const KParams& p, const DevState& s, int src, const FusedShape& sh,
                       cudaStream_t st);
size_t fused_smem_bytes(int bx);
// Fused step with bulk-tensor staging (lbm_sweep_tma.cu).
bool tma_available();
bool make_tensor_map(CUtensorMap* map, float* alloc, const KParams& p, int nplanes, int bx);
size_t tma_smem_bytes(int bx, bool coupled);
cudaError_t configure_tma_smem();
void launch_step_tma(const KParams& p, const DevState& s, int src, const FusedShape& sh,
                     const CUtensorMap* maps, int* err, cudaStream_t st);
// Batched step: one persistent launch over `nitems` tiles (int4: run, strip,
// segment, unused) of runs sharing block width bx and lattice count.
void launch_step_tma_batch(const RunDesc* runs, const int4* items, int nitems, int blocks,
                           int bx, bool coupled, int src, int* err, cudaStream_t st);
int tma_batch_blocks_per_sm(int bx, bool coupled);
int tma_blocks_per_sm(int bx, bool coupled);
// Fused TMA step with 16-bit storage (lbm_sweep_tma16.cu; block width 128 or 192).
// st: ST_F16 or ST_BF16 (lbm_store16.cuh); buffers hold store_planes(st, .)
// word planes, pointers to column 0 like the FP32 ones.
size_t tma16_smem_bytes(int bx, bool coupled);
cudaError_t configure_tma16_smem();
int tma16_blocks_per_sm(int bx, bool coupled, int st);
void launch_step_tma16(const KParams& p, float* src16, float* dst16, const float* fields,
                       const FusedShape& sh, const CUtensorMap& map, int st, int* err,
                       cudaStream_t s);
// Advance the device step counter of the stochastic rounding by n.
void launch_step_advance(unsigned* ctr, unsigned n, cudaStream_t s);
// Whole-buffer conversions between the FP32 deviation-form layout and the
// 16-bit layout (allocation base pointers; ghost columns included).
void launch_pack16(const KParams& p, const float* src32_alloc, float* dst16_alloc, int st,
                   cudaStream_t s);
void launch_unpack16(const KParams& p, const float* src16_alloc, float* dst32_alloc, int st,
                     cudaStream_t s);
// Fill the field planes (phi, c, dP*, sigma, n, |grad phi|) of the current state.
void launch_fields(const KParams& p, const DevState& s, int src, cudaStream_t st);
// Macroscopic outputs (float64, dense [ny][nx]) of the current state; needs launch_fields first.
void launch_macro_out(const KParams& p, const DevState& s, int src, double* phi, double* c,
                      double* ux, double* uy, double* P, cudaStream_t st);
// Initialisation from float64 fields (dense); writes buffer `dst` (uses the other as scratch).
void launch_init(const KParams& p, const DevState& s, int dst, const double* phi,
                 const double* c, const double* ux, const double* uy, const double* P,
                 cudaStream_t st);
// Post-streaming populations of buffer src as float64 dense [nlat*9][ny][nx].
void launch_get_pops(const KParams& p, const DevState& s, int src, double* out, cudaStream_t st);
// Replace buffer dst by given post-streaming populations (float64 dense [nlat*9][ny][nx]);
// lattices with a NULL pointer are taken from the current state of dst.
void launch_set_pops(const KParams& p, const DevState& s, int dst, const double* f,
                     const double* h, const double* g, cudaStream_t st);

// Connected components of {phi > level} (4-neighbour, periodic in x, and in
// y without walls) on the FP_PHI field plane: label init, one propagation
// sweep (sets *changed when a label moved), root count.
void launch_label_init(const KParams& p, const float* fields, float level, int* label,
                       cudaStream_t st);
void launch_label_step(const KParams& p, int* label, int* changed, cudaStream_t st);
void launch_label_roots(const KParams& p, const int* label, int* count, cudaStream_t st);
// FP64 reductions: partial sums per block into `partial`, then a fixed-order finish.
constexpr int DIAG_NSUM = 12;
int diag_blocks(const KParams& p);
void launch_diag(const KParams& p, const double* phi, const double* c, const double* ux,
                 const double* uy, double* partial, int nblocks, double* result,
                 cudaStream_t st);

}  // namespace lbm
