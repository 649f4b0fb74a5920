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

// Store modes of the bulk-tensor sweep (lbm_sweep2.cuh): direct stores from
// registers, or staged rows written by bulk-tensor stores.
constexpr int OUT_DIRECT = 0;
constexpr int OUT_STAGED = 1;

// Fused-kernel launch shape.
struct FusedShape {
    int bx;       // columns per block (interior columns + 4)
    int seg;      // rows per block
    int cpt = 1;  // cells (adjacent columns) per thread of the bulk-tensor sweep
    int out = 0;  // its store mode: 0 direct stores, 1 staged bulk-tensor stores
};

// Bulk-tensor store maps of one population buffer (bulk-tensor sweep): the
// scalar lattices' word planes and the flow lattice's, boxes {own columns,
// 1 row, planes}, over the columns -4 .. nx-1 of each row.
struct StoreMaps {
    CUtensorMap s, f;
};

// One run of a batch: its tensor maps (in global memory, where the
// persistent batch kernel reads them), buffers and buffer parity.
struct alignas(128) RunDesc {
    CUtensorMap tmap[2];    // bulk-tensor load maps over the run's two population buffers
    StoreMaps smap[2];      // bulk-tensor store maps over the same buffers
    float* pop[2];          // column 0 of each buffer
    float* fields;
    int seg;                // rows per tile
    int flip;               // the run reads buffer (parity ^ flip) at batch parity `parity`
};

// Tiling of up to BATCH_TABLE_RUNS runs, passed to the persistent batch
// kernel as one kernel parameter; larger batches take one launch per table
// per step.  Entry e covers the tiles first .. first + tiles - 1 of the
// launch, strip-major within its run (tile t: strip (t - first) % nsx,
// segment (t - first) / nsx); the run's parameters are slot slot0 + e of the
// batch parameter bank (constant memory, see batch_params_*).
constexpr int BATCH_TABLE_RUNS = 64;
struct BatchEntry {
    const CUtensorMap* tmap[2];   // the run's load maps (in its RunDesc, global memory)
    const StoreMaps* smap[2];     // its store maps (same)
    float* pop[2];                // column 0 of each of its buffers
    const float* fields;
    int first;      // first tile of this entry in the launch
    int nsx;        // strips (tiles across)
    int seg;        // rows per tile
    int flip;       // the run reads buffer (parity ^ flip) at batch parity `parity`
};
struct BatchTable {
    BatchEntry e[BATCH_TABLE_RUNS];
    int nentries;
    int ntiles;     // tiles of the launch
    int slot0;      // parameter-bank slot of entry 0
};
static_assert(sizeof(BatchTable) <= 32764, "kernel parameters are limited to 32764 bytes");

// The batch parameter bank: run parameters of the persistent batch kernel in
// constant memory, BATCH_PARAM_SLOTS slots per device, handed out in
// contiguous ranges (a kernel reads them with indexed constant loads, which
// the constant cache serves as it serves kernel parameters).
constexpr int BATCH_PARAM_SLOTS = 256;
int batch_params_alloc(int dev, int n);      // first slot of n free ones on device dev, or -1
void batch_params_free(int dev, int first, int n);
cudaError_t batch_params_upload(int first, const KParams* kp, int n, cudaStream_t st);

// Launchers (all asynchronous on `st`).
void launch_step_split(const KParams& p, const DevState& s, int src, cudaStream_t st);
void launch_step_fused(const KParams& p, const DevState& s, int src, const FusedShape& sh,
                       cudaStream_t st);
size_t fused_smem_bytes(int bx);
// Bulk-tensor load map over one population buffer: dims {pitch, ny, planes},
// box {bx + 4, 1, planes} (lbm_sweep_tma.cu).
bool tma_available();
bool make_tensor_map(CUtensorMap* map, float* alloc, const KParams& p, int nplanes, int bx);
// Bulk-tensor sweep with staged stores and cells per thread (lbm_sweep2.cuh):
// FP32 kernels in lbm_sweep_tma.cu, 16-bit ones in lbm_sweep_tma16.cu.
bool sweep2_shape_ok(int bx, int cpt, int st);
size_t sweep2_smem_bytes(int bx, int cpt, int out, bool coupled, int st);
int sweep2_blocks_per_sm(int bx, int cpt, int out, bool coupled, int st);
cudaError_t configure_sweep2_smem();
bool make_store_maps(StoreMaps* m, float* alloc, const KParams& p, int st, int bx);
void launch_step_sweep2(const KParams& p, float* dst, const float* fields, const FusedShape& sh,
                        const CUtensorMap& load_map, const StoreMaps& store_maps, int st,
                        int* err, cudaStream_t s);
// (per storage format)
bool sweep2_f32_shape_ok(int bx, int cpt);
size_t sweep2_f32_smem_bytes(int bx, int cpt, int out, bool coupled);
int sweep2_f32_blocks_per_sm(int bx, int cpt, int out, bool coupled);
cudaError_t configure_sweep2_f32_smem();
void launch_sweep2_f32(const KParams& p, float* dst, const float* fields, const FusedShape& sh,
                       const CUtensorMap& load_map, const StoreMaps& store_maps, int* err,
                       cudaStream_t s);
bool sweep2_16_shape_ok(int bx, int cpt);
size_t sweep2_16_smem_bytes(int bx, int cpt, int out, bool coupled);
int sweep2_16_blocks_per_sm(int bx, int cpt, int out, bool coupled, int st);
cudaError_t configure_sweep2_16_smem();
void launch_sweep2_16(const KParams& p, float* dst, const float* fields, const FusedShape& sh,
                      const CUtensorMap& load_map, const StoreMaps& store_maps, int st, int* err,
                      cudaStream_t s);
// Batched step: one persistent launch over the tab.ntiles tiles of the runs
// in `tab`, which share the launch shape (FP32 storage); step_off is the
// launch's offset within its graph (the stochastic roundings' step).
void launch_sweep2_batch(const BatchTable& tab, int blocks, const FusedShape& sh, bool coupled,
                         int parity, int step_off, int* err, cudaStream_t st);
int sweep2_batch_blocks_per_sm(int bx, int cpt, int out, bool coupled);
// Advance the device step counter of the stochastic roundings by n (one
// counter, or the counters of nctr runs).
void launch_step_advance(unsigned* ctr, unsigned n, cudaStream_t s);
void launch_step_advance_many(unsigned* const* ctrs, int nctr, unsigned n, cudaStream_t s);
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
