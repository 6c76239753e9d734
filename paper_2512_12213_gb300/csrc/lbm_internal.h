// lbm_internal.h -- host-side context of the C ABI and the per-storage-format
// dispatch table of kernel launchers.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// one boundary link (x_f, a'): node in the padded layout, direction a'
// pointing into the wall, and the wall id (8 bytes)
struct Link {
    uint32_t node;
    uint16_t dir;
    uint16_t wall;
};

// out_on_host of a reduction: LBM_OUT_DEVICE / LBM_OUT_HOST always; the
// asynchronous host copy only into page-locked memory and without
// accumulation (the host value would be read before the copy lands)
inline bool out_mode_ok(int mode, bool accumulate, const void* out, std::string& err)
{
    if (mode < LBM_OUT_DEVICE || mode > LBM_OUT_HOST_ASYNC) {
        err = "out_on_host must be LBM_OUT_DEVICE, LBM_OUT_HOST or LBM_OUT_HOST_ASYNC";
        return false;
    }
    if (mode != LBM_OUT_HOST_ASYNC) return true;
    if (accumulate) {
        err = "LBM_OUT_HOST_ASYNC cannot be combined with LBM_ACCUMULATE";
        return false;
    }
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, out) != cudaSuccess) {
        cudaGetLastError();
        err = "LBM_OUT_HOST_ASYNC: cannot query the output pointer";
        return false;
    }
    if (a.type != cudaMemoryTypeHost) {
        err = "LBM_OUT_HOST_ASYNC needs page-locked host memory";
        return false;
    }
    return true;
}

constexpr int MAX_PARTIAL_ROWS = 1024;   // block partials of one reduction
constexpr int ADJ_BLOCKS = 2048;         // fixed grid of the adjoint kernel
constexpr int PARTIAL_WIDTH = 8;         // doubles per partial row
// scratch layout (doubles): [reduction rows | adjoint rows | 8 result slots]
constexpr size_t SCRATCH_RED_OFF = 0;
constexpr size_t SCRATCH_ADJ_OFF = (size_t)MAX_PARTIAL_ROWS * PARTIAL_WIDTH;
constexpr size_t SCRATCH_OUT_OFF = SCRATCH_ADJ_OFF + (size_t)ADJ_BLOCKS * 6;
constexpr size_t SCRATCH_FLAG_OFF = SCRATCH_OUT_OFF + 8;   // device error flags (unsigned)
constexpr size_t SCRATCH_TICKET_OFF = SCRATCH_FLAG_OFF + 1; // last-block ticket of the fused wall force (unsigned)
constexpr size_t SCRATCH_DOUBLES = SCRATCH_FLAG_OFF + 8;
// insulating walls only, after the above: the field block (E, the sum of v,
// the force coefficient in FP64, FP32 and FP32 storage units, the ticket of
// the last-block reduction), the stage-one rows of the velocity sum, then one
// row of 3 doubles per warp of the step grid
constexpr size_t SCRATCH_INS_OFF = SCRATCH_DOUBLES;
constexpr int INS_E = 0, INS_VSUM = 3, INS_AEB_D = 6, INS_AEB_F = 9, INS_AEB_S = 11;   // doubles into the block
constexpr int INS_TICKET = 14;                                                         // unsigned in a double slot
constexpr int INS_RED_ROWS = 1024;
constexpr size_t SCRATCH_INS_RED = SCRATCH_INS_OFF + 16;
constexpr size_t SCRATCH_INS_ROWS = SCRATCH_INS_RED + (size_t)INS_RED_ROWS * 3;

struct Ctx;
struct StgForce;

struct Dispatch {
    cudaError_t (*step)(const Ctx&, const void* src, void* dst, uint32_t seed, cudaStream_t);
    // the staged step with the wall force of the stored state's step fused in
    cudaError_t (*step_force)(const Ctx&, const void* src, void* dst, uint32_t seed, const StgForce& fw,
                              cudaStream_t);
    cudaError_t (*import_f)(const Ctx&, const void* src, int dtype, void* dst, cudaStream_t);
    cudaError_t (*init_fields)(const Ctx&, const double* rho, const double* u, const double* xi, void* dst,
                               cudaStream_t);
    cudaError_t (*export_f)(const Ctx&, const void* P, void* out, int dtype, cudaStream_t);
    cudaError_t (*links)(const Ctx&, const void* P, long long begin, long long end, unsigned flags,
                         double* partials, int* nblocks, cudaStream_t);
    cudaError_t (*balance)(const Ctx&, const void* P, double* partials, int* nblocks, cudaStream_t);
    cudaError_t (*residual)(const Ctx&, const void* P, double* vref, int update, double* partials, int* nblocks,
                            cudaStream_t);
    cudaError_t (*stress)(const Ctx&, const void* cur, const void* prev, int variant, void* sig, void* S,
                          void* rho, void* v, cudaStream_t);
    // induced field: the coupled step, both field buffers at rest in the
    // external field, B(x, T) in canonical order
    cudaError_t (*mhd_step)(const Ctx&, const void* src, void* dst, const void* G, void* Gn, uint32_t seed,
                            cudaStream_t);
    cudaError_t (*mag_init)(const Ctx&, cudaStream_t);
    cudaError_t (*mag_field)(const Ctx&, double* B, cudaStream_t);
    cudaError_t (*adjoint)(const Ctx&, const void* Pprev, const void* phin, void* phio, int wall,
                           const double* dir, double seedw, double* partials, cudaStream_t);
};

const Dispatch& dispatch_f64();
const Dispatch& dispatch_f32();
const Dispatch& dispatch_f16();
const Dispatch& dispatch_bf16();

cudaError_t launch_reduce_rows(const double* partials, int nb, int W, double* out, double weight, int accumulate,
                               cudaStream_t st);
cudaError_t launch_zero(double* p, long long n, cudaStream_t st);
// out[2] = out[0] / out[1] (0 when out[1] is 0), on the device
cudaError_t launch_ratio(double* out, cudaStream_t st);
// insulating walls: set the field from the last step's mean flow velocity /
// reset it to the configured field
cudaError_t ins_update(const Ctx& x, cudaStream_t st);
cudaError_t ins_reset(const Ctx& x, cudaStream_t st);

struct Ctx {
    lbm_config cfg;
    int device;
    int ext;                 // Lorentz force, Maxwell equilibrium or LES present
    int les_pair;            // LES alone among the EXT terms, FP32 compute: the FP32x2 LES pair code
    int sr;                  // stochastic rounding of 16-bit stores
    Geo geo;
    KP<double> kpd;          // physical units
    KP<float> kpf;           // physical units, float
    KP<float> kps;           // storage units (d times the format's scale), float
    const Dispatch* ops;
    size_t elem;             // bytes per stored population
    size_t relem;            // bytes per compute value
    void* pop[2];
    int cur;                 // index of the buffer holding f^rel(T-1) (and, induced, G(T-1))
    void* mag[2];            // induced field: post-collision field distributions, null otherwise
    uint8_t* cls;
    const uint32_t* special;  // first nodes of the 4-node chunks with a non-bulk node (staged step), or null
    long long n_special;
    Link* links;
    long long wall_begin[LBM_MAX_WALLS + 2];   // link ranges per wall id (sorted)
    long long n_links;
    double* scratch;
    void* stage;
    size_t stage_bytes;
    int64_t t;
    bool prev_valid;
    std::string err;
    int sm_count;
    int smem_optin;
    // staged step (stage_R = 0: the register-tiled k_step serves the context)
    int stage_R;             // rows per tile
    int stage_n;             // pipeline stages
    long long stage_tiles;   // tiles per step
    size_t stage_smem;       // dynamic shared memory per block
    mutable bool stage_ready;
    mutable int adj_blocks;  // grid of the adjoint kernel (0: not yet sized)
    unsigned* errflag;
    // curved walls: the wall ids of the geometry (host), to check distances
    std::vector<uint8_t> host_wid;
    // insulating walls: rows of the velocity sum (warps of the step grid) and fluid nodes
    bool insulating;
    long long ins_rows;
    long long n_fluid;
};

// blocks of the staged step: one per SM, at most one per tile (each writes
// one partial row of the fused wall force)
inline int staged_blocks(const Ctx& c) { return (int)(c.stage_tiles < c.sm_count ? c.stage_tiles : c.sm_count); }

}  // namespace lbm

struct lbm_ctx {
    lbm::Ctx c;
};
