// internal.h -- types shared by the libwave translation units (not part of the ABI).
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder comes from the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "wave.h"

namespace wave {

// 8th-order centred second-derivative weights (unit spacing), the solution of
// the Taylor moment conditions sum_j c_|j| j^p = 2 [p == 2], p = 0,2,4,6,8.
constexpr float kC0 = -205.0f / 72.0f;
constexpr float kC1 = 8.0f / 5.0f;
constexpr float kC2 = -1.0f / 5.0f;
constexpr float kC3 = 8.0f / 315.0f;
constexpr float kC4 = -1.0f / 560.0f;

// Device error word bits.
enum : int {
    kErrNonFinite = 1,  // velocity not finite/positive or NaN in a result
    kErrTimeout = 2,    // a bounded wait ran out
    kErrCfl = 4         // dt vmax / h above the stability limit
};

// Padded geometry of one shot's field.  Fields are stored [Nz][Ny][P] floats
// (Ny = 1 in 2D) with the row pitch P = Nx rounded up to 32 floats (128 B);
// columns Nx..P-1 stay zero and stand for the Dirichlet exterior.
struct Dims {
    int ndim, nx, ny, nz, nb, nt;
    int Nx, Ny, Nz, P;
    long long cell;  // floats per field per shot = Nz * Ny * P
    long long phys;  // physical points
    float h, dt, vref;
};

Dims make_dims(const wave_grid_t& g);

// Partition of the padded grid.  Interpolation taps are grouped per "cell"
// (TX x TY x TZc points) in the order (shot, cx, cy, cz) with cz fastest, so
// that a kernel tile covering k consecutive cells along z owns one contiguous
// range of taps.
struct Tiling {
    int TX, TY, TZc;
    int ncx, ncy, ncz;
    int vf, va;  // 2D kernel variants for the forward / adjoint steps
    int v3;      // 3D kernel variant
    long long cells_per_shot() const { return (long long)ncx * ncy * ncz; }
};

// One list of interpolation taps (sources or receivers) in device memory,
// grouped per (shot, cell).
struct TapList {
    const int* cell_start = nullptr;  // [nshot * cells_per_shot + 1]
    const int* idx = nullptr;         // flat index inside the shot's field
    const float* fac = nullptr;       // injection factor (filled on device)
    const float* gw = nullptr;        // gather weight
    const int* ab = nullptr;          // amplitude base: (shot * nt) * npts + point
    const int* slot = nullptr;        // gather slot (position in point order)
    const float* w = nullptr;         // plain interpolation weight
    int npts = 0;                     // points per shot
    int ntap = 0;                     // total taps (all shots)
    const int* pt_start = nullptr;    // [nshot * npts + 1] taps of each point (point order)
};

struct HostTaps {
    std::vector<int> cell_start, idx, ab, slot, pt_start;
    std::vector<float> w;
    int npts = 0;
};

// Builds taps for nshot * npts points; WAVE_ERR_GEOMETRY for a point outside
// the physical grid.
wave_status_t build_taps(const Dims& d, const Tiling& t, int nshot, int npts, const float* xyz, HostTaps& out);

// TMA descriptors.  Every field batch ([nshot][Nz][P]) of a call lives in one
// pool of equally sized buffers, so one 4D map addresses any of them through a
// buffer-index coordinate.  halo: box of the stencil input with its 4-point
// halo; tile: box of a pointwise input; kap: the model; tile16: the BF16 store.
// _f / _a: boxes for the forward / adjoint tile heights.
struct StepMaps {
    CUtensorMap halo_f, tile_f, kap_f, halo_a, tile_a, kap_a, tile16_a;
    CUtensorMap halo3;  // 3D: (x, y, z, shot, buffer) over the pool, box 136 x (TY+8) x 1 x 1 x 1
};

// Arguments of one time step of the stencil kernels.
struct StepArgs {
    const float* u;      // [nshot][cell] field at the current level
    const float* uprev;  // [nshot][cell] previous level
    float* unew;         // [nshot][cell] next level (may alias uprev)
    const float* kap;    // [cell] (v dt / h)^2
    int Nx, Ny, Nz, P;
    long long cell;
    int nb, nx, ny, nz;
    int nshot;
    float ceps;          // eps = kap * ceps * depth^2 is eta dt v^2 / 2
    int ncx, ncy, ncz;   // tap cells per shot
    int TZc;             // tap cell height
    // injection into unew (forward: sources with q^n; adjoint: receivers with r^k)
    TapList inj;
    const float* amp_a;  // amplitude array [nshot][nt][npts]
    const float* amp_b;  // subtracted from amp_a (NULL = none)
    int amp_row;         // time index of the amplitudes
    // gather from unew after injection (forward: receivers, adjoint: sources)
    TapList gat;
    float* slots;        // [nt][ntap] gather slots
    int slot_row;
    // forward: optional copy of unew to a store row
    __nv_bfloat16* st16;
    float* st32;
    // adjoint: forward field u^k for the imaging condition, gradient accumulators
    const __nv_bfloat16* uf16;
    const float* uf32;
    float* gacc;         // [nshot][cell]
    int* err;
    // Born scattering source: unew gets -dmv .* (bs_a - 2 bs_b + bs_c) / (1 + eps)
    // added, dmv = Extend(dm) v^2 (kind 0 2D kernel and the 3D kernel only)
    const float* dmv;
    const float *bs_a, *bs_b, *bs_c;
    // pool indices of the same buffers for the TMA kernels (-1: none)
    int u_buf, prev_buf, uf_buf, g_buf, uf16_row;
};

// Kernel launchers (kernels.cu).
void launch_step(const Tiling& t, int ndim, bool adjoint, const StepArgs& a, const StepMaps* maps, cudaStream_t s);
void launch_prep(const Dims& d, const float* vel, float* kap, float* vmax, int* err, cudaStream_t s);
// Sets kErrCfl in *err when dt * (*vmax) / h exceeds limit (one thread).
void launch_check_cfl(const float* vmax, double dt_over_h, double limit, int* err, cudaStream_t s);
void launch_tapfac(const Dims& d, const TapList& l, const float* kap, float scale_inj, float ceps,
                   cudaStream_t s);
void launch_finalize(const TapList& l, const float* slots, int nshot, int nt, float* out, cudaStream_t s);
void launch_misfit(const float* a, const float* b, long long n, double* partial, int npart, double* out,
                   cudaStream_t s);
void launch_grad_reduce(const Dims& d, const float* gacc, int nshot, float* tmp, float* grad, const float* vel_chain,
                        cudaStream_t s);
void launch_ricker(float f0, float dt, int nt, float* out, cudaStream_t s);
void launch_prep_dm(const Dims& d, const float* dm, const float* kap, float* dmv, cudaStream_t s);
void launch_nan_scan(const float* a, long long n, int* err, cudaStream_t s);

// Tile geometry of the 2D steps (kernels.cu).
constexpr int kTX = 128;          // x points per tile (32 lanes x 4)
constexpr int kTZc2 = 8;          // 2D tap-cell height: divides every 2D tile height

// 2D kernel variants: direct loads (kind 0), the persistent TMA pipeline
// (kind 1) with tile height TZ, R rows per warp and NST stages, shot groups
// (kind 2): one CTA runs its tile for G shots (R = thread rows), the
// z-march (kind 3): one warp per TZ-row strip, R warps per CTA, prefetch
// distance NST rows, shot groups fed by TMA (kind 4, fields as kind 2; NST bit
// 0: the previous level's tile comes by TMA too, bit 1: the sponge factors sit
// in shared memory instead of registers, bit 2: the adjoint's forward level
// comes by TMA too, bits 3 / 4: a 3- / 4-stage ring instead of 2), or
// the persistent kernel over (tile, shot) items (kind 5, R = thread rows), or
// the z-window kernel (kind 7, below).
// With kinds 2 and 4 in the adjoint, the gradient buffer holds one
// accumulator per shot group; with kind 5, one per CTA segment of a tile.
struct Variant2D {
    int kind, TZ, R, NST, G;
};
// Kind 7: shot groups fed by TMA with the z window of each thread's
// consecutive rows in registers (G shots per CTA; NST = configuration index
// of launch_step2d_zw, step2d_zw.cu).
void launch_step2d_zw(int config, bool adjoint, const StepArgs& a, const StepMaps* maps, cudaStream_t s);
// Number of per-shot/per-group gradient accumulators the adjoint step fills.
int gradient_accumulators(const struct Tiling& t, int ndim, int nshot);
int persistent_slots(int v, int ncx, int ntz, int nshot);  // adjoint variant v of kind 5
int variant_count(int which);             // which: 0 2D forward, 1 2D adjoint, 2 3D
Variant2D variant_info(int which, int v);
int current_variant(int which);           // the selected or default variant
int select_variant(int which, int v);     // v = -1 restores the default; 0 on success
bool variant_forced(int which);           // true after wave_set_variant(which, v >= 0)

// Remembers the last failing CUDA call of this thread (profile.cu).
void note_cuda_error(cudaError_t e);

// Launch accounting and sampled per-launch timing of the stencil kernels
// (profile.cu).  Every launcher above calls count_launch(); launch_step wraps
// sampled launches in a pair of CUDA events on the launching stream.
void count_launch(int n = 1);
void count_step_launch();  // a stencil time step (launch_step)
bool profile_sample(bool adjoint, cudaStream_t s, cudaEvent_t* stop);
void profile_close(cudaEvent_t stop, cudaStream_t s);

// Tiling choice (plan.cu): the 2D variants come from wave_set_variant, else
// from a wave_autotune result for this (grid, nshot), else the defaults.
Tiling choose_tiling(const Dims& d, int nshot);
void remember_tuning(const Dims& d, int nshot, int vf, int va);

// Binomial checkpoint schedule (plan.cu).
enum ActionKind { kAdvance = 0, kSave = 1, kRestore = 2, kAdjointPair = 3, kFinalize = 4 };
struct Action {
    int kind;
    int a;     // advance: from macro position; save/restore: slot (-1 = zero state)
    int b;     // advance: to macro position; save/restore: macro position
};
// Macro positions p = 0..L map to forward states S_j = (u^j, u^{j-1}) with
// j(0) = 0 and j(p) = jmin + 2 (p - 1); every state j(p), p >= 1, serves the
// adjoint steps j and j - 1.
struct Schedule {
    int K = 0, L = 0, jmin = 0, nsnap = 0;
    long long advances = 0;  // macro advances in the whole schedule
    long long fwd_steps = 0; // forward time steps in the whole schedule
    std::vector<Action> actions;
    int state_of(int p) const { return p == 0 ? 0 : jmin + 2 * (p - 1); }
};
Schedule make_schedule(int nt, int nsnap);

}  // namespace wave
