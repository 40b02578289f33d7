// internal.h -- types shared by the libwave translation units (not part of the ABI).
#pragma once

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
    kErrNonFinite = 1,  // velocity not finite/positive or NaN in a field
    kErrTimeout = 2,    // a bounded wait ran out
    kErrIndex = 4       // an internal index check failed (a tap outside its tile)
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

// Tiling of the padded grid used by the stencil kernels.  A tile is the set of
// points whose update one CTA writes: TX x TY x TZ (TY = 1 in 2D).
struct Tiling {
    int TX, TY, TZ;
    int ntx, nty, ntz;  // tiles per shot along each axis
    int kind;           // kernel variant id (see kernels)
    long long tiles_per_shot() const { return (long long)ntx * nty * ntz; }
};

// One list of interpolation taps (sources or receivers) in device memory,
// grouped per (shot, tile) so that the CTA updating a tile handles exactly the
// taps that fall in it.
struct TapList {
    const int* tile_start = nullptr;  // [nshot * tiles_per_shot + 1]
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

// Host-side tap tables before upload.
struct HostTaps {
    std::vector<int> tile_start, idx, ab, slot, pt_start;
    std::vector<float> w;
    int npts = 0;
};

// Builds taps for nshot * npts points; returns WAVE_ERR_GEOMETRY for a point
// outside the physical grid.
wave_status_t build_taps(const Dims& d, const Tiling& t, int nshot, int npts, const float* xyz,
                         HostTaps& out);

// Arguments of one time step of the stencil kernels.
struct StepArgs {
    const float* u;      // [nshot][cell] field at the current time level
    float* unew;         // [nshot][cell] in: previous level, out: next level
    const float* kap;    // [cell] (v dt / h)^2
    int Nx, Ny, Nz, P;
    long long cell;
    int nb, nx, ny, nz;
    float ceps;          // eps = kap * ceps * depth^2 is eta dt v^2 / 2
    int ntx, nty, ntz;
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
    // adjoint: forward field u^k for the imaging condition, per-shot accumulators
    const __nv_bfloat16* uf16;
    const float* uf32;
    float* gacc;         // [nshot][cell]
    int* err;
};

// Kernel launchers (kernels.cu).
void launch_step(const Tiling& t, int ndim, bool adjoint, int nshot, const StepArgs& a, cudaStream_t s);
void launch_prep(const Dims& d, const float* vel, float* kap, float* vmax, int* err, cudaStream_t s);
void launch_tapfac(const Dims& d, const TapList& l, const float* kap, float scale_inj, float ceps,
                   cudaStream_t s);
void launch_finalize(const TapList& l, const float* slots, int nshot, int nt, float* out, cudaStream_t s);
void launch_misfit(const float* a, const float* b, long long n, double* partial, int npart, double* out,
                   cudaStream_t s);
void launch_grad_reduce(const Dims& d, const float* gacc, int nshot, float* grad, cudaStream_t s);
void launch_ricker(float f0, float dt, int nt, float* out, cudaStream_t s);
void launch_nan_scan(const float* a, long long n, int* err, cudaStream_t s);

// Launch accounting and sampled per-launch timing of the stencil kernels
// (profile.cu).  Every launcher above calls count_launch(); launch_step wraps
// sampled launches in a pair of CUDA events on the launching stream.
void count_launch(int n = 1);
bool profile_sample(bool adjoint, cudaStream_t s, cudaEvent_t* stop);
void profile_close(cudaEvent_t stop, cudaStream_t s);

// Tiling choice (plan.cu).
Tiling choose_tiling(const Dims& d, int nshot);

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
