// step_common.cuh -- device pieces shared by the 2D/3D step kernels: the
// sponge depth of a grid index and the sparse part of a step (injection into
// the new level, then gathers of it).
#pragma once

#include "internal.h"
#include "tma.cuh"

namespace wave {

__device__ __forceinline__ int sponge_depth(int i, int nb, int n)
{
    int d = max(nb - i, i - (nb + n - 1));
    return max(d, 0);
}

// ---------------------------------------------------------------------------
// Sparse part of a step, run by the CTA that owns a tile after its points are
// written: injection into unew, then gathers of unew into slots.  [ib, ie)
// and [gb, ge) are the tile's ranges in the injection and gather tap lists;
// sgt, if given, is the tile's gradient accumulator in shared memory, with
// its first point at (z0, x0).  WARP: the caller is one warp that owns the
// tile (warp barrier instead of a block barrier).
// bar() synchronises the nthr threads that run it (the version below uses the
// block barrier, or the warp barrier with WARP).
template <bool ADJ, class Bar>
__device__ __forceinline__ void sparse_phase_bar(const StepArgs& a, int ib, int ie, int gb, int ge, long long so,
                                                 int tid, int nthr, float* sgt, int z0, int x0, Bar bar)
{
    float* un = a.unew + so;
    if (a.inj.cell_start) {
        // Taps are sorted by grid point inside each cell: the thread holding the
        // first tap of a point sums that point's taps in a fixed order and owns
        // the update, so no atomics are needed and results are repeatable.
        for (int j = ib + tid; j < ie; j += nthr) {
            const int i = a.inj.idx[j];
            if (j > ib && a.inj.idx[j - 1] == i) continue;
            float add = 0.0f;
            for (int jj = j; jj < ie && a.inj.idx[jj] == i; ++jj) {
                const long long ai = (long long)a.inj.ab[jj] + (long long)a.amp_row * a.inj.npts;
                float amp = a.amp_a[ai];
                if (a.amp_b) amp -= a.amp_b[ai];
                add = fmaf(a.inj.fac[jj], amp, add);
            }
            const float v = un[i] + add;
            un[i] = v;
            if (!ADJ) {
                // the stored copy of the new level must include the injection
                if (a.st16) a.st16[so + i] = __float2bfloat16_rn(v);
                if (a.st32) a.st32[so + i] = v;
            } else if (a.gacc) {
                const float uf = a.uf16 ? __bfloat162float(a.uf16[so + i]) : a.uf32[so + i];
                if (sgt) {
                    // the tile's gradient accumulator lives in shared memory (2D, shot-group kernel)
                    const int z = i / a.P, x = i - z * a.P;
                    sgt[(z - z0) * kTX + (x - x0)] -= uf * add;
                } else {
                    a.gacc[so + i] -= uf * add;
                }
            }
        }
    }
    if (a.gat.cell_start) {
        bar();
        float* row = a.slots + (long long)a.slot_row * a.gat.ntap;
        for (int j = gb + tid; j < ge; j += nthr) row[a.gat.slot[j]] = a.gat.gw[j] * un[a.gat.idx[j]];
    }
}

template <bool ADJ, bool WARP = false>
__device__ __forceinline__ void sparse_phase(const StepArgs& a, int ib, int ie, int gb, int ge, long long so, int tid,
                                             int nthr, float* sgt = nullptr, int z0 = 0, int x0 = 0)
{
    sparse_phase_bar<ADJ>(a, ib, ie, gb, ge, so, tid, nthr, sgt, z0, x0, [] {
        if (WARP) __syncwarp();
        else __syncthreads();
    });
}

}  // namespace wave
