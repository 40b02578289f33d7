// stencil.cuh -- the per-point arithmetic of the 2D step, shared by every 2D
// kernel so that all of them produce the same bits.  The evaluation order is
// fixed by explicit fmaf calls rather than left to contraction.
#pragma once

#include "internal.h"

namespace wave {

// 8th-order Laplacian (unit spacing) of 4 consecutive x points.  w[0..11] are
// the row values x-4 .. x+7 (the points are w[4..7]); zn(k) returns the pair
// (values k rows above, values k rows below) of the 4 points, k = 1..4, and is
// called in the loop so that the loads interleave with the arithmetic.
// Evaluation order: 2 c0 w, then + c_k (w_{-k} + w_{+k}) for k = 1..4 along x,
// then along z.
template <class ZN>
__device__ __forceinline__ void lap4(const float* w, ZN zn, float* lap)
{
    const float ck[5] = {kC0, kC1, kC2, kC3, kC4};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float acc = (2.0f * kC0) * w[e + 4];
#pragma unroll
        for (int k = 1; k <= 4; ++k) acc = fmaf(ck[k], w[e + 4 - k] + w[e + 4 + k], acc);
        lap[e] = acc;
    }
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        float4 U, D;
        zn(k, U, D);
        lap[0] = fmaf(ck[k], U.x + D.x, lap[0]);
        lap[1] = fmaf(ck[k], U.y + D.y, lap[1]);
        lap[2] = fmaf(ck[k], U.z + D.z, lap[2]);
        lap[3] = fmaf(ck[k], U.w + D.w, lap[3]);
    }
}

// 3D Laplacian of 4 consecutive x points: w as in lap4; zn(k, Up, Dn, Zu, Zd)
// returns the 4 points' values k rows away in y (Up, Dn) and k planes away in
// z (Zu, Zd).  Order: 3 c0 w, + c_k (w_{-k} + w_{+k}) along x, then
// + c_k ((Up + Dn) + (Zu + Zd)) for k = 1..4.
template <class ZN>
__device__ __forceinline__ void lap4_3d(const float* w, ZN zn, float* lap)
{
    const float ck[5] = {kC0, kC1, kC2, kC3, kC4};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float acc = (3.0f * kC0) * w[e + 4];
#pragma unroll
        for (int k = 1; k <= 4; ++k) acc = fmaf(ck[k], w[e + 4 - k] + w[e + 4 + k], acc);
        lap[e] = acc;
    }
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        float4 Up, Dn, Zu, Zd;
        zn(k, Up, Dn, Zu, Zd);
        lap[0] = fmaf(ck[k], (Up.x + Dn.x) + (Zu.x + Zd.x), lap[0]);
        lap[1] = fmaf(ck[k], (Up.y + Dn.y) + (Zu.y + Zd.y), lap[1]);
        lap[2] = fmaf(ck[k], (Up.z + Dn.z) + (Zu.z + Zd.z), lap[2]);
        lap[3] = fmaf(ck[k], (Up.w + Dn.w) + (Zu.w + Zd.w), lap[3]);
    }
}

// 1 / x for the sponge factor (x = 1 + eps >= 1): the hardware approximation
// refined by one Newton-Raphson step for the reciprocal, r <- r + r (1 - x r).
// The result is within about 2^-24 relative of 1 / x before its rounding, so it
// is the rounded reciprocal except next to a rounding boundary, and unbiased
// there.  Three instructions instead of the correctly rounded sequence: the
// 3D steps and the batch sweeps evaluate it for every point at every step.
__device__ __forceinline__ float rcp_sponge(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// Leapfrog update of one point: (kap lap + eps um + 2 c - um - src) * inv,
// inv = 1 / (1 + eps); src is the Born secondary source (zero elsewhere).
__device__ __forceinline__ float leap1(float c, float um, float lap, float kap, float eps, float inv, float src)
{
    const float t = fmaf(kap, lap, fmaf(eps, um, fmaf(2.0f, c, -um)));
    return (t - src) * inv;
}

// The same for 4 points.
__device__ __forceinline__ void update4(const float* c, const float* um, const float* lap, const float* kap,
                                        const float* eps, const float* inv, const float* src, float* out)
{
#pragma unroll
    for (int e = 0; e < 4; ++e) out[e] = leap1(c[e], um[e], lap[e], kap[e], eps[e], inv[e], src[e]);
}

// The same update where the sponge is absent (eps = 0, inv = 1) and there is no
// secondary source: equal to update4 up to the sign of zero results.
__device__ __forceinline__ void update4_interior(const float* c, const float* um, const float* lap, const float* kap,
                                                 float* out)
{
#pragma unroll
    for (int e = 0; e < 4; ++e) out[e] = fmaf(kap[e], lap[e], fmaf(2.0f, c[e], -um[e]));
}

}  // namespace wave
