// kernels.cu -- the stencil time step (2D and 3D, forward and adjoint) and the
// small kernels around it (model preparation, tap factors, gathers, misfit,
// shot reduction of the gradient, Ricker wavelet).
//
// All of it is memory bound: FP32 arithmetic on CUDA cores, 128-bit accesses,
// halo tiles in shared memory.  Tensor cores play no part (the stencil is not
// a dense contraction).  The 2D step comes in two families selected per call:
// a direct-load kernel with a shared-memory halo tile, and a persistent kernel
// that streams tiles through shared memory with TMA (cp.async.bulk.tensor) and
// mbarriers, keeping one to three tiles of loads in flight per SM.
#include <math.h>

#include <algorithm>

#include "internal.h"
#include "stencil.cuh"
#include "tma.cuh"
#include "step_common.cuh"

namespace wave {


// One leapfrog update in Courant units:
//   (1+eps) u+ = 2u - (1-eps) u- + kap * lap,  kap = (v dt/h)^2, eps = eta dt v^2 / 2.
__device__ __forceinline__ float leap(float c, float um, float lap, float kap, float eps)
{
    float num = fmaf(kap, lap, fmaf(eps, um, 2.0f * c - um));
    return num * rcp_sponge(1.0f + eps);
}

// The same update with an extra source term subtracted before the damping
// factor (the Born secondary source); src = 0 gives exactly leap().
__device__ __forceinline__ float leap_src(float c, float um, float lap, float kap, float eps, float src)
{
    float num = fmaf(kap, lap, fmaf(eps, um, 2.0f * c - um)) - src;
    return num * rcp_sponge(1.0f + eps);
}

// Born secondary source of four points: dmv .* (u^{n+1} - 2 u^n + u^{n-1}),
// with dmv = dm v^2 (it enters the update as kap * lap - src).
__device__ __forceinline__ void born_source(const StepArgs& a, long long so, long long off, float* src)
{
    const float4 d = ld4(a.dmv + off);
    const float4 pa = ld4(a.bs_a + so + off), pb = ld4(a.bs_b + so + off), pc = ld4(a.bs_c + so + off);
    src[0] = d.x * (pa.x - 2.0f * pb.x + pc.x);
    src[1] = d.y * (pa.y - 2.0f * pb.y + pc.y);
    src[2] = d.z * (pa.z - 2.0f * pb.z + pc.z);
    src[3] = d.w * (pa.w - 2.0f * pb.w + pc.w);
}

// Writes one thread's four updated points (zeros past Nx) and, in the forward
// pass, their stored copies; in the adjoint pass adds the imaging term
// g -= u^k (mu^k - 2 mu^{k+1} + mu^{k+2}) to the loaded accumulator values.
template <bool ADJ>
__device__ __forceinline__ void write4(const StepArgs& a, long long so, long long off, int nvalid, const float* out,
                                       const float* cen, const float* um, bool imaging, const float* uf, float4 gv)
{
    float* un = a.unew + so;
    // Always a full float4: points past Nx are the zero exterior that the next
    // step's halo loads read, so every output buffer keeps them zero.
    *reinterpret_cast<float4*>(un + off) = make_float4(out[0], nvalid > 1 ? out[1] : 0.0f,
                                                       nvalid > 2 ? out[2] : 0.0f, nvalid > 3 ? out[3] : 0.0f);
    if (!ADJ) {
        if (a.st16) {
            if (nvalid == 4) {
                store_bf16x4(a.st16 + so + off, out);
            } else {
                for (int i = 0; i < nvalid; ++i) a.st16[so + off + i] = __float2bfloat16_rn(out[i]);
            }
        }
        if (a.st32) {
            if (nvalid == 4) {
                *reinterpret_cast<float4*>(a.st32 + so + off) = make_float4(out[0], out[1], out[2], out[3]);
            } else {
                for (int i = 0; i < nvalid; ++i) a.st32[so + off + i] = out[i];
            }
        }
    } else if (imaging) {
        float g[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) g[i] -= uf[i] * (out[i] - 2.0f * cen[i] + um[i]);
        float* gp = a.gacc + so + off;
        if (nvalid == 4) {
            *reinterpret_cast<float4*>(gp) = make_float4(g[0], g[1], g[2], g[3]);
        } else {
            for (int i = 0; i < nvalid; ++i) gp[i] = g[i];
        }
    }
}


// A thread whose 4 points all lie in the pitch padding [Nx, P) writes zeros
// there, so that a buffer that is only ever written by steps still reads as
// the zero exterior.
__device__ __forceinline__ void zero_padding(const StepArgs& a, long long so, long long off, int gx)
{
    if (gx < a.P) *reinterpret_cast<float4*>(a.unew + so + off) = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// 2D step, direct loads.  Tile = 128 (x) by TZ (z) points, CTA = 32 x BZ
// threads, each thread updates 4 consecutive x points on TZ/BZ rows.  The
// (TZ+8) x 136 halo tile of u is staged in shared memory with 128-bit loads;
// values outside the padded grid read as zero.  The pointwise inputs of the
// thread's rows are loaded before the halo tile so that their latency overlaps.
template <int TZ, int BZ, bool ADJ>
__global__ void __launch_bounds__(32 * BZ, 1024 / (32 * BZ)) k_step2d(const StepArgs a)
{
    constexpr int SW = kTX + 8;
    constexpr int RB = TZ / BZ;
    __shared__ __align__(16) float s[TZ + 8][SW];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int x0 = blockIdx.x * kTX, z0 = blockIdx.y * TZ;
    const int shot = blockIdx.z;
    const long long so = (long long)shot * a.cell;
    const float* __restrict__ u = a.u + so;
    const int lx = 4 * threadIdx.x;
    const int gx = x0 + lx;
    const int nvalid = min(4, a.Nx - gx);
    const bool imaging = ADJ && a.gacc != nullptr;

    float4 kp[RB], uo[RB];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        const int gz = z0 + threadIdx.y + rr * BZ;
        kp[rr] = uo[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gz < a.Nz && nvalid > 0) {
            const long long off = (long long)gz * a.P + gx;
            kp[rr] = ld4(a.kap + off);
            uo[rr] = *reinterpret_cast<const float4*>(a.uprev + so + off);
        }
    }
    for (int i = tid; i < (TZ + 8) * (SW / 4); i += 32 * BZ) {
        const int r = i / (SW / 4), c4 = i - r * (SW / 4);
        const int gz = z0 - 4 + r, gxx = x0 - 4 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gz >= 0 && gz < a.Nz && gxx >= 0 && gxx < a.P) v = ld4(u + (long long)gz * a.P + gxx);
        *reinterpret_cast<float4*>(&s[r][4 * c4]) = v;
    }
    __syncthreads();

#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        const int r = threadIdx.y + rr * BZ;
        const int gz = z0 + r;
        if (gz >= a.Nz) continue;
        if (nvalid <= 0) {
            zero_padding(a, so, (long long)gz * a.P + gx, gx);
            continue;
        }
        const float* row = &s[r + 4][lx];
        const float4 A = lds4(row), B = lds4(row + 4), C = lds4(row + 8);
        const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
        float lap[4];
        lap4(w, [&](int k, float4& Up, float4& Dn) {
            Up = lds4(&s[r + 4 - k][lx + 4]);
            Dn = lds4(&s[r + 4 + k][lx + 4]);
        }, lap);
        const long long off = (long long)gz * a.P + gx;
        const int dz = sponge_depth(gz, a.nb, a.nz);
        float out[4], cen[4], um[4], uf[4] = {0.f, 0.f, 0.f, 0.f};
        float bsrc[4] = {0.f, 0.f, 0.f, 0.f};
        if (a.dmv) born_source(a, so, off, bsrc);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int dd = max(sponge_depth(gx + i, a.nb, a.nx), dz);
            const float kap = f4(kp[rr], i);
            const float eps = kap * a.ceps * (float)(dd * dd);
            cen[i] = w[i + 4];
            um[i] = f4(uo[rr], i);
            out[i] = leap1(cen[i], um[i], lap[i], kap, eps, rcp_sponge(1.0f + eps), bsrc[i]);
        }
        float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (imaging) {
            if (a.uf16) {
                unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + so + off), uf);
            } else {
                const float4 v = ld4(a.uf32 + so + off);
                uf[0] = v.x;
                uf[1] = v.y;
                uf[2] = v.z;
                uf[3] = v.w;
            }
            gv = *reinterpret_cast<const float4*>(a.gacc + so + off);
        }
        write4<ADJ>(a, so, off, nvalid, out, cen, um, imaging, uf, gv);
    }
    if (a.inj.cell_start || a.gat.cell_start) {
        __syncthreads();
        const int kcell = TZ / a.TZc;
        const int cbase = (shot * a.ncx + (int)blockIdx.x) * a.ncz;
        const int c0 = (int)blockIdx.y * kcell, c1 = min(c0 + kcell, a.ncz);
        int ib = 0, ie = 0, gb = 0, ge = 0;
        if (a.inj.cell_start) {
            ib = a.inj.cell_start[cbase + c0];
            ie = a.inj.cell_start[cbase + c1];
        }
        if (a.gat.cell_start) {
            gb = a.gat.cell_start[cbase + c0];
            ge = a.gat.cell_start[cbase + c1];
        }
        sparse_phase<ADJ>(a, ib, ie, gb, ge, so, tid, 32 * BZ);
    }
}

// ---------------------------------------------------------------------------
// 2D step, shot groups.  A CTA owns one 128 x TZ tile and runs it for G
// consecutive shots of the batch (blockIdx.z = group).  Everything that does
// not depend on the shot -- the model, the sponge factors and their
// reciprocal -- is computed once per CTA; the next shot's halo tile is
// prefetched with cp.async into the second of two shared-memory buffers while
// the current shot is computed; in the adjoint the imaging condition is
// accumulated over the group in a shared-memory tile and written back once,
// into the group's gradient accumulator (buffer G holds one per group).
template <int TZ, int BZ, int G, bool ADJ>
__global__ void __launch_bounds__(32 * BZ) k_step2d_sg(const StepArgs a)
{
    constexpr int SW = kTX + 8;
    constexpr int RB = TZ / BZ;
    extern __shared__ __align__(16) float dsm[];
    float(*s)[TZ + 8][SW] = reinterpret_cast<float(*)[TZ + 8][SW]>(dsm);
    float* sg = dsm + 2 * (TZ + 8) * SW;  // [TZ][kTX], adjoint only
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * kTX, z0 = blockIdx.y * TZ;
    const int grp = blockIdx.z, s0 = grp * G, s1 = min(s0 + G, a.nshot);
    const int lx = 4 * tx, gx = x0 + lx;
    const int nvalid = min(4, a.Nx - gx);
    const bool imaging = ADJ && a.gacc != nullptr;
    const bool sparse = a.inj.cell_start != nullptr || a.gat.cell_start != nullptr;

    float4 kp[RB];
    float eps[RB][4], inv[RB][4];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        const int gz = z0 + ty + rr * BZ;
        kp[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gz < a.Nz && nvalid > 0) kp[rr] = ld4(a.kap + (long long)gz * a.P + gx);
        const int dz = sponge_depth(gz, a.nb, a.nz);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int dd = max(sponge_depth(gx + e, a.nb, a.nx), dz);
            eps[rr][e] = f4(kp[rr], e) * a.ceps * (float)(dd * dd);
            inv[rr][e] = rcp_sponge(1.0f + eps[rr][e]);
        }
    }
    float* gq = imaging ? a.gacc + (long long)grp * a.cell : nullptr;
    if (imaging) {
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int r = ty + rr * BZ, gz = z0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gz < a.Nz && nvalid > 0) v = *reinterpret_cast<const float4*>(gq + (long long)gz * a.P + gx);
            *reinterpret_cast<float4*>(sg + r * kTX + lx) = v;
        }
    }

    auto load_tile = [&](int buf, int shot) {
        const float* u = a.u + (long long)shot * a.cell;
        for (int r = ty; r < TZ + 8; r += BZ) {
            const int gz = z0 - 4 + r;
            for (int c4 = tx; c4 < SW / 4; c4 += 32) {
                const int gxx = x0 - 4 + 4 * c4;
                const bool ok = gz >= 0 && gz < a.Nz && gxx >= 0 && gxx < a.P;
                cp_async16(&s[buf][r][4 * c4], ok ? u + (long long)gz * a.P + gxx : a.u, ok ? 16 : 0);
            }
        }
        cp_async_commit();
    };

    load_tile(0, s0);
    for (int shot = s0; shot < s1; ++shot) {
        const int cur = (shot - s0) & 1;
        if (shot + 1 < s1) load_tile(cur ^ 1, shot + 1);
        else cp_async_commit();  // keep one group per iteration
        const long long so = (long long)shot * a.cell;
        float4 uo[RB];
        float uf[RB][4];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int gz = z0 + ty + rr * BZ;
            uo[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 4; ++e) uf[rr][e] = 0.f;
            if (gz < a.Nz && nvalid > 0) {
                const long long off = so + (long long)gz * a.P + gx;
                uo[rr] = *reinterpret_cast<const float4*>(a.uprev + off);
                if (imaging) {
                    if (a.uf16) {
                        unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + off), uf[rr]);
                    } else {
                        const float4 v = ld4(a.uf32 + off);
                        uf[rr][0] = v.x;
                        uf[rr][1] = v.y;
                        uf[rr][2] = v.z;
                        uf[rr][3] = v.w;
                    }
                }
            }
        }
        cp_async_wait_prev();
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int r = ty + rr * BZ;
            const int gz = z0 + r;
            if (gz >= a.Nz) continue;
            if (nvalid <= 0) {
                zero_padding(a, so, (long long)gz * a.P + gx, gx);
                continue;
            }
            const float* row = &s[cur][r + 4][lx];
            const float4 A = lds4(row), B = lds4(row + 4), C = lds4(row + 8);
            const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
            float lap[4];
            lap4(w, [&](int k, float4& Up, float4& Dn) {
                Up = lds4(&s[cur][r + 4 - k][lx + 4]);
                Dn = lds4(&s[cur][r + 4 + k][lx + 4]);
            }, lap);
            float out[4], cen[4], um[4], kv[4];
            const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                cen[e] = w[e + 4];
                um[e] = f4(uo[rr], e);
                kv[e] = f4(kp[rr], e);
            }
            update4(cen, um, lap, kv, eps[rr], inv[rr], zero4, out);
            write4<ADJ>(a, so, (long long)gz * a.P + gx, nvalid, out, cen, um, false, nullptr,
                        make_float4(0.f, 0.f, 0.f, 0.f));
            if (imaging) {
                float* g = sg + r * kTX + lx;
#pragma unroll
                for (int e = 0; e < 4; ++e) g[e] -= uf[rr][e] * (out[e] - 2.0f * cen[e] + um[e]);
            }
        }
        __syncthreads();
        if (sparse) {
            const int kcell = TZ / a.TZc;
            const int cbase = (shot * a.ncx + (int)blockIdx.x) * a.ncz;
            const int c0 = (int)blockIdx.y * kcell, c1 = min(c0 + kcell, a.ncz);
            int ib = 0, ie = 0, gb = 0, ge = 0;
            if (a.inj.cell_start) {
                ib = a.inj.cell_start[cbase + c0];
                ie = a.inj.cell_start[cbase + c1];
            }
            if (a.gat.cell_start) {
                gb = a.gat.cell_start[cbase + c0];
                ge = a.gat.cell_start[cbase + c1];
            }
            sparse_phase<ADJ>(a, ib, ie, gb, ge, so, tid, 32 * BZ, imaging ? sg : nullptr, z0, x0);
        }
    }
    if (imaging) {
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int r = ty + rr * BZ, gz = z0 + r;
            if (gz < a.Nz && nvalid > 0)
                *reinterpret_cast<float4*>(gq + (long long)gz * a.P + gx) =
                    *reinterpret_cast<const float4*>(sg + r * kTX + lx);
        }
    }
}

// ---------------------------------------------------------------------------
// 2D step, shot groups fed by TMA.  As the shot-group kernel, but each shot's
// (TZ+8) x 136 halo tile of u arrives by one TMA load (zero fill outside the
// padded grid) into a ring of NS stages (2 by default, 3 or 4 with FL bits 8
// or 16): one thread keeps the loads of the next NS - 1 shots in flight while
// shot i is computed.  FL bit 1 adds the previous level's tile to a stage,
// bit 4 (adjoint) the forward level u^k; bit 32 orders the grid so that the
// top tile rows, which hold the source and receiver taps and take longest,
// are dispatched first; bit 64 sizes registers for 3 CTAs per SM (what the
// shared memory of the adjoint's 2-stage u^k ring allows anyway).  Row offsets, the model and the sponge
// factors are set up once per CTA in 32-bit form, so the per-shot work is the
// stencil arithmetic, one load of the previous level and one store per 4
// points.  Waits on the ring are bounded; on a timeout the CTA records
// kErrTimeout, lets its issued copies land and returns.
template <int TZ, int BZ, int G, int FL, bool ADJ>
__global__ void __launch_bounds__(32 * BZ, (FL & 16) ? 512 / (32 * BZ)
                                          : ((FL & 8) || (FL & 64)) ? 768 / (32 * BZ)
                                          : (FL & 2) ? 1280 / (32 * BZ)
                                          : ((TZ / BZ) <= 2 ? 1024 / (32 * BZ) : 512 / (32 * BZ)))
    k_step2d_sgt(const __grid_constant__ StepMaps mp, const StepArgs a)
{
    constexpr bool PT = (FL & 1) != 0;  // the previous level's tile comes by TMA
    constexpr bool SE = (FL & 2) != 0;  // sponge factors kept in shared memory, not registers
    constexpr bool FT = ADJ && (FL & 4) != 0;  // adjoint: the forward level u^k comes by TMA too
    constexpr int NS = (FL & 16) ? 4 : ((FL & 8) ? 3 : 2);  // ring stages: copies run NS - 1 shots ahead
    constexpr int SW = kTX + 8;
    constexpr int RB = TZ / BZ;
    constexpr int SU = (TZ + 8) * SW;          // halo tile of u
    constexpr int SP = PT ? TZ * kTX : 0;      // previous level's tile (PT)
    constexpr int SU2 = SU + SP + (FT ? TZ * kTX : 0);  // one stage (+ u^k, FP32 or BF16 in the first half)
    static_assert(SU % 32 == 0 && SU2 % 32 == 0, "stages must stay 128-byte aligned");
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar[NS];
    __shared__ int taprng[G][4];  // per shot of the group: injection and gather tap ranges
    float* st = reinterpret_cast<float*>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));
    float* sg = st + NS * SU2;                        // [TZ][kTX] gradient tile (adjoint with imaging)
    float* se = sg + (ADJ ? TZ * kTX : 0);            // [2][TZ][kTX] eps and 1/(1+eps) (SE)
    const CUtensorMap* mh = ADJ ? &mp.halo_a : &mp.halo_f;
    const CUtensorMap* mt = ADJ ? &mp.tile_a : &mp.tile_f;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    // grid (x tiles, z tiles, groups), or with FL bit 32 (x tiles, groups, z
    // tiles): CTAs are dispatched in linear block order, so the second form
    // runs every group of the top tile rows (where sources and receivers sit)
    // in the first wave
    constexpr bool GM = (FL & 32) != 0;
    const int tzi = GM ? (int)blockIdx.z : (int)blockIdx.y;
    const int x0 = blockIdx.x * kTX, z0 = tzi * TZ;
    const int grp = GM ? (int)blockIdx.y : (int)blockIdx.z, s0 = grp * G, ns = min(G, a.nshot - s0);
    const int lx = 4 * tx, gx = x0 + lx;
    const int nvalid = min(4, a.Nx - gx);
    const bool imaging = ADJ && a.gacc != nullptr;
    const bool sparse = a.inj.cell_start != nullptr || a.gat.cell_start != nullptr;
    const bool ft = FT && imaging && (a.uf16 ? a.uf16_row >= 0 : a.uf_buf >= 0);
    const uint32_t kBytes = (uint32_t)(SU + SP) * 4u + (ft ? (uint32_t)(TZ * kTX) * (a.uf16 ? 2u : 4u) : 0u);
    // copies of shot i into ring stage i % NS
    auto issue = [&](int i) {
        const int sj = i % NS;
        float* sb = st + sj * SU2;
        mbar_expect_tx(&bar[sj], kBytes);
        tma_load_4d(sb, mh, &bar[sj], x0 - 4, z0 - 4, s0 + i, a.u_buf);
        if (PT) tma_load_4d(sb + SU, mt, &bar[sj], x0, z0, s0 + i, a.prev_buf);
        if (ft) {
            if (a.uf16) tma_load_4d(sb + SU + SP, &mp.tile16_a, &bar[sj], x0, z0, s0 + i, a.uf16_row);
            else tma_load_4d(sb + SU + SP, &mp.tile_a, &bar[sj], x0, z0, s0 + i, a.uf_buf);
        }
    };

    if (tid == 0) {
        for (int j = 0; j < NS; ++j) mbar_init(&bar[j], 1);
        fence_mbar_init();
    }
    // The tap tables are written before the call's first step and never by a
    // step, so the group's tap ranges are read here, ahead of
    // griddepcontrol.wait, one thread per shot.
    if (sparse && tid < ns) {
        const int kcell = TZ / a.TZc;
        const int cbase = ((s0 + tid) * a.ncx + (int)blockIdx.x) * a.ncz;
        const int c0 = tzi * kcell, c1 = min(c0 + kcell, a.ncz);
        taprng[tid][0] = a.inj.cell_start ? a.inj.cell_start[cbase + c0] : 0;
        taprng[tid][1] = a.inj.cell_start ? a.inj.cell_start[cbase + c1] : 0;
        taprng[tid][2] = a.gat.cell_start ? a.gat.cell_start[cbase + c0] : 0;
        taprng[tid][3] = a.gat.cell_start ? a.gat.cell_start[cbase + c1] : 0;
    }
    __syncthreads();
    // Programmatic dependent launch: the next step's CTAs may be scheduled once
    // every CTA of this grid has started.  Until griddepcontrol.wait (below)
    // this grid reads only the model, which no step writes and whose writer
    // finished before the first step of the call started; the fields are read
    // only after the previous kernel in the stream has finished and its writes
    // are visible (both are no-ops for a launch without the attribute).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    int off[RB];
    bool live[RB], pad[RB];
    float4 kp[RB];
    float eps[SE ? 1 : RB][4], inv[SE ? 1 : RB][4];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        const int gz = z0 + ty + rr * BZ;
        off[rr] = gz * a.P + gx;
        live[rr] = gz < a.Nz && nvalid > 0;
        pad[rr] = gz < a.Nz && nvalid <= 0 && gx < a.P;
        kp[rr] = live[rr] ? ld4(a.kap + off[rr]) : make_float4(0.f, 0.f, 0.f, 0.f);
        const int dz = sponge_depth(gz, a.nb, a.nz);
        float ev[4], iv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int dd = max(sponge_depth(gx + e, a.nb, a.nx), dz);
            ev[e] = f4(kp[rr], e) * a.ceps * (float)(dd * dd);
            iv[e] = rcp_sponge(1.0f + ev[e]);
        }
        if (SE) {
            // each thread reads back only its own entries: no barrier needed
            const int r = ty + rr * BZ;
            *reinterpret_cast<float4*>(se + r * kTX + lx) = make_float4(ev[0], ev[1], ev[2], ev[3]);
            *reinterpret_cast<float4*>(se + (TZ + r) * kTX + lx) = make_float4(iv[0], iv[1], iv[2], iv[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                eps[SE ? 0 : rr][e] = ev[e];
                inv[SE ? 0 : rr][e] = iv[e];
            }
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0)
        for (int j = 0; j < NS - 1 && j < ns; ++j) issue(j);
    float* gq = imaging ? a.gacc + (size_t)grp * a.cell : nullptr;
    if (imaging) {
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int r = ty + rr * BZ;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live[rr]) v = *reinterpret_cast<const float4*>(gq + off[rr]);
            *reinterpret_cast<float4*>(sg + r * kTX + lx) = v;
        }
    }

    // the stencil's imaging terms of this thread's points, summed over the
    // group's shots in registers; the taps' terms (other threads' points) go to
    // the shared tile sg, added at the end
    float gr[RB][4];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr)
#pragma unroll
        for (int e = 0; e < 4; ++e) gr[rr][e] = 0.0f;

    // A thread whose wait for a stage gives up records the timeout and does no
    // further work, but passes every block barrier below (they are uniform), so
    // the CTA never splits; thread 0, which issues the copies, first waits
    // (bounded) for the copies it has in flight and issues no more.
    bool alive = true;
    for (int i = 0; i < ns; ++i) {
        const int shot = s0 + i, stage = i % NS;
        if (tid == 0 && alive && i + NS - 1 < ns) {
            fence_proxy_async();
            issue(i + NS - 1);  // into the stage shot i - 1 used (released by the barrier after it)
        }
        const size_t so = (size_t)shot * a.cell;
        float4 uo[RB];
        if (!PT) {
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
                uo[rr] = live[rr] ? *reinterpret_cast<const float4*>(a.uprev + so + off[rr])
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (alive && !mbar_wait(&bar[stage], (uint32_t)(i / NS) & 1u)) {
            alive = false;
            atomicOr(a.err, kErrTimeout);
            if (tid == 0) {
                // copies issued by this CTA may still land in its shared memory
                for (int j = i; j < i + NS && j < ns; ++j) mbar_wait(&bar[j % NS], (uint32_t)(j / NS) & 1u);
            }
        }
        const float* sb = st + stage * SU2;
        if (PT && alive) {
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) uo[rr] = lds4(sb + SU + (ty + rr * BZ) * kTX + lx);
        }
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            if (!alive) break;
            const int r = ty + rr * BZ;
            float* un = a.unew + so + off[rr];
            if (!live[rr]) {
                if (pad[rr]) *reinterpret_cast<float4*>(un) = make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            const float* row = sb + (r + 4) * SW + lx;
            const float4 A = lds4(row), B = lds4(row + 4), C = lds4(row + 8);
            const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
            float lap[4];
            lap4(w, [&](int k, float4& Up, float4& Dn) {
                Up = lds4(row + 4 - k * SW);
                Dn = lds4(row + 4 + k * SW);
            }, lap);
            const float cen[4] = {B.x, B.y, B.z, B.w};
            const float um[4] = {uo[rr].x, uo[rr].y, uo[rr].z, uo[rr].w};
            const float kv[4] = {kp[rr].x, kp[rr].y, kp[rr].z, kp[rr].w};
            const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
            float out[4];
            if (SE) {
                const float4 E = lds4(se + r * kTX + lx), I = lds4(se + (TZ + r) * kTX + lx);
                const float ev[4] = {E.x, E.y, E.z, E.w}, iv[4] = {I.x, I.y, I.z, I.w};
                update4(cen, um, lap, kv, ev, iv, zero4, out);
            } else {
                update4(cen, um, lap, kv, eps[SE ? 0 : rr], inv[SE ? 0 : rr], zero4, out);
            }
            // a full float4: points past Nx stay the zero exterior
            *reinterpret_cast<float4*>(un) = make_float4(out[0], nvalid > 1 ? out[1] : 0.0f,
                                                         nvalid > 2 ? out[2] : 0.0f, nvalid > 3 ? out[3] : 0.0f);
            if (!ADJ) {
                if (a.st16) {
                    if (nvalid == 4) {
                        store_bf16x4(a.st16 + so + off[rr], out);
                    } else {
                        for (int e = 0; e < nvalid; ++e) a.st16[so + off[rr] + e] = __float2bfloat16_rn(out[e]);
                    }
                }
                if (a.st32) {
                    if (nvalid == 4) {
                        *reinterpret_cast<float4*>(a.st32 + so + off[rr]) = make_float4(out[0], out[1], out[2], out[3]);
                    } else {
                        for (int e = 0; e < nvalid; ++e) a.st32[so + off[rr] + e] = out[e];
                    }
                }
            } else if (imaging) {
                float uf[4];
                if (ft && a.uf16) {
                    unpack_bf16x4(*reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(sb + SU + SP) +
                                                                  r * kTX + lx),
                                  uf);
                } else if (ft) {
                    const float4 v = lds4(sb + SU + SP + r * kTX + lx);
                    uf[0] = v.x;
                    uf[1] = v.y;
                    uf[2] = v.z;
                    uf[3] = v.w;
                } else if (a.uf16) {
                    unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + so + off[rr]), uf);
                } else {
                    const float4 v = ld4(a.uf32 + so + off[rr]);
                    uf[0] = v.x;
                    uf[1] = v.y;
                    uf[2] = v.z;
                    uf[3] = v.w;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) gr[rr][e] -= uf[e] * (out[e] - 2.0f * cen[e] + um[e]);
            }
        }
        // This CTA's taps for the shot (the same values in every thread, so the
        // decisions below are uniform over the CTA).
        int ib = 0, ie = 0, gb = 0, ge = 0;
        if (sparse) {
            ib = taprng[i][0];
            ie = taprng[i][1];
            gb = taprng[i][2];
            ge = taprng[i][3];
        }
        const bool taps = ie > ib || ge > gb;
        // the stage is refilled by shot i + NS's copies, and taps touch other threads' points
        if (taps || i + NS < ns) __syncthreads();
        if (taps) {
            // (its terms go to sg, which the stencil no longer touches before the end)
            sparse_phase<ADJ>(a, ib, ie, gb, ge, (long long)so, tid, 32 * BZ, imaging ? sg : nullptr, z0, x0);
        }
    }
    if (imaging) {
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int r = ty + rr * BZ;
            if (live[rr]) {
                const float4 t = *reinterpret_cast<const float4*>(sg + r * kTX + lx);
                *reinterpret_cast<float4*>(gq + off[rr]) =
                    make_float4(t.x + gr[rr][0], t.y + gr[rr][1], t.z + gr[rr][2], t.w + gr[rr][3]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 2D step, persistent over (tile, shot) items.  The items of a step, taken
// tile-major, are split into gridDim.x contiguous ranges, one per CTA, with as
// many CTAs as fit on the GPU at once.  A CTA therefore keeps one tile for
// several consecutive shots: the model, the sponge factors and, in the
// adjoint, the gradient tile are set up when its tile changes rather than per
// shot.  Each item's halo tile of u and its tile of the previous level arrive
// by TMA into a two-stage ring; the next item's copies are issued as soon as
// every thread is done with the stage they overwrite, one block barrier per
// item.  The adjoint sums the imaging term of the CTA's shots of one tile in
// shared memory and writes it to accumulator slot (CTA - first CTA of the
// tile): each slot has a single writer, so the gradient is deterministic.
__host__ __device__ inline int pst_owner(long long j, int C, long long W)
{
    return (int)(((j + 1) * C - 1) / W);  // the CTA whose range holds item j
}

template <int TZ, int BZ, bool ADJ>
__global__ void __launch_bounds__(32 * BZ, (TZ / BZ) <= 2 ? 1024 / (32 * BZ) : 512 / (32 * BZ))
    k_step2d_pst(const __grid_constant__ StepMaps mp, const StepArgs a)
{
    constexpr int SW = kTX + 8;
    constexpr int RB = TZ / BZ;
    constexpr int SU = (TZ + 8) * SW;  // halo tile of u
    constexpr int ST = TZ * kTX;       // tile of the previous level
    constexpr int STAGE = SU + ST;
    static_assert(SU % 32 == 0 && ST % 32 == 0, "sub-buffers must stay 128-byte aligned");
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar[2];
    float* st = reinterpret_cast<float*>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));
    float* sg = st + 2 * STAGE;  // [TZ][kTX] gradient tile (adjoint with imaging)
    const CUtensorMap* mh = ADJ ? &mp.halo_a : &mp.halo_f;
    const CUtensorMap* mt = ADJ ? &mp.tile_a : &mp.tile_f;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int lx = 4 * tx;
    const int ntz = (a.Nz + TZ - 1) / TZ;
    const long long W = (long long)ntz * a.ncx * a.nshot;
    const int C = gridDim.x;
    const int j0 = (int)((long long)blockIdx.x * W / C), j1 = (int)((long long)(blockIdx.x + 1) * W / C);
    if (j0 >= j1) return;  // CTA-uniform, before any barrier or copy
    const bool imaging = ADJ && a.gacc != nullptr;
    const bool sparse = a.inj.cell_start != nullptr || a.gat.cell_start != nullptr;
    constexpr uint32_t kBytes = STAGE * 4u;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int stage, int j) {
        const int tile = j / a.nshot, shot = j - tile * a.nshot;
        const int tz = tile / a.ncx, txi = tile - tz * a.ncx;
        float* d = st + stage * STAGE;
        mbar_expect_tx(&bar[stage], kBytes);
        tma_load_4d(d, mh, &bar[stage], txi * kTX - 4, tz * TZ - 4, shot, a.u_buf);
        tma_load_4d(d + SU, mt, &bar[stage], txi * kTX, tz * TZ, shot, a.prev_buf);
    };
    if (tid == 0) issue(0, j0);

    int cur_tile = -1, x0 = 0, z0 = 0, nvalid = 0;
    int off[RB];
    bool live[RB], pad[RB];
    float4 kp[RB];
    float eps[RB][4], inv[RB][4];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        off[rr] = 0;
        live[rr] = pad[rr] = false;
    }
    float* gq = nullptr;
    auto flush = [&]() {
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
            if (live[rr])
                *reinterpret_cast<float4*>(gq + off[rr]) =
                    *reinterpret_cast<const float4*>(sg + (ty + rr * BZ) * kTX + lx);
    };

    for (int j = j0; j < j1; ++j) {
        const int i = j - j0, stage = i & 1;
        const int tile = j / a.nshot, shot = j - tile * a.nshot;
        const bool ok = mbar_wait(&bar[stage], (uint32_t)(i >> 1) & 1u);
        // also: every thread is done with item j-1 (its stage and its sparse phase)
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(a.err, kErrTimeout);
                mbar_wait(&bar[stage], (uint32_t)(i >> 1) & 1u);  // let the copy land first
            }
            return;
        }
        if (tid == 0 && j + 1 < j1) {
            fence_proxy_async();
            issue(stage ^ 1, j + 1);
        }
        if (tile != cur_tile) {
            if (imaging && cur_tile >= 0) flush();
            cur_tile = tile;
            const int tz = tile / a.ncx, txi = tile - tz * a.ncx;
            x0 = txi * kTX;
            z0 = tz * TZ;
            const int gx = x0 + lx;
            nvalid = min(4, a.Nx - gx);
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
                const int gz = z0 + ty + rr * BZ;
                off[rr] = gz * a.P + gx;
                live[rr] = gz < a.Nz && nvalid > 0;
                pad[rr] = gz < a.Nz && nvalid <= 0 && gx < a.P;
                kp[rr] = live[rr] ? ld4(a.kap + off[rr]) : make_float4(0.f, 0.f, 0.f, 0.f);
                const int dz = sponge_depth(gz, a.nb, a.nz);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int dd = max(sponge_depth(gx + e, a.nb, a.nx), dz);
                    eps[rr][e] = f4(kp[rr], e) * a.ceps * (float)(dd * dd);
                    inv[rr][e] = rcp_sponge(1.0f + eps[rr][e]);
                }
            }
            if (imaging) {
                const int slot = (int)blockIdx.x - pst_owner((long long)tile * a.nshot, C, W);
                gq = a.gacc + (size_t)slot * a.cell;
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (live[rr]) v = *reinterpret_cast<const float4*>(gq + off[rr]);
                    *reinterpret_cast<float4*>(sg + (ty + rr * BZ) * kTX + lx) = v;
                }
            }
        }
        const size_t so = (size_t)shot * a.cell;
        const float* sb = st + stage * STAGE;
        const float* sp = sb + SU;
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int r = ty + rr * BZ;
            float* un = a.unew + so + off[rr];
            if (!live[rr]) {
                if (pad[rr]) *reinterpret_cast<float4*>(un) = make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            const float* row = sb + (r + 4) * SW + lx;
            const float4 A = lds4(row), B = lds4(row + 4), Cc = lds4(row + 8);
            const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, Cc.x, Cc.y, Cc.z, Cc.w};
            float lap[4];
            lap4(w, [&](int k, float4& Up, float4& Dn) {
                Up = lds4(row + 4 - k * SW);
                Dn = lds4(row + 4 + k * SW);
            }, lap);
            const float4 uo = lds4(sp + r * kTX + lx);
            const float cen[4] = {B.x, B.y, B.z, B.w};
            const float um[4] = {uo.x, uo.y, uo.z, uo.w};
            const float kv[4] = {kp[rr].x, kp[rr].y, kp[rr].z, kp[rr].w};
            const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
            float out[4];
            update4(cen, um, lap, kv, eps[rr], inv[rr], zero4, out);
            // a full float4: points past Nx stay the zero exterior
            *reinterpret_cast<float4*>(un) = make_float4(out[0], nvalid > 1 ? out[1] : 0.0f,
                                                         nvalid > 2 ? out[2] : 0.0f, nvalid > 3 ? out[3] : 0.0f);
            if (!ADJ) {
                if (a.st16) {
                    if (nvalid == 4) {
                        store_bf16x4(a.st16 + so + off[rr], out);
                    } else {
                        for (int e = 0; e < nvalid; ++e) a.st16[so + off[rr] + e] = __float2bfloat16_rn(out[e]);
                    }
                }
                if (a.st32) {
                    if (nvalid == 4) {
                        *reinterpret_cast<float4*>(a.st32 + so + off[rr]) = make_float4(out[0], out[1], out[2], out[3]);
                    } else {
                        for (int e = 0; e < nvalid; ++e) a.st32[so + off[rr] + e] = out[e];
                    }
                }
            } else if (imaging) {
                float uf[4];
                if (a.uf16) {
                    unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + so + off[rr]), uf);
                } else {
                    const float4 v = ld4(a.uf32 + so + off[rr]);
                    uf[0] = v.x;
                    uf[1] = v.y;
                    uf[2] = v.z;
                    uf[3] = v.w;
                }
                float* g = sg + r * kTX + lx;
#pragma unroll
                for (int e = 0; e < 4; ++e) g[e] -= uf[e] * (out[e] - 2.0f * cen[e] + um[e]);
            }
        }
        if (sparse) {
            const int kcell = TZ / a.TZc;
            const int tz = tile / a.ncx, txi = tile - tz * a.ncx;
            const int cbase = (shot * a.ncx + txi) * a.ncz;
            const int c0 = tz * kcell, c1 = min(c0 + kcell, a.ncz);
            int ib = 0, ie = 0, gb = 0, ge = 0;
            if (a.inj.cell_start) {
                ib = a.inj.cell_start[cbase + c0];
                ie = a.inj.cell_start[cbase + c1];
            }
            if (a.gat.cell_start) {
                gb = a.gat.cell_start[cbase + c0];
                ge = a.gat.cell_start[cbase + c1];
            }
            if (ib < ie || gb < ge) {  // CTA-uniform
                __syncthreads();       // this item's points are written
                sparse_phase<ADJ>(a, ib, ie, gb, ge, (long long)so, tid, 32 * BZ, imaging ? sg : nullptr, z0, x0);
            }
        }
    }
    if (imaging) {
        __syncthreads();
        flush();
    }
}

// ---------------------------------------------------------------------------
// 2D step, z-march.  Each warp owns a 128-column strip of TZ consecutive rows
// of one shot (a CTA stacks NW such warps in z) and walks down it: lane l
// keeps the 9-row z window of its 4 columns in registers, takes its x
// neighbours from lanes l-1 and l+1 by shuffles (lanes 0 and 31 load the
// 4-column halo of the strip), and prefetches the previous level, the model
// and, in the adjoint, the forward field and the gradient D rows ahead.  No
// shared memory and no block barriers: warps stream independently.  Rows in
// the interior of the grid skip the sponge factors.
template <int TZ, int NW, int D, bool ADJ>
__global__ void __launch_bounds__(32 * NW) k_step2d_zm(const StepArgs a)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = blockIdx.x * kTX;
    const int zs = ((int)blockIdx.y * NW + warp) * TZ;
    if (zs >= a.Nz) return;  // warp-uniform; no block barrier follows
    const int ze = min(zs + TZ, a.Nz);
    const int shot = blockIdx.z;
    const long long so = (long long)shot * a.cell;
    const float* __restrict__ u = a.u + so;
    const int gx = x0 + 4 * lane;
    const int nvalid = min(4, a.Nx - gx);
    const bool in_p = gx < a.P;
    const int hx = lane == 0 ? x0 - 4 : x0 + kTX;
    const bool hok = (lane == 0 || lane == 31) && hx >= 0 && hx < a.P;
    const bool imaging = ADJ && a.gacc != nullptr;
    const bool xin = x0 >= a.nb && x0 + kTX - 1 <= a.nb + a.nx - 1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

    auto ldu = [&](int z) { return (z >= 0 && z < a.Nz && in_p) ? ld4(u + (long long)z * a.P + gx) : z4; };
    auto ldh = [&](int z) { return (hok && z < ze) ? ld4(u + (long long)z * a.P + hx) : z4; };
    auto ldp = [&](int z) {
        return (z < ze && nvalid > 0) ? *reinterpret_cast<const float4*>(a.uprev + so + (long long)z * a.P + gx) : z4;
    };
    auto ldk = [&](int z) { return (z < ze && nvalid > 0) ? ld4(a.kap + (long long)z * a.P + gx) : z4; };
    auto ldf = [&](int z) {
        if (!imaging || z >= ze || nvalid <= 0) return z4;
        const long long off = so + (long long)z * a.P + gx;
        if (a.uf16) {
            float t[4];
            unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + off), t);
            return make_float4(t[0], t[1], t[2], t[3]);
        }
        return ld4(a.uf32 + off);
    };
    auto ldg = [&](int z) {
        return (imaging && z < ze && nvalid > 0)
                   ? *reinterpret_cast<const float4*>(a.gacc + so + (long long)z * a.P + gx)
                   : z4;
    };

    float4 q[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = ldu(zs - 4 + k);
    float4 hq[D], pq[D], kq[D], fq[D], gq[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        hq[d] = ldh(zs + d);
        pq[d] = ldp(zs + d);
        kq[d] = ldk(zs + d);
        fq[d] = ldf(zs + d);
        gq[d] = ldg(zs + d);
    }
    for (int z = zs; z < ze; ++z) {
        q[8] = ldu(z + 4);
        const float4 hc = hq[0], pc = pq[0], kc = kq[0], fc = fq[0], gc = gq[0];
#pragma unroll
        for (int d = 0; d + 1 < D; ++d) {
            hq[d] = hq[d + 1];
            pq[d] = pq[d + 1];
            kq[d] = kq[d + 1];
            fq[d] = fq[d + 1];
            gq[d] = gq[d + 1];
        }
        hq[D - 1] = ldh(z + D);
        pq[D - 1] = ldp(z + D);
        kq[D - 1] = ldk(z + D);
        fq[D - 1] = ldf(z + D);
        gq[D - 1] = ldg(z + D);

        const float4 B = q[4];
        float4 A, C;
        A.x = __shfl_up_sync(FULL, B.x, 1);
        A.y = __shfl_up_sync(FULL, B.y, 1);
        A.z = __shfl_up_sync(FULL, B.z, 1);
        A.w = __shfl_up_sync(FULL, B.w, 1);
        C.x = __shfl_down_sync(FULL, B.x, 1);
        C.y = __shfl_down_sync(FULL, B.y, 1);
        C.z = __shfl_down_sync(FULL, B.z, 1);
        C.w = __shfl_down_sync(FULL, B.w, 1);
        if (lane == 0) A = hc;
        if (lane == 31) C = hc;
        const long long off = (long long)z * a.P + gx;
        if (nvalid > 0) {
            const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
            float lap[4];
            lap4(w, [&](int k, float4& Up, float4& Dn) {
                Up = q[4 - k];
                Dn = q[4 + k];
            }, lap);
            float out[4], kv[4];
            const float cen[4] = {B.x, B.y, B.z, B.w}, um[4] = {pc.x, pc.y, pc.z, pc.w};
            const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int e = 0; e < 4; ++e) kv[e] = f4(kc, e);
            if (xin && z >= a.nb && z <= a.nb + a.nz - 1) {
                update4_interior(cen, um, lap, kv, out);
            } else {
                float ev[4], iv[4];
                const int dz = sponge_depth(z, a.nb, a.nz);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int dd = max(sponge_depth(gx + e, a.nb, a.nx), dz);
                    ev[e] = kv[e] * a.ceps * (float)(dd * dd);
                    iv[e] = rcp_sponge(1.0f + ev[e]);
                }
                update4(cen, um, lap, kv, ev, iv, zero4, out);
            }
            const float uf[4] = {fc.x, fc.y, fc.z, fc.w};
            write4<ADJ>(a, so, off, nvalid, out, cen, um, imaging, uf, gc);
        } else if (in_p) {
            zero_padding(a, so, off, gx);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
    }
    if (a.inj.cell_start || a.gat.cell_start) {
        __syncwarp();
        const int cbase = (shot * a.ncx + (int)blockIdx.x) * a.ncz;
        const int c0 = zs / a.TZc, c1 = min(c0 + TZ / a.TZc, a.ncz);
        int ib = 0, ie = 0, gb = 0, ge = 0;
        if (a.inj.cell_start) {
            ib = a.inj.cell_start[cbase + c0];
            ie = a.inj.cell_start[cbase + c1];
        }
        if (a.gat.cell_start) {
            gb = a.gat.cell_start[cbase + c0];
            ge = a.gat.cell_start[cbase + c1];
        }
        sparse_phase<ADJ, true>(a, ib, ie, gb, ge, so, lane, 32);
    }
}

// ---------------------------------------------------------------------------
// 2D step: persistent, TMA-fed.  Tile = 128 (x) by TZ (z) points; the CTA has
// TZ/R warps and warp w owns the R consecutive rows w*R .. w*R+R-1 of a tile,
// keeping the 9-row z window of its lane's 4 x points in registers (so shared
// memory is read once per row for the z neighbours).  Per tile one elected
// thread issues TMA loads of the halo tile of u ((TZ+8) x 136), the previous
// level, the model and, in the adjoint, the forward field and the gradient
// accumulators into an NST-deep ring of stages; out-of-range boxes read as
// zero, which is the Dirichlet exterior.  Results are stored straight from
// registers.  Tiles are dealt round-robin to the CTAs (one per SM).
template <int TZ, int R, int NST, bool ADJ>
__global__ void __launch_bounds__(32 * (TZ / R), 1) k_step2d_tma(const __grid_constant__ StepMaps mp, const StepArgs a)
{
    constexpr int NTHR = 32 * (TZ / R);
    constexpr int SW = kTX + 8;
    constexpr int SU = (TZ + 8) * SW;  // floats in the halo tile
    constexpr int ST = TZ * kTX;       // floats in a point tile
    constexpr int NT = ADJ ? 4 : 2;
    constexpr int STAGE = SU + NT * ST;
    static_assert(SU % 32 == 0 && ST % 32 == 0, "sub-buffers must stay 128-byte aligned");
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t bars[NST];
    float* base = reinterpret_cast<float*>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));

    const CUtensorMap* mh = ADJ ? &mp.halo_a : &mp.halo_f;
    const CUtensorMap* mt = ADJ ? &mp.tile_a : &mp.tile_f;
    const CUtensorMap* mk = ADJ ? &mp.kap_a : &mp.kap_f;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntz = (a.Nz + TZ - 1) / TZ;
    const int per_shot = ntz * a.ncx;
    const int ntile = a.nshot * per_shot;
    const bool imaging = ADJ && a.g_buf >= 0;
    const bool uf_bf16 = ADJ && a.uf_buf < 0;
    const uint32_t bytes = (SU + 2 * ST) * 4u + (imaging ? (uf_bf16 ? ST * 2u : ST * 4u) + ST * 4u : 0u);
    const int kcell = TZ / a.TZc;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int s, int t) {
        float* st = base + s * STAGE;
        const int shot = t / per_shot, r = t - shot * per_shot, tz = r / a.ncx, tx = r - tz * a.ncx;
        const int x0 = tx * kTX, z0 = tz * TZ;
        mbar_expect_tx(&bars[s], bytes);
        tma_load_4d(st, mh, &bars[s], x0 - 4, z0 - 4, shot, a.u_buf);
        tma_load_4d(st + SU, mt, &bars[s], x0, z0, shot, a.prev_buf);
        tma_load_2d(st + SU + ST, mk, &bars[s], x0, z0);
        if (imaging) {
            if (uf_bf16)
                tma_load_4d(st + SU + 2 * ST, &mp.tile16_a, &bars[s], x0, z0, shot, a.uf16_row);
            else
                tma_load_4d(st + SU + 2 * ST, mt, &bars[s], x0, z0, shot, a.uf_buf);
            tma_load_4d(st + SU + 3 * ST, mt, &bars[s], x0, z0, shot, a.g_buf);
        }
    };

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < ntile) issue(s, t);
        }
    }

    const bool sparse = a.inj.cell_start != nullptr || a.gat.cell_start != nullptr;
    for (int i = 0;; ++i) {
        const int t = blockIdx.x + i * gridDim.x;
        if (t >= ntile) break;
        const int s = i % NST;
        const bool ok = mbar_wait(&bars[s], (uint32_t)(i / NST) & 1u);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(a.err, kErrTimeout);
                // let copies still in flight land before the CTA's shared memory is released
                for (int j = 0; j < NST; ++j) {
                    const int ii = i + j;
                    if ((long long)blockIdx.x + (long long)ii * gridDim.x < ntile)
                        mbar_wait(&bars[ii % NST], (uint32_t)(ii / NST) & 1u);
                }
            }
            return;
        }
        const float* su = base + s * STAGE;
        const float* sp = su + SU;
        const float* sk = sp + ST;
        const float* sf = sk + ST;
        const float* sg = sf + ST;
        const int shot = t / per_shot, rt = t - shot * per_shot, tz = rt / a.ncx, txi = rt - tz * a.ncx;
        const int x0 = txi * kTX, z0 = tz * TZ;
        const int gx = x0 + 4 * lane;
        const int nvalid = min(4, a.Nx - gx);
        const long long so = (long long)shot * a.cell;
        const int r0 = warp * R;
        float4 q[9];
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = lds4(su + (r0 + k) * SW + 4 * lane + 4);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int r = r0 + j;
            q[8] = lds4(su + (r + 8) * SW + 4 * lane + 4);
            const int gz = z0 + r;
            if (gz < a.Nz && nvalid <= 0) zero_padding(a, so, (long long)gz * a.P + gx, gx);
            if (gz < a.Nz && nvalid > 0) {
                const float4 A = lds4(su + (r + 4) * SW + 4 * lane);
                const float4 C = lds4(su + (r + 4) * SW + 4 * lane + 8);
                const float4 B = q[4];
                const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
                float lap[4];
                lap4(w, [&](int k, float4& Up, float4& Dn) {
                    Up = q[4 - k];
                    Dn = q[4 + k];
                }, lap);
                const float4 kp = lds4(sk + r * kTX + 4 * lane);
                const float4 uo = lds4(sp + r * kTX + 4 * lane);
                const int dz = sponge_depth(gz, a.nb, a.nz);
                float out[4], cen[4], um[4], uf[4] = {0.f, 0.f, 0.f, 0.f}, kv[4], ev[4], iv[4];
                const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
                float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int dd = max(sponge_depth(gx + e, a.nb, a.nx), dz);
                    kv[e] = f4(kp, e);
                    ev[e] = kv[e] * a.ceps * (float)(dd * dd);
                    iv[e] = rcp_sponge(1.0f + ev[e]);
                    cen[e] = w[e + 4];
                    um[e] = f4(uo, e);
                }
                update4(cen, um, lap, kv, ev, iv, zero4, out);
                if (imaging) {
                    if (uf_bf16) {
                        unpack_bf16x4(*reinterpret_cast<const uint2*>(
                                          reinterpret_cast<const __nv_bfloat16*>(sf) + r * kTX + 4 * lane),
                                      uf);
                    } else {
                        const float4 v = lds4(sf + r * kTX + 4 * lane);
                        uf[0] = v.x;
                        uf[1] = v.y;
                        uf[2] = v.z;
                        uf[3] = v.w;
                    }
                    gv = lds4(sg + r * kTX + 4 * lane);
                }
                write4<ADJ>(a, so, (long long)gz * a.P + gx, nvalid, out, cen, um, imaging, uf, gv);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
        }
        __syncthreads();  // stage s has been read and tile t's points are written
        if (tid == 0) {
            const int t2 = blockIdx.x + (i + NST) * gridDim.x;
            if (t2 < ntile) {
                fence_proxy_async();
                issue(s, t2);
            }
        }
        if (sparse) {
            const int cbase = (shot * a.ncx + txi) * a.ncz;  // ncy = 1 in 2D
            const int c0 = tz * kcell, c1 = min(c0 + kcell, a.ncz);
            int ib = 0, ie = 0, gb = 0, ge = 0;
            if (a.inj.cell_start) {
                ib = a.inj.cell_start[cbase + c0];
                ie = a.inj.cell_start[cbase + c1];
            }
            if (a.gat.cell_start) {
                gb = a.gat.cell_start[cbase + c0];
                ge = a.gat.cell_start[cbase + c1];
            }
            sparse_phase<ADJ>(a, ib, ie, gb, ge, so, tid, NTHR);
        }
    }
}

// ---------------------------------------------------------------------------
// 3D step.  Tile = 128 (x) by TY (y) by TZC (z) points; CTA = 32 x TY threads
// marching in z.  Each thread keeps its 4 x points of the 9 planes z-4..z+4 in
// registers; the current xy plane with its 4-point halo sits in shared memory.
template <int TY, int TZC, bool ADJ>
__global__ void __launch_bounds__(32 * TY) k_step3d(const StepArgs a)
{
    constexpr int SW = kTX + 8;
    __shared__ __align__(16) float s[TY + 8][SW];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * TY;
    const int ntz = (a.Nz + TZC - 1) / TZC;
    const int shot = blockIdx.z / ntz, tzi = blockIdx.z - shot * ntz;
    const int z0 = tzi * TZC;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const long long so = (long long)shot * a.cell;
    const long long plane = (long long)a.Ny * a.P;
    const float* __restrict__ u = a.u + so;
    const int nvalid = min(4, a.Nx - gx);
    const bool imaging = ADJ && a.gacc != nullptr;

    auto ld = [&](int z, int y, int x) -> float4 {
        if (z < 0 || z >= a.Nz || y < 0 || y >= a.Ny || x < 0 || x >= a.P) return make_float4(0.f, 0.f, 0.f, 0.f);
        return ld4(u + z * plane + (long long)y * a.P + x);
    };

    float4 q[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = ld(z0 - 4 + k, gy, gx);

    for (int zz = 0; zz < TZC; ++zz) {
        const int gz = z0 + zz;
        if (gz >= a.Nz) break;
        q[8] = ld(gz + 4, gy, gx);
        *reinterpret_cast<float4*>(&s[ty + 4][4 + 4 * tx]) = q[4];
        if (tx == 0) *reinterpret_cast<float4*>(&s[ty + 4][0]) = ld(gz, gy, x0 - 4);
        if (tx == 31) *reinterpret_cast<float4*>(&s[ty + 4][132]) = ld(gz, gy, x0 + kTX);
        for (int i = tid; i < 8 * (SW / 4); i += 32 * TY) {
            const int r = i / (SW / 4), c4 = i - r * (SW / 4);
            const int yy = r < 4 ? y0 - 4 + r : y0 + TY + (r - 4);
            const int sr = r < 4 ? r : TY + r;
            *reinterpret_cast<float4*>(&s[sr][4 * c4]) = ld(gz, yy, x0 - 4 + 4 * c4);
        }
        __syncthreads();
        if (gy < a.Ny && nvalid <= 0) zero_padding(a, so, gz * plane + (long long)gy * a.P + gx, gx);
        if (gy < a.Ny && nvalid > 0) {
            const float* row = &s[ty + 4][4 * tx];
            const float4 A = lds4(row), B = lds4(row + 4), C = lds4(row + 8);
            const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
            float lap[4];
            lap4_3d(w, [&](int k, float4& Up, float4& Dn, float4& Zu, float4& Zd) {
                Up = lds4(&s[ty + 4 - k][4 * tx + 4]);
                Dn = lds4(&s[ty + 4 + k][4 * tx + 4]);
                Zu = q[4 - k];
                Zd = q[4 + k];
            }, lap);
            const long long off = gz * plane + (long long)gy * a.P + gx;
            const float4 kp = ld4(a.kap + off);
            const float4 uo = *reinterpret_cast<const float4*>(a.uprev + so + off);
            const int dzy = max(sponge_depth(gz, a.nb, a.nz), sponge_depth(gy, a.nb, a.ny));
            float out[4], cen[4], um[4], uf[4] = {0.f, 0.f, 0.f, 0.f};
            float bsrc[4] = {0.f, 0.f, 0.f, 0.f};
            if (a.dmv) born_source(a, so, off, bsrc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int dd = max(sponge_depth(gx + i, a.nb, a.nx), dzy);
                const float kap = f4(kp, i);
                const float eps = kap * a.ceps * (float)(dd * dd);
                cen[i] = w[i + 4];
                um[i] = f4(uo, i);
                out[i] = leap1(cen[i], um[i], lap[i], kap, eps, rcp_sponge(1.0f + eps), bsrc[i]);
            }
            float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (imaging) {
                if (a.uf16) {
                    unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + so + off), uf);
                } else {
                    const float4 v = ld4(a.uf32 + so + off);
                    uf[0] = v.x;
                    uf[1] = v.y;
                    uf[2] = v.z;
                    uf[3] = v.w;
                }
                gv = *reinterpret_cast<const float4*>(a.gacc + so + off);
            }
            write4<ADJ>(a, so, off, nvalid, out, cen, um, imaging, uf, gv);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
    }
    if (a.inj.cell_start || a.gat.cell_start) {
        const int kcell = TZC / a.TZc;
        const int cbase = ((shot * a.ncx + (int)blockIdx.x) * a.ncy + (int)blockIdx.y) * a.ncz;
        const int c0 = tzi * kcell, c1 = min(c0 + kcell, a.ncz);
        int ib = 0, ie = 0, gb = 0, ge = 0;
        if (a.inj.cell_start) {
            ib = a.inj.cell_start[cbase + c0];
            ie = a.inj.cell_start[cbase + c1];
        }
        if (a.gat.cell_start) {
            gb = a.gat.cell_start[cbase + c0];
            ge = a.gat.cell_start[cbase + c1];
        }
        sparse_phase<ADJ>(a, ib, ie, gb, ge, so, tid, 32 * TY);
    }
}

// ---------------------------------------------------------------------------
// 3D step fed by TMA.  Tile = 128 (x) by TY (y) points, CTA = 32 x TY threads
// (4 x points per thread) marching over TZC planes in z.  Every xy plane of u
// with its 4-point halo ((TY+8) x 136 floats) arrives by one 5D bulk tensor
// load into a ring of NR shared-memory slots: planes z..z+4 are resident
// while planes up to z+NR-1 are in flight.  Each thread keeps the 9 planes
// z-4..z+4 of its 4 points in registers (read once from the ring when a plane
// arrives) and takes x and y neighbours from the centre plane's slot.  A slot
// is refilled right after the block barrier that ends the plane that used it
// as centre: one barrier per plane.  Sponge depths in x and y are fixed per
// thread.  Waits are bounded; on a timeout the CTA records kErrTimeout, lets
// its issued copies land and returns.
template <int TY, int TZC, int NR, bool ADJ, int PF = 0>
__global__ void __launch_bounds__(32 * TY, TY <= 8 ? 2 : 1) k_step3d_tma(const __grid_constant__ StepMaps mp,
                                                                        const StepArgs a)
{
    constexpr int SW = kTX + 8, SP = (TY + 8) * SW;
    static_assert(SP % 32 == 0, "ring slots must stay 128-byte aligned");
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar[NR];
    float* ring = reinterpret_cast<float*>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * TY;
    const int ntz = (a.Nz + TZC - 1) / TZC;
    const int shot = blockIdx.z / ntz, tzi = blockIdx.z - shot * ntz;
    const int z0 = tzi * TZC, z1 = min(z0 + TZC, a.Nz);
    const int nplanes = z1 - z0 + 8;  // planes z0-4 .. z1+3, index j = z - (z0 - 4)
    const int lx = 4 * tx, gx = x0 + lx, gy = y0 + ty;
    const int nvalid = min(4, a.Nx - gx);
    const bool live = gy < a.Ny && nvalid > 0;
    const bool pad = gy < a.Ny && nvalid <= 0 && gx < a.P;
    const size_t so = (size_t)shot * a.cell;
    const size_t plane = (size_t)a.Ny * a.P;
    const size_t roff = (size_t)gy * a.P + gx;
    const bool imaging = ADJ && a.gacc != nullptr;
    constexpr uint32_t kBytes = SP * 4u;
    // PF > 0: the model and the previous level of the thread's 4 points arrive
    // PF planes ahead by cp.async into PF + 1 per-thread slots of shared memory
    // ([slot][kap, uprev][thread] float4s: conflict-free), without registers
    constexpr int NT = 32 * TY, PS = PF + 1;
    float4* pre = reinterpret_cast<float4*>(ring + NR * SP);
    auto prefetch = [&](int i) {  // plane z0 + i
        const int gz = z0 + i;
        if (PF > 0 && live && gz < z1) {
            const int sl = i % PS;
            cp_async16(pre + (2 * sl) * NT + tid, a.kap + gz * plane + roff, 16);
            cp_async16(pre + (2 * sl + 1) * NT + tid, a.uprev + so + gz * plane + roff, 16);
        }
        if (PF > 0) cp_async_commit();
    };

    auto issue = [&](int j) {
        const int sl = j % NR;
        mbar_expect_tx(&bar[sl], kBytes);
        tma_load_5d(ring + sl * SP, &mp.halo3, &bar[sl], x0 - 4, y0 - 4, z0 - 4 + j, shot, a.u_buf);
    };
    auto waitp = [&](int j) { return mbar_wait(&bar[j % NR], (uint32_t)(j / NR) & 1u); };
    auto own = [&](int j) { return lds4(ring + (j % NR) * SP + (ty + 4) * SW + lx + 4); };
    int issued = -1;  // highest plane index issued (thread 0)
    auto drain = [&](int from) {
        // copies issued by this CTA may still land in its shared memory
        if (PF > 0) cp_async_wait_all();
        if (tid == 0) {
            atomicOr(a.err, kErrTimeout);
            for (int j = from; j <= issued; ++j) waitp(j);
        }
    };

    if (tid == 0) {
        for (int k = 0; k < NR; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j < min(NR, nplanes); ++j) issue(j);
        issued = min(NR, nplanes) - 1;
    }

    int dxy[4];
    {
        const int dy = sponge_depth(gy, a.nb, a.ny);
#pragma unroll
        for (int e = 0; e < 4; ++e) dxy[e] = max(sponge_depth(gx + e, a.nb, a.nx), dy);
    }
    float4 q[9];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ok = waitp(j) && ok;
        q[j] = own(j);
    }
    if (__syncthreads_or(!ok)) {
        drain(0);
        return;
    }
    if (tid == 0) {
        for (int j = NR; j < min(NR + 4, nplanes); ++j) issue(j);
        issued = max(issued, min(NR + 4, nplanes) - 1);
    }
#pragma unroll
    for (int j = 4; j < 8; ++j) {
        ok = waitp(j) && ok;
        q[j] = own(j);
    }

    // the model and the previous level of the next plane are loaded one plane
    // ahead (PF = 0), or PF planes ahead into shared memory
    float4 kp = make_float4(0.f, 0.f, 0.f, 0.f), uo = kp;
    if (PF == 0 && live) {
        kp = ld4(a.kap + z0 * plane + roff);
        uo = *reinterpret_cast<const float4*>(a.uprev + so + z0 * plane + roff);
    }
    for (int j = 0; j < PF; ++j) prefetch(j);
    for (int i = 0; i < z1 - z0; ++i) {
        const int gz = z0 + i;
        const size_t off = gz * plane + roff;
        float4 kpn = make_float4(0.f, 0.f, 0.f, 0.f), uon = kpn;
        if (PF == 0 && live && gz + 1 < z1) {
            kpn = ld4(a.kap + off + plane);
            uon = *reinterpret_cast<const float4*>(a.uprev + so + off + plane);
        }
        if (PF > 0) {
            prefetch(i + PF);    // into the slot plane i - 1 used
            cp_async_wait<PF>();  // plane i's copies (PF groups younger than it may stay pending)
            if (live) {
                kp = pre[(2 * (i % PS)) * NT + tid];
                uo = pre[(2 * (i % PS) + 1) * NT + tid];
            }
        }
        ok = waitp(i + 8) && ok;
        q[8] = own(i + 8);
        const float* cs = ring + ((i + 4) % NR) * SP + (ty + 4) * SW + lx;  // centre plane, this thread's row
        float* un = a.unew + so + off;
        if (live) {
            const float4 A = lds4(cs), B = lds4(cs + 4), C = lds4(cs + 8);
            const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
            float lap[4];
            lap4_3d(w, [&](int k, float4& Up, float4& Dn, float4& Zu, float4& Zd) {
                Up = lds4(cs + 4 - k * SW);
                Dn = lds4(cs + 4 + k * SW);
                Zu = q[4 - k];
                Zd = q[4 + k];
            }, lap);
            const int dz = sponge_depth(gz, a.nb, a.nz);
            const float cen[4] = {B.x, B.y, B.z, B.w};
            const float um[4] = {uo.x, uo.y, uo.z, uo.w};
            float out[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int dd = max(dxy[e], dz);
                const float kap = f4(kp, e);
                const float eps = kap * a.ceps * (float)(dd * dd);
                out[e] = leap1(cen[e], um[e], lap[e], kap, eps, rcp_sponge(1.0f + eps), 0.0f);
            }
            float uf[4] = {0.f, 0.f, 0.f, 0.f};
            float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (imaging) {
                if (a.uf16) {
                    unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + so + off), uf);
                } else {
                    const float4 v = ld4(a.uf32 + so + off);
                    uf[0] = v.x;
                    uf[1] = v.y;
                    uf[2] = v.z;
                    uf[3] = v.w;
                }
                gv = *reinterpret_cast<const float4*>(a.gacc + so + off);
            }
            write4<ADJ>(a, so, off, nvalid, out, cen, um, imaging, uf, gv);
        } else if (pad) {
            *reinterpret_cast<float4*>(un) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
        if (PF == 0) {
            kp = kpn;
            uo = uon;
        }
        // every thread is done with the centre slot of this plane: refill it
        if (__syncthreads_or(!ok)) {
            drain(0);
            return;
        }
        if (tid == 0 && i + 4 + NR < nplanes) {
            fence_proxy_async();
            issue(i + 4 + NR);
            issued = i + 4 + NR;
        }
    }
    if (a.inj.cell_start || a.gat.cell_start) {
        // the tile covers TY / TY_cell tap cells in y and TZC / TZc in z
        const int kcell = TZC / a.TZc;
        const int c0 = tzi * kcell, c1 = min(c0 + kcell, a.ncz);
        for (int cy = blockIdx.y * (TY / 8); cy < min((int)(blockIdx.y + 1) * (TY / 8), a.ncy); ++cy) {
            const int cbase = ((shot * a.ncx + (int)blockIdx.x) * a.ncy + cy) * a.ncz;
            int ib = 0, ie = 0, gb = 0, ge = 0;
            if (a.inj.cell_start) {
                ib = a.inj.cell_start[cbase + c0];
                ie = a.inj.cell_start[cbase + c1];
            }
            if (a.gat.cell_start) {
                gb = a.gat.cell_start[cbase + c0];
                ge = a.gat.cell_start[cbase + c1];
            }
            sparse_phase<ADJ>(a, ib, ie, gb, ge, (long long)so, tid, 32 * TY);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// 3D step, TMA plane ring without block barriers in the z loop.  As
// k_step3d_tma, but each ring slot also has an "empty" barrier on which every
// warp arrives once it is done with the slot (planes z0-4..z0-1 right after the
// prologue, every other plane after its turn as centre plane).  Thread 0
// refills a slot LAG = 2 planes after its release, waiting on that barrier, so
// warps never wait for one another, only for their data.  Every wait is
// bounded; a thread whose wait gives up raises a shared abort flag, all threads
// leave the loop and meet at one final barrier, thread 0 records kErrTimeout,
// waits for the copies still in flight (at most one per slot) and the CTA
// returns.
template <int TY, int TZC, int NR, bool ADJ>
__global__ void __launch_bounds__(32 * TY, 2) k_step3d_ws(const __grid_constant__ StepMaps mp, const StepArgs a)
{
    constexpr int SW = kTX + 8, SP = (TY + 8) * SW, LAG = 2;
    static_assert(SP % 32 == 0, "ring slots must stay 128-byte aligned");
    static_assert(NR >= 8 + LAG, "planes 0..7 are issued up front and the lag must leave slots to refill");
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t full[NR], empty[NR];
    __shared__ volatile int sabort;
    float* ring = reinterpret_cast<float*>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * TY;
    const int ntz = (a.Nz + TZC - 1) / TZC;
    const int shot = blockIdx.z / ntz, tzi = blockIdx.z - shot * ntz;
    const int z0 = tzi * TZC, z1 = min(z0 + TZC, a.Nz);
    const int nplanes = z1 - z0 + 8;  // planes z0-4 .. z1+3, index j = z - (z0 - 4)
    const int lx = 4 * tx, gx = x0 + lx, gy = y0 + ty;
    const int nvalid = min(4, a.Nx - gx);
    const bool live = gy < a.Ny && nvalid > 0;
    const bool pad = gy < a.Ny && nvalid <= 0 && gx < a.P;
    const size_t so = (size_t)shot * a.cell;
    const size_t plane = (size_t)a.Ny * a.P;
    const size_t roff = (size_t)gy * a.P + gx;
    const bool imaging = ADJ && a.gacc != nullptr;
    constexpr uint32_t kBytes = SP * 4u;

    auto issue = [&](int j) {
        const int sl = j % NR;
        mbar_expect_tx(&full[sl], kBytes);
        tma_load_5d(ring + sl * SP, &mp.halo3, &full[sl], x0 - 4, y0 - 4, z0 - 4 + j, shot, a.u_buf);
    };
    auto waitp = [&](int j) { return mbar_wait(&full[j % NR], (uint32_t)(j / NR) & 1u); };
    auto own = [&](int j) { return lds4(ring + (j % NR) * SP + (ty + 4) * SW + lx + 4); };
    auto release = [&](int j) {
        __syncwarp();
        if (tx == 0) mbar_arrive(&empty[j % NR]);
    };

    if (tid == 0) {
        for (int k = 0; k < NR; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], TY);
        }
        sabort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    int next = 0;  // next plane to issue (thread 0)
    if (tid == 0) {
        for (; next < min(NR, nplanes); ++next) issue(next);
    }
    // thread 0 refills the slot of every plane released at least LAG planes ago
    auto refill = [&](int released) {
        while (next < nplanes && next - NR <= released - LAG) {
            if (!mbar_wait(&empty[next % NR], (uint32_t)((next - NR) / NR) & 1u)) return false;
            fence_proxy_async();
            issue(next);
            ++next;
        }
        return true;
    };

    int dxy[4];
    {
        const int dy = sponge_depth(gy, a.nb, a.ny);
#pragma unroll
        for (int e = 0; e < 4; ++e) dxy[e] = max(sponge_depth(gx + e, a.nb, a.nx), dy);
    }
    float4 q[9];
    bool fail = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        fail = fail || !waitp(j);
        q[j] = own(j);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) release(j);  // below the tile's first plane: never a centre

    float4 kp = make_float4(0.f, 0.f, 0.f, 0.f), uo = kp;
    if (live) {
        kp = ld4(a.kap + z0 * plane + roff);
        uo = *reinterpret_cast<const float4*>(a.uprev + so + z0 * plane + roff);
    }
    for (int i = 0; i < z1 - z0 && !fail; ++i) {
        if (sabort) break;
        const int gz = z0 + i;
        const size_t off = gz * plane + roff;
        float4 kpn = make_float4(0.f, 0.f, 0.f, 0.f), uon = kpn;
        if (live && gz + 1 < z1) {
            kpn = ld4(a.kap + off + plane);
            uon = *reinterpret_cast<const float4*>(a.uprev + so + off + plane);
        }
        if (!waitp(i + 8)) {
            fail = true;
            break;
        }
        q[8] = own(i + 8);
        const float* cs = ring + ((i + 4) % NR) * SP + (ty + 4) * SW + lx;  // centre plane, this thread's row
        float* un = a.unew + so + off;
        if (live) {
            const float4 A = lds4(cs), B = lds4(cs + 4), C = lds4(cs + 8);
            const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
            float lap[4];
            lap4_3d(w, [&](int k, float4& Up, float4& Dn, float4& Zu, float4& Zd) {
                Up = lds4(cs + 4 - k * SW);
                Dn = lds4(cs + 4 + k * SW);
                Zu = q[4 - k];
                Zd = q[4 + k];
            }, lap);
            const int dz = sponge_depth(gz, a.nb, a.nz);
            const float cen[4] = {B.x, B.y, B.z, B.w};
            const float um[4] = {uo.x, uo.y, uo.z, uo.w};
            float out[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int dd = max(dxy[e], dz);
                const float kap = f4(kp, e);
                const float eps = kap * a.ceps * (float)(dd * dd);
                out[e] = leap1(cen[e], um[e], lap[e], kap, eps, rcp_sponge(1.0f + eps), 0.0f);
            }
            float uf[4] = {0.f, 0.f, 0.f, 0.f};
            float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (imaging) {
                if (a.uf16) {
                    unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + so + off), uf);
                } else {
                    const float4 v = ld4(a.uf32 + so + off);
                    uf[0] = v.x;
                    uf[1] = v.y;
                    uf[2] = v.z;
                    uf[3] = v.w;
                }
                gv = *reinterpret_cast<const float4*>(a.gacc + so + off);
            }
            write4<ADJ>(a, so, off, nvalid, out, cen, um, imaging, uf, gv);
        } else if (pad) {
            *reinterpret_cast<float4*>(un) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
        kp = kpn;
        uo = uon;
        release(i + 4);
        if (tid == 0 && !refill(i + 4)) {
            fail = true;
            break;
        }
    }
    if (fail) sabort = 1;
    if (__syncthreads_or(fail || sabort)) {
        if (tid == 0) {
            atomicOr(a.err, kErrTimeout);
            // at most one copy per slot can be in flight: the last NR issued
            for (int j = max(0, next - NR); j < next; ++j) waitp(j);
        }
        return;
    }
    if (a.inj.cell_start || a.gat.cell_start) {
        const int kcell = TZC / a.TZc;
        const int c0 = tzi * kcell, c1 = min(c0 + kcell, a.ncz);
        for (int cy = blockIdx.y * (TY / 8); cy < min((int)(blockIdx.y + 1) * (TY / 8), a.ncy); ++cy) {
            const int cbase = ((shot * a.ncx + (int)blockIdx.x) * a.ncy + cy) * a.ncz;
            int ib = 0, ie = 0, gb = 0, ge = 0;
            if (a.inj.cell_start) {
                ib = a.inj.cell_start[cbase + c0];
                ie = a.inj.cell_start[cbase + c1];
            }
            if (a.gat.cell_start) {
                gb = a.gat.cell_start[cbase + c0];
                ge = a.gat.cell_start[cbase + c1];
            }
            sparse_phase<ADJ>(a, ib, ie, gb, ge, (long long)so, tid, 32 * TY);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------

static int num_sms()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        n = v;
    }
    return n;
}

// True on the first call for the current device with this flag array (one
// flag per device): kernel attributes such as the dynamic shared-memory limit
// are per device, so each device gets its own first call.
constexpr int kMaxDev = 64;
static bool first_on_device(bool* done)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        (void)cudaGetLastError();
        return true;
    }
    if (done[dev]) return false;
    done[dev] = true;
    return true;
}

template <int TZ, int R, int NST, bool ADJ>
static void launch_2d(const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
    constexpr int STAGE = (TZ + 8) * (kTX + 8) + (ADJ ? 4 : 2) * TZ * kTX;
    constexpr size_t smem = (size_t)NST * STAGE * 4 + 128;
    static bool configured[kMaxDev] = {};
    if (first_on_device(configured)) {
        cudaFuncSetAttribute(k_step2d_tma<TZ, R, NST, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    const int ntz = (a.Nz + TZ - 1) / TZ;
    const long long ntile = (long long)a.nshot * ntz * a.ncx;
    const int grid = (int)std::min<long long>(ntile, num_sms());
    k_step2d_tma<TZ, R, NST, ADJ><<<grid, 32 * (TZ / R), smem, s>>>(*maps, a);
}

// 2D variants (which = 0 forward, 1 adjoint).  The TMA map boxes and the
// launch below must agree on TZ; plan/api read TZ from this table.
static const Variant2D kFwd2D[] = {{0, 32, 4, 0, 0}, {1, 48, 6, 2, 0}, {1, 32, 4, 3, 0}, {1, 24, 3, 4, 0},
                                   {1, 16, 2, 4, 0}, {1, 32, 2, 3, 0}, {2, 32, 8, 0, 4}, {2, 16, 8, 0, 4},
                                   {2, 32, 8, 0, 8}, {2, 16, 8, 0, 2}, {3, 24, 4, 1, 0}, {3, 24, 4, 2, 0},
                                   {3, 48, 4, 2, 0}, {3, 16, 8, 2, 0}, {1, 32, 1, 3, 0}, {2, 16, 8, 0, 8},
                                   {2, 16, 8, 0, 16}, {2, 8, 8, 0, 8}, {4, 16, 8, 0, 2}, {4, 16, 8, 0, 4},
                                   {4, 16, 8, 0, 8}, {4, 32, 8, 0, 2}, {4, 32, 8, 0, 4}, {4, 8, 8, 0, 4},
                                   {5, 16, 8, 0, 0}, {5, 8, 8, 0, 0}, {5, 32, 8, 0, 0}, {4, 16, 8, 1, 2},
                                   {4, 16, 8, 1, 4}, {4, 8, 8, 1, 4}, {4, 16, 8, 2, 2}, {4, 16, 8, 3, 2},
                                   {4, 16, 8, 2, 4},  {7, 16, 4, 0, 2}, {7, 16, 4, 1, 4}, {7, 16, 2, 2, 2},
                                   {7, 32, 8, 3, 2},  {7, 32, 4, 4, 2}, {7, 16, 8, 5, 2}, {4, 16, 8, 9, 2},
                                   {4, 16, 8, 9, 4},  {4, 16, 8, 17, 4}, {4, 16, 8, 9, 8}, {4, 16, 8, 17, 8}, {4, 16, 8, 41, 4},
                                   {4, 16, 8, 33, 2},  {4, 16, 8, 41, 8}, {4, 16, 8, 49, 4}};
static const Variant2D kAdj2D[] = {{0, 32, 4, 0, 0}, {1, 24, 3, 3, 0}, {1, 16, 2, 4, 0}, {1, 32, 4, 2, 0},
                                   {2, 32, 8, 0, 4}, {2, 16, 8, 0, 4}, {2, 32, 8, 0, 8}, {2, 16, 8, 0, 2},
                                   {3, 24, 4, 1, 0}, {3, 24, 4, 2, 0}, {3, 48, 4, 2, 0}, {3, 16, 8, 2, 0},
                                   {1, 16, 1, 4, 0}, {2, 16, 8, 0, 8}, {2, 16, 8, 0, 16}, {2, 8, 8, 0, 8},
                                   {4, 16, 8, 0, 2}, {4, 16, 8, 0, 4}, {4, 16, 8, 0, 8}, {4, 32, 8, 0, 2},
                                   {4, 32, 8, 0, 4}, {4, 8, 8, 0, 4}, {5, 16, 8, 0, 0}, {5, 8, 8, 0, 0},
                                   {5, 32, 8, 0, 0}, {4, 16, 8, 1, 2}, {4, 16, 8, 1, 4}, {4, 8, 8, 1, 4},
                                   {4, 16, 8, 2, 2}, {4, 16, 8, 3, 2}, {4, 16, 8, 2, 4},  {7, 16, 4, 0, 2},
                                   {7, 16, 4, 1, 4}, {7, 16, 2, 2, 2}, {7, 32, 8, 3, 2},  {7, 32, 4, 4, 2},
                                   {7, 16, 8, 5, 2}, {4, 16, 8, 5, 2}, {4, 16, 8, 13, 2}, {4, 16, 8, 13, 4},
                                   {4, 16, 8, 5, 4}, {4, 16, 8, 69, 4}, {4, 16, 8, 101, 4}, {4, 16, 8, 37, 4},
                                   {4, 16, 8, 101, 8}, {4, 16, 8, 45, 4}, {4, 16, 8, 101, 2}};
// 3D variants (which = 2; TZ = planes per CTA, R = tile rows in y, NST = ring
// slots, G = 1 for the ring without block barriers, G = PF + 1 for the ring
// whose model and previous level arrive PF planes ahead by cp.async): kind 0
// is the z-march with a shared-memory halo plane, kind 6 the TMA plane ring.
static const Variant2D k3D[] = {{0, 32, 8, 0, 0},  {6, 32, 8, 7, 0},  {6, 64, 8, 7, 0},  {6, 32, 16, 7, 0},
                                {6, 64, 16, 7, 0}, {6, 64, 8, 10, 0}, {6, 32, 8, 10, 0}, {6, 96, 8, 10, 0},
                                {6, 64, 8, 10, 1}, {6, 64, 8, 12, 1}, {6, 96, 8, 12, 1}, {6, 64, 8, 8, 4},
                                {6, 64, 8, 7, 5},  {6, 96, 8, 8, 4},  {6, 76, 8, 10, 0},
                                {6, 76, 8, 12, 0}, {6, 76, 8, 8, 0}};
static int g_selected[3] = {-1, -1, -1};
static const int kDefaultVariant[3] = {44, 42, 16};

int variant_count(int which)
{
    switch (which) {
    case 0: return (int)(sizeof(kFwd2D) / sizeof(kFwd2D[0]));
    case 1: return (int)(sizeof(kAdj2D) / sizeof(kAdj2D[0]));
    case 2: return (int)(sizeof(k3D) / sizeof(k3D[0]));
    default: return 0;
    }
}

Variant2D variant_info(int which, int v)
{
    if (v < 0 || v >= variant_count(which)) return Variant2D{-1, 0, 0, 0, 0};
    return which == 0 ? kFwd2D[v] : (which == 1 ? kAdj2D[v] : k3D[v]);
}

int current_variant(int which)
{
    if (which < 0 || which > 2) return -1;
    return g_selected[which] >= 0 ? g_selected[which] : kDefaultVariant[which];
}

bool variant_forced(int which) { return which >= 0 && which <= 2 && g_selected[which] >= 0; }

int select_variant(int which, int v)
{
    if (which < 0 || which > 2 || v < -1 || v >= variant_count(which)) return -1;
    g_selected[which] = v;
    return 0;
}

template <int TY, int TZC, int NR>
static void launch_3d_ws(bool adjoint, const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
    constexpr size_t smem = (size_t)NR * (TY + 8) * (kTX + 8) * 4 + 128;
    static bool configured[kMaxDev] = {};
    if (first_on_device(configured)) {
        cudaFuncSetAttribute(k_step3d_ws<TY, TZC, NR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_step3d_ws<TY, TZC, NR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    const int ntz = (a.Nz + TZC - 1) / TZC;
    dim3 grid(a.ncx, (a.Ny + TY - 1) / TY, ntz * a.nshot);
    if (adjoint) k_step3d_ws<TY, TZC, NR, true><<<grid, dim3(32, TY), smem, s>>>(*maps, a);
    else k_step3d_ws<TY, TZC, NR, false><<<grid, dim3(32, TY), smem, s>>>(*maps, a);
}

template <int TY, int TZC, int NR, int PF = 0>
static void launch_3d_tma(bool adjoint, const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
    constexpr size_t smem = (size_t)NR * (TY + 8) * (kTX + 8) * 4 + (size_t)(PF > 0 ? (PF + 1) * 2 * 32 * TY * 16 : 0) +
                            128;
    static bool configured[kMaxDev] = {};
    if (first_on_device(configured)) {
        cudaFuncSetAttribute(k_step3d_tma<TY, TZC, NR, false, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cudaFuncSetAttribute(k_step3d_tma<TY, TZC, NR, true, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    }
    const int ntz = (a.Nz + TZC - 1) / TZC;
    dim3 grid(a.ncx, (a.Ny + TY - 1) / TY, ntz * a.nshot);
    if (adjoint) k_step3d_tma<TY, TZC, NR, true, PF><<<grid, dim3(32, TY), smem, s>>>(*maps, a);
    else k_step3d_tma<TY, TZC, NR, false, PF><<<grid, dim3(32, TY), smem, s>>>(*maps, a);
}

template <int TZ, int BZ, int G, bool ADJ>
static void launch_2d_group(const StepArgs& a, cudaStream_t s)
{
    constexpr size_t smem = (size_t)(2 * (TZ + 8) * (kTX + 8) + (ADJ ? TZ * kTX : 0)) * 4;
    static bool configured[kMaxDev] = {};
    if (first_on_device(configured)) {
        cudaFuncSetAttribute(k_step2d_sg<TZ, BZ, G, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    dim3 grid(a.ncx, (a.Nz + TZ - 1) / TZ, (a.nshot + G - 1) / G);
    k_step2d_sg<TZ, BZ, G, ADJ><<<grid, dim3(32, BZ), smem, s>>>(a);
}

template <int TZ, int BZ, int G, bool ADJ, int FL = 0>
static void launch_2d_group_tma(const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
    constexpr int NS = (FL & 16) ? 4 : ((FL & 8) ? 3 : 2);
    constexpr size_t smem = (size_t)(NS * ((TZ + 8) * (kTX + 8) + ((FL & 1) ? TZ * kTX : 0) +
                                           ((ADJ && (FL & 4)) ? TZ * kTX : 0)) +
                                     (ADJ ? TZ * kTX : 0) + ((FL & 2) ? 2 * TZ * kTX : 0)) * 4 + 128;
    static bool configured[kMaxDev] = {};
    if (first_on_device(configured)) {
        cudaFuncSetAttribute(k_step2d_sgt<TZ, BZ, G, FL, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    // launched with programmatic stream serialization: consecutive steps overlap the
    // launch and set-up of one with the last CTAs of the other (see the kernel)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = (FL & 32) ? dim3(a.ncx, (a.nshot + G - 1) / G, (a.Nz + TZ - 1) / TZ)
                            : dim3(a.ncx, (a.Nz + TZ - 1) / TZ, (a.nshot + G - 1) / G);
    cfg.blockDim = dim3(32, BZ);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_step2d_sgt<TZ, BZ, G, FL, ADJ>, *maps, a);
    if (e != cudaSuccess) note_cuda_error(e);  // the caller's cudaGetLastError check reports it
}

template <int TZ, int BZ, bool ADJ>
static size_t pst_smem()
{
    return (size_t)(2 * ((TZ + 8) * (kTX + 8) + TZ * kTX) + (ADJ ? TZ * kTX : 0)) * 4 + 128;
}

// CTAs of the persistent 2D kernel on the current device: as many as are
// resident at once, at most one per item.
template <int TZ, int BZ, bool ADJ>
static int pst_ctas(long long items)
{
    static int per_sm[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (per_sm[dev] == 0) {
        const size_t smem = pst_smem<TZ, BZ, ADJ>();
        cudaFuncSetAttribute(k_step2d_pst<TZ, BZ, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 0, nsm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step2d_pst<TZ, BZ, ADJ>, 32 * BZ, smem);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        per_sm[dev] = max(1, occ) * max(1, nsm);
    }
    return (int)std::min<long long>(items, per_sm[dev]);
}

template <int TZ, int BZ, bool ADJ>
static void launch_2d_persistent(const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
    const long long W = (long long)((a.Nz + TZ - 1) / TZ) * a.ncx * a.nshot;
    const int C = pst_ctas<TZ, BZ, ADJ>(W);
    k_step2d_pst<TZ, BZ, ADJ><<<C, dim3(32, BZ), pst_smem<TZ, BZ, ADJ>(), s>>>(*maps, a);
}

// Gradient accumulator slots the persistent adjoint variant v fills: for each
// tile, the number of CTAs whose item ranges cover its shots.
int persistent_slots(int v, int ncx, int ntz, int nshot)
{
    const long long W = (long long)ncx * ntz * nshot;
    int C = 0;
    switch (v) {
    case 22: C = pst_ctas<16, 8, true>(W); break;
    case 23: C = pst_ctas<8, 8, true>(W); break;
    case 24: C = pst_ctas<32, 8, true>(W); break;
    default: return nshot;
    }
    int n = 1;
    for (long long t = 0; t < (long long)ncx * ntz; ++t)
        n = std::max(n, pst_owner((t + 1) * nshot - 1, C, W) - pst_owner(t * nshot, C, W) + 1);
    return n;
}

template <int TZ, int NW, int D, bool ADJ>
static void launch_2d_march(const StepArgs& a, cudaStream_t s)
{
    dim3 grid(a.ncx, (a.Nz + TZ * NW - 1) / (TZ * NW), a.nshot);
    k_step2d_zm<TZ, NW, D, ADJ><<<grid, 32 * NW, 0, s>>>(a);
}

template <int TZ, int BZ, bool ADJ>
static void launch_2d_direct(const StepArgs& a, cudaStream_t s)
{
    dim3 grid(a.ncx, (a.Nz + TZ - 1) / TZ, a.nshot);
    k_step2d<TZ, BZ, ADJ><<<grid, dim3(32, BZ), 0, s>>>(a);
}

static void launch_step_raw(const Tiling& t, int ndim, bool adjoint, const StepArgs& a, const StepMaps* maps,
                            cudaStream_t s)
{
    if (ndim == 2) {
        const Variant2D vi = variant_info(adjoint ? 1 : 0, adjoint ? t.va : t.vf);
        if (vi.kind == 7) {  // z window in registers (step2d_zw.cu); NST holds its configuration index
            launch_step2d_zw(vi.NST, adjoint, a, maps, s);
            return;
        }
        if (!adjoint) {
            switch (t.vf) {
            case 1: launch_2d<48, 6, 2, false>(a, maps, s); break;
            case 2: launch_2d<32, 4, 3, false>(a, maps, s); break;
            case 3: launch_2d<24, 3, 4, false>(a, maps, s); break;
            case 4: launch_2d<16, 2, 4, false>(a, maps, s); break;
            case 5: launch_2d<32, 2, 3, false>(a, maps, s); break;
            case 6: launch_2d_group<32, 8, 4, false>(a, s); break;
            case 7: launch_2d_group<16, 8, 4, false>(a, s); break;
            case 8: launch_2d_group<32, 8, 8, false>(a, s); break;
            case 9: launch_2d_group<16, 8, 2, false>(a, s); break;
            case 10: launch_2d_march<24, 4, 1, false>(a, s); break;
            case 11: launch_2d_march<24, 4, 2, false>(a, s); break;
            case 12: launch_2d_march<48, 4, 2, false>(a, s); break;
            case 13: launch_2d_march<16, 8, 2, false>(a, s); break;
            case 14: launch_2d<32, 1, 3, false>(a, maps, s); break;
            case 15: launch_2d_group<16, 8, 8, false>(a, s); break;
            case 16: launch_2d_group<16, 8, 16, false>(a, s); break;
            case 17: launch_2d_group<8, 8, 8, false>(a, s); break;
            case 18: launch_2d_group_tma<16, 8, 2, false>(a, maps, s); break;
            case 19: launch_2d_group_tma<16, 8, 4, false>(a, maps, s); break;
            case 20: launch_2d_group_tma<16, 8, 8, false>(a, maps, s); break;
            case 21: launch_2d_group_tma<32, 8, 2, false>(a, maps, s); break;
            case 22: launch_2d_group_tma<32, 8, 4, false>(a, maps, s); break;
            case 23: launch_2d_group_tma<8, 8, 4, false>(a, maps, s); break;
            case 24: launch_2d_persistent<16, 8, false>(a, maps, s); break;
            case 25: launch_2d_persistent<8, 8, false>(a, maps, s); break;
            case 26: launch_2d_persistent<32, 8, false>(a, maps, s); break;
            case 27: launch_2d_group_tma<16, 8, 2, false, 1>(a, maps, s); break;
            case 28: launch_2d_group_tma<16, 8, 4, false, 1>(a, maps, s); break;
            case 29: launch_2d_group_tma<8, 8, 4, false, 1>(a, maps, s); break;
            case 30: launch_2d_group_tma<16, 8, 2, false, 2>(a, maps, s); break;
            case 31: launch_2d_group_tma<16, 8, 2, false, 3>(a, maps, s); break;
            case 32: launch_2d_group_tma<16, 8, 4, false, 2>(a, maps, s); break;
            case 39: launch_2d_group_tma<16, 8, 2, false, 9>(a, maps, s); break;
            case 40: launch_2d_group_tma<16, 8, 4, false, 9>(a, maps, s); break;
            case 41: launch_2d_group_tma<16, 8, 4, false, 17>(a, maps, s); break;
            case 42: launch_2d_group_tma<16, 8, 8, false, 9>(a, maps, s); break;
            case 43: launch_2d_group_tma<16, 8, 8, false, 17>(a, maps, s); break;
            case 44: launch_2d_group_tma<16, 8, 4, false, 9 | 32>(a, maps, s); break;
            case 45: launch_2d_group_tma<16, 8, 2, false, 1 | 32>(a, maps, s); break;
            case 46: launch_2d_group_tma<16, 8, 8, false, 9 | 32>(a, maps, s); break;
            case 47: launch_2d_group_tma<16, 8, 4, false, 17 | 32>(a, maps, s); break;
            default: launch_2d_direct<32, 8, false>(a, s); break;
            }
        } else {
            switch (t.va) {
            case 1: launch_2d<24, 3, 3, true>(a, maps, s); break;
            case 2: launch_2d<16, 2, 4, true>(a, maps, s); break;
            case 3: launch_2d<32, 4, 2, true>(a, maps, s); break;
            case 4: launch_2d_group<32, 8, 4, true>(a, s); break;
            case 5: launch_2d_group<16, 8, 4, true>(a, s); break;
            case 6: launch_2d_group<32, 8, 8, true>(a, s); break;
            case 7: launch_2d_group<16, 8, 2, true>(a, s); break;
            case 8: launch_2d_march<24, 4, 1, true>(a, s); break;
            case 9: launch_2d_march<24, 4, 2, true>(a, s); break;
            case 10: launch_2d_march<48, 4, 2, true>(a, s); break;
            case 11: launch_2d_march<16, 8, 2, true>(a, s); break;
            case 12: launch_2d<16, 1, 4, true>(a, maps, s); break;
            case 13: launch_2d_group<16, 8, 8, true>(a, s); break;
            case 14: launch_2d_group<16, 8, 16, true>(a, s); break;
            case 15: launch_2d_group<8, 8, 8, true>(a, s); break;
            case 16: launch_2d_group_tma<16, 8, 2, true>(a, maps, s); break;
            case 17: launch_2d_group_tma<16, 8, 4, true>(a, maps, s); break;
            case 18: launch_2d_group_tma<16, 8, 8, true>(a, maps, s); break;
            case 19: launch_2d_group_tma<32, 8, 2, true>(a, maps, s); break;
            case 20: launch_2d_group_tma<32, 8, 4, true>(a, maps, s); break;
            case 21: launch_2d_group_tma<8, 8, 4, true>(a, maps, s); break;
            case 22: launch_2d_persistent<16, 8, true>(a, maps, s); break;
            case 23: launch_2d_persistent<8, 8, true>(a, maps, s); break;
            case 24: launch_2d_persistent<32, 8, true>(a, maps, s); break;
            case 25: launch_2d_group_tma<16, 8, 2, true, 1>(a, maps, s); break;
            case 26: launch_2d_group_tma<16, 8, 4, true, 1>(a, maps, s); break;
            case 27: launch_2d_group_tma<8, 8, 4, true, 1>(a, maps, s); break;
            case 28: launch_2d_group_tma<16, 8, 2, true, 2>(a, maps, s); break;
            case 29: launch_2d_group_tma<16, 8, 2, true, 3>(a, maps, s); break;
            case 30: launch_2d_group_tma<16, 8, 4, true, 2>(a, maps, s); break;
            case 37: launch_2d_group_tma<16, 8, 2, true, 5>(a, maps, s); break;
            case 38: launch_2d_group_tma<16, 8, 2, true, 13>(a, maps, s); break;
            case 39: launch_2d_group_tma<16, 8, 4, true, 13>(a, maps, s); break;
            case 40: launch_2d_group_tma<16, 8, 4, true, 5>(a, maps, s); break;
            case 41: launch_2d_group_tma<16, 8, 4, true, 5 | 64>(a, maps, s); break;
            case 42: launch_2d_group_tma<16, 8, 4, true, 5 | 32 | 64>(a, maps, s); break;
            case 43: launch_2d_group_tma<16, 8, 4, true, 5 | 32>(a, maps, s); break;
            case 44: launch_2d_group_tma<16, 8, 8, true, 5 | 32 | 64>(a, maps, s); break;
            case 45: launch_2d_group_tma<16, 8, 4, true, 13 | 32>(a, maps, s); break;
            case 46: launch_2d_group_tma<16, 8, 2, true, 5 | 32 | 64>(a, maps, s); break;
            default: launch_2d_direct<32, 8, true>(a, s); break;
            }
        }
    } else {
        switch (a.dmv ? 0 : t.v3) {  // the Born source is carried by the z-march kernel only
        case 1: launch_3d_tma<8, 32, 7>(adjoint, a, maps, s); break;
        case 2: launch_3d_tma<8, 64, 7>(adjoint, a, maps, s); break;
        case 3: launch_3d_tma<16, 32, 7>(adjoint, a, maps, s); break;
        case 4: launch_3d_tma<16, 64, 7>(adjoint, a, maps, s); break;
        case 5: launch_3d_tma<8, 64, 10>(adjoint, a, maps, s); break;
        case 6: launch_3d_tma<8, 32, 10>(adjoint, a, maps, s); break;
        case 7: launch_3d_tma<8, 96, 10>(adjoint, a, maps, s); break;
        case 8: launch_3d_ws<8, 64, 10>(adjoint, a, maps, s); break;
        case 9: launch_3d_ws<8, 64, 12>(adjoint, a, maps, s); break;
        case 10: launch_3d_ws<8, 96, 12>(adjoint, a, maps, s); break;
        case 11: launch_3d_tma<8, 64, 8, 3>(adjoint, a, maps, s); break;
        case 12: launch_3d_tma<8, 64, 7, 4>(adjoint, a, maps, s); break;
        case 13: launch_3d_tma<8, 96, 8, 3>(adjoint, a, maps, s); break;
        case 14: launch_3d_tma<8, 76, 10>(adjoint, a, maps, s); break;
        case 15: launch_3d_tma<8, 76, 12>(adjoint, a, maps, s); break;
        case 16: launch_3d_tma<8, 76, 8>(adjoint, a, maps, s); break;
        default: {
            const int ntz = (a.Nz + 31) / 32;
            dim3 grid(t.ncx, t.ncy, ntz * a.nshot);
            dim3 block(32, 8);
            if (adjoint) k_step3d<8, 32, true><<<grid, block, 0, s>>>(a);
            else k_step3d<8, 32, false><<<grid, block, 0, s>>>(a);
        }
        }
    }
}

void launch_step(const Tiling& t, int ndim, bool adjoint, const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
    count_step_launch();
    cudaEvent_t stop;
    const bool timed = profile_sample(adjoint, s, &stop);
    launch_step_raw(t, ndim, adjoint, a, maps, s);
    if (timed) profile_close(stop, s);
}

// ---------------------------------------------------------------------------
// kap = (v dt / h)^2 on the padded grid, copied outward from the nearest
// physical cell; pitch columns get 0.  Flags non-finite or non-positive
// velocities and records the maximum velocity.
__global__ void k_prep(Dims d, const float* __restrict__ vel, float* __restrict__ kap, float* vmax, int* err)
{
    const long long n = d.cell;
    const float c = d.dt / d.h;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % d.P);
        const long long r = i / d.P;
        const int y = (int)(r % d.Ny);
        const int z = (int)(r / d.Ny);
        if (x >= d.Nx) {
            kap[i] = 0.0f;
            continue;
        }
        const int jx = min(max(x - d.nb, 0), d.nx - 1);
        const int jz = min(max(z - d.nb, 0), d.nz - 1);
        const int jy = d.ndim == 3 ? min(max(y - d.nb, 0), d.ny - 1) : 0;
        const long long j = ((long long)jz * (d.ndim == 3 ? d.ny : 1) + jy) * d.nx + jx;
        const float v = vel[j];
        if (!(v > 0.0f) || !isfinite(v)) {
            atomicOr(err, kErrNonFinite);
            kap[i] = 0.0f;
            continue;
        }
        const float cv = v * c;
        kap[i] = cv * cv;
        atomicMax(reinterpret_cast<int*>(vmax), __float_as_int(v));
    }
}

void launch_prep(const Dims& d, const float* vel, float* kap, float* vmax, int* err, cudaStream_t s)
{
    long long blocks = (d.cell + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    count_launch();
    k_prep<<<(int)blocks, 256, 0, s>>>(d, vel, kap, vmax, err);
}

// The stability check on the device, so that a call need not wait for the
// model's maximum velocity on the host: compares in double, as the host did.
__global__ void k_check_cfl(const float* vmax, double dt_over_h, double limit, int* err)
{
    if (threadIdx.x == 0 && dt_over_h * (double)*vmax > limit) atomicOr(err, kErrCfl);
}

void launch_check_cfl(const float* vmax, double dt_over_h, double limit, int* err, cudaStream_t s)
{
    count_launch();
    k_check_cfl<<<1, 32, 0, s>>>(vmax, dt_over_h, limit, err);
}

// fac = w * scale * kap / (1 + eps) at each tap's grid point: the amount that
// a unit amplitude adds to the updated field.
__global__ void k_tapfac(Dims d, int ntap, const int* __restrict__ idx, const float* __restrict__ w,
                         float* __restrict__ fac, const float* __restrict__ kap, float scale, float ceps)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ntap) return;
    const int i = idx[j];
    const int x = i % d.P;
    const int r = i / d.P;
    const int y = r % d.Ny;
    const int z = r / d.Ny;
    int dd = max(sponge_depth(x, d.nb, d.nx), sponge_depth(z, d.nb, d.nz));
    if (d.ndim == 3) dd = max(dd, sponge_depth(y, d.nb, d.ny));
    const float k = kap[i];
    const float eps = k * ceps * (float)(dd * dd);
    fac[j] = w[j] * scale * k * rcp_sponge(1.0f + eps);
}

void launch_tapfac(const Dims& d, const TapList& l, const float* kap, float scale_inj, float ceps, cudaStream_t s)
{
    if (l.ntap == 0) return;
    count_launch();
    k_tapfac<<<(l.ntap + 255) / 256, 256, 0, s>>>(d, l.ntap, l.idx, l.w, const_cast<float*>(l.fac), kap, scale_inj,
                                                   ceps);
}

// out[s][n][p] = sum of the point's gather slots at time row n.
__global__ void k_finalize(const int* __restrict__ pt_start, const float* __restrict__ slots, int npts_all, int npts,
                           int nt, int ntap, float* __restrict__ out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long total = (long long)nt * npts_all;
    if (i >= total) return;
    const int pt = (int)(i % npts_all);
    const int n = (int)(i / npts_all);
    const float* row = slots + (long long)n * ntap;
    float acc = 0.0f;
    for (int t = pt_start[pt]; t < pt_start[pt + 1]; ++t) acc += row[t];
    const int shot = pt / npts, p = pt - shot * npts;
    out[((long long)shot * nt + n) * npts + p] = acc;
}

void launch_finalize(const TapList& l, const float* slots, int nshot, int nt, float* out, cudaStream_t s)
{
    const int npts_all = nshot * l.npts;
    const long long total = (long long)nt * npts_all;
    if (total == 0) return;
    count_launch();
    k_finalize<<<(int)((total + 255) / 256), 256, 0, s>>>(l.pt_start, slots, npts_all, l.npts, nt, l.ntap, out);
}

// Misfit 1/2 sum (a - b)^2 in double, in a fixed reduction order.
__global__ void k_sq_partial(const float* __restrict__ a, const float* __restrict__ b, long long n, double* part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const double r = (double)a[i] - (double)b[i];
        acc += r * r;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_partial(const double* part, int npart, double* out)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < npart; i += 256) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0.5 * sh[0];
}

void launch_misfit(const float* a, const float* b, long long n, double* partial, int npart, double* out,
                   cudaStream_t s)
{
    count_launch(2);
    k_sq_partial<<<npart, 256, 0, s>>>(a, b, n, partial);
    k_sum_partial<<<1, 256, 0, s>>>(partial, npart, out);
}

// Gradient on the physical grid: sum over shots, then the adjoint of the
// edge-replicating extension one axis at a time (each physical edge cell
// collects the sponge cells that were copied from it).
__global__ void k_shot_sum(const float* __restrict__ gacc, long long cell, int nshot, float* __restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cell; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int s = 0; s < nshot; ++s) acc += gacc[(long long)s * cell + i];
        out[i] = acc;
    }
}

// in [rows][P] (padded x) -> out [rows][nx]
__global__ void k_collapse_x(const float* __restrict__ in, long long rows, int P, int nx, int nb, int Nx,
                             float* __restrict__ out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows * nx) return;
    const int jx = (int)(i % nx);
    const long long r = i / nx;
    const int lo = jx == 0 ? 0 : jx + nb, hi = jx == nx - 1 ? Nx - 1 : jx + nb;
    float acc = 0.0f;
    for (int x = lo; x <= hi; ++x) acc += in[r * P + x];
    out[i] = acc;
}

// in [outer][N][M] (padded middle axis) -> out [outer][n][M]
__global__ void k_collapse_mid(const float* __restrict__ in, long long outer, int N, int n, int nb, long long M,
                               float* __restrict__ out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= outer * n * M) return;
    const long long m = i % M;
    const long long r = i / M;
    const int j = (int)(r % n);
    const long long o = r / n;
    const int lo = j == 0 ? 0 : j + nb, hi = j == n - 1 ? N - 1 : j + nb;
    float acc = 0.0f;
    for (int k = lo; k <= hi; ++k) acc += in[(o * N + k) * M + m];
    out[i] = acc;
}

// grad *= -2 / v^3: the gradient with respect to velocity from the one with
// respect to squared slowness (m = 1/v^2).
__global__ void k_chain_velocity(const float* __restrict__ vel, long long n, float* __restrict__ grad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = vel[i];
        grad[i] *= -2.0f / (v * v * v);
    }
}

void launch_grad_reduce(const Dims& d, const float* gacc, int nshot, float* tmp, float* grad, const float* vel_chain,
                        cudaStream_t s)
{
    // tmp holds 2 * cell floats: [0, cell) the shot sum, [cell, 2 cell) the x-collapsed sum.
    float* t0 = tmp;
    float* t1 = tmp + d.cell;
    const int bs = 256;
    count_launch(d.ndim == 3 ? 4 : 3);
    k_shot_sum<<<152 * 8, bs, 0, s>>>(gacc, d.cell, nshot, t0);
    const long long rows = (long long)d.Nz * d.Ny;
    k_collapse_x<<<(int)((rows * d.nx + bs - 1) / bs), bs, 0, s>>>(t0, rows, d.P, d.nx, d.nb, d.Nx, t1);
    if (d.ndim == 3) {
        const long long n1 = (long long)d.Nz * d.ny * d.nx;
        k_collapse_mid<<<(int)((n1 + bs - 1) / bs), bs, 0, s>>>(t1, d.Nz, d.Ny, d.ny, d.nb, d.nx, t0);
        k_collapse_mid<<<(int)((d.phys + bs - 1) / bs), bs, 0, s>>>(t0, 1, d.Nz, d.nz, d.nb,
                                                                     (long long)d.ny * d.nx, grad);
    } else {
        k_collapse_mid<<<(int)((d.phys + bs - 1) / bs), bs, 0, s>>>(t1, 1, d.Nz, d.nz, d.nb, d.nx, grad);
    }
    if (vel_chain) {
        count_launch();
        k_chain_velocity<<<(int)std::min<long long>((d.phys + bs - 1) / bs, 152 * 8), bs, 0, s>>>(vel_chain, d.phys,
                                                                                                grad);
    }
}

// dmv = Extend(dm) * v^2 on the padded grid (v^2 = kap h^2 / dt^2); pitch columns 0.
__global__ void k_prep_dm(Dims d, const float* __restrict__ dm, const float* __restrict__ kap, float* __restrict__ dmv)
{
    const float s = (d.h / d.dt) * (d.h / d.dt);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.cell; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % d.P);
        const long long r = i / d.P;
        const int y = (int)(r % d.Ny);
        const int z = (int)(r / d.Ny);
        if (x >= d.Nx) {
            dmv[i] = 0.0f;
            continue;
        }
        const int jx = min(max(x - d.nb, 0), d.nx - 1);
        const int jz = min(max(z - d.nb, 0), d.nz - 1);
        const int jy = d.ndim == 3 ? min(max(y - d.nb, 0), d.ny - 1) : 0;
        const long long j = ((long long)jz * (d.ndim == 3 ? d.ny : 1) + jy) * d.nx + jx;
        dmv[i] = dm[j] * kap[i] * s;
    }
}

void launch_prep_dm(const Dims& d, const float* dm, const float* kap, float* dmv, cudaStream_t s)
{
    long long blocks = (d.cell + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    count_launch();
    k_prep_dm<<<(int)blocks, 256, 0, s>>>(d, dm, kap, dmv);
}

__global__ void k_ricker(double f0, double dt, int nt, float* out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nt) return;
    const double t0 = 1.0 / f0;
    double a = 3.14159265358979323846 * f0 * (n * dt - t0);
    a *= a;
    out[n] = (float)((1.0 - 2.0 * a) * exp(-a));
}

void launch_ricker(float f0, float dt, int nt, float* out, cudaStream_t s)
{
    count_launch();
    k_ricker<<<(nt + 255) / 256, 256, 0, s>>>((double)f0, (double)dt, nt, out);
}

__global__ void k_nan_scan(const float* __restrict__ a, long long n, int* err)
{
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(a[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNonFinite);
}

void launch_nan_scan(const float* a, long long n, int* err, cudaStream_t s)
{
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    count_launch();
    k_nan_scan<<<(int)blocks, 256, 0, s>>>(a, n, err);
}

}  // namespace wave
