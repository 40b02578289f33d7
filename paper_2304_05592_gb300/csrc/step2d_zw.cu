// step2d_zw.cu -- 2D time step, shot groups fed by TMA with the z window in
// registers.
//
// Same work split as the shot-group TMA kernel (one CTA runs a 128 x TZ tile
// for G shots; each shot's halo tile of the current level and its tile of the
// previous level arrive by TMA into a two-stage ring, the next shot's copies
// issued while this one is computed), but each thread owns RB = TZ/BZ
// *consecutive* rows of 4 points and walks down them with the 9 rows of its
// z stencil held in registers: per row it reads one new row of its window and
// the two x neighbours from shared memory (3 + 1 loads of 16 bytes per 4
// points instead of 11 + 1).  The model is read once per CTA; tiles that touch
// the sponge recompute its factors per shot from indices, interior tiles skip
// them.  In the adjoint the forward level u^k also arrives by TMA and the
// imaging term is summed over the group in a shared-memory gradient tile.
// Arithmetic order per point is that of every other 2D step kernel
// (stencil.cuh), so shot records are the same bits.
#include <math.h>

#include "internal.h"
#include "stencil.cuh"
#include "step_common.cuh"
#include "tma.cuh"

namespace wave {
namespace {

template <int TZ, bool ADJ>
struct ZwLayout {
    static constexpr int SW = kTX + 8;
    static constexpr int H = (TZ + 8) * SW;      // halo tile of the current level
    static constexpr int U = TZ * kTX;           // previous level
    static constexpr int F = ADJ ? TZ * kTX : 0; // forward level u^k (FP32, or BF16 in its first half)
    static constexpr int stage = H + U + F;
    static_assert(H % 32 == 0 && U % 32 == 0, "sub-buffers stay 128-byte aligned");
};

template <int TZ, int BZ, int G, bool ADJ>
__global__ void __launch_bounds__(32 * BZ, 16 / BZ) k_step2d_zw(const __grid_constant__ StepMaps mp, const StepArgs a)
{
    using L = ZwLayout<TZ, ADJ>;
    constexpr int SW = L::SW;
    constexpr int RB = TZ / BZ;
    static_assert(TZ % BZ == 0, "rows split evenly over the thread rows");
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar[2];
    float* st = reinterpret_cast<float*>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));
    float* sg = st + 2 * L::stage;  // [TZ][kTX] gradient tile of the group (adjoint with imaging)
    const CUtensorMap* mh = ADJ ? &mp.halo_a : &mp.halo_f;
    const CUtensorMap* mt = ADJ ? &mp.tile_a : &mp.tile_f;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * kTX, z0 = blockIdx.y * TZ;
    const int grp = blockIdx.z, s0 = grp * G, ns = min(G, a.nshot - s0);
    const int lx = 4 * tx, gx = x0 + lx;
    const int nvalid = min(4, a.Nx - gx);
    const int r0 = ty * RB;
    const bool imaging = ADJ && a.gacc != nullptr;
    const bool uf_tma = imaging && (a.uf16 ? a.uf16_row >= 0 : a.uf_buf >= 0);
    const bool sparse = a.inj.cell_start != nullptr || a.gat.cell_start != nullptr;
    const uint32_t kBytes =
        (uint32_t)(L::H + L::U) * 4u + (uf_tma ? (uint32_t)(TZ * kTX) * (a.uf16 ? 2u : 4u) : 0u);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // programmatic dependent launch, as in the other shot-group kernels: only
    // the model (never written by a step) is read before griddepcontrol.wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    auto issue = [&](int i) {
        float* sb = st + (i & 1) * L::stage;
        const int shot = s0 + i;
        mbar_expect_tx(&bar[i & 1], kBytes);
        tma_load_4d(sb, mh, &bar[i & 1], x0 - 4, z0 - 4, shot, a.u_buf);
        tma_load_4d(sb + L::H, mt, &bar[i & 1], x0, z0, shot, a.prev_buf);
        if (uf_tma) {
            if (a.uf16) tma_load_4d(sb + L::H + L::U, &mp.tile16_a, &bar[i & 1], x0, z0, shot, a.uf16_row);
            else tma_load_4d(sb + L::H + L::U, &mp.tile_a, &bar[i & 1], x0, z0, shot, a.uf_buf);
        }
    };
    // per CTA: the model of the thread's rows, the sponge depth of its columns
    const bool sponge_tile = a.ceps != 0.0f && (x0 < a.nb || x0 + kTX > a.nb + a.nx || z0 < a.nb ||
                                                z0 + TZ > a.nb + a.nz);
    float4 kp[RB];
    int dxe[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) dxe[e] = sponge_depth(gx + e, a.nb, a.nx);
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        const int gz = z0 + r0 + rr;
        kp[rr] = (gz < a.Nz && nvalid > 0) ? ld4(a.kap + gz * a.P + gx) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0) issue(0);
    float* gq = imaging ? a.gacc + (size_t)grp * a.cell : nullptr;
    if (imaging) {
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int gz = z0 + r0 + rr;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gz < a.Nz && nvalid > 0) v = *reinterpret_cast<const float4*>(gq + gz * a.P + gx);
            *reinterpret_cast<float4*>(sg + (r0 + rr) * kTX + lx) = v;
        }
    }

    // A thread whose wait for a stage gives up records the timeout and does no
    // further work but passes every block barrier below (they are uniform);
    // thread 0 first waits (bounded) for the copies it has in flight.
    bool alive = true;
    for (int i = 0; i < ns; ++i) {
        const int shot = s0 + i, stage = i & 1;
        if (tid == 0 && alive && i + 1 < ns) {
            fence_proxy_async();
            issue(i + 1);
        }
        if (alive && !mbar_wait(&bar[stage], (uint32_t)(i >> 1) & 1u)) {
            alive = false;
            atomicOr(a.err, kErrTimeout);
            if (tid == 0) {
                mbar_wait(&bar[stage], (uint32_t)(i >> 1) & 1u);
                if (i + 1 < ns) mbar_wait(&bar[stage ^ 1], (uint32_t)((i + 1) >> 1) & 1u);
            }
        }
        const size_t so = (size_t)shot * a.cell;
        if (alive) {
            const float* H = st + stage * L::stage;
            const float* U = H + L::H;
            const float* F = U + L::U;
            float4 zw[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) zw[j] = lds4(H + (r0 + j) * SW + lx + 4);
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
                const int r = r0 + rr, gz = z0 + r;
                const float* row = H + (r + 4) * SW + lx;
                const float4 A = lds4(row), C = lds4(row + 8);
                const float4 B = zw[4];
                const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
                float lap[4];
                lap4(w, [&](int k, float4& Up, float4& Dn) {
                    Up = zw[4 - k];
                    Dn = zw[4 + k];
                }, lap);
                const float4 uo = lds4(U + r * kTX + lx);
                const float cen[4] = {B.x, B.y, B.z, B.w};
                const float um[4] = {uo.x, uo.y, uo.z, uo.w};
                const float kv[4] = {kp[rr].x, kp[rr].y, kp[rr].z, kp[rr].w};
                float out[4];
                if (sponge_tile) {
                    const int dz = sponge_depth(gz, a.nb, a.nz);
                    float ev[4], iv[4];
                    const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int dd = max(dxe[e], dz);
                        ev[e] = kv[e] * a.ceps * (float)(dd * dd);
                        iv[e] = rcp_sponge(1.0f + ev[e]);
                    }
                    update4(cen, um, lap, kv, ev, iv, zero4, out);
                } else {
                    update4_interior(cen, um, lap, kv, out);
                }
                float uf[4] = {0.f, 0.f, 0.f, 0.f};
                if (imaging) {
                    if (uf_tma && a.uf16) {
                        unpack_bf16x4(*reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(F) +
                                                                      r * kTX + lx),
                                      uf);
                    } else if (uf_tma) {
                        const float4 v = lds4(F + r * kTX + lx);
                        uf[0] = v.x;
                        uf[1] = v.y;
                        uf[2] = v.z;
                        uf[3] = v.w;
                    } else if (gz < a.Nz && nvalid > 0) {
                        const int off = gz * a.P + gx;
                        if (a.uf16) {
                            unpack_bf16x4(*reinterpret_cast<const uint2*>(a.uf16 + so + off), uf);
                        } else {
                            const float4 v = ld4(a.uf32 + so + off);
                            uf[0] = v.x;
                            uf[1] = v.y;
                            uf[2] = v.z;
                            uf[3] = v.w;
                        }
                    }
                }
                if (rr + 1 < RB) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) zw[j] = zw[j + 1];
                    zw[8] = lds4(H + (r + 9) * SW + lx + 4);
                }
                if (gz >= a.Nz) continue;
                const int off = gz * a.P + gx;
                float* un = a.unew + so + off;
                if (nvalid <= 0) {
                    if (gx < a.P) *reinterpret_cast<float4*>(un) = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                // a full float4: points past Nx stay the zero exterior
                *reinterpret_cast<float4*>(un) = make_float4(out[0], nvalid > 1 ? out[1] : 0.0f,
                                                             nvalid > 2 ? out[2] : 0.0f, nvalid > 3 ? out[3] : 0.0f);
                if (!ADJ) {
                    if (a.st16) {
                        if (nvalid == 4) {
                            store_bf16x4(a.st16 + so + off, out);
                        } else {
                            for (int e = 0; e < nvalid; ++e) a.st16[so + off + e] = __float2bfloat16_rn(out[e]);
                        }
                    }
                    if (a.st32) {
                        if (nvalid == 4) {
                            *reinterpret_cast<float4*>(a.st32 + so + off) = make_float4(out[0], out[1], out[2], out[3]);
                        } else {
                            for (int e = 0; e < nvalid; ++e) a.st32[so + off + e] = out[e];
                        }
                    }
                } else if (imaging) {
                    float* g = sg + r * kTX + lx;
#pragma unroll
                    for (int e = 0; e < 4; ++e) g[e] -= uf[e] * (out[e] - 2.0f * cen[e] + um[e]);
                }
            }
        }
        // this CTA's taps for the shot (the same values in every thread: uniform decisions)
        int ib = 0, ie = 0, gb = 0, ge = 0;
        if (sparse) {
            const int kcell = TZ / a.TZc;
            const int cbase = (shot * a.ncx + (int)blockIdx.x) * a.ncz;
            const int c0 = (int)blockIdx.y * kcell, c1 = min(c0 + kcell, a.ncz);
            if (a.inj.cell_start) {
                ib = a.inj.cell_start[cbase + c0];
                ie = a.inj.cell_start[cbase + c1];
            }
            if (a.gat.cell_start) {
                gb = a.gat.cell_start[cbase + c0];
                ge = a.gat.cell_start[cbase + c1];
            }
        }
        const bool taps = ie > ib || ge > gb;
        // the stage is refilled by shot i + 2's copies, and taps touch other threads' points
        if (taps || i + 2 < ns) __syncthreads();
        if (taps) sparse_phase<ADJ>(a, ib, ie, gb, ge, (long long)so, tid, 32 * BZ, imaging ? sg : nullptr, z0, x0);
        if (taps && imaging) __syncthreads();  // injection terms land in the gradient tile before the next shot
    }
    if (imaging) {
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int gz = z0 + r0 + rr;
            if (gz < a.Nz && nvalid > 0)
                *reinterpret_cast<float4*>(gq + gz * a.P + gx) =
                    *reinterpret_cast<const float4*>(sg + (r0 + rr) * kTX + lx);
        }
    }
}

template <int TZ, int BZ, int G, bool ADJ>
void launch_zw(const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
    constexpr size_t smem = (size_t)(2 * ZwLayout<TZ, ADJ>::stage + (ADJ ? TZ * kTX : 0)) * 4 + 128;
    static bool configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        dev = 0;
        configured[0] = false;
    }
    if (!configured[dev]) {
        cudaFuncSetAttribute(k_step2d_zw<TZ, BZ, G, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured[dev] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.ncx, (a.Nz + TZ - 1) / TZ, (a.nshot + G - 1) / G);
    cfg.blockDim = dim3(32, BZ);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_step2d_zw<TZ, BZ, G, ADJ>, *maps, a);
    if (e != cudaSuccess) note_cuda_error(e);  // the caller's cudaGetLastError check reports it
}

}  // namespace

// Configurations (TZ, BZ, G) of the z-window kernel, by index.
void launch_step2d_zw(int config, bool adjoint, const StepArgs& a, const StepMaps* maps, cudaStream_t s)
{
#define ZW(i, tz, bz, g)                                                                           \
    case i:                                                                                        \
        if (adjoint) launch_zw<tz, bz, g, true>(a, maps, s);                                       \
        else launch_zw<tz, bz, g, false>(a, maps, s);                                              \
        return;
    switch (config) {
        ZW(0, 16, 4, 2)
        ZW(1, 16, 4, 4)
        ZW(2, 16, 2, 2)
        ZW(3, 32, 8, 2)
        ZW(4, 32, 4, 2)
        ZW(5, 16, 8, 2)
    default: return;
    }
#undef ZW
}

}  // namespace wave
