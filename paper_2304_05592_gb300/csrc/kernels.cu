// kernels.cu -- the stencil time step (2D and 3D, forward and adjoint) and the
// small kernels around it (model preparation, tap factors, gathers, misfit,
// shot reduction of the gradient, Ricker wavelet).
//
// Every kernel here is HBM/L2-bandwidth bound: FP32 arithmetic on CUDA cores,
// 128-bit loads and stores, halo tiles in shared memory.  Tensor cores play no
// part (the stencil is not a dense contraction).
#include <math.h>

#include "internal.h"

namespace wave {

__device__ __forceinline__ int sponge_depth(int i, int nb, int n)
{
    int d = max(nb - i, i - (nb + n - 1));
    return max(d, 0);
}

// One leapfrog update in Courant units:
//   (1+eps) u+ = 2u - (1-eps) u- + kap * lap,  kap = (v dt/h)^2, eps = eta dt v^2 / 2.
__device__ __forceinline__ float leap(float c, float um, float lap, float kap, float eps)
{
    float num = fmaf(kap, lap, fmaf(eps, um, 2.0f * c - um));
    return num * __frcp_rn(1.0f + eps);
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float f4(const float4& v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

__device__ __forceinline__ void store_bf16x4(__nv_bfloat16* p, const float* o)
{
    __nv_bfloat162 lo = __floats2bfloat162_rn(o[0], o[1]);
    __nv_bfloat162 hi = __floats2bfloat162_rn(o[2], o[3]);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t*>(&lo);
    v.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(p) = v;
}

__device__ __forceinline__ void load_bf16x4(const __nv_bfloat16* p, float* o)
{
    uint2 v = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&v.x);
    __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&v.y);
    float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

// Writes the four updated points of one thread (x .. x+3 of one row) and, in
// the forward pass, their stored copy; in the adjoint pass accumulates the
// imaging condition g -= u^k (mu^k - 2 mu^{k+1} + mu^{k+2}).
template <bool ADJ>
__device__ __forceinline__ void finish4(const StepArgs& a, long long so, long long off, int nvalid,
                                        const float* out, const float* cen, const float* um)
{
    float* un = a.unew + so;
    if (nvalid == 4) {
        *reinterpret_cast<float4*>(un + off) = make_float4(out[0], out[1], out[2], out[3]);
    } else {
        for (int i = 0; i < nvalid; ++i) un[off + i] = out[i];
    }
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
    } else if (a.gacc) {
        float uf[4];
        if (a.uf16) {
            if (nvalid == 4) {
                load_bf16x4(a.uf16 + so + off, uf);
            } else {
                for (int i = 0; i < nvalid; ++i) uf[i] = __bfloat162float(a.uf16[so + off + i]);
            }
        } else {
            if (nvalid == 4) {
                float4 v = ld4(a.uf32 + so + off);
                uf[0] = v.x;
                uf[1] = v.y;
                uf[2] = v.z;
                uf[3] = v.w;
            } else {
                for (int i = 0; i < nvalid; ++i) uf[i] = a.uf32[so + off + i];
            }
        }
        float* g = a.gacc + so + off;
        if (nvalid == 4) {
            float4 gv = *reinterpret_cast<float4*>(g);
            gv.x -= uf[0] * (out[0] - 2.0f * cen[0] + um[0]);
            gv.y -= uf[1] * (out[1] - 2.0f * cen[1] + um[1]);
            gv.z -= uf[2] * (out[2] - 2.0f * cen[2] + um[2]);
            gv.w -= uf[3] * (out[3] - 2.0f * cen[3] + um[3]);
            *reinterpret_cast<float4*>(g) = gv;
        } else {
            for (int i = 0; i < nvalid; ++i) g[i] -= uf[i] * (out[i] - 2.0f * cen[i] + um[i]);
        }
    }
}

// Sparse part of a step, run by the CTA that owns the tile after its points
// are written: injection into unew (atomic: taps of different points may
// share a grid point), then gathers of unew into slots.
template <bool ADJ>
__device__ __forceinline__ void sparse_phase(const StepArgs& a, long long tile, long long so, int tid,
                                             int nthr)
{
    float* un = a.unew + so;
    if (a.inj.tile_start) {
        const int b = a.inj.tile_start[tile], e = a.inj.tile_start[tile + 1];
        for (int j = b + tid; j < e; j += nthr) {
            const int i = a.inj.idx[j];
            const long long ai = (long long)a.inj.ab[j] + (long long)a.amp_row * a.inj.npts;
            float amp = a.amp_a[ai];
            if (a.amp_b) amp -= a.amp_b[ai];
            const float add = a.inj.fac[j] * amp;
            atomicAdd(un + i, add);
            if (ADJ && a.gacc) {
                const float uf = a.uf16 ? __bfloat162float(a.uf16[so + i]) : a.uf32[so + i];
                atomicAdd(a.gacc + so + i, -uf * add);
            }
        }
        if (!ADJ && (a.st16 || a.st32)) {
            // the stored copy of the new level must include the injection
            __syncthreads();
            for (int j = b + tid; j < e; j += nthr) {
                const int i = a.inj.idx[j];
                const float v = un[i];
                if (a.st16) a.st16[so + i] = __float2bfloat16_rn(v);
                if (a.st32) a.st32[so + i] = v;
            }
        }
    }
    if (a.gat.tile_start) {
        __syncthreads();
        const int b = a.gat.tile_start[tile], e = a.gat.tile_start[tile + 1];
        float* row = a.slots + (long long)a.slot_row * a.gat.ntap;
        for (int j = b + tid; j < e; j += nthr) row[a.gat.slot[j]] = a.gat.gw[j] * un[a.gat.idx[j]];
    }
}

// ---------------------------------------------------------------------------
// 2D step.  Tile = 128 (x) by TZ (z) points, CTA = 32 x BZ threads, each
// thread updates 4 consecutive x points on TZ/BZ rows.  The (TZ+8) x 136 halo
// tile of u is staged in shared memory with 128-bit loads; values outside the
// padded grid read as zero.
template <int TZ, int BZ, bool ADJ>
__global__ void __launch_bounds__(32 * BZ) k_step2d(const StepArgs a)
{
    constexpr int SW = 136;
    __shared__ __align__(16) float s[TZ + 8][SW];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int x0 = blockIdx.x * 128, z0 = blockIdx.y * TZ;
    const long long so = (long long)blockIdx.z * a.cell;
    const float* __restrict__ u = a.u + so;

    for (int i = tid; i < (TZ + 8) * (SW / 4); i += 32 * BZ) {
        const int r = i / (SW / 4), c4 = i - r * (SW / 4);
        const int gz = z0 - 4 + r, gx = x0 - 4 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gz >= 0 && gz < a.Nz && gx >= 0 && gx < a.P) v = ld4(u + (long long)gz * a.P + gx);
        *reinterpret_cast<float4*>(&s[r][4 * c4]) = v;
    }
    __syncthreads();

    const int lx = 4 * threadIdx.x;
    const int gx = x0 + lx;
    const int nvalid = min(4, a.Nx - gx);
#pragma unroll
    for (int rr = 0; rr < TZ / BZ; ++rr) {
        const int r = threadIdx.y + rr * BZ;
        const int gz = z0 + r;
        if (gz >= a.Nz || nvalid <= 0) continue;
        const float* row = &s[r + 4][lx];
        float w[12];
        {
            float4 A = *reinterpret_cast<const float4*>(row);
            float4 B = *reinterpret_cast<const float4*>(row + 4);
            float4 C = *reinterpret_cast<const float4*>(row + 8);
            w[0] = A.x; w[1] = A.y; w[2] = A.z; w[3] = A.w;
            w[4] = B.x; w[5] = B.y; w[6] = B.z; w[7] = B.w;
            w[8] = C.x; w[9] = C.y; w[10] = C.z; w[11] = C.w;
        }
        float lap[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            lap[i] = 2.0f * kC0 * w[i + 4] + kC1 * (w[i + 3] + w[i + 5]) + kC2 * (w[i + 2] + w[i + 6]) +
                     kC3 * (w[i + 1] + w[i + 7]) + kC4 * (w[i] + w[i + 8]);
        const float ck[5] = {kC0, kC1, kC2, kC3, kC4};
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            float4 U = *reinterpret_cast<const float4*>(&s[r + 4 - k][lx + 4]);
            float4 D = *reinterpret_cast<const float4*>(&s[r + 4 + k][lx + 4]);
            lap[0] += ck[k] * (U.x + D.x);
            lap[1] += ck[k] * (U.y + D.y);
            lap[2] += ck[k] * (U.z + D.z);
            lap[3] += ck[k] * (U.w + D.w);
        }
        const long long off = (long long)gz * a.P + gx;
        const float4 kp = ld4(a.kap + off);
        const float4 uo = *reinterpret_cast<const float4*>(a.unew + so + off);
        const int dz = sponge_depth(gz, a.nb, a.nz);
        float out[4], cen[4], um[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int dd = max(sponge_depth(gx + i, a.nb, a.nx), dz);
            const float kap = f4(kp, i);
            const float eps = kap * a.ceps * (float)(dd * dd);
            cen[i] = w[i + 4];
            um[i] = f4(uo, i);
            out[i] = leap(cen[i], um[i], lap[i], kap, eps);
        }
        finish4<ADJ>(a, so, off, nvalid, out, cen, um);
    }
    if (a.inj.tile_start || a.gat.tile_start) {
        __syncthreads();
        const long long tile = ((long long)blockIdx.z * a.ntz + blockIdx.y) * a.ntx + blockIdx.x;
        sparse_phase<ADJ>(a, tile, so, tid, 32 * BZ);
    }
}

// ---------------------------------------------------------------------------
// 3D step.  Tile = 128 (x) by TY (y) by TZC (z) points; CTA = 32 x TY threads
// marching in z.  Each thread keeps its 4 x points of the 9 planes z-4..z+4 in
// registers; the current xy plane with its 4-point halo sits in shared memory.
template <int TY, int TZC, bool ADJ>
__global__ void __launch_bounds__(32 * TY) k_step3d(const StepArgs a)
{
    constexpr int SW = 136;
    __shared__ __align__(16) float s[TY + 8][SW];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * TY;
    const int shot = blockIdx.z / a.ntz, tzi = blockIdx.z - shot * a.ntz;
    const int z0 = tzi * TZC;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const long long so = (long long)shot * a.cell;
    const long long plane = (long long)a.Ny * a.P;
    const float* __restrict__ u = a.u + so;
    const int nvalid = min(4, a.Nx - gx);

    auto ld = [&](int z, int y, int x) -> float4 {
        if (z < 0 || z >= a.Nz || y < 0 || y >= a.Ny || x < 0 || x >= a.P) return make_float4(0.f, 0.f, 0.f, 0.f);
        return ld4(u + z * plane + (long long)y * a.P + x);
    };

    float4 q[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = ld(z0 - 4 + k, gy, gx);

    const float ck[5] = {kC0, kC1, kC2, kC3, kC4};
    for (int zz = 0; zz < TZC; ++zz) {
        const int gz = z0 + zz;
        if (gz >= a.Nz) break;
        q[8] = ld(gz + 4, gy, gx);
        *reinterpret_cast<float4*>(&s[ty + 4][4 + 4 * tx]) = q[4];
        if (tx == 0) *reinterpret_cast<float4*>(&s[ty + 4][0]) = ld(gz, gy, x0 - 4);
        if (tx == 31) *reinterpret_cast<float4*>(&s[ty + 4][132]) = ld(gz, gy, x0 + 128);
        for (int i = tid; i < 8 * (SW / 4); i += 32 * TY) {
            const int r = i / (SW / 4), c4 = i - r * (SW / 4);
            const int yy = r < 4 ? y0 - 4 + r : y0 + TY + (r - 4);
            const int sr = r < 4 ? r : TY + r;
            *reinterpret_cast<float4*>(&s[sr][4 * c4]) = ld(gz, yy, x0 - 4 + 4 * c4);
        }
        __syncthreads();
        if (gy < a.Ny && nvalid > 0) {
            const float* row = &s[ty + 4][4 * tx];
            float w[12];
            {
                float4 A = *reinterpret_cast<const float4*>(row);
                float4 B = *reinterpret_cast<const float4*>(row + 4);
                float4 C = *reinterpret_cast<const float4*>(row + 8);
                w[0] = A.x; w[1] = A.y; w[2] = A.z; w[3] = A.w;
                w[4] = B.x; w[5] = B.y; w[6] = B.z; w[7] = B.w;
                w[8] = C.x; w[9] = C.y; w[10] = C.z; w[11] = C.w;
            }
            float lap[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                lap[i] = 3.0f * kC0 * w[i + 4] + kC1 * (w[i + 3] + w[i + 5]) + kC2 * (w[i + 2] + w[i + 6]) +
                         kC3 * (w[i + 1] + w[i + 7]) + kC4 * (w[i] + w[i + 8]);
#pragma unroll
            for (int k = 1; k <= 4; ++k) {
                float4 U = *reinterpret_cast<const float4*>(&s[ty + 4 - k][4 * tx + 4]);
                float4 D = *reinterpret_cast<const float4*>(&s[ty + 4 + k][4 * tx + 4]);
                const float4 zu = q[4 - k], zd = q[4 + k];
                lap[0] += ck[k] * (U.x + D.x + zu.x + zd.x);
                lap[1] += ck[k] * (U.y + D.y + zu.y + zd.y);
                lap[2] += ck[k] * (U.z + D.z + zu.z + zd.z);
                lap[3] += ck[k] * (U.w + D.w + zu.w + zd.w);
            }
            const long long off = gz * plane + (long long)gy * a.P + gx;
            const float4 kp = ld4(a.kap + off);
            const float4 uo = *reinterpret_cast<const float4*>(a.unew + so + off);
            const int dzy = max(sponge_depth(gz, a.nb, a.nz), sponge_depth(gy, a.nb, a.ny));
            float out[4], cen[4], um[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int dd = max(sponge_depth(gx + i, a.nb, a.nx), dzy);
                const float kap = f4(kp, i);
                const float eps = kap * a.ceps * (float)(dd * dd);
                cen[i] = w[i + 4];
                um[i] = f4(uo, i);
                out[i] = leap(cen[i], um[i], lap[i], kap, eps);
            }
            finish4<ADJ>(a, so, off, nvalid, out, cen, um);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
    }
    if (a.inj.tile_start || a.gat.tile_start) {
        const long long tile = (((long long)shot * a.ntz + tzi) * a.nty + blockIdx.y) * a.ntx + blockIdx.x;
        sparse_phase<ADJ>(a, tile, so, tid, 32 * TY);
    }
}

static void launch_step_raw(const Tiling& t, int ndim, bool adjoint, int nshot, const StepArgs& a, cudaStream_t s);

void launch_step(const Tiling& t, int ndim, bool adjoint, int nshot, const StepArgs& a, cudaStream_t s)
{
    count_launch();
    cudaEvent_t stop;
    const bool timed = profile_sample(adjoint, s, &stop);
    launch_step_raw(t, ndim, adjoint, nshot, a, s);
    if (timed) profile_close(stop, s);
}

static void launch_step_raw(const Tiling& t, int ndim, bool adjoint, int nshot, const StepArgs& a, cudaStream_t s)
{
    if (ndim == 2) {
        dim3 grid(t.ntx, t.ntz, nshot);
        if (t.TZ == 32) {
            dim3 block(32, 8);
            if (adjoint) k_step2d<32, 8, true><<<grid, block, 0, s>>>(a);
            else k_step2d<32, 8, false><<<grid, block, 0, s>>>(a);
        } else if (t.TZ == 16) {
            dim3 block(32, 8);
            if (adjoint) k_step2d<16, 8, true><<<grid, block, 0, s>>>(a);
            else k_step2d<16, 8, false><<<grid, block, 0, s>>>(a);
        } else {
            dim3 block(32, 8);
            if (adjoint) k_step2d<64, 8, true><<<grid, block, 0, s>>>(a);
            else k_step2d<64, 8, false><<<grid, block, 0, s>>>(a);
        }
    } else {
        dim3 grid(t.ntx, t.nty, t.ntz * nshot);
        dim3 block(32, 8);
        if (adjoint) k_step3d<8, 32, true><<<grid, block, 0, s>>>(a);
        else k_step3d<8, 32, false><<<grid, block, 0, s>>>(a);
    }
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
    fac[j] = w[j] * scale * k * __frcp_rn(1.0f + eps);
}

void launch_tapfac(const Dims& d, const TapList& l, const float* kap, float scale_inj, float ceps, cudaStream_t s)
{
    if (l.ntap == 0) return;
    count_launch();
    k_tapfac<<<(l.ntap + 255) / 256, 256, 0, s>>>(d, l.ntap, l.idx, l.w, const_cast<float*>(l.fac), kap,
                                                   scale_inj, ceps);
}

// out[s][n][p] = sum of the point's gather slots at time row n.
__global__ void k_finalize(const int* __restrict__ pt_start, const float* __restrict__ slots, int npts_all,
                           int npts, int nt, int ntap, float* __restrict__ out)
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

// grad[j] = sum over shots and over the padded cells whose model value was
// copied from physical cell j (the adjoint of the edge extension).
__global__ void k_grad_reduce(Dims d, const float* __restrict__ gacc, int nshot, float* __restrict__ grad)
{
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= d.phys) return;
    const int jx = (int)(j % d.nx);
    const long long r = j / d.nx;
    const int nyp = d.ndim == 3 ? d.ny : 1;
    const int jy = (int)(r % nyp);
    const int jz = (int)(r / nyp);
    const int x_lo = jx == 0 ? 0 : jx + d.nb, x_hi = jx == d.nx - 1 ? d.Nx - 1 : jx + d.nb;
    const int z_lo = jz == 0 ? 0 : jz + d.nb, z_hi = jz == d.nz - 1 ? d.Nz - 1 : jz + d.nb;
    int y_lo = 0, y_hi = 0;
    if (d.ndim == 3) {
        y_lo = jy == 0 ? 0 : jy + d.nb;
        y_hi = jy == d.ny - 1 ? d.Ny - 1 : jy + d.nb;
    }
    float acc = 0.0f;
    for (int s = 0; s < nshot; ++s) {
        const float* g = gacc + (long long)s * d.cell;
        for (int z = z_lo; z <= z_hi; ++z)
            for (int y = y_lo; y <= y_hi; ++y)
                for (int x = x_lo; x <= x_hi; ++x) acc += g[((long long)z * d.Ny + y) * d.P + x];
    }
    grad[j] = acc;
}

void launch_grad_reduce(const Dims& d, const float* gacc, int nshot, float* grad, cudaStream_t s)
{
    count_launch();
    k_grad_reduce<<<(int)((d.phys + 255) / 256), 256, 0, s>>>(d, gacc, nshot, grad);
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
