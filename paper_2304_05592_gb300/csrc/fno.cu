// fno.cu -- kernels of the Fourier neural operator used as a learned
// preconditioner: twiddle tables, the truncated DFT along x and z and their
// inverse directions, the per-mode complex channel mix (alone, and fused with
// the inverse z transform) and its backward, the fused pointwise channel mix +
// spectral inverse + GELU, the fused projection head, weight gradients, the MSE
// loss and the Adam update.  BF16 inference runs the channel mix, the
// projection head and the x transform on the 5th-generation tensor cores
// (tcgen05, operands in shared memory, accumulators in tensor memory).  The
// operations and layouts are those of include/fno.h; the network is the FNO of
// Li et al. (2020) that the paper uses as a learned surrogate (section "Fourier
// neural operator surrogates").
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "fno.h"
#include "internal.h"

namespace wave {
namespace {

__device__ __forceinline__ float ldf(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void stf(float* p, size_t i, float v) { p[i] = v; }
__device__ __forceinline__ void stf(__nv_bfloat16* p, size_t i, float v) { p[i] = __float2bfloat16_rn(v); }

// GELU(x) = x Phi(x) with Phi the standard normal distribution function.
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// --- tables -------------------------------------------------------------------

__global__ void k_tables(int Nz, int Nx, int mz, int mx, float* tf, float* ti, float* tb, float* ta, float* tz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Nx * mx) {
        const int x = i / mx, kx = i - x * mx;
        const long long r = ((long long)kx * x) % Nx;  // exact argument reduction
        double s, c;
        sincospi(2.0 * (double)r / (double)Nx, &s, &c);
        const double w = (kx == 0 ? 1.0 : 2.0) / ((double)Nz * (double)Nx);
        tf[2 * i] = (float)c;
        tf[2 * i + 1] = (float)(-s);
        ti[2 * i] = (float)(w * c);
        ti[2 * i + 1] = (float)(w * s);
        tb[2 * i] = (float)(w * c);
        tb[2 * i + 1] = (float)(-w * s);
        ta[2 * i] = (float)c;
        ta[2 * i + 1] = (float)s;
    }
    const int KZ = 2 * mz;
    if (i < Nz * KZ) {
        const int z = i / KZ, a = i - z * KZ;
        const int kz = a < mz ? a : Nz - KZ + a;  // rows 0..mz-1, then Nz-mz..Nz-1
        const long long r = ((long long)kz * z) % Nz;
        double s, c;
        sincospi(2.0 * (double)r / (double)Nz, &s, &c);
        tz[2 * i] = (float)c;
        tz[2 * i + 1] = (float)s;
    }
}

// --- along x: out[r][n] = sum_x in[r][x] tab[x][n], n < 2 mx ------------------
// CTA = 256 threads, kDxRows rows; thread (tr, tn) owns rows kDxRq tr ..
// kDxRq tr + kDxRq - 1 and outputs 4 tn .. 4 tn + 3, accumulated over x in
// chunks of 32 staged in shared memory (rows padded to 33 floats: conflict-free
// in both directions).  The chunks are double-buffered: chunk c + 1 is loaded
// into registers while chunk c is summed, then stored to the other buffer, one
// block barrier per chunk.  128 rows per CTA put a 65536-row transform on the
// GPU in one wave.
constexpr int kDxRows = 128, kDxChunk = 32, kDxRq = kDxRows / 32;
constexpr int kDxPv = kDxRows * kDxChunk / 256, kDxPt = kDxChunk * 32 / 256;  // elements per thread and chunk

template <typename T>
__global__ void __launch_bounds__(256, 4) k_dft_x(long long rows, int Nx, int n2, const T* __restrict__ in,
                                               const float* __restrict__ tab, float* __restrict__ out)
{
    __shared__ float sv[2][kDxRows][kDxChunk + 1];
    __shared__ __align__(16) float st[2][kDxChunk][32];
    const int tid = threadIdx.x, tn = tid & 7, tr = tid >> 3;
    const long long r0 = (long long)blockIdx.x * kDxRows;
    float acc[kDxRq][4];
#pragma unroll
    for (int q = 0; q < kDxRq; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = 0.0f;
    float pv[kDxPv], pt[kDxPt];
    auto load = [&](int xc) {
#pragma unroll
        for (int k = 0; k < kDxPv; ++k) {
            const int e = tid + 256 * k, row = e / kDxChunk, x = e - row * kDxChunk;
            const long long gr = r0 + row;
            pv[k] = (gr < rows && xc + x < Nx) ? ldf(in, (size_t)gr * Nx + xc + x) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kDxPt; ++k) {
            const int e = tid + 256 * k, x = e >> 5, n = e & 31;
            pt[k] = (xc + x < Nx && n < n2) ? tab[(size_t)(xc + x) * n2 + n] : 0.0f;
        }
    };
    auto store = [&](int q) {
#pragma unroll
        for (int k = 0; k < kDxPv; ++k) {
            const int e = tid + 256 * k, row = e / kDxChunk, x = e - row * kDxChunk;
            sv[q][row][x] = pv[k];
        }
#pragma unroll
        for (int k = 0; k < kDxPt; ++k) {
            const int e = tid + 256 * k;
            st[q][e >> 5][e & 31] = pt[k];
        }
    };
    load(0);
    store(0);
    __syncthreads();
    int q = 0;
    for (int xc = 0; xc < Nx; xc += kDxChunk, q ^= 1) {
        const bool more = xc + kDxChunk < Nx;
        if (more) load(xc + kDxChunk);  // in flight during the sums below
#pragma unroll 4
        for (int x = 0; x < kDxChunk; ++x) {
            const float4 t = *reinterpret_cast<const float4*>(&st[q][x][4 * tn]);
#pragma unroll
            for (int r = 0; r < kDxRq; ++r) {
                const float a = sv[q][kDxRq * tr + r][x];
                acc[r][0] = fmaf(a, t.x, acc[r][0]);
                acc[r][1] = fmaf(a, t.y, acc[r][1]);
                acc[r][2] = fmaf(a, t.z, acc[r][2]);
                acc[r][3] = fmaf(a, t.w, acc[r][3]);
            }
        }
        if (more) store(q ^ 1);  // the buffer chunk c - 1 used: free since the last barrier
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < kDxRq; ++r) {
        const long long gr = r0 + kDxRq * tr + r;
        if (gr >= rows) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (4 * tn + c < n2) out[(size_t)gr * n2 + 4 * tn + c] = acc[r][c];
    }
}

// --- along z -------------------------------------------------------------------

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
// acc + a b and acc + a conj(b) as four FMAs each
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b)
{
    return make_float2(fmaf(-a.y, b.y, fmaf(a.x, b.x, acc.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, acc.y)));
}
__device__ __forceinline__ float2 cfmac(float2 acc, float2 a, float2 b)
{
    return make_float2(fmaf(a.y, b.y, fmaf(a.x, b.x, acc.x)), fmaf(-a.x, b.y, fmaf(a.y, b.x, acc.y)));
}

// out[b][a][kx] = sum_z in[b][z][kx] conj(E[z][a]); CTA per (b, 16 values of a).
// Thread (h, q, kx) computes outputs (a0 + 4 q .. a0 + 4 q + 3, kx) over quarter h
// of every 64-row chunk of z, so each in[z][kx] read from shared memory feeds
// four outputs; the quarters are added at the end in a fixed order.
__global__ void __launch_bounds__(256) k_dft_z(int Nz, int KZ, int mx, const float2* __restrict__ in,
                                               const float2* __restrict__ tz, float2* __restrict__ out)
{
    __shared__ float2 si[64][16];
    __shared__ __align__(16) float2 se[64][16];
    __shared__ float2 red[3][16][16];
    const int b = blockIdx.x, a0 = blockIdx.y * 16, tid = threadIdx.x;
    const int kx = tid & 15, q = (tid >> 4) & 3, h = tid >> 6;
    float2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int z0 = 0; z0 < Nz; z0 += 64) {
        const int zc = min(64, Nz - z0);
        for (int e = tid; e < 64 * 16; e += 256) {
            const int zz = e >> 4, k = e & 15;
            si[zz][k] = (zz < zc && k < mx) ? in[((size_t)b * Nz + z0 + zz) * mx + k] : make_float2(0.f, 0.f);
            se[zz][k] = (zz < zc && a0 + k < KZ) ? tz[(size_t)(z0 + zz) * KZ + a0 + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int zz = 16 * h; zz < 16 * h + 16; ++zz) {
            const float2 v = si[zz][kx];
            const float4 e01 = *reinterpret_cast<const float4*>(&se[zz][4 * q]);
            const float4 e23 = *reinterpret_cast<const float4*>(&se[zz][4 * q + 2]);
            acc[0] = cfmac(acc[0], v, make_float2(e01.x, e01.y));
            acc[1] = cfmac(acc[1], v, make_float2(e01.z, e01.w));
            acc[2] = cfmac(acc[2], v, make_float2(e23.x, e23.y));
            acc[3] = cfmac(acc[3], v, make_float2(e23.z, e23.w));
        }
        __syncthreads();
    }
    if (h > 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) red[h - 1][4 * q + j][kx] = acc[j];
    __syncthreads();
    if (h == 0 && kx < mx)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int aa = a0 + 4 * q + j;
            if (aa < KZ)
                out[((size_t)b * KZ + aa) * mx + kx] =
                    cadd(cadd(acc[j], red[0][4 * q + j][kx]), cadd(red[1][4 * q + j][kx], red[2][4 * q + j][kx]));
        }
}

// out[b][z][kx] = sum_a in[b][a][kx] E[z][a]; CTA per (b, 64 rows of z).
// Thread (zr, kx) computes rows zr, zr+16, zr+32, zr+48 of its kx, so that each
// in[a][kx] read from shared memory feeds four outputs.
__global__ void __launch_bounds__(256) k_idft_z(int Nz, int KZ, int mx, const float2* __restrict__ in,
                                                const float2* __restrict__ tz, float2* __restrict__ out)
{
    __shared__ float2 sx[64][16];
    __shared__ float2 se[64][65];
    const int b = blockIdx.x, z0 = blockIdx.y * 64, tid = threadIdx.x;
    const int kx = tid & 15, zr = tid >> 4;
    for (int e = tid; e < 64 * 16; e += 256) {
        const int a = e >> 4, k = e & 15;
        sx[a][k] = (a < KZ && k < mx) ? in[((size_t)b * KZ + a) * mx + k] : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < 64 * KZ; e += 256) {
        const int zz = e / KZ, a = e - zz * KZ;
        se[zz][a] = z0 + zz < Nz ? tz[(size_t)(z0 + zz) * KZ + a] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int a = 0; a < KZ; ++a) {
        const float2 y = sx[a][kx];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = cfma(acc[q], y, se[zr + 16 * q][a]);
    }
    if (kx < mx)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int z = z0 + zr + 16 * q;
            if (z < Nz) out[((size_t)b * Nz + z) * mx + kx] = acc[q];
        }
}

// --- per-mode channel mix ---------------------------------------------------------

__global__ void k_mix(int B, int Ci, int Co, int nm, const float2* __restrict__ X, const float2* __restrict__ R,
                      float2* __restrict__ Y)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * Co * nm) return;
    const int m = (int)(t % nm);
    const long long bo = t / nm;
    const int o = (int)(bo % Co), b = (int)(bo / Co);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int i = 0; i < Ci; ++i)  // unrolled: eight loads of each operand in flight
        acc = cfma(acc, X[((size_t)b * Ci + i) * nm + m], R[((size_t)i * Co + o) * nm + m]);
    Y[t] = acc;
}

// k_mix followed by k_idft_z for one (b, o) per CTA, the mixed spectrum kept in
// shared memory: out[b][o][z][kx] = sum_a Y[a][kx] E[z][a] with
// Y[a][kx] = sum_i X[b][i][a][kx] R[i][o][a][kx] (both sums in the same order as
// the two separate kernels).
__global__ void __launch_bounds__(256) k_mix_idft_z(int Ci, int Co, int Nz, int KZ, int mx, const float2* __restrict__ X,
                                                    const float2* __restrict__ R, const float2* __restrict__ tz,
                                                    float2* __restrict__ out)
{
    __shared__ float2 sy[64][16];
    __shared__ float2 se[64][65];
    const int bo = blockIdx.x, b = bo / Co, o = bo - b * Co, tid = threadIdx.x;
    const int nm = KZ * mx;
    for (int m = tid; m < 64 * 16; m += 256) {
        const int a = m >> 4, k = m & 15;
        float2 acc = make_float2(0.f, 0.f);
        if (a < KZ && k < mx) {
            const int mm = a * mx + k;
#pragma unroll 8
            for (int i = 0; i < Ci; ++i)
                acc = cfma(acc, X[((size_t)b * Ci + i) * nm + mm], R[((size_t)i * Co + o) * nm + mm]);
        }
        sy[a][k] = acc;
    }
    const int kx = tid & 15, zr = tid >> 4;
    for (int z0 = 0; z0 < Nz; z0 += 64) {
        __syncthreads();  // the spectrum is complete; the previous chunk's table has been read
        for (int e = tid; e < 64 * KZ; e += 256) {
            const int zz = e / KZ, a = e - zz * KZ;
            se[zz][a] = z0 + zz < Nz ? tz[(size_t)(z0 + zz) * KZ + a] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int a = 0; a < KZ; ++a) {
            const float2 y = sy[a][kx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = cfma(acc[q], y, se[zr + 16 * q][a]);
        }
        if (kx < mx)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int z = z0 + zr + 16 * q;
                if (z < Nz) out[((size_t)bo * Nz + z) * mx + kx] = acc[q];
            }
    }
}

__global__ void k_mix_dx(int B, int Ci, int Co, int nm, const float2* __restrict__ dY, const float2* __restrict__ R,
                         float2* __restrict__ dX)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * Ci * nm) return;
    const int m = (int)(t % nm);
    const long long bi = t / nm;
    const int i = (int)(bi % Ci), b = (int)(bi / Ci);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int o = 0; o < Co; ++o)
        acc = cfmac(acc, dY[((size_t)b * Co + o) * nm + m], R[((size_t)i * Co + o) * nm + m]);
    dX[t] = acc;
}

__global__ void k_mix_dr(int B, int Ci, int Co, int nm, const float2* __restrict__ X, const float2* __restrict__ dY,
                         float2* __restrict__ dR)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)Ci * Co * nm) return;
    const int m = (int)(t % nm);
    const long long io = t / nm;
    const int o = (int)(io % Co), i = (int)(io / Co);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int b = 0; b < B; ++b)  // conj(X) dY, summed over the batch in order
        acc = cfmac(acc, dY[((size_t)b * Co + o) * nm + m], X[((size_t)b * Ci + i) * nm + m]);
    dR[t] = acc;
}

// --- fused pointwise mix + spectral inverse + activation ------------------------------
// CTA = 256 pixels of one (b, z) row; M (padded to CIMAX per row), bias and the
// row's spectral coefficients T[b][o][z][:] are staged in shared memory and read
// as broadcasts; each thread keeps its pixel's ci inputs and the 2 mx table
// factors of its x in registers and produces all co outputs.
template <int CIMAX, typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_combine(int ci, int co, int Nz, int Nx, int mx, const Tin* __restrict__ in,
                                                 const float* __restrict__ M, int mtrans,
                                                 const float* __restrict__ bias, const float* __restrict__ T,
                                                 const float* __restrict__ tab, int act, float* __restrict__ pre,
                                                 Tout* __restrict__ out)
{
    extern __shared__ __align__(16) float sm[];
    float* sM = sm;                  // [co][CIMAX]
    float* sT = sM + co * CIMAX;     // [co][32]
    float* sB = sT + co * 32;        // [co]
    const int b = blockIdx.z, z = blockIdx.y, tid = threadIdx.x;
    const int x = blockIdx.x * 256 + tid;
    const int n2 = 2 * mx;
#pragma unroll 4
    for (int e = tid; e < co * CIMAX; e += 256) {
        const int o = e / CIMAX, i = e - o * CIMAX;
        sM[e] = i < ci ? (mtrans ? M[(size_t)i * co + o] : M[(size_t)o * ci + i]) : 0.0f;
    }
#pragma unroll 4
    for (int e = tid; e < co * 32; e += 256) {
        const int o = e >> 5, r = e & 31;
        sT[e] = (T && r < n2) ? T[(((size_t)b * co + o) * Nz + z) * n2 + r] : 0.0f;
    }
    for (int e = tid; e < co; e += 256) sB[e] = bias ? bias[e] : 0.0f;
    __syncthreads();
    if (x >= Nx) return;  // no barrier follows
    const size_t npix = (size_t)Nz * Nx, pix = (size_t)z * Nx + x;
    float v[CIMAX];
#pragma unroll
    for (int i = 0; i < CIMAX; ++i) v[i] = i < ci ? ldf(in, ((size_t)b * ci + i) * npix + pix) : 0.0f;
    float tc[16], ts[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        tc[k] = (T && k < mx) ? tab[((size_t)x * mx + k) * 2] : 0.0f;
        ts[k] = (T && k < mx) ? tab[((size_t)x * mx + k) * 2 + 1] : 0.0f;
    }
    for (int o = 0; o < co; ++o) {
        float acc = sB[o];
        // weights by 16-byte loads (the same address in every thread: broadcasts)
        const float4* mr = reinterpret_cast<const float4*>(sM + o * CIMAX);
#pragma unroll
        for (int i4 = 0; i4 < CIMAX / 4; ++i4) {
            const float4 w = mr[i4];
            acc = fmaf(w.x, v[4 * i4], acc);
            acc = fmaf(w.y, v[4 * i4 + 1], acc);
            acc = fmaf(w.z, v[4 * i4 + 2], acc);
            acc = fmaf(w.w, v[4 * i4 + 3], acc);
        }
        if (T) {  // uniform over the grid
            const float4* tr = reinterpret_cast<const float4*>(sT + o * 32);
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) {
                const float4 t = tr[k2];
                acc = fmaf(t.x, tc[2 * k2], acc);
                acc = fmaf(-t.y, ts[2 * k2], acc);
                acc = fmaf(t.z, tc[2 * k2 + 1], acc);
                acc = fmaf(-t.w, ts[2 * k2 + 1], acc);
            }
        }
        const size_t oi = ((size_t)b * co + o) * npix + pix;
        if (pre) pre[oi] = acc;
        stf(out, oi, act == FNO_ACT_GELU ? gelu(acc) : acc);
    }
}

// The same combine as a register-tiled product, for CO = 32 or 64 output
// channels: out[o][p] = bias[o] + sum_k A[k][o] B[k][p] with A = [M^T; the
// row's spectral coefficients (sine terms negated, zero past 2 mx, 32 rows)]
// and B = [the input tile; the x inverse-transform table of the tile's
// pixels], k ascending, so every output is the same fmaf sequence as in
// k_combine (bitwise the same).  A block takes 128 pixels of one row; thread
// (oq, pq) holds outputs 4 oq .. 4 oq + 3 at pixels 4 pq .. 4 pq + 3 and
// 64 + 4 pq .. 64 + 4 pq + 3: per k one 16-byte load of A (a broadcast) and
// two of B feed 32 FMAs.
constexpr int kRtP = 128, kRtS = kRtP + 4;  // pixels per block, B row stride
template <int CO, typename Tin, typename Tout>
__global__ void __launch_bounds__(CO * 4) k_combine_rt(int ci, int Nz, int Nx, int mx, const Tin* __restrict__ in,
                                                   const float* __restrict__ M, int mtrans,
                                                   const float* __restrict__ bias, const float* __restrict__ T,
                                                   const float* __restrict__ tab, int act, float* __restrict__ pre,
                                                   Tout* __restrict__ out)
{
    extern __shared__ __align__(16) float sm[];
    constexpr int NT = CO * 4;
    const int K = ci + (T ? 32 : 0);
    float* sA = sm;                // [K][CO]
    float* sB = sA + K * CO;       // [K][kRtS]
    float* sBias = sB + K * kRtS;  // [CO]
    const int b = blockIdx.z, z = blockIdx.y, x0 = blockIdx.x * kRtP, tid = threadIdx.x;
    const int n2 = 2 * mx;
    const size_t npix = (size_t)Nz * Nx, row = (size_t)z * Nx;
    for (int e = tid; e < K * CO; e += NT) {
        const int k = e / CO, o = e - k * CO;
        float a;
        if (k < ci) {
            a = mtrans ? M[(size_t)k * CO + o] : M[(size_t)o * ci + k];
        } else {
            const int r = k - ci;
            a = r < n2 ? T[(((size_t)b * CO + o) * Nz + z) * n2 + r] : 0.0f;
            if (r & 1) a = -a;
        }
        sA[e] = a;
    }
    for (int e = tid; e < ci * kRtP; e += NT) {
        const int i = e / kRtP, p = e - i * kRtP;
        sB[i * kRtS + p] = x0 + p < Nx ? ldf(in, ((size_t)b * ci + i) * npix + row + x0 + p) : 0.0f;
    }
    if (T) {
        for (int e = tid; e < 32 * kRtP; e += NT) {
            const int p = e >> 5, r = e & 31;
            sB[(ci + r) * kRtS + p] = (x0 + p < Nx && r < n2) ? tab[(size_t)(x0 + p) * n2 + r] : 0.0f;
        }
    }
    for (int e = tid; e < CO; e += NT) sBias[e] = bias ? bias[e] : 0.0f;
    __syncthreads();
    const int oq = tid / 16, pq = tid % 16;
    float acc[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = sBias[4 * oq + u];
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(sA + k * CO + 4 * oq);
        const float4 b0 = *reinterpret_cast<const float4*>(sB + k * kRtS + 4 * pq);
        const float4 b1 = *reinterpret_cast<const float4*>(sB + k * kRtS + 64 + 4 * pq);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const size_t ob = ((size_t)b * CO + 4 * oq + u) * npix + row;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = x0 + 64 * h + 4 * pq;
            float y[4], g[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                y[j] = acc[u][4 * h + j];
                g[j] = act == FNO_ACT_GELU ? gelu(y[j]) : y[j];
            }
            if (x + 3 < Nx && ((ob + x) & 3) == 0) {  // 16-byte (8-byte for BF16) stores
                if (pre) *reinterpret_cast<float4*>(pre + ob + x) = make_float4(y[0], y[1], y[2], y[3]);
                if constexpr (std::is_same<Tout, float>::value) {
                    *reinterpret_cast<float4*>(out + ob + x) = make_float4(g[0], g[1], g[2], g[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) stf(out, ob + x + j, g[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (x + j >= Nx) continue;
                    if (pre) pre[ob + x + j] = y[j];
                    stf(out, ob + x + j, g[j]);
                }
            }
        }
    }
}

// The same channel mix for few input channels and no spectral term (the lift):
// each thread takes 4 consecutive pixels of one sample (16-byte input loads) and
// writes 4 pixels of every output channel at once; the sum over i runs in the
// order of k_combine, so results are identical.  Needs Nz Nx a multiple of 4.
template <int CIMAX, typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_combine_px4(int ci, int co, long long npix, const Tin* __restrict__ in,
                                                     const float* __restrict__ M, int mtrans,
                                                     const float* __restrict__ bias, int act, float* __restrict__ pre,
                                                     Tout* __restrict__ out)
{
    __shared__ float sM[64][CIMAX];
    __shared__ float sB[64];
    const int tid = threadIdx.x, b = blockIdx.y;
    for (int e = tid; e < co * CIMAX; e += 256) {
        const int o = e / CIMAX, i = e - o * CIMAX;
        sM[o][i] = i < ci ? (mtrans ? M[(size_t)i * co + o] : M[(size_t)o * ci + i]) : 0.0f;
    }
    for (int o = tid; o < co; o += 256) sB[o] = bias ? bias[o] : 0.0f;
    __syncthreads();
    const long long p = 4 * ((long long)blockIdx.x * 256 + tid);
    if (p >= npix) return;  // no barrier follows
    float v[CIMAX][4];
#pragma unroll
    for (int i = 0; i < CIMAX; ++i) {
        if (i < ci) {
            const size_t base = ((size_t)b * ci + i) * npix + p;
            if constexpr (sizeof(Tin) == 4) {
                const float4 t = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(in) + base);
                v[i][0] = t.x, v[i][1] = t.y, v[i][2] = t.z, v[i][3] = t.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[i][q] = ldf(in, base + q);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[i][q] = 0.0f;
        }
    }
    for (int o = 0; o < co; ++o) {
        float r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float acc = sB[o];
#pragma unroll
            for (int i = 0; i < CIMAX; ++i) acc = fmaf(sM[o][i], v[i][q], acc);
            r[q] = acc;
        }
        const size_t oi = ((size_t)b * co + o) * npix + p;
        if (pre) *reinterpret_cast<float4*>(pre + oi) = make_float4(r[0], r[1], r[2], r[3]);
        if (act == FNO_ACT_GELU)
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q] = gelu(r[q]);
        if constexpr (sizeof(Tout) == 4) {
            *reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + oi) = make_float4(r[0], r[1], r[2], r[3]);
        } else {
            const __nv_bfloat162 lo = __floats2bfloat162_rn(r[0], r[1]), hi = __floats2bfloat162_rn(r[2], r[3]);
            uint2 u;
            u.x = *reinterpret_cast<const uint32_t*>(&lo);
            u.y = *reinterpret_cast<const uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(out) + oi) = u;
        }
    }
}

// --- the same channel mix on the 5th-generation tensor cores (BF16 inference) -----------
// One CTA (4 warps) computes 128-pixel pieces of rw consecutive rows (b, z) for
// all co outputs, one row at a time, as
//   D[128 x co] = A1 B1^T + A2 B2^T + A3 B3^T
// with tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in tensor memory):
//   A1[p][i] = in[b][i][z][x0+p]        B1[o][i] = M[o][i]
//   A2[p][k] = table[x0+p][k]           B2[o][k] = (T re, -T im)[b][o][z][k]
//   A3[p][k] = (1, 1, 0, ...)           B3[o][k] = (hi, lo, 0, ...) with
// (k = 2 kx + {0, 1} in A2, B2) so that A2 B2^T is the x part of the spectral
// inverse and A3 B3^T adds the bias, split into two BF16 parts hi + lo (bias
// to about 16 significant bits) so that the epilogue reads finished sums.
// Operands sit in shared memory without swizzle, in core matrices of 8 rows x
// 16 bytes: B1, A2, B2 K-major (element (r, k) at (r/8)*512 + (k/8)*128 +
// (r%8)*16 + (k%8)*2 bytes), A3, B3 K-major with 256 bytes between row
// groups, A1 pixel-major (element (p, i) at (p/8)*512 + (i/8)*128 + (i%8)*16 +
// (p%8)*2), which is how the activations lie in memory: every 16-byte piece of
// 8 pixels of one channel is copied as it is (cp.async) and the MMA reads A1
// transposed.  In all layouts the descriptor's leading offset (128 B) steps
// along K and its stride offset along rows.  Pipeline, for row it: row it+1's
// activations and T arrived during row it-1; T is converted to BF16 and row
// it+1's MMAs go to the second accumulator; row it's MMAs are waited for, row
// it+2's copies go into the buffers row it has finished with, and row it's
// accumulator is read (tcgen05.ld), passed through GELU and stored BF16 straight
// from registers: lane = pixel, so a warp writes 64 contiguous bytes of each
// output channel.  Requires ci = 32, co in {32, 64}, mx <= 16.

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc_sbo(uint32_t saddr, uint32_t sbo)
{
    // start address, leading (K) offset 128 B, stride (row-group) offset sbo,
    // descriptor version 1, no swizzle
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
           ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) { return umma_desc_sbo(saddr, 512); }

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t ta, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ uint4 pack8_bf16(const float* f)
{
    uint4 u;
    __nv_bfloat162 h0 = __floats2bfloat162_rn(f[0], f[1]), h1 = __floats2bfloat162_rn(f[2], f[3]),
                   h2 = __floats2bfloat162_rn(f[4], f[5]), h3 = __floats2bfloat162_rn(f[6], f[7]);
    u.x = *reinterpret_cast<uint32_t*>(&h0);
    u.y = *reinterpret_cast<uint32_t*>(&h1);
    u.z = *reinterpret_cast<uint32_t*>(&h2);
    u.w = *reinterpret_cast<uint32_t*>(&h3);
    return u;
}

__device__ __forceinline__ bool mbar_wait_parity(uint64_t* bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
// all but the kDxtStages - 1 most recent groups complete (kDxtStages = 3)
__device__ __forceinline__ void cp_async_wait_stages() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }

// k_combine_rt for FP32 inputs with rows of a multiple of 4 pixels, a block
// marching over kRzRows rows of one 128-pixel column strip: the weights, the
// strip's x inverse table and the bias are staged once, the next row's input
// tile arrives by cp.async and its spectral coefficients through registers
// while the current row is computed.  The same k order and fmaf sequence as
// k_combine (bitwise the same outputs).
constexpr int kRzRows = 8;
template <int CO, typename Tout>
__global__ void __launch_bounds__(CO * 4) k_combine_rz(int ci, int Nz, int Nx, int mx, const float* __restrict__ in,
                                                   const float* __restrict__ M, int mtrans,
                                                   const float* __restrict__ bias, const float* __restrict__ T,
                                                   const float* __restrict__ tab, int act, float* __restrict__ pre,
                                                   Tout* __restrict__ out)
{
    extern __shared__ __align__(16) float sm[];
    constexpr int NT = CO * 4, TPT = 32 * CO / NT;  // spectral coefficients per thread and row (8)
    const bool spec = T != nullptr;
    float* sW = sm;                           // [ci][CO]
    float* sT = sW + ci * CO;                 // [2][32][CO] (spec)
    float* sX = sT + (spec ? 2 * 32 * CO : 0);  // [2][ci][kRtS]
    float* sTab = sX + 2 * ci * kRtS;         // [32][kRtS] (spec)
    float* sBias = sTab + (spec ? 32 * kRtS : 0);  // [CO]
    const int b = blockIdx.z, x0 = blockIdx.x * kRtP, tid = threadIdx.x;
    const int z0 = blockIdx.y * kRzRows, z1 = min(z0 + kRzRows, Nz);
    const int n2 = 2 * mx;
    const size_t npix = (size_t)Nz * Nx;
    for (int e = tid; e < ci * CO; e += NT) {
        const int k = e / CO, o = e - k * CO;
        sW[e] = mtrans ? M[(size_t)k * CO + o] : M[(size_t)o * ci + k];
    }
    if (spec) {
        for (int e = tid; e < 32 * kRtP; e += NT) {
            const int r = e / kRtP, p = e - r * kRtP;
            sTab[r * kRtS + p] = (x0 + p < Nx && r < n2) ? tab[(size_t)(x0 + p) * n2 + r] : 0.0f;
        }
    }
    for (int e = tid; e < CO; e += NT) sBias[e] = bias ? bias[e] : 0.0f;
    // row z's input tile into buffer q (16-byte copies, zero past Nx)
    auto issue = [&](int z, int q) {
        float* dst = sX + q * ci * kRtS;
        for (int e = tid; e < ci * (kRtP / 4); e += NT) {
            const int i = e / (kRtP / 4), p = 4 * (e - i * (kRtP / 4));
            const float* src = in + ((size_t)b * ci + i) * npix + (size_t)z * Nx;
            const int bytes = x0 + p < Nx ? 16 : 0;  // Nx is a multiple of 4
            cp_async16(su32(dst + i * kRtS + p), bytes ? src + x0 + p : src, bytes);
        }
        cp_async_commit();
    };
    // row z's spectral coefficients (o, r) of this thread: e = tid + j NT
    float tn[TPT];
    auto load_t = [&](int z) {
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int e = tid + j * NT, o = e >> 5, r = e & 31;
            tn[j] = r < n2 ? T[(((size_t)b * CO + o) * Nz + z) * n2 + r] : 0.0f;
        }
    };
    auto store_t = [&](int q) {
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int e = tid + j * NT, o = e >> 5, r = e & 31;
            sT[(q * 32 + r) * CO + o] = (r & 1) ? -tn[j] : tn[j];
        }
    };
    if (z0 < z1) {
        issue(z0, 0);
        if (spec) {
            load_t(z0);
            store_t(0);
        }
    }
    const int oq = tid / 16, pq = tid % 16;
    for (int z = z0; z < z1; ++z) {
        const int q = (z - z0) & 1;
        const bool next = z + 1 < z1;
        if (next) {
            issue(z + 1, q ^ 1);  // the buffer row z - 1 used (barrier at the end of it)
            if (spec) load_t(z + 1);
            cp_async_wait_prev();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const float* X = sX + q * ci * kRtS;
        const float* A2 = sT + q * 32 * CO;
        float acc[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = sBias[4 * oq + u];
        auto step = [&](const float* Ak, const float* Bk) {
            const float4 a = *reinterpret_cast<const float4*>(Ak + 4 * oq);
            const float4 b0 = *reinterpret_cast<const float4*>(Bk + 4 * pq);
            const float4 b1 = *reinterpret_cast<const float4*>(Bk + 64 + 4 * pq);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        };
#pragma unroll 4
        for (int k = 0; k < ci; ++k) step(sW + k * CO, X + k * kRtS);
        if (spec) {
#pragma unroll 4
            for (int r = 0; r < 32; ++r) step(A2 + r * CO, sTab + r * kRtS);
        }
        const size_t row = (size_t)z * Nx;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t ob = ((size_t)b * CO + 4 * oq + u) * npix + row;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = x0 + 64 * h + 4 * pq;
                if (x >= Nx) continue;  // Nx is a multiple of 4: the 4 pixels are all in or all out
                float y[4], g[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    y[j] = acc[u][4 * h + j];
                    g[j] = act == FNO_ACT_GELU ? gelu(y[j]) : y[j];
                }
                if (pre) *reinterpret_cast<float4*>(pre + ob + x) = make_float4(y[0], y[1], y[2], y[3]);
                if constexpr (std::is_same<Tout, float>::value) {
                    *reinterpret_cast<float4*>(out + ob + x) = make_float4(g[0], g[1], g[2], g[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) stf(out, ob + x + j, g[j]);
                }
            }
        }
        if (next && spec) store_t(q ^ 1);  // read after the barrier at the top of row z + 1
        __syncthreads();
    }
}

// GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 with erf from Abramowitz and
// Stegun, Handbook of Mathematical Functions, formula 7.1.26 (after Hastings):
// erf(a) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-a^2), t = 1 / (1 + p a),
// a >= 0, |error| <= 1.5e-7.  The exponential and the reciprocal are the
// hardware approximations (ex2.approx, rcp.approx; relative errors near 2^-22),
// which keeps this at about 15 instructions.  Used by the BF16 tensor-core
// epilogues, whose outputs carry 8 significant bits.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_as(float x)
{
    const float a = fabsf(x) * 0.70710678118654752f;
    const float t = rcp_approx(fmaf(0.3275911f, a, 1.0f));
    float q = fmaf(t, 1.061405429f, -1.453152027f);
    q = fmaf(t, q, 1.421413741f);
    q = fmaf(t, q, -0.284496736f);
    q = fmaf(t, q, 0.254829592f);
    // half of erfc(a) = q t exp(-a^2) / 2, exp(-a^2) = 2^(-a^2 log2 e), a^2 = x^2 / 2
    const float h = 0.5f * q * t * ex2_approx(-0.72134752044448170f * x * x);
    return x * (x >= 0.0f ? 1.0f - h : h);
}

constexpr int kTcCi = 32;

// Set by the tensor-core kernels if a wait for their MMAs gives up; read and
// cleared by fno_tensor_core_status.
__device__ int g_tc_err;

// dynamic shared memory of k_combine_tc<co, proj>, in bytes (all pieces 16-byte
// aligned; the projection needs no table and no spectral term)
__host__ __device__ constexpr int tc_smem_bytes(int co, bool proj)
{
    return 2 * 8192 /*A1 x2*/ + co * 64 /*B1*/ + 4096 /*A3*/ + co * 32 /*B3*/ +
           (proj ? 0 : 8192 /*A2*/ + 2 * co * 64 /*B2 x2*/ + 2 * co * 32 * 4 /*raw T x2*/);
}

// PROJ: the projection head instead of a BF16 output -- out (float, one channel)
// = q2 + sum_o Q2[o] GELU(D[p][o]); T must be NULL.
template <int CO, bool PROJ>
__global__ void __launch_bounds__(128) k_combine_tc(int Nz, int Nx, int mx, int rw, const __nv_bfloat16* __restrict__ in,
                                                    const float* __restrict__ M, const float* __restrict__ bias,
                                                    const float* __restrict__ T, const float* __restrict__ tab,
                                                    int act, const float* __restrict__ Q2, const float* __restrict__ q2,
                                                    void* __restrict__ out_)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* const sA1 = smem;               // [2][8192]
    unsigned char* const sB1 = smem + 2 * 8192;    // [CO * 64]
    unsigned char* const sA3 = sB1 + CO * 64;      // [4096]
    unsigned char* const sB3 = sA3 + 4096;         // [CO * 32]
    unsigned char* const sA2 = sB3 + CO * 32;      // [8192]            (not PROJ)
    unsigned char* const sB2 = sA2 + 8192;         // [2][CO * 64]      (not PROJ)
    float* const sT = reinterpret_cast<float*>(sB2 + 2 * CO * 64);  // [2][CO][32] (not PROJ)
    __shared__ float sq2[CO + 1];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z, x0 = blockIdx.x * 128;
    const int z0 = blockIdx.y * rw, nrows = min(rw, Nz - z0);
    const size_t npix = (size_t)Nz * Nx;
    const int n2 = 2 * mx;
    const bool spectral = !PROJ && T != nullptr;
    const bool vecA = (Nx & 7) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    const bool vecT = (n2 & 3) == 0 && (reinterpret_cast<uintptr_t>(T) & 15) == 0;
    if (nrows <= 0) return;  // uniform over the CTA

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"((uint32_t)(2 * CO))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }

    // row r of this CTA -> buffers `slot`: activations (pixel-major A1) and raw T
    auto prefetch = [&](int r, int slot) {
        const int z = z0 + r;
        unsigned char* a = sA1 + slot * 8192;
        if (vecA) {
            // a quarter-warp copies one 8-pixel group of 8 channels: 128 contiguous bytes
            // in shared memory, 16 bytes from each of 8 channel rows in global memory
            const int g = tid >> 3, x = x0 + 8 * g;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = 8 * i + (tid & 7);
                const __nv_bfloat16* src = in + ((size_t)b * kTcCi + c) * npix + (size_t)z * Nx + min(x, Nx - 8);
                cp_async16(su32(a + g * 512 + i * 128 + (tid & 7) * 16), src, x < Nx ? 16 : 0);
            }
        } else {
            for (int e = tid; e < kTcCi * 128; e += 128) {
                const int c = e >> 7, p = e & 127, x = x0 + p;
                const __nv_bfloat16 v =
                    x < Nx ? in[((size_t)b * kTcCi + c) * npix + (size_t)z * Nx + x] : __float2bfloat16_rn(0.0f);
                *reinterpret_cast<__nv_bfloat16*>(a + (p >> 3) * 512 + (c >> 3) * 128 + (c & 7) * 16 + (p & 7) * 2) = v;
            }
        }
        if (spectral) {
            float* t = sT + slot * CO * 32;
            if (vecT) {
                for (int e = tid; e < CO * 8; e += 128) {
                    const int o = e >> 3, j = e & 7;
                    if (4 * j < n2) cp_async16(su32(t + o * 32 + 4 * j), T + (((size_t)b * CO + o) * Nz + z) * n2 + 4 * j, 16);
                }
            } else {
                for (int e = tid; e < CO * 32; e += 128) {
                    const int o = e >> 5, k = e & 31;
                    if (k < n2) t[o * 32 + k] = T[(((size_t)b * CO + o) * Nz + z) * n2 + k];
                }
            }
        }
        cp_async_commit();
    };
    // raw T of buffers `slot` -> B2 (BF16, K-major, odd entries negated)
    auto convert = [&](int slot) {
        const float* t = sT + slot * CO * 32;
        unsigned char* bb = sB2 + slot * CO * 64;
        for (int e = tid; e < CO * 4; e += 128) {
            const int o = e >> 2, kg = e & 3;
            float g[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = 8 * kg + j;
                const float v = k < n2 ? t[o * 32 + k] : 0.0f;
                g[j] = (k & 1) ? -v : v;
            }
            *reinterpret_cast<uint4*>(bb + (o >> 3) * 512 + kg * 128 + (o & 7) * 16) = pack8_bf16(g);
        }
    };
    const uint32_t idesc_k = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t idesc_a1 = idesc_k | (1u << 15);  // A read transposed (pixel-major)
    auto issue = [&](int slot, uint32_t tm) {
#pragma unroll
        for (int j = 0; j < kTcCi / 16; ++j)
            umma_bf16(tm, umma_desc(su32(sA1 + slot * 8192) + j * 256), umma_desc(su32(sB1) + j * 256), idesc_a1, j > 0);
        umma_bf16(tm, umma_desc_sbo(su32(sA3), 256), umma_desc_sbo(su32(sB3), 256), idesc_k, 1u);
        if (spectral) {
#pragma unroll
            for (int j = 0; j < 2; ++j)
                umma_bf16(tm, umma_desc(su32(sA2) + j * 256), umma_desc(su32(sB2 + slot * CO * 64) + j * 256), idesc_k, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar[slot]))
                     : "memory");
    };

    prefetch(0, 0);
    if (nrows > 1) prefetch(1, 1);
    // set up once per CTA while the first rows are in flight: weights, bias, table
    for (int e = tid; e < CO * 4; e += 128) {
        const int o = e >> 2, kg = e & 3;
        float g[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) g[j] = M[(size_t)o * kTcCi + 8 * kg + j];
        *reinterpret_cast<uint4*>(sB1 + (o >> 3) * 512 + kg * 128 + (o & 7) * 16) = pack8_bf16(g);
    }
    {
        // A3: ones in k = 0, 1 of every pixel row; B3: the bias as hi + lo in k = 0, 1
        float g[8] = {1.0f, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        const float z8[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        *reinterpret_cast<uint4*>(sA3 + (tid >> 3) * 256 + (tid & 7) * 16) = pack8_bf16(g);
        *reinterpret_cast<uint4*>(sA3 + (tid >> 3) * 256 + 128 + (tid & 7) * 16) = pack8_bf16(z8);
        if (tid < CO) {
            const float bo = bias ? bias[tid] : 0.0f;
            g[0] = __bfloat162float(__float2bfloat16_rn(bo));
            g[1] = bo - g[0];
            *reinterpret_cast<uint4*>(sB3 + (tid >> 3) * 256 + (tid & 7) * 16) = pack8_bf16(g);
            *reinterpret_cast<uint4*>(sB3 + (tid >> 3) * 256 + 128 + (tid & 7) * 16) = pack8_bf16(z8);
        }
    }
    if (spectral) {
        const int x = x0 + tid;
        float f[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) f[k] = (x < Nx && k < n2) ? tab[(size_t)x * n2 + k] : 0.0f;
#pragma unroll
        for (int kg = 0; kg < 4; ++kg)
            *reinterpret_cast<uint4*>(sA2 + (tid >> 3) * 512 + kg * 128 + (tid & 7) * 16) = pack8_bf16(f + 8 * kg);
    }
    if (PROJ)
        for (int o = tid; o <= CO; o += 128) sq2[o] = o < CO ? Q2[o] : (q2 ? q2[0] : 0.0f);
    if (nrows > 1) cp_async_wait_prev();
    else cp_async_wait_all();
    __syncthreads();  // row 0's raw T visible to every thread
    if (spectral) convert(0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = tmem_base;
    if (tid == 0) issue(0, tm);

    bool ok = true;
    const int x = x0 + warp * 32 + lane;  // accumulator lane = pixel of the tile
    for (int it = 0; it < nrows; ++it) {
        const int cur = it & 1, nxt = cur ^ 1;
        if (it + 1 < nrows) {
            cp_async_wait_all();  // this thread's copies of row it+1
            if (spectral) {
                __syncthreads();  // every thread's raw T before the conversion
                convert(nxt);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // row it+1's operands complete; row it-1's accumulator has been read
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (it + 1 < nrows && tid == 0) issue(nxt, tm + (uint32_t)(nxt * CO));
        ok = mbar_wait_parity(&bar[cur], (uint32_t)(it >> 1) & 1u) && ok;  // row it's MMAs are done
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (it + 2 < nrows) prefetch(it + 2, cur);  // into the buffers row it's MMAs have finished reading
        if (!ok) continue;
        const uint32_t ta = tm + (uint32_t)(cur * CO) + ((uint32_t)(warp * 32) << 16);
        const size_t row = (size_t)b * (PROJ ? 1 : CO) * npix + (size_t)(z0 + it) * Nx + x;
        float y = PROJ ? sq2[CO] : 0.0f;
#pragma unroll
        for (int half = 0; half < CO / 32; ++half) {
            float v[32];
            tmem_ld32(ta + half * 32, v);
            if (PROJ) {
#pragma unroll
                for (int c = 0; c < 32; ++c) y = fmaf(sq2[half * 32 + c], gelu_as(v[c]), y);
            } else if (x < Nx) {
                __nv_bfloat16* dst = static_cast<__nv_bfloat16*>(out_) + row + (size_t)(half * 32) * npix;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    dst[(size_t)c * npix] = __float2bfloat16_rn(act == FNO_ACT_GELU ? gelu_as(v[c]) : v[c]);
            }
        }
        if (PROJ && x < Nx) static_cast<float*>(out_)[row] = y;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");  // ordered before the next row's barrier
    }
    if (!ok && tid == 0) atomicOr(&g_tc_err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"((uint32_t)(2 * CO))
                     : "memory");
}

// x transform on the tensor cores (BF16 input): D[128 rows x 32] = A B^T with
// A[r][x] = in[r0 + r][x] and B[n][x] = table[x][n] (zero for n >= 2 mx), K = Nx
// in chunks of 64 staged K-major (stride offset 1024 B between 8-row groups)
// into two alternating buffers; the MMAs of a chunk are committed to that
// buffer's mbarrier, which is waited on before the buffer is refilled.  Used
// for rows whose length is not a multiple of 8 (k_dft_x_tc2 below otherwise).
constexpr int kTcKc = 64;



__global__ void __launch_bounds__(128) k_dft_x_tc(long long rows, int Nx, int n2, const __nv_bfloat16* __restrict__ in,
                                                  const float* __restrict__ tab, float* __restrict__ out)
{
    constexpr int SA = 128 * kTcKc * 2, SB = 32 * kTcKc * 2;  // bytes per buffer
    __shared__ __align__(1024) unsigned char sA[2][SA];
    __shared__ __align__(1024) unsigned char sB[2][SB];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long r0 = (long long)blockIdx.x * 128;
    const long long row = r0 + tid;
    const bool rin = row < rows;
    const int nchunk = (Nx + kTcKc - 1) / kTcKc;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    bool ok = true;
    uint32_t tm = 0;
    for (int c = 0; c < nchunk; ++c) {
        const int buf = c & 1, k0 = c * kTcKc;
        if (c >= 2) ok = mbar_wait_parity(&bar[buf], (uint32_t)((c - 2) >> 1) & 1u) && ok;  // MMAs of chunk c-2 done
        // A: 128 rows x 64 x values
        if ((Nx & 7) == 0) {
            // 16-byte pieces, consecutive threads along a row (coalesced), copied as they are
            for (int e = tid; e < 128 * (kTcKc / 8); e += 128) {
                const int rr = e >> 3, kg = e & 7;
                const long long gr = r0 + rr;
                const int xk = k0 + 8 * kg;
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                if (gr < rows && xk < Nx) val = *reinterpret_cast<const uint4*>(in + gr * Nx + xk);
                *reinterpret_cast<uint4*>(sA[buf] + (rr >> 3) * 1024 + kg * 128 + (rr & 7) * 16) = val;
            }
        } else {
            for (int kg = 0; kg < kTcKc / 8; ++kg) {
                float f[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int xk = k0 + 8 * kg + j;
                    f[j] = (rin && xk < Nx) ? __bfloat162float(in[row * Nx + xk]) : 0.0f;
                }
                *reinterpret_cast<uint4*>(sA[buf] + (tid >> 3) * 1024 + kg * 128 + (tid & 7) * 16) = pack8_bf16(f);
            }
        }
        // B: 32 outputs x 64 x values of the table
        for (int e = tid; e < 32 * (kTcKc / 8); e += 128) {
            const int n = e & 31, kg = e >> 5;
            float g[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int xk = k0 + 8 * kg + j;
                g[j] = (n < n2 && xk < Nx) ? tab[(size_t)xk * n2 + n] : 0.0f;
            }
            *reinterpret_cast<uint4*>(sB[buf] + (n >> 3) * 1024 + kg * 128 + (n & 7) * 16) = pack8_bf16(g);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tm = tmem_base;
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < kTcKc / 16; ++j)
                umma_bf16(tm, umma_desc_sbo(su32(sA[buf]) + j * 256, 1024), umma_desc_sbo(su32(sB[buf]) + j * 256, 1024),
                          idesc, (c > 0 || j > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar[buf]))
                         : "memory");
        }
    }
    // the last chunk's commit covers all earlier MMAs
    {
        const int c = nchunk - 1;
        ok = mbar_wait_parity(&bar[c & 1], (uint32_t)(c >> 1) & 1u) && ok;
        if (nchunk >= 2) ok = mbar_wait_parity(&bar[(c - 1) & 1], (uint32_t)((c - 1) >> 1) & 1u) && ok;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        float v[32];
        tmem_ld32(tm + ((uint32_t)(warp * 32) << 16), v);
        const long long r = r0 + warp * 32 + lane;
        if (r < rows) {
#pragma unroll
            for (int n = 0; n < 32; ++n)
                if (n < n2) out[r * n2 + n] = v[n];
        }
    } else if (tid == 0) {
        atomicOr(&g_tc_err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tm) : "memory");
}

// The same x transform with the activations streamed through a kDxtStages-deep
// cp.async ring (Nx a multiple of 8): each 64-wide K chunk of the 128-row tile
// is copied in 16-byte pieces, a quarter-warp filling 128 contiguous bytes of
// shared memory (rows 8 g .. 8 g + 7 of one 8-column group), while the MMAs of
// earlier chunks run.  The table chunk (BF16, K-major) is double-buffered: its
// floats are loaded into registers one chunk ahead and stored just before the
// chunk's MMAs.  A stage is refilled once the MMAs that read it have committed.
constexpr int kDxtStages = 3;
constexpr int kDxtSA = 128 * kTcKc * 2, kDxtSB = 32 * kTcKc * 2;  // bytes per A stage, per B buffer
constexpr int kDxtSmem = kDxtStages * kDxtSA + 2 * kDxtSB;

__global__ void __launch_bounds__(128) k_dft_x_tc2(long long rows, int Nx, int n2, const __nv_bfloat16* __restrict__ in,
                                                   const float* __restrict__ tab, float* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* const sA = smem;                          // [kDxtStages][kDxtSA]
    unsigned char* const sB = smem + kDxtStages * kDxtSA;    // [2][kDxtSB]
    __shared__ __align__(8) uint64_t bar[kDxtStages];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long r0 = (long long)blockIdx.x * 128;
    const int nchunk = (Nx + kTcKc - 1) / kTcKc;

    if (tid == 0) {
        for (int j = 0; j < kDxtStages; ++j)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[j])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // chunk c -> stage c % kDxtStages: piece (g, kg, r8) = rows 8 g + r8, x = 64 c + 8 kg .. + 7
    auto issue_chunk = [&](int c) {
        if (c < nchunk) {
            unsigned char* a = sA + (c % kDxtStages) * kDxtSA;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = tid + 128 * u, r8 = e & 7, kg = (e >> 3) & 7, g = e >> 6;
                const long long gr = r0 + 8 * g + r8;
                const int x = c * kTcKc + 8 * kg;
                const bool ok = gr < rows && x < Nx;
                const __nv_bfloat16* src = in + (ok ? gr * Nx + x : 0);
                cp_async16(su32(a + g * 1024 + kg * 128 + r8 * 16), src, ok ? 16 : 0);
            }
        }
        cp_async_commit();  // one group per chunk slot, empty past the end
    };
    // table chunk c: thread owns pieces (n, kg) = (tid & 31, 2 (tid >> 5) + {0, 1}), 8 x each
    float tb[2][8];
    auto load_table = [&](int c) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int n = tid & 31, kg = 2 * (tid >> 5) + q;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int x = c * kTcKc + 8 * kg + j;
                tb[q][j] = (c < nchunk && n < n2 && x < Nx) ? tab[(size_t)x * n2 + n] : 0.0f;
            }
        }
    };
    auto store_table = [&](int c) {
        unsigned char* bb = sB + (c & 1) * kDxtSB;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int n = tid & 31, kg = 2 * (tid >> 5) + q;
            *reinterpret_cast<uint4*>(bb + (n >> 3) * 1024 + kg * 128 + (n & 7) * 16) = pack8_bf16(tb[q]);
        }
    };
#pragma unroll
    for (int c = 0; c < kDxtStages; ++c) issue_chunk(c);
    load_table(0);
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    bool ok = true;
    uint32_t tm = 0;
    for (int c = 0; c < nchunk; ++c) {
        const int st = c % kDxtStages;
        store_table(c);  // buffer c & 1 was last read by chunk c - 2's MMAs, waited for below
        cp_async_wait_stages();  // this thread's pieces of chunk c have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tm = tmem_base;
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < kTcKc / 16; ++j)
                umma_bf16(tm, umma_desc_sbo(su32(sA + st * kDxtSA) + j * 256, 1024),
                          umma_desc_sbo(su32(sB + (c & 1) * kDxtSB) + j * 256, 1024), idesc, (c > 0 || j > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar[st]))
                         : "memory");
        }
        if (c + 1 < nchunk) load_table(c + 1);  // in flight during the wait below
        // chunk c's MMAs done: stage st may be refilled and table buffer c & 1 rewritten
        ok = mbar_wait_parity(&bar[st], (uint32_t)(c / kDxtStages) & 1u) && ok;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_chunk(c + kDxtStages);
    }
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
        float v[32];
        tmem_ld32(tm + ((uint32_t)(warp * 32) << 16), v);
        const long long r = r0 + warp * 32 + lane;
        if (r < rows) {
            if ((n2 & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
#pragma unroll
                for (int n = 0; n < 32; n += 4)
                    if (n < n2) *reinterpret_cast<float4*>(out + r * n2 + n) = make_float4(v[n], v[n + 1], v[n + 2], v[n + 3]);
            } else {
#pragma unroll
                for (int n = 0; n < 32; ++n)
                    if (n < n2) out[r * n2 + n] = v[n];
            }
        }
    } else if (lane == 0) {
        atomicOr(&g_tc_err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tm) : "memory");
}

// --- projection head on the CUDA cores ------------------------------------------------
// out[b][p] = q2 + sum_h Q2[h] GELU(q1[h] + sum_i Q1[h][i] in[b][i][p]): the
// two pointwise layers of the head in one pass, the hidden channels kept in
// registers.  One thread per pixel; the weights in shared memory.
template <int CIMAX, typename Tin>
__global__ void __launch_bounds__(256) k_project(int ci, int H, long long npix, const Tin* __restrict__ in,
                                                 const float* __restrict__ Q1, const float* __restrict__ q1,
                                                 const float* __restrict__ Q2, const float* __restrict__ q2,
                                                 float* __restrict__ out)
{
    extern __shared__ float w[];  // Q1 [H][ci], then q1 [H] and Q2 [H]
    const int tid = threadIdx.x, b = blockIdx.y;
    for (int e = tid; e < H * ci; e += 256) w[e] = Q1[e];
    for (int h = tid; h < H; h += 256) {
        w[H * ci + h] = q1 ? q1[h] : 0.0f;
        w[H * ci + H + h] = Q2[h];
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * 256 + tid;
    if (p >= npix) return;
    float x[CIMAX];
#pragma unroll
    for (int i = 0; i < CIMAX; ++i) x[i] = i < ci ? ldf(in, ((size_t)b * ci + i) * npix + p) : 0.0f;
    float y = q2 ? q2[0] : 0.0f;
    for (int h = 0; h < H; ++h) {
        float acc = w[H * ci + h];
#pragma unroll
        for (int i = 0; i < CIMAX; ++i)
            if (i < ci) acc = fmaf(w[h * ci + i], x[i], acc);
        y = fmaf(w[H * ci + H + h], gelu(acc), y);
    }
    out[(size_t)b * npix + p] = y;
}

// --- weight gradients ---------------------------------------------------------------
// Block (k, b) sums pixels [k chunk, (k+1) chunk) of sample b into
// partial[b nchunk + k][o][0..cip) (column ci is the bias, fed by a constant
// 1); k_wgrad_reduce adds the blocks in index order.
// The host sizes chunk (a multiple of kWgTile, at least kWgMinChunk) so that
// the B x nchunk blocks fill the GPU in one wave.
constexpr int kWgTile = 64, kWgMinChunk = 512;

__host__ __device__ inline int wg_cip(int ci) { return ((ci + 1) + 3) & ~3; }
inline long long wg_max_blocks(int B, long long npix) { return B * ((npix + kWgMinChunk - 1) / kWgMinChunk); }

// Channel-major tiles of kWgTile pixels in shared memory (row stride kWgS,
// padded so that 8 consecutive rows start in different banks): rows 0..cop-1
// hold dU (zero past co), then cip rows of the input (row ci all ones, the
// bias; zero past it).  Thread (task, slice) accumulates 4 x 4 outputs, o =
// oq + u cop/4 and i = iq + v cip/4 (strided, so that the threads of a warp
// read consecutive rows: no bank conflicts), over the 4-pixel groups slice,
// slice + nslice, ... of each tile: 8 16-byte loads per 64 FMAs.
constexpr int kWgS = kWgTile + 4;
__host__ __device__ inline int wg_cop(int co) { return (co + 3) & ~3; }

__global__ void k_wgrad(int ci, int co, long long npix, long long chunk, const float* __restrict__ dU,
                        const float* __restrict__ in, float* __restrict__ partial)
{
    extern __shared__ __align__(16) float sm[];
    const int cip = wg_cip(ci), cop = wg_cop(co), g4 = cip / 4, ntask = (cop / 4) * g4;
    const int nslice = blockDim.x / ntask;  // divides kWgTile / 4 (host)
    const int nrow = cop + cip;
    // each tile buffer: [cop][kWgS] rows of dU, then [cip][kWgS] rows of the input
    const int b = blockIdx.y, tid = threadIdx.x;
    const int task = tid % ntask, slice = tid / ntask;
    const int oq = task / g4, iq = task % g4, og = cop / 4;
    const long long p0 = (long long)blockIdx.x * chunk, p1 = min(p0 + chunk, npix);
    const float* dUb = dU + (size_t)b * co * npix;
    const float* inb = in + (size_t)b * ci * npix;
    const bool vec = (npix & 3) == 0 && (reinterpret_cast<uintptr_t>(dU) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    // Tiles are double-buffered: the copies of tile k + 1 (cp.async, or plain
    // loads when the rows are not 16-byte aligned) are issued before the
    // arithmetic of tile k.
    float* buf[2] = {sm, sm + nrow * kWgS};
    const int npiece = nrow * (kWgTile / 4);
    auto fill = [&](float* dst, long long g) {
        const int n = (int)min((long long)kWgTile, p1 - g);
        for (int e = tid; e < npiece; e += blockDim.x) {
            const int r = e / (kWgTile / 4), p = 4 * (e % (kWgTile / 4));
            float* d = dst + r * kWgS + p;
            const float* src = r < co ? dUb + (size_t)r * npix
                                      : (r < cop ? nullptr : (r - cop < ci ? inb + (size_t)(r - cop) * npix : nullptr));
            if (src && vec) {
                const int bytes = 4 * max(0, min(4, n - p));
                cp_async16(su32(d), bytes ? src + g + p : src, bytes);  // zero fill past the pixels
            } else if (src) {
                *reinterpret_cast<float4*>(d) =
                    make_float4(p < n ? src[g + p] : 0.0f, p + 1 < n ? src[g + p + 1] : 0.0f,
                                p + 2 < n ? src[g + p + 2] : 0.0f, p + 3 < n ? src[g + p + 3] : 0.0f);
            } else {
                const float one = r - cop == ci ? 1.0f : 0.0f;
                *reinterpret_cast<float4*>(d) = make_float4(p < n ? one : 0.f, p + 1 < n ? one : 0.f,
                                                            p + 2 < n ? one : 0.f, p + 3 < n ? one : 0.f);
            }
        }
        cp_async_commit();
    };
    if (p0 < p1) fill(buf[0], p0);
    int cur = 0;
    for (long long g = p0; g < p1; g += kWgTile, cur ^= 1) {
        if (g + kWgTile < p1) {
            fill(buf[cur ^ 1], g + kWgTile);  // the buffer tile k - 1 used (barrier below)
            cp_async_wait_prev();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const float* tD = buf[cur];
        const float* tI = buf[cur] + cop * kWgS;
        if (slice < nslice) {
            for (int q = slice; q < kWgTile / 4; q += nslice) {
                float4 d[4], x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) d[u] = *reinterpret_cast<const float4*>(tD + (oq + u * og) * kWgS + 4 * q);
#pragma unroll
                for (int v = 0; v < 4; ++v) x[v] = *reinterpret_cast<const float4*>(tI + (iq + v * g4) * kWgS + 4 * q);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        acc[u][v] = fmaf(d[u].x, x[v].x, acc[u][v]);
                        acc[u][v] = fmaf(d[u].y, x[v].y, acc[u][v]);
                        acc[u][v] = fmaf(d[u].z, x[v].z, acc[u][v]);
                        acc[u][v] = fmaf(d[u].w, x[v].w, acc[u][v]);
                    }
            }
        }
        __syncthreads();
    }
    // sum the slices in index order through shared memory, then one row per block
    float* red = sm;  // [nslice][cop][cip]
    if (slice < nslice) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) red[((size_t)slice * cop + oq + u * og) * cip + iq + v * g4] = acc[u][v];
    }
    __syncthreads();
    const size_t blk = (size_t)b * gridDim.x + blockIdx.x;
    for (int e = tid; e < co * cip; e += blockDim.x) {
        const int o = e / cip, i = e - o * cip;
        float t = 0.0f;
        for (int k = 0; k < nslice; ++k) t += red[((size_t)k * cop + o) * cip + i];
        partial[(blk * co + o) * cip + i] = t;
    }
}

__global__ void k_wgrad_reduce(int ci, int co, long long nblk, const float* __restrict__ partial,
                               float* __restrict__ dM, float* __restrict__ dbias)
{
    // one warp per output: lane l sums blocks l, l + 32, ... in order, then a
    // fixed shuffle tree (the same order on every run)
    const int cip = wg_cip(ci);
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (t >= co * (ci + 1)) return;
    const int o = t / (ci + 1), i = t - o * (ci + 1);
    float s = 0.0f;
    for (long long k = lane; k < nblk; k += 32) s += partial[((size_t)k * co + o) * cip + i];
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) s += __shfl_down_sync(0xffffffffu, s, w);
    if (lane == 0) {
        if (i < ci) dM[(size_t)o * ci + i] = s;
        else if (dbias) dbias[o] = s;
    }
}

// --- elementwise ------------------------------------------------------------------------

__global__ void k_gelu_bwd(long long n, const float* __restrict__ dout, const float* __restrict__ pre,
                           float* __restrict__ dpre)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dpre[i] = dout[i] * gelu_grad(pre[i]);
}

// The same, 4 elements per thread and 16-byte accesses (n4 = n / 4, aligned arrays).
__global__ void k_gelu_bwd4(long long n4, const float4* __restrict__ dout, const float4* __restrict__ pre,
                            float4* __restrict__ dpre)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 d = dout[i], x = pre[i];
        dpre[i] = make_float4(d.x * gelu_grad(x.x), d.y * gelu_grad(x.y), d.z * gelu_grad(x.z), d.w * gelu_grad(x.w));
    }
}

constexpr int kMseBlocks = 256;

__global__ void __launch_bounds__(256) k_mse(long long n, const float* __restrict__ pred,
                                             const float* __restrict__ target, float* __restrict__ dpred,
                                             double* __restrict__ part)
{
    __shared__ double s[256];
    double acc = 0.0;
    const float scale = (float)(2.0 / (double)n);
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
        const float r = pred[i] - target[i];
        acc += (double)r * (double)r;
        if (dpred) dpred[i] = scale * r;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_mse_final(long long n, const double* __restrict__ part, double* __restrict__ loss)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < kMseBlocks; ++k) s += part[k];
    *loss = s / (double)n;
}

// omb1 = 1 - b1 and omb2 = 1 - b2 are formed in double and then rounded: 1 - b2
// formed in float from b2 = 0.999f would be off by 1.3e-5 relative.
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float omb1, float omb2, float eps, float c1,
                       float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + omb1 * gi;
        const float vi = b2 * v[i] + omb2 * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

long long nblk128(long long rows) { return (rows + 127) / 128; }

int g_tensor_cores = 1;  // fno_combine's BF16 path uses tcgen05 when set and the shape allows

wave_status_t launched()
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return WAVE_ERR_CUDA;
    }
    return WAVE_OK;
}

bool modes_ok(int Nz, int Nx, int mz, int mx)
{
    return Nz > 0 && Nx > 0 && mz >= 1 && mz <= 32 && 2 * mz <= Nz && mx >= 1 && mx <= 16 && 2 * mx <= Nx;
}

template <int CIMAX, typename Tin, typename Tout>
void combine_launch(int B, int ci, int co, int Nz, int Nx, int mx, const void* in, const float* M, int mt,
                    const float* bias, const float* T, const float* tab, int act, float* pre, void* out,
                    cudaStream_t s)
{
    const size_t smem = (size_t)(co * CIMAX + co * 32 + co) * sizeof(float);
    dim3 grid((Nx + 255) / 256, Nz, B);
    k_combine<CIMAX, Tin, Tout><<<grid, 256, smem, s>>>(ci, co, Nz, Nx, mx, static_cast<const Tin*>(in), M, mt, bias,
                                                         T, tab, act, pre, static_cast<Tout*>(out));
}

// Resident CTAs of k_combine_tc<CO, PROJ> on the whole device (per device, found
// once), from the kernel's registers and shared memory against the SM's limits.
template <int CO, bool PROJ>
int tc_slots()
{
    static int slots[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (slots[dev] == 0) {
        cudaFuncAttributes fa;
        int nsm = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0, thr_sm = 0;
        // all of the unified L1 as shared memory
        const int smem_dyn = tc_smem_bytes(CO, PROJ);
        if (cudaFuncSetAttribute(k_combine_tc<CO, PROJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_dyn) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_combine_tc<CO, PROJ>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, k_combine_tc<CO, PROJ>) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
            return 0;
        const int smem_cta = smem_dyn + (int)fa.sharedSizeBytes + smem_rsv;
        const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
        int occ = std::min(smem_sm / smem_cta, thr_sm / 128);
        if (regs_warp > 0) occ = std::min(occ, regs_sm / (4 * regs_warp));
        // a CTA holds 2 CO columns of tensor memory out of 512
        occ = std::min(occ, 512 / (2 * CO));
        if (occ < 1) return 0;
        slots[dev] = nsm * occ;
    }
    return slots[dev];
}

// One wave: rows per CTA so that the (x tiles) x (row chunks) x B grid fills
// the resident slots once.
template <int CO, bool PROJ>
wave_status_t combine_tc_launch(int B, int Nz, int Nx, int mx, const void* in, const float* M, const float* bias,
                                const float* T, const float* tab, int act, const float* Q2, const float* q2, void* out,
                                cudaStream_t s)
{
    const int slots = tc_slots<CO, PROJ>();
    if (slots <= 0) return WAVE_ERR_CUDA;
    const long long xt = (Nx + 127) / 128, tiles = xt * Nz * (long long)B;
    int rw = (int)std::min<long long>(Nz, std::max<long long>(1, (tiles + slots - 1) / slots));
    while (rw < Nz && xt * ((Nz + rw - 1) / rw) * B > slots) ++rw;  // rounding must not spill into a second wave
    dim3 grid((unsigned)xt, (unsigned)((Nz + rw - 1) / rw), B);
    k_combine_tc<CO, PROJ><<<grid, 128, tc_smem_bytes(CO, PROJ), s>>>(
        Nz, Nx, mx, rw, static_cast<const __nv_bfloat16*>(in), M, bias, T, tab, act, Q2, q2, out);
    return launched();
}

template <typename Tin, typename Tout>
void combine_dispatch(int B, int ci, int co, int Nz, int Nx, int mx, const void* in, const float* M, int mt,
                      const float* bias, const float* T, const float* tab, int act, float* pre, void* out,
                      cudaStream_t s)
{
    const long long npix = (long long)Nz * Nx;
    const bool al16 = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) |
                        reinterpret_cast<uintptr_t>(pre)) & 15) == 0;
    if (!T && ci <= 4 && (npix & 3) == 0 && al16 && npix / 4 / 256 < 0x7fffffffLL) {
        const dim3 grid((unsigned)((npix / 4 + 255) / 256), B);
        k_combine_px4<4, Tin, Tout><<<grid, 256, 0, s>>>(ci, co, npix, static_cast<const Tin*>(in), M, mt, bias, act,
                                                         pre, static_cast<Tout*>(out));
        return;
    }
    if constexpr (std::is_same<Tin, float>::value) {
        if ((co == 32 || co == 64) && ci <= 64 && (!T || mx <= 16) && (Nx & 3) == 0 && al16 &&
            (reinterpret_cast<uintptr_t>(T) & 15) == 0) {
            const size_t smem = (size_t)(ci * co + (T ? 2 * 32 * co : 0) + 2 * ci * kRtS + (T ? 32 * kRtS : 0) + co) *
                                sizeof(float);
            const dim3 grid((unsigned)((Nx + kRtP - 1) / kRtP), (unsigned)((Nz + kRzRows - 1) / kRzRows), (unsigned)B);
            if (co == 32) {
                cudaFuncSetAttribute(k_combine_rz<32, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                k_combine_rz<32, Tout><<<grid, 128, smem, s>>>(ci, Nz, Nx, mx, static_cast<const float*>(in), M, mt, bias,
                                                               T, tab, act, pre, static_cast<Tout*>(out));
            } else {
                cudaFuncSetAttribute(k_combine_rz<64, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                k_combine_rz<64, Tout><<<grid, 256, smem, s>>>(ci, Nz, Nx, mx, static_cast<const float*>(in), M, mt, bias,
                                                               T, tab, act, pre, static_cast<Tout*>(out));
            }
            return;
        }
    }
    if ((co == 32 || co == 64) && ci <= 64 && (!T || mx <= 16)) {
        const int K = ci + (T ? 32 : 0);
        const size_t smem = (size_t)(K * co + K * kRtS + co) * sizeof(float);
        const dim3 grid((unsigned)((Nx + kRtP - 1) / kRtP), (unsigned)Nz, (unsigned)B);
        if (co == 32) {
            cudaFuncSetAttribute(k_combine_rt<32, Tin, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_combine_rt<32, Tin, Tout><<<grid, 128, smem, s>>>(ci, Nz, Nx, mx, static_cast<const Tin*>(in), M, mt, bias,
                                                                 T, tab, act, pre, static_cast<Tout*>(out));
        } else {
            cudaFuncSetAttribute(k_combine_rt<64, Tin, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_combine_rt<64, Tin, Tout><<<grid, 256, smem, s>>>(ci, Nz, Nx, mx, static_cast<const Tin*>(in), M, mt, bias,
                                                                 T, tab, act, pre, static_cast<Tout*>(out));
        }
        return;
    }
    if (ci <= 4) combine_launch<4, Tin, Tout>(B, ci, co, Nz, Nx, mx, in, M, mt, bias, T, tab, act, pre, out, s);
    else if (ci <= 8) combine_launch<8, Tin, Tout>(B, ci, co, Nz, Nx, mx, in, M, mt, bias, T, tab, act, pre, out, s);
    else if (ci <= 16) combine_launch<16, Tin, Tout>(B, ci, co, Nz, Nx, mx, in, M, mt, bias, T, tab, act, pre, out, s);
    else if (ci <= 32) combine_launch<32, Tin, Tout>(B, ci, co, Nz, Nx, mx, in, M, mt, bias, T, tab, act, pre, out, s);
    else combine_launch<64, Tin, Tout>(B, ci, co, Nz, Nx, mx, in, M, mt, bias, T, tab, act, pre, out, s);
}

}  // namespace
}  // namespace wave

using namespace wave;

extern "C" {

wave_status_t fno_tables(int Nz, int Nx, int mz, int mx, float* tx_fwd, float* tx_inv, float* tx_bwd, float* tx_adj,
                         float* tz, void* stream)
{
    if (!modes_ok(Nz, Nx, mz, mx) || !tx_fwd || !tx_inv || !tx_bwd || !tx_adj || !tz) return WAVE_ERR_ARG;
    const int n = max(Nx * mx, Nz * 2 * mz);
    k_tables<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(Nz, Nx, mz, mx, tx_fwd, tx_inv, tx_bwd, tx_adj, tz);
    return launched();
}

wave_status_t fno_dft_x(long long rows, int Nx, int mx, const void* in, int in_bf16, const float* table, float* out,
                        void* stream)
{
    if (rows < 0 || Nx <= 0 || mx < 1 || mx > 16 || !in || !table || !out) return WAVE_ERR_ARG;
    if (rows == 0) return WAVE_OK;
    const long long nblk = (rows + kDxRows - 1) / kDxRows;
    if (nblk > 0x7fffffffLL) return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (in_bf16 && g_tensor_cores) {
        if ((Nx & 7) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
            static bool attr[64] = {false};  // per device
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WAVE_ERR_CUDA;
            if (!attr[dev]) {
                if (cudaFuncSetAttribute(k_dft_x_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, kDxtSmem) != cudaSuccess)
                    return WAVE_ERR_CUDA;
                attr[dev] = true;
            }
            k_dft_x_tc2<<<(unsigned)nblk128(rows), 128, kDxtSmem, s>>>(
                rows, Nx, 2 * mx, static_cast<const __nv_bfloat16*>(in), table, out);
        } else {
            k_dft_x_tc<<<(unsigned)nblk128(rows), 128, 0, s>>>(rows, Nx, 2 * mx, static_cast<const __nv_bfloat16*>(in),
                                                               table, out);
        }
        return launched();
    }
    if (in_bf16)
        k_dft_x<__nv_bfloat16><<<(unsigned)nblk, 256, 0, s>>>(rows, Nx, 2 * mx, static_cast<const __nv_bfloat16*>(in),
                                                              table, out);
    else
        k_dft_x<float><<<(unsigned)nblk, 256, 0, s>>>(rows, Nx, 2 * mx, static_cast<const float*>(in), table, out);
    return launched();
}

wave_status_t fno_dft_z(int nb, int Nz, int mz, int mx, const float* in, const float* tz, float* out, void* stream)
{
    if (nb < 0 || !modes_ok(Nz, 2 * mx, mz, mx) || !in || !tz || !out) return WAVE_ERR_ARG;
    if (nb == 0) return WAVE_OK;
    k_dft_z<<<dim3(nb, (2 * mz + 15) / 16), 256, 0, (cudaStream_t)stream>>>(Nz, 2 * mz, mx, reinterpret_cast<const float2*>(in),
                                                  reinterpret_cast<const float2*>(tz), reinterpret_cast<float2*>(out));
    return launched();
}

wave_status_t fno_idft_z(int nb, int Nz, int mz, int mx, const float* in, const float* tz, float* out, void* stream)
{
    if (nb < 0 || !modes_ok(Nz, 2 * mx, mz, mx) || !in || !tz || !out) return WAVE_ERR_ARG;
    if (nb == 0) return WAVE_OK;
    dim3 grid(nb, (Nz + 63) / 64);
    k_idft_z<<<grid, 256, 0, (cudaStream_t)stream>>>(Nz, 2 * mz, mx, reinterpret_cast<const float2*>(in),
                                                     reinterpret_cast<const float2*>(tz),
                                                     reinterpret_cast<float2*>(out));
    return launched();
}

wave_status_t fno_mix(int B, int Ci, int Co, int nmode, const float* X, const float* R, float* Y, void* stream)
{
    if (B < 0 || Ci < 1 || Co < 1 || Ci > 64 || Co > 64 || nmode < 1 || !X || !R || !Y) return WAVE_ERR_ARG;
    const long long n = (long long)B * Co * nmode;
    if (n == 0) return WAVE_OK;
    k_mix<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        B, Ci, Co, nmode, reinterpret_cast<const float2*>(X), reinterpret_cast<const float2*>(R),
        reinterpret_cast<float2*>(Y));
    return launched();
}

wave_status_t fno_mix_idft_z(int B, int Ci, int Co, int Nz, int mz, int mx, const float* X, const float* R,
                             const float* tz, float* out, void* stream)
{
    if (B < 0 || Ci < 1 || Co < 1 || Ci > 64 || Co > 64 || !modes_ok(Nz, 2 * mx, mz, mx) || !X || !R || !tz || !out)
        return WAVE_ERR_ARG;
    const long long nb = (long long)B * Co;
    if (nb == 0) return WAVE_OK;
    if (nb > 0x7fffffffLL) return WAVE_ERR_ARG;
    k_mix_idft_z<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>(
        Ci, Co, Nz, 2 * mz, mx, reinterpret_cast<const float2*>(X), reinterpret_cast<const float2*>(R),
        reinterpret_cast<const float2*>(tz), reinterpret_cast<float2*>(out));
    return launched();
}

wave_status_t fno_mix_backward(int B, int Ci, int Co, int nmode, const float* X, const float* R, const float* dY,
                               float* dX, float* dR, void* stream)
{
    if (B < 0 || Ci < 1 || Co < 1 || Ci > 64 || Co > 64 || nmode < 1 || !dY) return WAVE_ERR_ARG;
    if ((dX && !R) || (dR && !X)) return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (dX && B > 0) {
        const long long n = (long long)B * Ci * nmode;
        k_mix_dx<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B, Ci, Co, nmode, reinterpret_cast<const float2*>(dY),
                                                            reinterpret_cast<const float2*>(R),
                                                            reinterpret_cast<float2*>(dX));
    }
    if (dR) {
        const long long n = (long long)Ci * Co * nmode;
        k_mix_dr<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B, Ci, Co, nmode, reinterpret_cast<const float2*>(X),
                                                            reinterpret_cast<const float2*>(dY),
                                                            reinterpret_cast<float2*>(dR));
    }
    return launched();
}

wave_status_t fno_combine(int B, int Ci, int Co, int Nz, int Nx, int mx, const void* in, int in_bf16,
                          const float* M, int m_trans, const float* bias, const float* T, const float* table,
                          int act, float* pre, void* out, int out_bf16, void* stream)
{
    if (B < 0 || Ci < 1 || Ci > 64 || Co < 1 || Co > 64 || Nz < 1 || Nx < 1 || !in || !M || !out) return WAVE_ERR_ARG;
    if (T && (!table || mx < 1 || mx > 16)) return WAVE_ERR_ARG;
    if (act != FNO_ACT_NONE && act != FNO_ACT_GELU) return WAVE_ERR_ARG;
    if (B == 0) return WAVE_OK;
    if (Nz > 65535 || B > 65535) return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int mxe = T ? mx : 1;
    if (g_tensor_cores && in_bf16 && out_bf16 && !pre && !m_trans && Ci == kTcCi && (Co == 32 || Co == 64)) {
        if (Co == 32)
            return combine_tc_launch<32, false>(B, Nz, Nx, mxe, in, M, bias, T, table, act, nullptr, nullptr, out, s);
        return combine_tc_launch<64, false>(B, Nz, Nx, mxe, in, M, bias, T, table, act, nullptr, nullptr, out, s);
    }
    if (in_bf16 && out_bf16)
        combine_dispatch<__nv_bfloat16, __nv_bfloat16>(B, Ci, Co, Nz, Nx, mxe, in, M, m_trans, bias, T, table, act, pre,
                                                       out, s);
    else if (in_bf16)
        combine_dispatch<__nv_bfloat16, float>(B, Ci, Co, Nz, Nx, mxe, in, M, m_trans, bias, T, table, act, pre, out, s);
    else if (out_bf16)
        combine_dispatch<float, __nv_bfloat16>(B, Ci, Co, Nz, Nx, mxe, in, M, m_trans, bias, T, table, act, pre, out, s);
    else
        combine_dispatch<float, float>(B, Ci, Co, Nz, Nx, mxe, in, M, m_trans, bias, T, table, act, pre, out, s);
    return launched();
}

wave_status_t fno_project(int B, int Ci, int H, int Nz, int Nx, const void* in, int in_bf16, const float* Q1,
                          const float* q1, const float* Q2, const float* q2, float* out, void* stream)
{
    if (B < 0 || Ci < 1 || Ci > 64 || H < 1 || H > 64 || Nz < 1 || Nx < 1 || !in || !Q1 || !Q2 || !out)
        return WAVE_ERR_ARG;
    if (B == 0) return WAVE_OK;
    if (B > 65535 || Nz > 65535) return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g_tensor_cores && in_bf16 && Ci == kTcCi && (H == 32 || H == 64)) {
        if (H == 32)
            return combine_tc_launch<32, true>(B, Nz, Nx, 1, in, Q1, q1, nullptr, nullptr, FNO_ACT_GELU, Q2, q2, out, s);
        return combine_tc_launch<64, true>(B, Nz, Nx, 1, in, Q1, q1, nullptr, nullptr, FNO_ACT_GELU, Q2, q2, out, s);
    }
    const long long npix = (long long)Nz * Nx, nblk = (npix + 255) / 256;
    if (nblk > 0x7fffffffLL) return WAVE_ERR_ARG;
    const dim3 grid((unsigned)nblk, B);
    const size_t smem = (size_t)(H * Ci + 2 * H) * sizeof(float);
#define WAVE_PROJECT(CIMAX)                                                                                        \
    do {                                                                                                           \
        if (in_bf16)                                                                                               \
            k_project<CIMAX, __nv_bfloat16><<<grid, 256, smem, s>>>(Ci, H, npix,                                   \
                                                                     static_cast<const __nv_bfloat16*>(in), Q1, q1, \
                                                                     Q2, q2, out);                                 \
        else                                                                                                       \
            k_project<CIMAX, float><<<grid, 256, smem, s>>>(Ci, H, npix, static_cast<const float*>(in), Q1, q1, Q2, \
                                                             q2, out);                                             \
    } while (0)
    if (Ci <= 4) WAVE_PROJECT(4);
    else if (Ci <= 8) WAVE_PROJECT(8);
    else if (Ci <= 16) WAVE_PROJECT(16);
    else if (Ci <= 32) WAVE_PROJECT(32);
    else WAVE_PROJECT(64);
#undef WAVE_PROJECT
    return launched();
}

wave_status_t fno_set_tensor_cores(int on)
{
    if (on != 0 && on != 1) return WAVE_ERR_ARG;
    g_tensor_cores = on;
    return WAVE_OK;
}

wave_status_t fno_tensor_core_status(void)
{
    int h = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_tc_err, sizeof(int)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(int)) != cudaSuccess)
        return WAVE_ERR_CUDA;
    return h ? WAVE_ERR_TIMEOUT : WAVE_OK;
}

size_t fno_wgrad_work_floats(int B, int Ci, int Co, long long npix)
{
    if (B < 0 || Ci < 1 || Co < 1 || npix < 0) return 0;
    return (size_t)wg_max_blocks(B, npix) * Co * wg_cip(Ci);
}

wave_status_t fno_wgrad(int B, int Ci, int Co, long long npix, const float* dU, const float* in, float* dM,
                        float* dbias, float* work, void* stream)
{
    if (B < 0 || Ci < 1 || Ci > 64 || Co < 1 || Co > 64 || npix < 0 || !dU || !in || !dM || !work)
        return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (wg_max_blocks(B, npix) > 0x7fffffffLL || B > 65535) return WAVE_ERR_ARG;
    long long nblk = 0;
    if (npix > 0 && B > 0) {
        // 4 x 4 output blocks times pixel slices (a power of two dividing the
        // tile's 16 groups of 4), about 256 threads
        const int ntask = (wg_cop(Co) / 4) * (wg_cip(Ci) / 4);
        int nslice = 1;
        while (nslice < kWgTile / 4 && ntask * nslice * 2 <= 320) nslice *= 2;
        const int threads = ntask * nslice;
        const size_t tile = (size_t)(wg_cop(Co) + wg_cip(Ci)) * kWgS;
        const size_t red = (size_t)nslice * wg_cop(Co) * wg_cip(Ci);
        const size_t smem = std::max(2 * tile, red) * sizeof(float);
        cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // chunks per sample so that all blocks are resident at once
        int per = 0, dev = 0, nsm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wgrad, threads, smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        (void)cudaGetLastError();
        const long long want = std::max(1LL, (long long)std::max(per, 1) * nsm / B);
        long long chunk = (npix + want - 1) / want;
        chunk = std::max<long long>(kWgMinChunk, (chunk + kWgTile - 1) / kWgTile * kWgTile);
        const long long nchunk = (npix + chunk - 1) / chunk;
        nblk = (long long)B * nchunk;
        const dim3 grid((unsigned)nchunk, B);
        k_wgrad<<<grid, threads, smem, s>>>(Ci, Co, npix, chunk, dU, in, work);
    }
    const int nout = Co * (Ci + 1);
    k_wgrad_reduce<<<(nout + 7) / 8, 256, 0, s>>>(Ci, Co, nblk, work, dM, dbias);
    return launched();
}

wave_status_t fno_gelu_backward(long long n, const float* dout, const float* pre, float* dpre, void* stream)
{
    if (n < 0 || !dout || !pre || !dpre) return WAVE_ERR_ARG;
    if (n == 0) return WAVE_OK;
    if ((n & 3) == 0 && ((reinterpret_cast<uintptr_t>(dout) | reinterpret_cast<uintptr_t>(pre) |
                          reinterpret_cast<uintptr_t>(dpre)) & 15) == 0) {
        const long long nb = std::min<long long>((n / 4 + 255) / 256, 16384);
        k_gelu_bwd4<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>(n / 4, reinterpret_cast<const float4*>(dout),
                                                                   reinterpret_cast<const float4*>(pre),
                                                                   reinterpret_cast<float4*>(dpre));
        return launched();
    }
    const long long nb = std::min<long long>((n + 255) / 256, 4096);
    k_gelu_bwd<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>(n, dout, pre, dpre);
    return launched();
}

wave_status_t fno_mse(long long n, const float* pred, const float* target, float* dpred, double* loss, double* work,
                      void* stream)
{
    if (n <= 0 || !pred || !target || !loss || !work) return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_mse<<<kMseBlocks, 256, 0, s>>>(n, pred, target, dpred, work);
    k_mse_final<<<1, 32, 0, s>>>(n, work, loss);
    return launched();
}

wave_status_t fno_adam(long long n, float* p, const float* g, float* m, float* v, double lr, double b1, double b2,
                       double eps, int t, void* stream)
{
    if (n < 0 || t < 1 || !p || !g || !m || !v) return WAVE_ERR_ARG;
    if (n == 0) return WAVE_OK;
    const float c1 = (float)(1.0 - pow(b1, t)), c2 = (float)(1.0 - pow(b2, t));
    const long long nb = std::min<long long>((n + 255) / 256, 4096);
    k_adam<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, (float)lr, (float)b1, (float)b2,
                                                           (float)(1.0 - b1), (float)(1.0 - b2), (float)eps, c1, c2);
    return launched();
}

}  // extern "C"
