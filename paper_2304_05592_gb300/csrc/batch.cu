// batch.cu -- FWI gradients of an uneven batch of independent 2D problems
// (each with its own grid, model, time axis, sources and receivers) in two
// persistent launches: one forward sweep that stores every level in BF16 or
// FP32, and one adjoint sweep with the imaging condition.
//
// The CTAs of a sweep stay resident (cooperative launch) and each owns a fixed
// set of 128 x TZ tiles of all problems.  A tile advances one time step as
// soon as its neighbours (same problem) have finished the previous one: tiles
// publish the number of steps they completed in a flag word, and waiters poll
// those words with a bounded wait.  Problems with few time steps simply drop
// out of the sweep; there is no global barrier between steps.
//
// Two sweep kernels exist, chosen per batch by wave_autotune_batch:
//  * kind 0 (direct): each CTA loads a tile's halo with plain loads through L2,
//    computes and publishes it, one tile after the other;
//  * kind 1 (producer / consumer): one producer warp waits for the neighbour
//    flags of the CTA's next tiles and fetches each tile's halo, previous
//    level, model (and in the adjoint the stored forward level and the
//    gradient accumulator) by TMA into a ring of NS shared-memory stages, so
//    that loads of later tiles overlap the arithmetic of the current one;
//    BZ consumer warps run the stencil with the 9-row z window of each
//    thread's 4 x 4... RB rows kept in registers; one releaser warp publishes
//    finished tiles (its GPU-scope fence stays off the consumers' path).
// Tile height TZ, consumer warps BZ, stage count NS and CTAs per SM are the
// tuned parameters.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "internal.h"
#include "stencil.cuh"
#include "tma.cuh"

namespace wave {

// TMA descriptors of one problem (indices into its block of kMaps maps).
enum : int {
    kMapHaloW = 0,  // + (level & 1): halo box of the forward levels w[0], w[1]
    kMapTileW = 2,  // + (level & 1): tile box of the forward levels
    kMapHaloA = 4,  // + (level & 1): halo box of the adjoint levels a[0], a[1]
    kMapTileA = 6,  // + (level & 1): tile box of the adjoint levels
    kMapKap = 8,    // tile box of the model
    kMapG = 9,      // tile box of the gradient accumulator
    kMapStore = 10, // (x, z, n) tile box of the wavefield store (BF16 or FP32)
    kMaps = 11
};

struct BProb {
    int Nx, Nz, P, nx, nz, nb, nt, ncx, ncz, ntz, tile0;
    long long cell;
    float ceps;
    float* w[2];  // forward levels: u^n lives in w[n & 1]
    float* a[2];  // adjoint levels: mu^k lives in a[k & 1]
    const float* kap;
    __nv_bfloat16* st16;  // [nt][cell] store (BF16) or null
    float* st32;          // [nt][cell] store (FP32) or null
    float* g;             // [cell] gradient accumulator
    const float* wavelet; // [nt][nsrc]
    const float* dobs;    // [nt][nrec]
    float* dsyn;          // [nt][nrec]
    float* slots;         // [nt][ntap of the receivers]
    TapList src, rec;
};

namespace {

// Sweep variants: kind 0 is the direct kernel (TZ = 32, BZ thread rows);
// kind 1 the producer / consumer kernel with TZ rows per tile, BZ consumer
// warps, NS stages and at most `cap` CTAs per SM (0: as many as fit).
struct BVariant {
    int kind, TZ, BZ, NS, cap;
};
// (Stages of the adjoint sweep hold five arrays: 45.8 KB at TZ = 16, 87.3 KB at TZ = 32.)
const BVariant kBatchVariants[] = {{0, 32, 8, 0, 0},  {1, 16, 4, 2, 0}, {1, 16, 4, 3, 0}, {1, 32, 8, 2, 0},
                                   {1, 32, 4, 2, 0},  {1, 16, 2, 3, 0}, {1, 16, 8, 2, 0}, {1, 16, 4, 2, 2},
                                   {1, 16, 8, 3, 0},  {1, 16, 2, 2, 0}, {1, 16, 8, 2, 1}};
constexpr int kNumBatchVariants = sizeof(kBatchVariants) / sizeof(kBatchVariants[0]);
constexpr int kDefaultBatchVariant = 1;
constexpr int kMinTZ = 16;  // smallest tile height of any variant (sizes the tile tables)

constexpr int kPollLimit = 1 << 22;
constexpr uint64_t kFlagWaitNs = 2000000000ull;  // a neighbour that has not moved for 2 s has failed
constexpr uint64_t kStageWaitNs = 4000000000ull; // longer than any flag wait a stage can be held up by

__device__ __forceinline__ float4 ldcg4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ int bdepth(int i, int nb, int n)
{
    int d = max(nb - i, i - (nb + n - 1));
    return max(d, 0);
}

// Polls flag >= want through L2; false on timeout or when another CTA aborted.
__device__ bool wait_flag(int* flag, int want, int* abort_word)
{
    for (int it = 0; it < kPollLimit; ++it) {
        if (atomicAdd(flag, 0) >= want) return true;
        if ((it & 255) == 255 && atomicAdd(abort_word, 0) != 0) return false;
    }
    return false;
}

// The same with an acquire load and a wall-clock bound (kind 1).
__device__ bool wait_flag_acq(const int* flag, int want, const int* abort_word)
{
    const uint64_t t0 = global_ns();
    for (int it = 0;; ++it) {
        if (ld_acquire_gpu(flag) >= want) return true;
        if ((it & 63) == 63) {
            if (ld_acquire_gpu(abort_word) != 0) return false;
            if (global_ns() - t0 > kFlagWaitNs) return false;
        }
    }
}

// Bounded wait on an mbarrier phase that also gives up when the sweep aborts.
__device__ bool mbar_wait_abort(uint64_t* b, uint32_t parity, const int* abort_word, uint64_t limit_ns)
{
    const uint64_t t0 = global_ns();
    for (int it = 0;; ++it) {
        if (mbar_try(b, parity)) return true;
        if ((it & 63) == 63) {
            if (ld_acquire_gpu(abort_word) != 0) return false;
            if (global_ns() - t0 > limit_ns) return false;
        }
    }
}

// One thread runs the sweep's bounded wait on a caller-given flag.
__global__ void k_wait_probe(int* flag, int want, int* abort_word, int* err)
{
    if (threadIdx.x == 0 && !wait_flag(flag, want, abort_word)) atomicOr(err, kErrTimeout);
}

// Sparse part of a tile's step, run by nthr threads (index tid) after the
// tile's points are written: injection (forward: sources with q^n; adjoint:
// the residual at the receivers) into un, then in the forward sweep the
// receiver gathers of u^{n+1}.  bar() synchronises those threads.
template <bool ADJ, class Bar>
__device__ __forceinline__ void batch_sparse(const BProb& p, int tz, int tx, int TZ, int n, float* un, int tid,
                                             int nthr, Bar bar)
{
    const TapList& inj = ADJ ? p.rec : p.src;
    const int kcell = TZ / kTZc2;
    const int cbase = tx * p.ncz;
    const int c0 = tz * kcell, c1 = min(c0 + kcell, p.ncz);
    const int ib = inj.ntap > 0 ? inj.cell_start[cbase + c0] : 0, ie = inj.ntap > 0 ? inj.cell_start[cbase + c1] : 0;
    const int gb = !ADJ && p.rec.ntap > 0 ? p.rec.cell_start[cbase + c0] : 0;
    const int ge = !ADJ && p.rec.ntap > 0 ? p.rec.cell_start[cbase + c1] : 0;
    if (ie > ib) {
        for (int j = ib + tid; j < ie; j += nthr) {
            const int i = inj.idx[j];
            if (j > ib && inj.idx[j - 1] == i) continue;
            float add = 0.0f;
            for (int jj = j; jj < ie && inj.idx[jj] == i; ++jj) {
                const long long ai = (long long)inj.ab[jj] + (long long)n * inj.npts;
                const float amp = ADJ ? p.dsyn[ai] - p.dobs[ai] : p.wavelet[ai];
                add = fmaf(inj.fac[jj], amp, add);
            }
            const float v = __ldcg(un + i) + add;
            un[i] = v;
            if (!ADJ) {
                const long long so = (long long)(n + 1) * p.cell + i;
                if (p.st16) p.st16[so] = __float2bfloat16_rn(v);
                else p.st32[so] = v;
            } else {
                const long long so = (long long)n * p.cell + i;
                const float uf = p.st16 ? __bfloat162float(p.st16[so]) : p.st32[so];
                p.g[i] = __ldcg(p.g + i) - uf * add;
            }
        }
    }
    if (ge > gb) {
        if (ie > ib) bar();
        float* row = p.slots + (long long)(n + 1) * p.rec.ntap;
        for (int j = gb + tid; j < ge; j += nthr) row[p.rec.slot[j]] = p.rec.gw[j] * __ldcg(un + p.rec.idx[j]);
    }
}

// ---------------------------------------------------------------------------
// Kind 0: direct loads, one tile at a time per CTA.
constexpr int kBTZ = 32;  // tile height
constexpr int kBBZ = 8;   // thread rows

template <bool ADJ>
__global__ void __launch_bounds__(32 * kBBZ, 2)
    k_batch_sweep(const BProb* __restrict__ probs, const int* __restrict__ tile_prob, int ntile, int nsteps,
                  int* flags, int* err, int* abort_word)
{
    constexpr int SW = kTX + 8;
    constexpr int RB = kBTZ / kBBZ;
    __shared__ __align__(16) float s[kBTZ + 8][SW];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int lx = 4 * threadIdx.x;
    for (int step = 0; step < nsteps; ++step) {
        for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
            const BProb& p = probs[tile_prob[t]];
            const int local = t - p.tile0;
            const int tz = local / p.ncx, tx = local - tz * p.ncx;
            // time index of this problem at this sweep step
            const int n = ADJ ? p.nt - 1 - step : step;
            if (ADJ ? n < 1 : n >= p.nt - 1) continue;  // block-uniform

            // wait until the 8 neighbour tiles have finished the previous step
            bool ok = true;
            if (tid < 9 && tid != 4) {
                const int nz = tz + tid / 3 - 1, nx = tx + tid % 3 - 1;
                if (nz >= 0 && nz < p.ntz && nx >= 0 && nx < p.ncx)
                    ok = wait_flag(flags + p.tile0 + nz * p.ncx + nx, step, abort_word);
            }
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(err, kErrTimeout);
                    atomicExch(abort_word, 1);
                }
                return;
            }
            __threadfence();

            const float* u = ADJ ? p.a[(n + 1) & 1] : p.w[n & 1];      // mu^{k+1} / u^n
            float* un = ADJ ? p.a[n & 1] : p.w[(n + 1) & 1];           // mu^k over mu^{k+2} / u^{n+1} over u^{n-1}
            const int x0 = tx * kTX, z0 = tz * kBTZ;
            for (int r = threadIdx.y; r < kBTZ + 8; r += kBBZ) {
                const int gz = z0 - 4 + r;
                for (int c4 = threadIdx.x; c4 < SW / 4; c4 += 32) {
                    const int gx = x0 - 4 + 4 * c4;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (gz >= 0 && gz < p.Nz && gx >= 0 && gx < p.P) v = ldcg4(u + (long long)gz * p.P + gx);
                    *reinterpret_cast<float4*>(&s[r][4 * c4]) = v;
                }
            }
            __syncthreads();

            const int gx = x0 + lx;
            const int nvalid = min(4, p.Nx - gx);
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
                const int r = threadIdx.y + rr * kBBZ;
                const int gz = z0 + r;
                if (gz >= p.Nz) continue;
                const long long off = (long long)gz * p.P + gx;
                if (nvalid <= 0) {
                    if (gx < p.P) *reinterpret_cast<float4*>(un + off) = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                const float* row = &s[r + 4][lx];
                const float4 A = *reinterpret_cast<const float4*>(row);
                const float4 B = *reinterpret_cast<const float4*>(row + 4);
                const float4 C = *reinterpret_cast<const float4*>(row + 8);
                const float w[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
                float lap[4];
                lap4(w, [&](int k, float4& Up, float4& Dn) {
                    Up = *reinterpret_cast<const float4*>(&s[r + 4 - k][lx + 4]);
                    Dn = *reinterpret_cast<const float4*>(&s[r + 4 + k][lx + 4]);
                }, lap);
                const float4 kp = __ldg(reinterpret_cast<const float4*>(p.kap + off));
                const float4 uo = ldcg4(un + off);
                const float kv[4] = {kp.x, kp.y, kp.z, kp.w};
                const float ov[4] = {uo.x, uo.y, uo.z, uo.w};
                const float cv[4] = {w[4], w[5], w[6], w[7]};
                const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
                const int dz = bdepth(gz, p.nb, p.nz);
                float out[4], ev[4], iv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int dd = max(bdepth(gx + e, p.nb, p.nx), dz);
                    ev[e] = kv[e] * p.ceps * (float)(dd * dd);
                    iv[e] = rcp_sponge(1.0f + ev[e]);
                }
                update4(cv, ov, lap, kv, ev, iv, zero4, out);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e >= nvalid) out[e] = 0.0f;
                *reinterpret_cast<float4*>(un + off) = make_float4(out[0], out[1], out[2], out[3]);
                if (!ADJ) {
                    const long long so = (long long)(n + 1) * p.cell + off;
                    if (p.st16) store_bf16x4(p.st16 + so, out);
                    else *reinterpret_cast<float4*>(p.st32 + so) = make_float4(out[0], out[1], out[2], out[3]);
                } else {
                    const long long so = (long long)n * p.cell + off;
                    float uf[4];
                    if (p.st16) {
                        unpack_bf16x4(*reinterpret_cast<const uint2*>(p.st16 + so), uf);
                    } else {
                        const float4 v = __ldg(reinterpret_cast<const float4*>(p.st32 + so));
                        uf[0] = v.x;
                        uf[1] = v.y;
                        uf[2] = v.z;
                        uf[3] = v.w;
                    }
                    const float4 gv = ldcg4(p.g + off);
                    float gg[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) gg[e] -= uf[e] * (out[e] - 2.0f * w[e + 4] + ov[e]);
                    if (nvalid == 4) {
                        *reinterpret_cast<float4*>(p.g + off) = make_float4(gg[0], gg[1], gg[2], gg[3]);
                    } else {
                        for (int e = 0; e < nvalid; ++e) p.g[off + e] = gg[e];
                    }
                }
            }
            __threadfence();
            __syncthreads();
            batch_sparse<ADJ>(p, tz, tx, kBTZ, n, un, tid, 32 * kBBZ, [] {
                __threadfence();
                __syncthreads();
            });
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicExch(flags + t, step + 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Kind 1: producer / consumer sweep.
//
// Warp 0 (producer) walks the CTA's items (step, tile) in order, skipping
// tiles of problems that have finished; for each it waits until the ring
// stage is free, polls the flags of the tile and its 8 neighbours (previous
// step done), and issues the TMA loads of the item into the stage.  Warps
// 2 .. BZ+1 (consumers) wait for the stage, compute the tile, apply its
// sources / receivers, and hand the item to warp 1 (releaser), which makes
// the tile's writes visible GPU-wide and publishes its flag.  Every wait is
// bounded; a wait that gives up sets kErrTimeout and the abort word, which
// makes every other wait of the sweep give up too, and each warp leaves only
// after the copies it issued have landed.
struct ItemInfo {
    int prob, tile, step, end, taps;  // taps: the tile has sources or receivers
};

template <int TZ, bool ADJ>
struct StageLayout {
    static constexpr int SW = kTX + 8;
    static constexpr int H = (TZ + 8) * SW;  // halo of the current level
    static constexpr int U = TZ * kTX;       // previous level
    static constexpr int K = TZ * kTX;       // model
    static constexpr int F = ADJ ? TZ * kTX : 0;  // stored forward level (FP32, or BF16 in its first half)
    static constexpr int G = ADJ ? TZ * kTX : 0;  // gradient accumulator
    static constexpr int floats = H + U + K + F + G;
    static_assert(H % 32 == 0 && U % 32 == 0, "sub-buffers stay 128-byte aligned");
};

constexpr int kRelSlots = 8;  // release ring between consumers and the releaser

template <int TZ, int BZ, int NS, bool ADJ>
__global__ void __launch_bounds__(32 * (BZ + 2))
    k_batch_sweep_tma(const BProb* __restrict__ probs, const CUtensorMap* __restrict__ maps,
                      const int* __restrict__ tile_prob, const int* __restrict__ order, int ntile, int nsteps,
                      int* flags, int* err, int* abort_word)
{
    using SL = StageLayout<TZ, ADJ>;
    constexpr int SW = SL::SW;
    constexpr int RB = TZ / BZ;  // consecutive rows per consumer warp
    static_assert(TZ % BZ == 0 && TZ % kTZc2 == 0, "tile rows split evenly");
    constexpr int NC = 32 * BZ;  // consumer threads
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], done[kRelSlots], freed[kRelSlots];
    __shared__ ItemInfo info[NS];
    __shared__ int rel_tile[kRelSlots], rel_step[kRelSlots];
    float* st = reinterpret_cast<float*>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NC);  // every consumer thread arrives
        }
        for (int i = 0; i < kRelSlots; ++i) {
            mbar_init(&done[i], NC);   // every consumer thread arrives after its last store
            mbar_init(&freed[i], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == 0) {
        // ---- producer
        int it = 0;
        bool ok = true;
        for (int step = 0; step < nsteps && ok; ++step) {
            for (int q = blockIdx.x; q < ntile && ok; q += gridDim.x) {
                const int t = order[q];  // position q of the round-robin holds tile t
                const int pi = tile_prob[t];
                const BProb& p = probs[pi];
                if (step >= p.nt - 1) continue;
                const int local = t - p.tile0;
                const int tz = local / p.ncx, tx = local - tz * p.ncx;
                // whether the consumers have a sparse phase for the tile: looked up
                // here, off their path (the loads overlap the waits below)
                const TapList& inj = ADJ ? p.rec : p.src;
                const int c0 = tz * (TZ / kTZc2), c1 = min(c0 + TZ / kTZc2, p.ncz), cb = tx * p.ncz;
                const int taps = (inj.ntap > 0 && inj.cell_start[cb + c1] > inj.cell_start[cb + c0]) ||
                                 (!ADJ && p.rec.ntap > 0 && p.rec.cell_start[cb + c1] > p.rec.cell_start[cb + c0]);
                const int stage = it % NS;
                if (it >= NS && !mbar_wait_abort(&empty[stage], (uint32_t)((it / NS) - 1) & 1u, abort_word,
                                                 kStageWaitNs)) {
                    ok = false;
                    break;
                }
                bool mine = true;
                if (lane < 9) {
                    const int nz = tz + lane / 3 - 1, nx = tx + lane % 3 - 1;
                    if (nz >= 0 && nz < p.ntz && nx >= 0 && nx < p.ncx)
                        mine = wait_flag_acq(flags + p.tile0 + nz * p.ncx + nx, step, abort_word);
                }
                __syncwarp();  // orders the lanes' acquire loads before lane 0's copies
                if (!__all_sync(0xffffffffu, mine)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    fence_proxy_async_global();  // other CTAs' plain stores before this CTA's TMA reads
                    info[stage] = ItemInfo{pi, t, step, 0, taps};
                    float* sb = st + stage * SL::floats;
                    const CUtensorMap* m = maps + (size_t)pi * kMaps;
                    const int x0 = tx * kTX, z0 = tz * TZ;
                    const int n = ADJ ? p.nt - 1 - step : step;
                    uint32_t bytes = (uint32_t)(SL::H + SL::U + SL::K) * 4u;
                    if (ADJ) bytes += (uint32_t)(TZ * kTX) * (p.st16 ? 2u : 4u) + (uint32_t)SL::G * 4u;
                    mbar_expect_tx(&full[stage], bytes);
                    // the maps are rewritten by the host between launches (another batch, tile height)
                    if (ADJ) {
                        tensormap_acquire(m + kMapHaloA + ((n + 1) & 1));
                        tensormap_acquire(m + kMapTileA + (n & 1));
                        tensormap_acquire(m + kMapKap);
                        tensormap_acquire(m + kMapStore);
                        tensormap_acquire(m + kMapG);
                    } else {
                        tensormap_acquire(m + kMapHaloW + (n & 1));
                        tensormap_acquire(m + kMapTileW + ((n + 1) & 1));
                        tensormap_acquire(m + kMapKap);
                    }
                    if (ADJ) {
                        tma_load_2d(sb, m + kMapHaloA + ((n + 1) & 1), &full[stage], x0 - 4, z0 - 4);
                        tma_load_2d(sb + SL::H, m + kMapTileA + (n & 1), &full[stage], x0, z0);
                        tma_load_2d(sb + SL::H + SL::U, m + kMapKap, &full[stage], x0, z0);
                        tma_load_3d(sb + SL::H + SL::U + SL::K, m + kMapStore, &full[stage], x0, z0, n);
                        tma_load_2d(sb + SL::H + SL::U + SL::K + SL::F, m + kMapG, &full[stage], x0, z0);
                    } else {
                        tma_load_2d(sb, m + kMapHaloW + (n & 1), &full[stage], x0 - 4, z0 - 4);
                        tma_load_2d(sb + SL::H, m + kMapTileW + ((n + 1) & 1), &full[stage], x0, z0);
                        tma_load_2d(sb + SL::H + SL::U, m + kMapKap, &full[stage], x0, z0);
                    }
                }
                __syncwarp();
                ++it;
            }
        }
        if (!ok && lane == 0) {
            if (ld_acquire_gpu(abort_word) == 0) atomicOr(err, kErrTimeout);
            atomicExch(abort_word, 1);
        }
        // end marker for the consumers
        bool posted = false;
        {
            const int stage = it % NS;
            if (it < NS ||
                mbar_wait_abort(&empty[stage], (uint32_t)((it / NS) - 1) & 1u, abort_word, kStageWaitNs)) {
                if (lane == 0) {
                    info[stage] = ItemInfo{-1, -1, -1, 1, 0};
                    mbar_arrive(&full[stage]);
                }
                posted = true;
            }
        }
        // the CTA must not finish while copies it issued can still land
        if (lane == 0) {
            int first = max(0, it - NS + (posted ? 1 : 0));
            for (int i = first; i < it; ++i) mbar_wait(&full[i % NS], (uint32_t)(i / NS) & 1u);
        }
        return;
    }

    if (warp == 1) {
        // ---- releaser
        if (lane != 0) return;
        for (int i = 0;; ++i) {
            const int slot = i % kRelSlots;
            if (!mbar_wait_abort(&done[slot], (uint32_t)(i / kRelSlots) & 1u, abort_word, 2 * kStageWaitNs)) {
                if (ld_acquire_gpu(abort_word) == 0) atomicOr(err, kErrTimeout);
                atomicExch(abort_word, 1);
                return;
            }
            const int t = rel_tile[slot], step = rel_step[slot];
            mbar_arrive(&freed[slot]);
            if (t < 0) return;
            __threadfence();             // the consumers' stores of the tile, GPU-wide
            fence_proxy_async_global();  // ... and before TMA reads of other CTAs
            st_release_gpu(flags + t, step + 1);
        }
    }

    // ---- consumers
    const int ctid = threadIdx.x - 64;
    const int cw = ctid >> 5;
    const int lx = 4 * lane;
    auto cbar = [] { named_barrier(1, NC); };
    bool failed = false;
    // Every consumer thread arrives on done[slot] after its last store of an
    // item (thread 0 first records which tile it was); the releaser waits for
    // all of them.  A slot is reused only after the releaser freed it.
    auto hand_over = [&](int idx, int t, int step) {
        const int slot = idx % kRelSlots;
        if (idx >= kRelSlots && !failed &&
            !mbar_wait_abort(&freed[slot], (uint32_t)((idx / kRelSlots) - 1) & 1u, abort_word, 2 * kStageWaitNs))
            failed = true;
        if (failed) return;
        if (ctid == 0) {
            rel_tile[slot] = t;
            rel_step[slot] = step;
        }
        mbar_arrive(&done[slot]);
    };
    for (int i = 0;; ++i) {
        const int stage = i % NS;
        bool ok = !failed && mbar_wait_abort(&full[stage], (uint32_t)(i / NS) & 1u, abort_word, 2 * kStageWaitNs);
        // one vote per item: either every consumer goes on or every one leaves
        if (named_barrier_or(1, NC, !ok)) {
            if (ctid == 0) {
                if (ld_acquire_gpu(abort_word) == 0) atomicOr(err, kErrTimeout);
                atomicExch(abort_word, 1);
            }
            return;
        }
        const ItemInfo it = info[stage];
        if (it.end) {
            hand_over(i, -1, 0);  // tells the releaser to stop
            return;
        }
        const BProb& p = probs[it.prob];
        const int local = it.tile - p.tile0;
        const int tz = local / p.ncx, tx = local - tz * p.ncx;
        const int n = ADJ ? p.nt - 1 - it.step : it.step;
        const int x0 = tx * kTX, z0 = tz * TZ;
        float* un = ADJ ? p.a[n & 1] : p.w[(n + 1) & 1];
        const float* sb = st + stage * SL::floats;
        const float* H = sb;
        const float* U = sb + SL::H;
        const float* K = U + SL::U;
        const int gx = x0 + lx;
        const int nvalid = min(4, p.Nx - gx);
        const int r0 = cw * RB;
        // sponge: depth along x of the thread's 4 columns, interior test for the tile
        const bool interior = p.ceps == 0.0f || (x0 >= p.nb && x0 + kTX <= p.nb + p.nx && z0 >= p.nb &&
                                                 z0 + TZ <= p.nb + p.nz);
        int dxe[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) dxe[e] = bdepth(gx + e, p.nb, p.nx);

        float4 zw[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) zw[j] = lds4(H + (r0 + j) * SW + lx + 4);
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            const int r = r0 + rr;
            const int gz = z0 + r;
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
            const float4 kp = lds4(K + r * kTX + lx);
            const float cen[4] = {B.x, B.y, B.z, B.w};
            const float um[4] = {uo.x, uo.y, uo.z, uo.w};
            const float kv[4] = {kp.x, kp.y, kp.z, kp.w};
            float out[4];
            if (interior) {
                update4_interior(cen, um, lap, kv, out);
            } else {
                const int dz = bdepth(gz, p.nb, p.nz);
                float ev[4], iv[4];
                const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int dd = max(dxe[e], dz);
                    ev[e] = kv[e] * p.ceps * (float)(dd * dd);
                    iv[e] = rcp_sponge(1.0f + ev[e]);
                }
                update4(cen, um, lap, kv, ev, iv, zero4, out);
            }
            float uf[4], gg[4];
            if (ADJ) {
                const float* F = K + SL::K;
                const float* G = F + SL::F;
                if (p.st16) {
                    const __nv_bfloat16* F16 = reinterpret_cast<const __nv_bfloat16*>(F);
                    unpack_bf16x4(*reinterpret_cast<const uint2*>(F16 + r * kTX + lx), uf);
                } else {
                    const float4 v = lds4(F + r * kTX + lx);
                    uf[0] = v.x;
                    uf[1] = v.y;
                    uf[2] = v.z;
                    uf[3] = v.w;
                }
                const float4 gv = lds4(G + r * kTX + lx);
                gg[0] = gv.x;
                gg[1] = gv.y;
                gg[2] = gv.z;
                gg[3] = gv.w;
            }
            if (rr + 1 < RB) {
#pragma unroll
                for (int j = 0; j < 8; ++j) zw[j] = zw[j + 1];
                zw[8] = lds4(H + (r + 9) * SW + lx + 4);
            }
            if (gz >= p.Nz || nvalid <= 0) continue;
            const long long off = (long long)gz * p.P + gx;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e >= nvalid) out[e] = 0.0f;  // points past Nx stay the zero exterior
            *reinterpret_cast<float4*>(un + off) = make_float4(out[0], out[1], out[2], out[3]);
            if (!ADJ) {
                const long long so = (long long)(n + 1) * p.cell + off;
                if (p.st16) store_bf16x4(p.st16 + so, out);
                else *reinterpret_cast<float4*>(p.st32 + so) = make_float4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) gg[e] -= uf[e] * (out[e] - 2.0f * cen[e] + um[e]);
                if (nvalid == 4) {
                    *reinterpret_cast<float4*>(p.g + off) = make_float4(gg[0], gg[1], gg[2], gg[3]);
                } else {
                    for (int e = 0; e < nvalid; ++e) p.g[off + e] = gg[e];
                }
            }
        }
        mbar_arrive(&empty[stage]);  // this thread is done with the stage
        // the tile's sources / receivers (block-uniform decision)
        if (it.taps) {
            cbar();  // the tile's points are written before taps touch them
            batch_sparse<ADJ>(p, tz, tx, TZ, n, un, ctid, NC, cbar);
        }
        hand_over(i, it.tile, it.step);
    }
}

// ---------------------------------------------------------------------------
// Host side.

struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t n)
    {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

struct HostProb {
    Dims d;
    Tiling t;
    HostTaps hs, hr;
    std::vector<float> gw_s, gw_r;
    int ntz = 0, tile0 = 0;
};

struct BatchLayout {
    std::vector<HostProb> hp;
    std::vector<BProb> bp;
    std::vector<int> tile_prob;
    int ntile = 0, maxnt = 0, ntile_cap = 0, TZ = 0;
    BProb* d_probs = nullptr;
    int* d_tile_prob = nullptr;
    // per sweep (forward, adjoint): position q of the round-robin -> tile
    std::vector<int> order[2];
    int* d_order[2] = {nullptr, nullptr};
    CUtensorMap* d_maps = nullptr;
    std::vector<CUtensorMap> maps;
    int* flags = nullptr;
    int* err = nullptr;  // [0] error bits, [1] abort word
    float* vmax = nullptr;
    double* part = nullptr;
    double* misfit = nullptr;
    size_t bytes = 0;
};

constexpr int kNumPartials = 256;

void carve_list(Carver& c, const HostTaps& h, TapList& l)
{
    const size_t ntap = h.idx.size();
    l.cell_start = c.take<int>(h.cell_start.size());
    l.idx = c.take<int>(ntap);
    l.fac = c.take<float>(ntap);
    l.gw = c.take<float>(ntap);
    l.ab = c.take<int>(ntap);
    l.slot = c.take<int>(ntap);
    l.w = c.take<float>(ntap);
    l.pt_start = c.take<int>(h.pt_start.size());
    l.npts = h.npts;
    l.ntap = (int)ntap;
}

bool valid_grid(const wave_grid_t& g)
{
    if (g.ndim != 2 || g.nx < 2 || g.nz < 2 || g.nb < 0 || g.nt < 1) return false;
    if (!(g.h > 0.0f) || !(g.dt > 0.0f) || !isfinite(g.h) || !isfinite(g.dt) || !isfinite(g.vref) || g.vref < 0.0f)
        return false;
    return make_dims(g).cell < (1LL << 31);
}

// Tiles of every problem for tile height TZ (the flag and tile tables are
// sized for the smallest tile height of any variant).  Problems take tile
// numbers in order of decreasing nt: the tiles still stepping at any time are
// then a prefix of the numbering, and the sweeps' round-robin assignment
// (tile t to CTA t mod grid) keeps every CTA within one tile of the others
// as the shorter problems finish.
void layout_tiles(BatchLayout& B, int TZ)
{
    B.TZ = TZ;
    B.ntile = 0;
    std::vector<int> order(B.hp.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return B.hp[x].d.nt > B.hp[y].d.nt; });
    for (const int i : order) {
        HostProb& h = B.hp[i];
        h.ntz = (h.d.Nz + TZ - 1) / TZ;
        h.tile0 = B.ntile;
        B.ntile += h.ntz * h.t.ncx;
        B.bp[i].ntz = h.ntz;
        B.bp[i].tile0 = h.tile0;
    }
    B.tile_prob.assign(B.ntile, 0);
    for (size_t i = 0; i < B.hp.size(); ++i)
        for (int k = 0; k < B.hp[i].ntz * B.hp[i].t.ncx; ++k) B.tile_prob[B.hp[i].tile0 + k] = (int)i;
}

wave_status_t plan_batch(const wave_problem_t* probs, int nprob, int store, void* base, BatchLayout& B)
{
    if (!probs || nprob < 0 || (store != WAVE_STORE_BF16 && store != WAVE_STORE_FP32)) return WAVE_ERR_ARG;
    B = BatchLayout();
    B.hp.resize(nprob);
    B.bp.resize(nprob);
    for (int i = 0; i < nprob; ++i) {
        const wave_problem_t& q = probs[i];
        if (!valid_grid(q.grid) || q.nsrc < 0 || q.nrec < 0 || (q.nsrc && !q.src_xyz) || (q.nrec && !q.rec_xyz))
            return WAVE_ERR_ARG;
        if ((long long)q.grid.nt * std::max(q.nsrc, q.nrec) >= (1LL << 31)) return WAVE_ERR_ARG;
        HostProb& h = B.hp[i];
        h.d = make_dims(q.grid);
        h.t.TX = kTX;
        h.t.TY = 1;
        h.t.TZc = kTZc2;
        h.t.ncx = (h.d.Nx + kTX - 1) / kTX;
        h.t.ncy = 1;
        h.t.ncz = (h.d.Nz + kTZc2 - 1) / kTZc2;
        h.t.vf = h.t.va = 0;
        wave_status_t st = build_taps(h.d, h.t, 1, q.nsrc, q.src_xyz, h.hs);
        if (st) return st;
        st = build_taps(h.d, h.t, 1, q.nrec, q.rec_xyz, h.hr);
        if (st) return st;
        B.ntile_cap += ((h.d.Nz + kMinTZ - 1) / kMinTZ) * h.t.ncx;
        B.maxnt = std::max(B.maxnt, q.grid.nt);
        const double h2 = (double)h.d.h * h.d.h;
        h.gw_r.assign(h.hr.w.begin(), h.hr.w.end());
        h.gw_s.resize(h.hs.w.size());
        for (size_t j = 0; j < h.hs.w.size(); ++j) h.gw_s[j] = (float)(h.hs.w[j] * (double)h.d.dt * h.d.dt / h2);
    }
    Carver c(base);
    B.d_probs = c.take<BProb>(nprob);
    B.d_tile_prob = c.take<int>(B.ntile_cap);
    B.d_order[0] = c.take<int>(B.ntile_cap);
    B.d_order[1] = c.take<int>(B.ntile_cap);
    B.flags = c.take<int>(B.ntile_cap);
    B.d_maps = c.take<CUtensorMap>((size_t)nprob * kMaps);
    B.err = c.take<int>(4);
    B.vmax = c.take<float>(std::max(nprob, 1));
    B.part = c.take<double>(kNumPartials);
    B.misfit = c.take<double>(std::max(nprob, 1));
    for (int i = 0; i < nprob; ++i) {
        const wave_problem_t& q = probs[i];
        HostProb& h = B.hp[i];
        BProb& p = B.bp[i];
        memset(&p, 0, sizeof(p));
        const Dims& d = h.d;
        p.Nx = d.Nx;
        p.Nz = d.Nz;
        p.P = d.P;
        p.nx = d.nx;
        p.nz = d.nz;
        p.nb = d.nb;
        p.nt = d.nt;
        p.ncx = h.t.ncx;
        p.ncz = h.t.ncz;
        p.cell = d.cell;
        p.ceps = 0.0f;
        if (d.nb > 0 && d.vref > 0.0f)
            p.ceps = (float)(3.0 * log(1000.0) * d.h / (4.0 * d.dt * d.vref * (double)d.nb * d.nb * d.nb));
        p.kap = c.take<float>(d.cell);
        for (int k = 0; k < 2; ++k) p.w[k] = c.take<float>(d.cell);
        p.a[0] = c.take<float>(2 * d.cell);  // a[0], a[1] contiguous: scratch of the gradient reduction
        p.a[1] = p.a[0] + d.cell;
        p.g = c.take<float>(d.cell);
        if (store == WAVE_STORE_BF16) p.st16 = c.take<__nv_bfloat16>((size_t)d.nt * d.cell);
        else p.st32 = c.take<float>((size_t)d.nt * d.cell);
        p.dsyn = c.take<float>((size_t)d.nt * q.nrec);
        p.slots = c.take<float>((size_t)d.nt * h.hr.idx.size());
        carve_list(c, h.hs, p.src);
        carve_list(c, h.hr, p.rec);
        p.wavelet = q.wavelet;
        p.dobs = q.d_obs;
    }
    B.bytes = c.off;
    layout_tiles(B, kBTZ);
    return WAVE_OK;
}

#define BCK(x)                        \
    do {                              \
        cudaError_t e_ = (x);         \
        if (e_ != cudaSuccess) {      \
            note_cuda_error(e_);      \
            (void)cudaGetLastError(); \
            return WAVE_ERR_CUDA;     \
        }                             \
    } while (0)

// --- TMA descriptors of the batch ------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn batch_encoder()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        (void)cudaGetLastError();
    });
    return fn;
}

// 2D (x, z) map over one [Nz][P] array (FP32), or the 3D (x, z, n) map of a
// store; box bx x bz (x 1).  Columns past Nx and rows past Nz read as zero.
bool encode_field(CUtensorMap* m, const void* ptr, const Dims& d, int bx, int bz, bool bf16 = false, int nt = 0)
{
    EncodeTiledFn fn = batch_encoder();
    if (!fn) return false;
    const int es = bf16 ? 2 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)d.Nx, (cuuint64_t)d.Nz, (cuuint64_t)nt};
    const cuuint64_t str[2] = {(cuuint64_t)d.P * es, (cuuint64_t)d.cell * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)bz, 1};
    const cuuint32_t ones[3] = {1, 1, 1};
    return fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nt > 0 ? 3 : 2,
              const_cast<void*>(ptr), dims, str, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

wave_status_t encode_batch_maps(BatchLayout& B, int TZ)
{
    const size_t np = B.bp.size();
    B.maps.assign(np * kMaps, CUtensorMap{});
    for (size_t i = 0; i < np; ++i) {
        const BProb& p = B.bp[i];
        const Dims& d = B.hp[i].d;
        CUtensorMap* m = &B.maps[i * kMaps];
        bool ok = true;
        for (int k = 0; k < 2; ++k) {
            ok = ok && encode_field(m + kMapHaloW + k, p.w[k], d, kTX + 8, TZ + 8) &&
                 encode_field(m + kMapTileW + k, p.w[k], d, kTX, TZ) &&
                 encode_field(m + kMapHaloA + k, p.a[k], d, kTX + 8, TZ + 8) &&
                 encode_field(m + kMapTileA + k, p.a[k], d, kTX, TZ);
        }
        ok = ok && encode_field(m + kMapKap, p.kap, d, kTX, TZ) && encode_field(m + kMapG, p.g, d, kTX, TZ);
        ok = ok && (p.st16 ? encode_field(m + kMapStore, p.st16, d, kTX, TZ, true, d.nt)
                           : encode_field(m + kMapStore, p.st32, d, kTX, TZ, false, d.nt));
        if (!ok) return WAVE_ERR_CUDA;
    }
    return WAVE_OK;
}

wave_status_t upload_list(const HostTaps& h, const std::vector<float>& gw, const TapList& l, cudaStream_t s)
{
    const size_t ntap = h.idx.size();
    BCK(cudaMemcpyAsync(const_cast<int*>(l.cell_start), h.cell_start.data(), h.cell_start.size() * sizeof(int),
                        cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(const_cast<int*>(l.pt_start), h.pt_start.data(), h.pt_start.size() * sizeof(int),
                        cudaMemcpyHostToDevice, s));
    if (ntap) {
        BCK(cudaMemcpyAsync(const_cast<int*>(l.idx), h.idx.data(), ntap * sizeof(int), cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(const_cast<int*>(l.ab), h.ab.data(), ntap * sizeof(int), cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(const_cast<int*>(l.slot), h.slot.data(), ntap * sizeof(int), cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(const_cast<float*>(l.w), h.w.data(), ntap * sizeof(float), cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(const_cast<float*>(l.gw), gw.data(), ntap * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    return WAVE_OK;
}

// --- sweep launches ----------------------------------------------------------

template <int TZ, int BZ, int NS, bool ADJ>
size_t tma_smem()
{
    return (size_t)NS * StageLayout<TZ, ADJ>::floats * 4 + 128;
}

// Occupancy and attributes of one kind-1 instantiation (per device).
template <int TZ, int BZ, int NS, bool ADJ>
int tma_per_sm()
{
    static int per[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return 0;
    }
    if (!per[dev]) {
        const size_t smem = tma_smem<TZ, BZ, NS, ADJ>();
        cudaFuncSetAttribute(k_batch_sweep_tma<TZ, BZ, NS, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_sweep_tma<TZ, BZ, NS, ADJ>, 32 * (BZ + 2), smem);
        (void)cudaGetLastError();
        per[dev] = std::max(n, 0) + 1;  // stored plus one: 0 means "not yet computed"
    }
    return per[dev] - 1;
}

int num_sms_batch()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    (void)cudaGetLastError();
    return std::max(sms, 1);
}

cudaLaunchConfig_t sweep_config(int grid, int threads, size_t smem, bool cooperative, cudaStream_t s,
                                cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = cooperative ? attr : nullptr;
    cfg.numAttrs = cooperative ? 1 : 0;
    return cfg;
}

// CTAs of a kind-1 sweep: as many as are resident at once (0: does not fit).
template <int TZ, int BZ, int NS, bool ADJ>
int tma_grid(const BatchLayout& B, int cap)
{
    const int per = tma_per_sm<TZ, BZ, NS, ADJ>();
    if (per < 1) return 0;
    return std::max(1, std::min(B.ntile, num_sms_batch() * (cap > 0 ? std::min(cap, per) : per)));
}

template <int TZ, int BZ, int NS, bool ADJ>
wave_status_t launch_tma_sweep(const BatchLayout& B, int nsteps, int cap, bool cooperative, cudaStream_t s)
{
    const int grid = tma_grid<TZ, BZ, NS, ADJ>(B, cap);
    if (grid < 1) return WAVE_ERR_CUDA;  // does not fit on an SM
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = sweep_config(grid, 32 * (BZ + 2), tma_smem<TZ, BZ, NS, ADJ>(), cooperative, s, attr);
    count_launch();
    BCK(cudaLaunchKernelEx(&cfg, k_batch_sweep_tma<TZ, BZ, NS, ADJ>, (const BProb*)B.d_probs,
                           (const CUtensorMap*)B.d_maps, (const int*)B.d_tile_prob, (const int*)B.d_order[ADJ ? 1 : 0],
                           B.ntile, nsteps, B.flags, B.err, B.err + 1));
    return WAVE_OK;
}

template <bool ADJ>
wave_status_t launch_direct_sweep(const BatchLayout& B, int nsteps, bool cooperative, cudaStream_t s)
{
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_sweep<ADJ>, 32 * kBBZ, 0);
    (void)cudaGetLastError();
    const int grid = std::max(1, std::min(B.ntile, num_sms_batch() * std::max(1, per)));
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = sweep_config(grid, 32 * kBBZ, 0, cooperative, s, attr);
    cfg.blockDim = dim3(32, kBBZ);
    count_launch();
    BCK(cudaLaunchKernelEx(&cfg, k_batch_sweep<ADJ>, (const BProb*)B.d_probs, (const int*)B.d_tile_prob, B.ntile,
                           nsteps, B.flags, B.err, B.err + 1));
    return WAVE_OK;
}

// cooperative: ask for co-residency through the launch attribute (eager
// calls); stream capture takes the launch without it, and the grid is sized
// by the occupancy calculator so that every CTA fits at once either way.
wave_status_t launch_sweep(const BatchLayout& B, int variant, bool adj, int nsteps, bool cooperative, cudaStream_t s)
{
    const BVariant v = kBatchVariants[variant];
    if (v.kind == 0) return adj ? launch_direct_sweep<true>(B, nsteps, cooperative, s)
                                : launch_direct_sweep<false>(B, nsteps, cooperative, s);
#define SWEEP(tz, bz, ns)                                                                   \
    if (v.TZ == tz && v.BZ == bz && v.NS == ns)                                             \
        return adj ? launch_tma_sweep<tz, bz, ns, true>(B, nsteps, v.cap, cooperative, s)  \
                   : launch_tma_sweep<tz, bz, ns, false>(B, nsteps, v.cap, cooperative, s);
    SWEEP(16, 4, 2)
    SWEEP(16, 4, 3)
    SWEEP(32, 8, 2)
    SWEEP(32, 4, 2)
    SWEEP(16, 2, 3)
    SWEEP(16, 8, 2)
    SWEEP(16, 8, 3)
    SWEEP(16, 2, 2)
#undef SWEEP
    return WAVE_ERR_ARG;
}

// CTAs of a variant's sweep (0 for the direct kernel, which takes tiles in
// numbering order).
int sweep_grid(const BatchLayout& B, int variant, bool adj)
{
    const BVariant v = kBatchVariants[variant];
    if (v.kind == 0) return 0;
#define GRID(tz, bz, ns) \
    if (v.TZ == tz && v.BZ == bz && v.NS == ns) return adj ? tma_grid<tz, bz, ns, true>(B, v.cap) : tma_grid<tz, bz, ns, false>(B, v.cap);
    GRID(16, 4, 2)
    GRID(16, 4, 3)
    GRID(32, 8, 2)
    GRID(32, 4, 2)
    GRID(16, 2, 3)
    GRID(16, 8, 2)
    GRID(16, 8, 3)
    GRID(16, 2, 2)
#undef GRID
    return 0;
}

// Round-robin order of a sweep: position q goes to CTA q mod grid.  The
// positions keep the tiles of layout_tiles' numbering (longest problems
// first) block by block (positions b grid .. b grid + grid - 1), so each CTA
// still holds one position per block and the active tiles stay balanced to
// one per CTA as problems finish.  Inside a block, tiles are handed out by
// cost: tiles touching the sponge (sponge factors computed per point) and
// tiles with sources or receivers (a sparse phase) cost more, and the dearest
// go to the CTAs with the least work so far.
void build_order(const BatchLayout& B, int grid, bool adj, std::vector<int>& order)
{
    order.resize(B.ntile);
    for (int q = 0; q < B.ntile; ++q) order[q] = q;
    if (grid <= 1 || grid >= B.ntile) return;
    // relative costs measured per item: sponge tiles 1.18 (adjoint) and 1.24
    // (forward) x an interior tile, tiles with taps about 2 x
    const float wsponge = adj ? 0.18f : 0.24f, wtaps = 1.0f;
    std::vector<float> cost(B.ntile, 1.0f);
    for (size_t i = 0; i < B.hp.size(); ++i) {
        const HostProb& h = B.hp[i];
        const BProb& p = B.bp[i];
        const HostTaps& inj = adj ? h.hr : h.hs;
        const int kcell = B.TZ / kTZc2;
        for (int tz = 0; tz < h.ntz; ++tz)
            for (int tx = 0; tx < p.ncx; ++tx) {
                const int x0 = tx * kTX, z0 = tz * B.TZ;
                const bool interior = p.ceps == 0.0f || (x0 >= p.nb && x0 + kTX <= p.nb + p.nx && z0 >= p.nb &&
                                                         z0 + B.TZ <= p.nb + p.nz);
                const int c0 = tz * kcell, c1 = std::min(c0 + kcell, p.ncz), cb = tx * p.ncz;
                const bool taps = (!inj.idx.empty() && inj.cell_start[cb + c1] > inj.cell_start[cb + c0]) ||
                                  (!adj && !h.hr.idx.empty() && h.hr.cell_start[cb + c1] > h.hr.cell_start[cb + c0]);
                cost[h.tile0 + tz * p.ncx + tx] = 1.0f + (interior ? 0.0f : wsponge) + (taps ? wtaps : 0.0f);
            }
    }
    std::vector<double> load(grid, 0.0);
    std::vector<int> tiles, ctas;
    for (int b0 = 0; b0 < B.ntile; b0 += grid) {
        const int n = std::min(grid, B.ntile - b0);
        tiles.resize(n);
        ctas.resize(n);
        for (int k = 0; k < n; ++k) {
            tiles[k] = b0 + k;
            ctas[k] = k;  // the CTAs that have a position in this block
        }
        std::stable_sort(tiles.begin(), tiles.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        std::stable_sort(ctas.begin(), ctas.end(), [&](int a, int b) { return load[a] < load[b]; });
        for (int k = 0; k < n; ++k) {
            order[b0 + ctas[k]] = tiles[k];
            load[ctas[k]] += cost[tiles[k]];
        }
    }
}

// Tile tables, round-robin orders of the two sweeps and TMA maps for a
// variant's tile height (host work, then stream-ordered uploads; the host
// vectors stay alive until the caller syncs).  vf and va share the tile height.
wave_status_t prepare_variant(BatchLayout& B, int vf, int va, cudaStream_t s)
{
    const BVariant v = kBatchVariants[vf];
    layout_tiles(B, v.TZ);
    BCK(cudaMemcpyAsync(B.d_probs, B.bp.data(), B.bp.size() * sizeof(BProb), cudaMemcpyHostToDevice, s));
    if (B.ntile)
        BCK(cudaMemcpyAsync(B.d_tile_prob, B.tile_prob.data(), B.ntile * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < 2; ++k) {
        build_order(B, sweep_grid(B, k ? va : vf, k == 1), k == 1, B.order[k]);
        if (B.ntile)
            BCK(cudaMemcpyAsync(B.d_order[k], B.order[k].data(), B.ntile * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    if (v.kind == 1) {
        wave_status_t st = encode_batch_maps(B, v.TZ);
        if (st) return st;
        BCK(cudaMemcpyAsync(B.d_maps, B.maps.data(), B.maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s));
    }
    return WAVE_OK;
}

// Zeroes the levels, accumulators, first store rows and receiver slots.
wave_status_t clear_state(const BatchLayout& B, cudaStream_t s)
{
    for (size_t i = 0; i < B.bp.size(); ++i) {
        const BProb& p = B.bp[i];
        const Dims& d = B.hp[i].d;
        BCK(cudaMemsetAsync(p.w[0], 0, d.cell * sizeof(float), s));
        BCK(cudaMemsetAsync(p.w[1], 0, d.cell * sizeof(float), s));
        BCK(cudaMemsetAsync(p.a[0], 0, 2 * d.cell * sizeof(float), s));
        BCK(cudaMemsetAsync(p.g, 0, d.cell * sizeof(float), s));
        if (p.st16) BCK(cudaMemsetAsync(p.st16, 0, d.cell * sizeof(__nv_bfloat16), s));
        if (p.st32) BCK(cudaMemsetAsync(p.st32, 0, d.cell * sizeof(float), s));
        if (p.rec.ntap) BCK(cudaMemsetAsync(p.slots, 0, p.rec.ntap * sizeof(float), s));
    }
    return WAVE_OK;
}

// Device work after the set-up: both sweeps and the per-problem reductions.
wave_status_t compute_phase(const BatchLayout& B, const wave_problem_t* probs, int nprob, int wrt, int vf, int va,
                            bool capture, cudaStream_t s)
{
    const int nsteps = std::max(0, B.maxnt - 1);
    BCK(cudaMemsetAsync(B.flags, 0, B.ntile_cap * sizeof(int), s));
    wave_status_t st = launch_sweep(B, vf, false, nsteps, !capture, s);
    if (st) return st;
    for (int i = 0; i < nprob; ++i) {
        const BProb& p = B.bp[i];
        if (probs[i].nrec == 0) {
            BCK(cudaMemsetAsync(B.misfit + i, 0, sizeof(double), s));
            continue;
        }
        launch_finalize(p.rec, p.slots, 1, p.nt, p.dsyn, s);
        launch_misfit(p.dsyn, p.dobs, (long long)p.nt * probs[i].nrec, B.part, kNumPartials, B.misfit + i, s);
    }
    BCK(cudaMemsetAsync(B.flags, 0, B.ntile_cap * sizeof(int), s));
    st = launch_sweep(B, va, true, nsteps, !capture, s);
    if (st) return st;
    for (int i = 0; i < nprob; ++i) {
        const BProb& p = B.bp[i];
        launch_grad_reduce(B.hp[i].d, p.g, 1, p.a[0], probs[i].grad, wrt == WAVE_WRT_VELOCITY ? probs[i].vel : nullptr,
                           s);
        launch_nan_scan(probs[i].grad, B.hp[i].d.phys, B.err, s);
    }
    BCK(cudaGetLastError());
    return WAVE_OK;
}

// Set-up shared by the gradient and the autotuner: tables, models, stability
// check, injection factors (synchronises once to check the models).
wave_status_t setup_batch(BatchLayout& B, const wave_problem_t* probs, int nprob, cudaStream_t s)
{
    BCK(cudaMemsetAsync(B.err, 0, 4 * sizeof(int), s));
    BCK(cudaMemsetAsync(B.vmax, 0, nprob * sizeof(float), s));
    for (int i = 0; i < nprob; ++i) {
        HostProb& h = B.hp[i];
        BProb& p = B.bp[i];
        wave_status_t st = upload_list(h.hs, h.gw_s, p.src, s);
        if (st) return st;
        if ((st = upload_list(h.hr, h.gw_r, p.rec, s))) return st;
        launch_prep(h.d, probs[i].vel, const_cast<float*>(p.kap), B.vmax + i, B.err, s);
    }
    std::vector<float> vmax(nprob);
    int herr = 0;
    BCK(cudaMemcpyAsync(vmax.data(), B.vmax, nprob * sizeof(float), cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (herr & kErrNonFinite) return WAVE_ERR_NONFINITE;
    const double lim = 2.0 / sqrt(2.0 * 2048.0 / 315.0);
    for (int i = 0; i < nprob; ++i)
        if ((double)B.hp[i].d.dt * vmax[i] / B.hp[i].d.h > lim) return WAVE_ERR_CFL;
    for (int i = 0; i < nprob; ++i) {
        const Dims& d = B.hp[i].d;
        BProb& p = B.bp[i];
        launch_tapfac(d, p.src, p.kap, 1.0f, p.ceps, s);
        launch_tapfac(d, p.rec, p.kap, (float)((double)d.h * d.h / ((double)d.dt * d.dt)), p.ceps, s);
    }
    BCK(cudaGetLastError());
    return WAVE_OK;
}

wave_status_t check_batch_args(const wave_problem_t* probs, int nprob, const BatchLayout& B, void* work,
                               size_t work_bytes)
{
    for (int i = 0; i < nprob; ++i) {
        const wave_problem_t& q = probs[i];
        if (!q.vel || (q.nsrc && !q.wavelet) || (q.nrec && !q.d_obs)) return WAVE_ERR_ARG;
    }
    if (B.bytes > 0 && (!work || work_bytes < B.bytes)) return WAVE_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(work) % 256) return WAVE_ERR_WORKSPACE;
    return WAVE_OK;
}

// Variants picked by wave_autotune_batch, keyed by the batch's shapes.
std::mutex g_pick_mu;
std::map<std::vector<long long>, std::pair<int, int>> g_picks;

std::vector<long long> batch_signature(const wave_problem_t* probs, int nprob, int store)
{
    std::vector<long long> k = {store, nprob};
    for (int i = 0; i < nprob; ++i) {
        const wave_grid_t& g = probs[i].grid;
        k.push_back(((long long)g.nx << 32) | (unsigned)g.nz);
        k.push_back(((long long)g.nt << 32) | (unsigned)g.nb);
        k.push_back(((long long)probs[i].nsrc << 32) | (unsigned)probs[i].nrec);
    }
    return k;
}

int g_forced[2] = {-1, -1};  // wave_set_batch_variant

std::pair<int, int> picked_variants(const wave_problem_t* probs, int nprob, int store)
{
    std::lock_guard<std::mutex> lock(g_pick_mu);
    if (g_forced[0] >= 0) return std::make_pair(g_forced[0], g_forced[1]);
    auto it = g_picks.find(batch_signature(probs, nprob, store));
    if (it != g_picks.end()) return it->second;
    return std::make_pair(kDefaultBatchVariant, kDefaultBatchVariant);
}

// Captured compute phases, replayed when a call repeats the same buffers.
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;

std::vector<uintptr_t> graph_key(const wave_problem_t* probs, int nprob, int store, int wrt, void* work, int vf,
                                 int va)
{
    std::vector<uintptr_t> k = {(uintptr_t)work, (uintptr_t)nprob, (uintptr_t)store, (uintptr_t)wrt,
                                (uintptr_t)vf, (uintptr_t)va};
    for (int i = 0; i < nprob; ++i) {
        const wave_problem_t& q = probs[i];
        k.push_back((uintptr_t)q.vel);
        k.push_back((uintptr_t)q.wavelet);
        k.push_back((uintptr_t)q.d_obs);
        k.push_back((uintptr_t)q.grad);
        k.push_back(((uintptr_t)q.grid.nx << 32) ^ (uintptr_t)q.grid.nz);
        k.push_back(((uintptr_t)q.grid.nt << 32) ^ (uintptr_t)q.grid.nb);
        k.push_back(((uintptr_t)q.nsrc << 32) ^ (uintptr_t)q.nrec);
    }
    return k;
}

void add_tap_counts(std::vector<uintptr_t>& k, const BatchLayout& B)
{
    for (const BProb& p : B.bp) k.push_back(((uintptr_t)p.src.ntap << 32) ^ (uintptr_t)p.rec.ntap);
}

}  // namespace
}  // namespace wave

using namespace wave;

extern "C" {

wave_status_t wave_workspace_size_batch(const wave_problem_t* probs, int nprob, int store, size_t* bytes)
{
    if (!bytes) return WAVE_ERR_ARG;
    BatchLayout B;
    wave_status_t st = plan_batch(probs, nprob, store, nullptr, B);
    if (st) return st;
    *bytes = B.bytes;
    return WAVE_OK;
}

int wave_batch_variant_count(void) { return kNumBatchVariants; }

wave_status_t wave_set_batch_variant(int fwd, int adj)
{
    if (fwd == -1 && adj == -1) {
        std::lock_guard<std::mutex> lock(g_pick_mu);
        g_forced[0] = g_forced[1] = -1;
        return WAVE_OK;
    }
    if (fwd < 0 || fwd >= kNumBatchVariants || adj < 0 || adj >= kNumBatchVariants) return WAVE_ERR_ARG;
    if (kBatchVariants[fwd].TZ != kBatchVariants[adj].TZ) return WAVE_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_pick_mu);
    g_forced[0] = fwd;
    g_forced[1] = adj;
    return WAVE_OK;
}

wave_status_t wave_gradient_batch(wave_problem_t* probs, int nprob, int store, int wrt, int use_graph, void* work,
                                  size_t work_bytes, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (wrt != WAVE_WRT_SLOWNESS2 && wrt != WAVE_WRT_VELOCITY) return WAVE_ERR_ARG;
    BatchLayout B;
    wave_status_t st = plan_batch(probs, nprob, store, work, B);
    if (st) return st;
    if (nprob == 0) return WAVE_OK;
    for (int i = 0; i < nprob; ++i)
        if (!probs[i].grad) return WAVE_ERR_ARG;
    if ((st = check_batch_args(probs, nprob, B, work, work_bytes))) return st;
    const std::pair<int, int> v = picked_variants(probs, nprob, store);
    // the two sweeps must agree on the tile tables: both use the forward pick's tile height
    // unless the adjoint pick has the same one
    const int vf = v.first;
    const int va = kBatchVariants[v.second].TZ == kBatchVariants[vf].TZ ? v.second : vf;

    if ((st = setup_batch(B, probs, nprob, s))) return st;
    if ((st = prepare_variant(B, vf, va, s))) return st;
    if ((st = clear_state(B, s))) return st;

    if (use_graph) {
        std::vector<uintptr_t> key = graph_key(probs, nprob, store, wrt, work, vf, va);
        add_tap_counts(key, B);
        cudaGraphExec_t exec = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_graph_mu);
            for (const GraphEntry& e : g_graphs)
                if (e.key == key) exec = e.exec;
        }
        if (!exec) {
            // Record on a private stream: capture runs nothing, and the caller's
            // stream may be the legacy default stream, which cannot be captured.
            static thread_local cudaStream_t cs = nullptr;
            if (!cs) BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            BCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            st = compute_phase(B, probs, nprob, wrt, vf, va, true, cs);
            cudaError_t e = cudaStreamEndCapture(cs, &graph);
            if (st || e != cudaSuccess) {
                note_cuda_error(e);
                if (graph) cudaGraphDestroy(graph);
                (void)cudaGetLastError();
                return st ? st : WAVE_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            BCK(e);
            std::lock_guard<std::mutex> lock(g_graph_mu);
            if (g_graphs.size() >= 8) {
                cudaGraphExecDestroy(g_graphs.front().exec);
                g_graphs.erase(g_graphs.begin());
            }
            g_graphs.push_back(GraphEntry{exec, key});
        }
        BCK(cudaGraphLaunch(exec, s));
    } else {
        if ((st = compute_phase(B, probs, nprob, wrt, vf, va, false, s))) return st;
    }
    std::vector<double> mf(nprob);
    int herr = 0;
    BCK(cudaMemcpyAsync(mf.data(), B.misfit, nprob * sizeof(double), cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (herr & kErrTimeout) return WAVE_ERR_TIMEOUT;
    if (herr & kErrNonFinite) return WAVE_ERR_NONFINITE;
    if (herr) return WAVE_ERR_CUDA;
    for (int i = 0; i < nprob; ++i) probs[i].misfit = mf[i];
    return WAVE_OK;
}

wave_status_t wave_autotune_batch(wave_problem_t* probs, int nprob, int store, int steps, void* work,
                                  size_t work_bytes, void* stream, int* best_fwd, int* best_adj)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (steps < 1) return WAVE_ERR_ARG;
    BatchLayout B;
    wave_status_t st = plan_batch(probs, nprob, store, work, B);
    if (st) return st;
    if (nprob == 0) return WAVE_ERR_ARG;
    if ((st = check_batch_args(probs, nprob, B, work, work_bytes))) return st;
    if ((st = setup_batch(B, probs, nprob, s))) return st;
    const int nsteps = std::max(1, std::min(steps, B.maxnt - 1));
    cudaEvent_t e0, e1, e2;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    BCK(cudaEventCreate(&e2));
    float tf[kNumBatchVariants], ta[kNumBatchVariants];
    for (int v = 0; v < kNumBatchVariants && st == WAVE_OK; ++v) {
        if ((st = prepare_variant(B, v, v, s))) break;
        if ((st = clear_state(B, s))) break;
        if (cudaMemsetAsync(B.flags, 0, B.ntile_cap * sizeof(int), s) != cudaSuccess) st = WAVE_ERR_CUDA;
        cudaEventRecord(e0, s);
        if (!st) st = launch_sweep(B, v, false, nsteps, true, s);
        cudaEventRecord(e1, s);
        if (!st && cudaMemsetAsync(B.flags, 0, B.ntile_cap * sizeof(int), s) != cudaSuccess) st = WAVE_ERR_CUDA;
        if (!st) st = launch_sweep(B, v, true, nsteps, true, s);
        cudaEventRecord(e2, s);
        if (cudaEventSynchronize(e2) != cudaSuccess) st = WAVE_ERR_CUDA;
        if (st) break;
        int herr = 0;
        if (cudaMemcpy(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) st = WAVE_ERR_CUDA;
        if (herr) {
            st = (herr & kErrTimeout) ? WAVE_ERR_TIMEOUT : WAVE_ERR_CUDA;
            break;
        }
        cudaEventElapsedTime(&tf[v], e0, e1);
        cudaEventElapsedTime(&ta[v], e1, e2);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (st) {
        (void)cudaGetLastError();
        return st;
    }
    // both sweeps of a call share the tile tables, so the pair must agree on the tile height
    int pick[2] = {kDefaultBatchVariant, kDefaultBatchVariant};
    float best = 1e30f;
    for (int f = 0; f < kNumBatchVariants; ++f)
        for (int a = 0; a < kNumBatchVariants; ++a)
            if (kBatchVariants[f].TZ == kBatchVariants[a].TZ && tf[f] + ta[a] < best) {
                best = tf[f] + ta[a];
                pick[0] = f;
                pick[1] = a;
            }
    {
        std::lock_guard<std::mutex> lock(g_pick_mu);
        g_picks[batch_signature(probs, nprob, store)] = std::make_pair(pick[0], pick[1]);
    }
    if (best_fwd) *best_fwd = pick[0];
    if (best_adj) *best_adj = pick[1];
    return WAVE_OK;
}

wave_status_t wave_wait_probe(int* flag, int want, int* abort_word, int* err, void* stream)
{
    if (!flag || !abort_word || !err) return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int herr = 0;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return WAVE_ERR_CUDA;
    k_wait_probe<<<1, 32, 0, s>>>(flag, want, abort_word, err);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return WAVE_ERR_CUDA;
    }
    return (herr & kErrTimeout) ? WAVE_ERR_TIMEOUT : WAVE_OK;
}

}  // extern "C"
