// batch.cu -- FWI gradients of an uneven batch of independent 2D problems
// (each with its own grid, model, time axis, sources and receivers) in two
// persistent launches: one forward sweep that stores every level in BF16 or
// FP32, and one adjoint sweep with the imaging condition.
//
// The CTAs of a sweep stay resident (cooperative launch) and each owns a fixed
// set of 128 x 32 tiles of all problems.  A tile advances one time step as
// soon as its neighbours (same problem) have finished the previous one: tiles
// publish the number of steps they completed in a flag word, and waiters poll
// those words with a bounded number of tries.  Problems with few time steps
// simply drop out of the sweep; there is no global barrier between steps.
// Mutable fields are read through L2 only (ld.global.cg) because other SMs
// rewrite them during the sweep.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "internal.h"
#include "stencil.cuh"

namespace wave {

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

constexpr int kBTZ = 32;       // tile height
constexpr int kBBZ = 8;        // thread rows
constexpr int kPollLimit = 1 << 22;

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

// One thread runs the sweep's bounded wait on a caller-given flag.
__global__ void k_wait_probe(int* flag, int want, int* abort_word, int* err)
{
    if (threadIdx.x == 0 && !wait_flag(flag, want, abort_word)) atomicOr(err, kErrTimeout);
}

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
                    iv[e] = __frcp_rn(1.0f + ev[e]);
                }
                update4(cv, ov, lap, kv, ev, iv, zero4, out);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e >= nvalid) out[e] = 0.0f;
                *reinterpret_cast<float4*>(un + off) = make_float4(out[0], out[1], out[2], out[3]);
                if (!ADJ) {
                    const long long so = (long long)(n + 1) * p.cell + off;
                    if (p.st16) {
                        __nv_bfloat162 lo = __floats2bfloat162_rn(out[0], out[1]);
                        __nv_bfloat162 hi = __floats2bfloat162_rn(out[2], out[3]);
                        uint2 v;
                        v.x = *reinterpret_cast<uint32_t*>(&lo);
                        v.y = *reinterpret_cast<uint32_t*>(&hi);
                        *reinterpret_cast<uint2*>(p.st16 + so) = v;
                    } else {
                        *reinterpret_cast<float4*>(p.st32 + so) = make_float4(out[0], out[1], out[2], out[3]);
                    }
                } else {
                    const long long so = (long long)n * p.cell + off;
                    float uf[4];
                    if (p.st16) {
                        const uint2 v = *reinterpret_cast<const uint2*>(p.st16 + so);
                        const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
                        const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
                        uf[0] = lo.x;
                        uf[1] = lo.y;
                        uf[2] = hi.x;
                        uf[3] = hi.y;
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

            // sparse part: injection (fwd: sources with q^n; adj: residual at the receivers),
            // then, in the forward sweep, the receiver gathers of u^{n+1}
            const TapList& inj = ADJ ? p.rec : p.src;
            const int kcell = kBTZ / kTZc2;
            const int cbase = tx * p.ncz;
            const int c0 = tz * kcell, c1 = min(c0 + kcell, p.ncz);
            if (inj.ntap > 0) {
                const int ib = inj.cell_start[cbase + c0], ie = inj.cell_start[cbase + c1];
                for (int j = ib + tid; j < ie; j += 32 * kBBZ) {
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
            if (!ADJ && p.rec.ntap > 0) {
                __threadfence();
                __syncthreads();
                const int gb = p.rec.cell_start[cbase + c0], ge = p.rec.cell_start[cbase + c1];
                float* row = p.slots + (long long)(n + 1) * p.rec.ntap;
                for (int j = gb + tid; j < ge; j += 32 * kBBZ) row[p.rec.slot[j]] = p.rec.gw[j] * __ldcg(un + p.rec.idx[j]);
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicExch(flags + t, step + 1);
        }
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
    int ntile = 0, maxnt = 0;
    BProb* d_probs = nullptr;
    int* d_tile_prob = nullptr;
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
        h.ntz = (h.d.Nz + kBTZ - 1) / kBTZ;
        wave_status_t st = build_taps(h.d, h.t, 1, q.nsrc, q.src_xyz, h.hs);
        if (st) return st;
        st = build_taps(h.d, h.t, 1, q.nrec, q.rec_xyz, h.hr);
        if (st) return st;
        h.tile0 = B.ntile;
        B.ntile += h.ntz * h.t.ncx;
        B.maxnt = std::max(B.maxnt, q.grid.nt);
        const double h2 = (double)h.d.h * h.d.h;
        h.gw_r.assign(h.hr.w.begin(), h.hr.w.end());
        h.gw_s.resize(h.hs.w.size());
        for (size_t j = 0; j < h.hs.w.size(); ++j) h.gw_s[j] = (float)(h.hs.w[j] * (double)h.d.dt * h.d.dt / h2);
    }
    B.tile_prob.resize(B.ntile);
    Carver c(base);
    B.d_probs = c.take<BProb>(nprob);
    B.d_tile_prob = c.take<int>(B.ntile);
    B.flags = c.take<int>(B.ntile);
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
        p.ntz = h.ntz;
        p.tile0 = h.tile0;
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
        for (int k = 0; k < h.ntz * h.t.ncx; ++k) B.tile_prob[h.tile0 + k] = i;
    }
    B.bytes = c.off;
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

int sweep_grid(int ntile, bool adj)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (adj) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_sweep<true>, 32 * kBBZ, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_sweep<false>, 32 * kBBZ, 0);
    (void)cudaGetLastError();
    return std::max(1, std::min(ntile, std::max(1, sms) * std::max(1, per)));
}

// cooperative: ask for co-residency through the launch attribute (eager
// calls); stream capture takes the launch without it, and the grid is sized
// by the occupancy calculator so that every CTA fits at once either way.
wave_status_t launch_sweep(const BatchLayout& B, bool adj, bool cooperative, cudaStream_t s)
{
    const int grid = sweep_grid(B.ntile, adj);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32, kBBZ);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = cooperative ? attr : nullptr;
    cfg.numAttrs = cooperative ? 1 : 0;
    const int nsteps = std::max(0, B.maxnt - 1);
    count_launch();
    cudaError_t e = adj ? cudaLaunchKernelEx(&cfg, k_batch_sweep<true>, (const BProb*)B.d_probs,
                                             (const int*)B.d_tile_prob, B.ntile, nsteps, B.flags, B.err, B.err + 1)
                        : cudaLaunchKernelEx(&cfg, k_batch_sweep<false>, (const BProb*)B.d_probs,
                                             (const int*)B.d_tile_prob, B.ntile, nsteps, B.flags, B.err, B.err + 1);
    BCK(e);
    return WAVE_OK;
}

// Device work after the set-up: both sweeps and the per-problem reductions.
wave_status_t compute_phase(const BatchLayout& B, const wave_problem_t* probs, int nprob, int wrt, bool capture,
                            cudaStream_t s)
{
    BCK(cudaMemsetAsync(B.flags, 0, B.ntile * sizeof(int), s));
    wave_status_t st = launch_sweep(B, false, !capture, s);
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
    BCK(cudaMemsetAsync(B.flags, 0, B.ntile * sizeof(int), s));
    st = launch_sweep(B, true, !capture, s);
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

// Captured compute phases, replayed when a call repeats the same buffers.
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;

std::vector<uintptr_t> graph_key(const wave_problem_t* probs, int nprob, int store, int wrt, void* work)
{
    std::vector<uintptr_t> k = {(uintptr_t)work, (uintptr_t)nprob, (uintptr_t)store, (uintptr_t)wrt};
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

wave_status_t wave_gradient_batch(wave_problem_t* probs, int nprob, int store, int wrt, int use_graph, void* work,
                                  size_t work_bytes, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (wrt != WAVE_WRT_SLOWNESS2 && wrt != WAVE_WRT_VELOCITY) return WAVE_ERR_ARG;
    BatchLayout B;
    wave_status_t st = plan_batch(probs, nprob, store, work, B);
    if (st) return st;
    if (nprob == 0) return WAVE_OK;
    for (int i = 0; i < nprob; ++i) {
        const wave_problem_t& q = probs[i];
        if (!q.vel || !q.grad || (q.nsrc && !q.wavelet) || (q.nrec && !q.d_obs)) return WAVE_ERR_ARG;
    }
    if (B.bytes > 0 && (!work || work_bytes < B.bytes)) return WAVE_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(work) % 256) return WAVE_ERR_WORKSPACE;

    // set-up: tables, models, stability check, injection factors
    BCK(cudaMemcpyAsync(B.d_probs, B.bp.data(), nprob * sizeof(BProb), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(B.d_tile_prob, B.tile_prob.data(), B.ntile * sizeof(int), cudaMemcpyHostToDevice, s));
    BCK(cudaMemsetAsync(B.err, 0, 4 * sizeof(int), s));
    BCK(cudaMemsetAsync(B.vmax, 0, nprob * sizeof(float), s));
    for (int i = 0; i < nprob; ++i) {
        HostProb& h = B.hp[i];
        BProb& p = B.bp[i];
        if ((st = upload_list(h.hs, h.gw_s, p.src, s))) return st;
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
        // levels, accumulators and the first rows of the store and the slots start at zero
        BCK(cudaMemsetAsync(p.w[0], 0, d.cell * sizeof(float), s));
        BCK(cudaMemsetAsync(p.w[1], 0, d.cell * sizeof(float), s));
        BCK(cudaMemsetAsync(p.a[0], 0, d.cell * sizeof(float), s));
        BCK(cudaMemsetAsync(p.a[1], 0, d.cell * sizeof(float), s));
        BCK(cudaMemsetAsync(p.g, 0, d.cell * sizeof(float), s));
        if (p.st16) BCK(cudaMemsetAsync(p.st16, 0, d.cell * sizeof(__nv_bfloat16), s));
        if (p.st32) BCK(cudaMemsetAsync(p.st32, 0, d.cell * sizeof(float), s));
        if (p.rec.ntap) BCK(cudaMemsetAsync(p.slots, 0, p.rec.ntap * sizeof(float), s));
    }
    BCK(cudaGetLastError());

    if (use_graph) {
        std::vector<uintptr_t> key = graph_key(probs, nprob, store, wrt, work);
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
            st = compute_phase(B, probs, nprob, wrt, true, cs);
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
        if ((st = compute_phase(B, probs, nprob, wrt, false, s))) return st;
    }
    std::vector<double> mf(nprob);
    BCK(cudaMemcpyAsync(mf.data(), B.misfit, nprob * sizeof(double), cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (herr & kErrTimeout) return WAVE_ERR_TIMEOUT;
    if (herr & kErrNonFinite) return WAVE_ERR_NONFINITE;
    if (herr) return WAVE_ERR_CUDA;
    for (int i = 0; i < nprob; ++i) probs[i].misfit = mf[i];
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
