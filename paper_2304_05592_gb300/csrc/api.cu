// api.cu -- the extern "C" entry points of libwave and the host orchestration
// of the time loops (forward sweep, adjoint sweep, checkpointed reversal).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>

#include "internal.h"

using namespace wave;

namespace {

constexpr int kNumPartials = 1024;

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

struct DevTaps {
    TapList l;
    int *cell_start = nullptr, *idx = nullptr, *ab = nullptr, *slot = nullptr, *pt_start = nullptr;
    float *fac = nullptr, *gw = nullptr, *w = nullptr;
    std::vector<float> gw_host;
};

// Workspace layout.  Every field batch ([nshot][cell] floats) is one buffer of
// a single pool with a fixed stride, so a buffer is named by its index (and one
// TMA map covers them all):
//   forward  : W0 W1
//   adjoint  : A0 A1
//   gradient : W0 W1 A0 A1 G Z S(0).cur S(0).prev ... [FP32 store rows 0..nt-1]
//   Born     : W0 W1 W2 (background levels) A0 A1 (scattered levels)
// W = forward levels, A = adjoint levels, G = per-shot gradient accumulators,
// Z = a zero batch (the state before the first step), S(k) = checkpoint slot k.
// The first 256 bytes of every workspace: the device error word of the last
// call queued on it and that call's misfit, read back by wave_status_wait.
struct WsHeader {
    int err[4];
    double misfit;
    float vmax;
};
static_assert(sizeof(WsHeader) <= 256, "the header fits the first carved block");

struct Layout {
    Dims d;
    Tiling t;
    int op = 0, nshot = 0, nsrc = 0, nrec = 0, store = 0, nsnap = 0;
    HostTaps hs, hr;
    DevTaps ts, tr;
    int* err = nullptr;
    float* vmax = nullptr;
    double* part = nullptr;
    double* misfit = nullptr;
    float* kap = nullptr;
    float* pool = nullptr;
    int nbuf = 0;
    int iW0 = -1, iA0 = -1, iG = -1, iZ = -1, iS0 = -1, iT0 = -1;
    float* slots_rec = nullptr;
    float* slots_src = nullptr;
    float* dsyn = nullptr;
    float* dmv = nullptr;
    __nv_bfloat16* st16 = nullptr;
    size_t bytes = 0;
    StepMaps maps;

    size_t field() const { return (size_t)nshot * d.cell; }
    float* buf(int i) const { return pool + (size_t)i * field(); }
};

bool finite_pos(float x) { return isfinite(x) && x > 0.0f; }

wave_status_t check_grid(const wave_grid_t* g)
{
    if (!g) return WAVE_ERR_ARG;
    if (g->ndim != 2 && g->ndim != 3) return WAVE_ERR_ARG;
    if (g->nx < 2 || g->nz < 2 || (g->ndim == 3 && g->ny < 2)) return WAVE_ERR_ARG;
    if (g->nb < 0 || g->nt < 1) return WAVE_ERR_ARG;
    if (!finite_pos(g->h) || !finite_pos(g->dt) || !isfinite(g->vref) || g->vref < 0.0f) return WAVE_ERR_ARG;
    const Dims d = make_dims(*g);
    if (d.cell >= (1LL << 31)) return WAVE_ERR_ARG;  // flat indices are 32-bit
    return WAVE_OK;
}

void carve_taps(Carver& c, const HostTaps& h, long long ncells_all, DevTaps& t)
{
    const size_t ntap = h.idx.size();
    t.cell_start = c.take<int>(ncells_all + 1);
    t.idx = c.take<int>(ntap);
    t.fac = c.take<float>(ntap);
    t.gw = c.take<float>(ntap);
    t.ab = c.take<int>(ntap);
    t.slot = c.take<int>(ntap);
    t.w = c.take<float>(ntap);
    t.pt_start = c.take<int>(h.pt_start.size());
    t.l.cell_start = t.cell_start;
    t.l.idx = t.idx;
    t.l.fac = t.fac;
    t.l.gw = t.gw;
    t.l.ab = t.ab;
    t.l.slot = t.slot;
    t.l.w = t.w;
    t.l.pt_start = t.pt_start;
    t.l.npts = h.npts;
    t.l.ntap = (int)ntap;
}

int macro_count(int nt)
{
    const int K = nt - 1;
    if (K < 1) return 0;
    const int jmin = (K % 2 == 1) ? 1 : 2;
    return (K - jmin) / 2 + 1;
}

// Builds the tap tables and carves the workspace (base may be NULL to size it).
wave_status_t plan(const wave_grid_t* g, int op, int nshot, int nsrc, const float* src_xyz, int nrec,
                   const float* rec_xyz, int store, int nsnap, void* base, Layout& L)
{
    wave_status_t st = check_grid(g);
    if (st) return st;
    if (op < 0 || op > 3 || nshot < 0 || nsrc < 0 || nrec < 0) return WAVE_ERR_ARG;
    if ((nshot && nsrc && !src_xyz) || (nshot && nrec && !rec_xyz)) return WAVE_ERR_ARG;
    if (op == 2 && (store < 0 || store > 2 || (store == WAVE_STORE_CHECKPOINT && nsnap < 1))) return WAVE_ERR_ARG;
    if ((long long)nshot * g->nt * std::max(nsrc, nrec) >= (1LL << 31)) return WAVE_ERR_ARG;
    L.d = make_dims(*g);
    L.t = choose_tiling(L.d, nshot);
    L.op = op;
    L.nshot = nshot;
    L.nsrc = nsrc;
    L.nrec = nrec;
    L.store = store;
    const Dims& d = L.d;
    st = build_taps(d, L.t, nshot, nsrc, src_xyz, L.hs);
    if (st) return st;
    st = build_taps(d, L.t, nshot, nrec, rec_xyz, L.hr);
    if (st) return st;

    const long long ncells_all = (long long)nshot * L.t.cells_per_shot();
    const size_t nt = (size_t)d.nt;
    if (op == 0) {
        L.iW0 = 0;
        L.nbuf = 2;
    } else if (op == 1) {
        L.iA0 = 0;
        L.nbuf = 2;
    } else if (op == 3) {
        L.iW0 = 0;  // three background levels W0 W1 W2, then the scattered field A0 A1
        L.iA0 = 3;
        L.nbuf = 5;
    } else {
        L.iW0 = 0;
        L.iA0 = 2;
        L.iG = 4;
        L.iZ = 5;
        L.iS0 = 6;
        L.nsnap = store == WAVE_STORE_CHECKPOINT ? std::max(0, std::min(nsnap, macro_count(d.nt))) : 0;
        L.nbuf = 6 + 2 * L.nsnap;
        if (store == WAVE_STORE_FP32) {
            L.iT0 = L.nbuf;
            L.nbuf += (int)nt;
        }
    }
    Carver c(base);
    WsHeader* hdr = c.take<WsHeader>(1);  // offset 0
    L.err = hdr ? hdr->err : nullptr;
    L.vmax = hdr ? &hdr->vmax : nullptr;
    L.misfit = hdr ? &hdr->misfit : nullptr;
    L.part = c.take<double>(kNumPartials);
    L.kap = c.take<float>(d.cell);
    carve_taps(c, L.hs, ncells_all, L.ts);
    carve_taps(c, L.hr, ncells_all, L.tr);
    L.pool = c.take<float>((size_t)L.nbuf * L.field());
    if (op == 0 || op == 2 || op == 3) L.slots_rec = c.take<float>(nt * L.hr.idx.size());
    if (op == 3) L.dmv = c.take<float>(d.cell);
    if (op == 1) L.slots_src = c.take<float>(nt * L.hs.idx.size());
    if (op == 2) {
        L.dsyn = c.take<float>((size_t)nshot * nt * nrec);
        if (store == WAVE_STORE_BF16) L.st16 = c.take<__nv_bfloat16>(nt * L.field());
    }
    L.bytes = c.off;
    // Gather weights: receivers sample with w; the source-side adjoint
    // gathers dt^2 w / h^ndim (the transpose of the injection).
    const double hd = d.ndim == 3 ? (double)d.h * d.h * d.h : (double)d.h * d.h;
    L.tr.gw_host.assign(L.hr.w.begin(), L.hr.w.end());
    L.ts.gw_host.resize(L.hs.w.size());
    for (size_t j = 0; j < L.hs.w.size(); ++j) L.ts.gw_host[j] = (float)(L.hs.w[j] * (double)d.dt * d.dt / hd);
    return WAVE_OK;
}

#define CK(x)                         \
    do {                              \
        cudaError_t e_ = (x);         \
        if (e_ != cudaSuccess) {      \
            note_cuda_error(e_);      \
            (void)cudaGetLastError(); \
            return WAVE_ERR_CUDA;     \
        }                             \
    } while (0)

// --- TMA descriptors -------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder()
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

bool encode(CUtensorMap* m, CUtensorMapDataType type, int rank, void* ptr, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box)
{
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return fn(m, type, (cuuint32_t)rank, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps over the field pool, the model and the BF16 store (the 2D kernels use them).
wave_status_t make_maps(Layout& L)
{
    memset(&L.maps, 0, sizeof(L.maps));
    const Dims& d = L.d;
    if (d.ndim == 3) {
        const Variant2D v = variant_info(2, L.t.v3);
        if (v.kind != 6) return WAVE_OK;
        const cuuint64_t dims[5] = {(cuuint64_t)d.Nx, (cuuint64_t)d.Ny, (cuuint64_t)d.Nz, (cuuint64_t)L.nshot,
                                    (cuuint64_t)L.nbuf};
        const cuuint64_t str[4] = {(cuuint64_t)d.P * 4, (cuuint64_t)d.Ny * d.P * 4, (cuuint64_t)d.cell * 4,
                                   (cuuint64_t)L.field() * 4};
        const cuuint32_t box[5] = {kTX + 8, (cuuint32_t)v.R + 8, 1, 1, 1};
        return encode(&L.maps.halo3, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, L.pool, dims, str, box) ? WAVE_OK
                                                                                                : WAVE_ERR_CUDA;
    }
    if (d.ndim != 2) return WAVE_OK;
    const cuuint64_t fdims[4] = {(cuuint64_t)d.Nx, (cuuint64_t)d.Nz, (cuuint64_t)L.nshot, (cuuint64_t)L.nbuf};
    const cuuint64_t fstr[3] = {(cuuint64_t)d.P * 4, (cuuint64_t)d.cell * 4, (cuuint64_t)L.field() * 4};
    const cuuint64_t kdims[2] = {(cuuint64_t)d.Nx, (cuuint64_t)d.Nz};
    const cuuint64_t kstr[1] = {(cuuint64_t)d.P * 4};
    const cuuint32_t tzf = (cuuint32_t)variant_info(0, L.t.vf).TZ, tza = (cuuint32_t)variant_info(1, L.t.va).TZ;
    const cuuint32_t hb_f[4] = {kTX + 8, tzf + 8, 1, 1}, tb_f[4] = {kTX, tzf, 1, 1};
    const cuuint32_t hb_a[4] = {kTX + 8, tza + 8, 1, 1}, tb_a[4] = {kTX, tza, 1, 1};
    bool ok = encode(&L.maps.halo_f, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.pool, fdims, fstr, hb_f) &&
              encode(&L.maps.tile_f, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.pool, fdims, fstr, tb_f) &&
              encode(&L.maps.halo_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.pool, fdims, fstr, hb_a) &&
              encode(&L.maps.tile_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.pool, fdims, fstr, tb_a) &&
              encode(&L.maps.kap_f, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, L.kap, kdims, kstr, tb_f) &&
              encode(&L.maps.kap_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, L.kap, kdims, kstr, tb_a);
    if (ok && L.st16) {
        const cuuint64_t sdims[4] = {(cuuint64_t)d.Nx, (cuuint64_t)d.Nz, (cuuint64_t)L.nshot, (cuuint64_t)d.nt};
        const cuuint64_t sstr[3] = {(cuuint64_t)d.P * 2, (cuuint64_t)d.cell * 2, (cuuint64_t)L.field() * 2};
        ok = encode(&L.maps.tile16_a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, L.st16, sdims, sstr, tb_a);
    }
    return ok ? WAVE_OK : WAVE_ERR_CUDA;
}

// --- set-up ----------------------------------------------------------------

// Pinned host staging for the set-up tables.  A copy from pageable host
// memory makes the host wait for the stream's earlier work, so each call
// instead writes its tables into a pinned buffer and uploads them with one
// asynchronous copy.  A buffer is handed out again once the event recorded
// after its copy has completed; at most kMaxStage buffers exist, after which
// the oldest is waited for.  These are host allocations (cudaHostAlloc) made
// the first few times a larger table is needed; device memory is never
// allocated.
struct StageBuf {
    char* p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    int dev = -1;
    bool busy = false;
    unsigned long long used = 0;  // order of last use
};
constexpr int kMaxStage = 8;
std::mutex g_stage_mu;
StageBuf g_stage[kMaxStage];
unsigned long long g_stage_clock = 0;

wave_status_t stage_acquire(size_t need, int* out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_stage_mu);
    int pick = -1, empty = -1, oldest = -1;
    for (int i = 0; i < kMaxStage; ++i) {
        StageBuf& b = g_stage[i];
        if (b.busy) continue;
        if (!b.p) {
            if (empty < 0) empty = i;
            continue;
        }
        if (b.dev != dev) continue;
        if (cudaEventQuery(b.ev) != cudaSuccess) {
            if (oldest < 0 || b.used < g_stage[oldest].used) oldest = i;
            continue;
        }
        if (b.cap >= need && (pick < 0 || b.cap < g_stage[pick].cap)) pick = i;
        else if (b.cap < need && empty < 0) empty = -2 - i;  // an idle buffer that is too small: replace it
    }
    if (pick < 0 && empty != -1) {
        const int i = empty >= 0 ? empty : -2 - empty;
        StageBuf& b = g_stage[i];
        if (b.p) {
            cudaFreeHost(b.p);
            cudaEventDestroy(b.ev);
            b = StageBuf();
        }
        const size_t cap = std::max<size_t>(need, 1 << 16);
        void* p = nullptr;
        CK(cudaHostAlloc(&p, cap, cudaHostAllocPortable));
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaFreeHost(p);
            (void)cudaGetLastError();
            return WAVE_ERR_CUDA;
        }
        b.p = static_cast<char*>(p);
        b.cap = cap;
        b.ev = ev;
        b.dev = dev;
        pick = i;
    }
    if (pick < 0) {
        // every buffer of this device is in flight (or none fits): wait for the oldest one
        if (oldest < 0) return WAVE_ERR_CUDA;  // all buffers belong to busy calls of other devices
        StageBuf& b = g_stage[oldest];
        CK(cudaEventSynchronize(b.ev));
        if (b.cap < need) {
            cudaFreeHost(b.p);
            void* p = nullptr;
            b.p = nullptr;
            b.cap = 0;
            CK(cudaHostAlloc(&p, need, cudaHostAllocPortable));
            b.p = static_cast<char*>(p);
            b.cap = need;
        }
        pick = oldest;
    }
    g_stage[pick].busy = true;
    g_stage[pick].used = ++g_stage_clock;
    *out = pick;
    return WAVE_OK;
}

void stage_release(int i, cudaStream_t s)
{
    std::lock_guard<std::mutex> lock(g_stage_mu);
    cudaEventRecord(g_stage[i].ev, s);
    g_stage[i].busy = false;
}

// Uploads both tap tables with one copy: the source and receiver arrays are
// carved back to back, so the staged image mirrors that whole region (the
// injection factors in it are filled on the device afterwards).
wave_status_t upload_taps(Layout& L, cudaStream_t s)
{
    char* base = reinterpret_cast<char*>(L.ts.cell_start);
    char* end = reinterpret_cast<char*>(L.tr.pt_start + L.hr.pt_start.size());
    const size_t n = (size_t)(end - base);
    int sb = -1;
    wave_status_t st = stage_acquire(n, &sb);
    if (st) return st;
    char* h = g_stage[sb].p;
    auto put = [&](const void* dst, const void* src, size_t bytes) {
        if (bytes) memcpy(h + (reinterpret_cast<const char*>(dst) - base), src, bytes);
    };
    for (int k = 0; k < 2; ++k) {
        const HostTaps& ht = k ? L.hr : L.hs;
        const DevTaps& t = k ? L.tr : L.ts;
        const size_t ntap = ht.idx.size();
        put(t.cell_start, ht.cell_start.data(), ht.cell_start.size() * sizeof(int));
        put(t.pt_start, ht.pt_start.data(), ht.pt_start.size() * sizeof(int));
        put(t.idx, ht.idx.data(), ntap * sizeof(int));
        put(t.ab, ht.ab.data(), ntap * sizeof(int));
        put(t.slot, ht.slot.data(), ntap * sizeof(int));
        put(t.w, ht.w.data(), ntap * sizeof(float));
        put(t.gw, t.gw_host.data(), ntap * sizeof(float));
    }
    const cudaError_t e = cudaMemcpyAsync(base, h, n, cudaMemcpyHostToDevice, s);
    stage_release(sb, s);
    CK(e);
    return WAVE_OK;
}

double courant_limit(int ndim)
{
    // 2048/315 is the largest magnitude of the 1D 8th-order symbol (at the
    // Nyquist wavenumber); leapfrog is stable for ndim K (v dt / h)^2 <= 4.
    if (ndim != 2 && ndim != 3) return 0.0;
    return 2.0 / sqrt(ndim * 2048.0 / 315.0);
}

// c_eps such that eps = kap * c_eps * depth^2 equals eta dt v^2 / 2 with
// eta = gamma0 (depth/nb)^2 / vref^2, gamma0 = 3 vref ln(1000) / (2 nb h).
float sponge_coefficient(const Dims& d)
{
    if (d.nb == 0 || d.vref <= 0.0f) return 0.0f;
    const double nb = d.nb;
    return (float)(3.0 * log(1000.0) * d.h / (4.0 * d.dt * d.vref * nb * nb * nb));
}

// Uploads tables, prepares the model, queues its validation (non-finite
// velocities and the stability limit set bits of the device error word; the
// host does not wait for them), fills the injection factors and encodes the
// TMA maps.
wave_status_t setup(Layout& L, const float* vel, cudaStream_t s)
{
    wave_status_t st = upload_taps(L, s);
    if (st) return st;
    CK(cudaMemsetAsync(L.err, 0, sizeof(WsHeader), s));  // error word, misfit and vmax
    launch_prep(L.d, vel, L.kap, L.vmax, L.err, s);
    launch_check_cfl(L.vmax, (double)L.d.dt / L.d.h, courant_limit(L.d.ndim), L.err, s);
    CK(cudaGetLastError());
    const float ceps = sponge_coefficient(L.d);
    const double h = L.d.h, dt = L.d.dt;
    // Forward source injection adds dt^2 w q / (h^ndim (m + e)) = kap h^(2-ndim) w q / (1 + eps).
    launch_tapfac(L.d, L.ts.l, L.kap, (float)(L.d.ndim == 3 ? 1.0 / h : 1.0), ceps, s);
    // Adjoint receiver injection adds w r / (m + e) = kap (h/dt)^2 w r / (1 + eps).
    launch_tapfac(L.d, L.tr.l, L.kap, (float)(h * h / (dt * dt)), ceps, s);
    CK(cudaGetLastError());
    return make_maps(L);
}

StepArgs base_args(const Layout& L)
{
    StepArgs a;
    memset(&a, 0, sizeof(a));
    const Dims& d = L.d;
    a.kap = L.kap;
    a.Nx = d.Nx;
    a.Ny = d.Ny;
    a.Nz = d.Nz;
    a.P = d.P;
    a.cell = d.cell;
    a.nb = d.nb;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.nshot = L.nshot;
    a.ceps = sponge_coefficient(d);
    a.ncx = L.t.ncx;
    a.ncy = L.t.ncy;
    a.ncz = L.t.ncz;
    a.TZc = L.t.TZc;
    a.err = L.err;
    a.u_buf = a.prev_buf = a.uf_buf = a.g_buf = a.uf16_row = -1;
    return a;
}

// Forward step n: reads u^n (buffer cur) and u^{n-1} (buffer prev), writes
// u^{n+1} into buffer out (which may be prev), injecting q^n; optionally
// records d^{n+1} and stores u^{n+1} (BF16 row or FP32 buffer).
void fwd_step(const Layout& L, int cur, int prev, int out, int n, const float* wavelet, bool record,
              __nv_bfloat16* st16, float* st32, cudaStream_t s)
{
    StepArgs a = base_args(L);
    a.u = L.buf(cur);
    a.uprev = L.buf(prev);
    a.unew = L.buf(out);
    a.u_buf = cur;
    a.prev_buf = prev;
    if (L.nsrc > 0 && L.ts.l.ntap > 0) {
        a.inj = L.ts.l;
        a.amp_a = wavelet;
        a.amp_row = n;
    }
    if (record && L.nrec > 0 && L.tr.l.ntap > 0) {
        a.gat = L.tr.l;
        a.slots = L.slots_rec;
        a.slot_row = n + 1;
    }
    a.st16 = st16;
    a.st32 = st32;
    launch_step(L.t, L.d.ndim, false, a, &L.maps, s);
}

// Adjoint step k: reads mu^{k+1} (buffer cur) and mu^{k+2} (buffer prev),
// writes mu^k over mu^{k+2}, injecting amp_a - amp_b at time k at the
// receivers; optionally gathers the source-side adjoint (F' r)^{k-1}; with a
// forward field (buffer uf, or BF16 row uf16_row) accumulates the imaging
// condition into the gradient buffer.
void adj_step(const Layout& L, int cur, int prev, int k, const float* amp_a, const float* amp_b, bool gather_src,
              int uf, int uf16_row, cudaStream_t s)
{
    StepArgs a = base_args(L);
    a.u = L.buf(cur);
    a.uprev = L.buf(prev);
    a.unew = L.buf(prev);
    a.u_buf = cur;
    a.prev_buf = prev;
    if (L.nrec > 0 && L.tr.l.ntap > 0) {
        a.inj = L.tr.l;
        a.amp_a = amp_a;
        a.amp_b = amp_b;
        a.amp_row = k;
    }
    if (gather_src && L.nsrc > 0 && L.ts.l.ntap > 0) {
        a.gat = L.ts.l;
        a.slots = L.slots_src;
        a.slot_row = k - 1;
    }
    if (uf >= 0 || uf16_row >= 0) {
        a.gacc = L.buf(L.iG);
        a.g_buf = L.iG;
        if (uf >= 0) {
            a.uf32 = L.buf(uf);
            a.uf_buf = uf;
        } else {
            a.uf16 = L.st16 + (size_t)uf16_row * L.field();
            a.uf16_row = uf16_row;
        }
    }
    launch_step(L.t, L.d.ndim, true, a, &L.maps, s);
}

wave_status_t check_work(const Layout& L, void* work, size_t work_bytes)
{
    if (L.bytes > 0 && (!work || work_bytes < L.bytes)) return WAVE_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(work) % 256) return WAVE_ERR_WORKSPACE;
    return WAVE_OK;
}

// Status of a device error word; the stability limit takes precedence over
// non-finite results, which an unstable run produces.
wave_status_t status_of(int herr)
{
    if (herr & kErrTimeout) return WAVE_ERR_TIMEOUT;
    if (herr & kErrCfl) return WAVE_ERR_CFL;
    if (herr & kErrNonFinite) return WAVE_ERR_NONFINITE;
    if (herr) return WAVE_ERR_CUDA;
    return WAVE_OK;
}

// Synchronous end of a call (autotuner): waits and reads the error word.
wave_status_t finish(const Layout& L, cudaStream_t s)
{
    CK(cudaGetLastError());
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, L.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return status_of(herr);
}

// A call with no shots queues no work; it still clears the header of a
// usable workspace, so that wave_status_wait reports success for it.
wave_status_t clear_header(const Layout& L, void* work, size_t work_bytes, cudaStream_t s)
{
    if (work && check_work(L, work, work_bytes) == WAVE_OK) CK(cudaMemsetAsync(L.err, 0, sizeof(WsHeader), s));
    return WAVE_OK;
}

// Asynchronous end of a call: launch errors are reported now, device-side
// errors through wave_status_wait.
wave_status_t queued()
{
    CK(cudaGetLastError());
    return WAVE_OK;
}


// Runs the binomial checkpoint schedule without copying states: a restore
// only renames which buffers hold (u^j, u^{j-1}), the last two steps of an
// advance that ends in a save write straight into the slot, and a step that
// starts from a slot writes out of place into W0/W1.
wave_status_t run_checkpointed(Layout& L, const float* wavelet, const float* amp_a, const float* amp_b,
                               bool record_data, const std::function<void()>& finalize_data, cudaStream_t s)
{
    const Dims& d = L.d;
    const Schedule sch = make_schedule(d.nt, L.nsnap);
    const int W0 = L.iW0, W1 = L.iW0 + 1, Z = L.iZ, A0 = L.iA0;
    auto slot_cur = [&](int k) { return L.iS0 + 2 * k; };
    auto slot_prev = [&](int k) { return L.iS0 + 2 * k + 1; };
    int cur = Z, prev = Z, state = 0, recorded = 0, acur = 0;
    const size_t fb = L.field() * sizeof(float);
    for (size_t ai = 0; ai < sch.actions.size(); ++ai) {
        const Action& act = sch.actions[ai];
        switch (act.kind) {
        case kAdvance: {
            const int j0 = sch.state_of(act.a), j1 = sch.state_of(act.b);
            if (j0 != state) return WAVE_ERR_ARG;  // inconsistent schedule (not reachable)
            const bool to_slot = ai + 1 < sch.actions.size() && sch.actions[ai + 1].kind == kSave;
            const int slot = to_slot ? sch.actions[ai + 1].a : -1;
            for (int n = j0; n < j1; ++n) {
                int out;
                if (to_slot && n == j1 - 1) out = slot_cur(slot);
                else if (to_slot && n == j1 - 2) out = slot_prev(slot);
                else if (prev == W0 || prev == W1) out = prev;
                else out = cur == W0 ? W1 : W0;
                const bool rec = record_data && n >= recorded;
                fwd_step(L, cur, prev, out, n, wavelet, rec, nullptr, nullptr, s);
                if (rec) recorded = n + 1;
                prev = cur;
                cur = out;
            }
            state = j1;
            break;
        }
        case kSave: {
            const int k = act.a;
            if (cur != slot_cur(k)) CK(cudaMemcpyAsync(L.buf(slot_cur(k)), L.buf(cur), fb, cudaMemcpyDeviceToDevice, s));
            if (prev != slot_prev(k))
                CK(cudaMemcpyAsync(L.buf(slot_prev(k)), L.buf(prev), fb, cudaMemcpyDeviceToDevice, s));
            cur = slot_cur(k);
            prev = slot_prev(k);
            break;
        }
        case kRestore:
            if (act.a < 0) {
                cur = prev = Z;
            } else {
                cur = slot_cur(act.a);
                prev = slot_prev(act.a);
            }
            state = sch.state_of(act.b);
            break;
        case kFinalize:
            if (record_data && recorded != sch.K) return WAVE_ERR_ARG;  // not reachable
            finalize_data();
            break;
        case kAdjointPair: {
            const int j = sch.state_of(act.a);
            if (j != state) return WAVE_ERR_ARG;  // not reachable
            adj_step(L, A0 + acur, A0 + 1 - acur, j, amp_a, amp_b, false, cur, -1, s);
            acur ^= 1;
            if (j - 1 >= 1) {
                adj_step(L, A0 + acur, A0 + 1 - acur, j - 1, amp_a, amp_b, false, prev, -1, s);
                acur ^= 1;
            }
            break;
        }
        }
    }
    return WAVE_OK;
}

}  // namespace

extern "C" {

const char* wave_status_str(wave_status_t s)
{
    switch (s) {
    case WAVE_OK: return "ok";
    case WAVE_ERR_ARG: return "invalid argument";
    case WAVE_ERR_CFL: return "time step above the stability limit";
    case WAVE_ERR_GEOMETRY: return "source or receiver outside the physical grid";
    case WAVE_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case WAVE_ERR_CUDA: return "CUDA error";
    case WAVE_ERR_TIMEOUT: return "device-side wait timed out";
    case WAVE_ERR_NONFINITE: return "non-finite or non-positive value";
    }
    return "unknown status";
}

double wave_courant_limit(int ndim) { return courant_limit(ndim); }

wave_status_t wave_workspace_size(const wave_grid_t* grid, int op, int nshot, int nsrc, const float* src_xyz,
                                  int nrec, const float* rec_xyz, int store, int nsnap, size_t* bytes)
{
    if (!bytes) return WAVE_ERR_ARG;
    Layout L;
    wave_status_t st = plan(grid, op, nshot, nsrc, src_xyz, nrec, rec_xyz, store, nsnap, nullptr, L);
    if (st) return st;
    *bytes = L.bytes;
    return WAVE_OK;
}

wave_status_t wave_status_wait(const void* work, void* stream, double* misfit)
{
    if (!work) return WAVE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader h;
    memset(&h, 0, sizeof(h));
    CK(cudaMemcpyAsync(&h, work, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (misfit) *misfit = h.misfit;
    return status_of(h.err[0]);
}

wave_status_t wave_forward(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                           const float* wavelet, int nrec, const float* rec_xyz, float* data, void* work,
                           size_t work_bytes, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Layout L;
    wave_status_t st = plan(grid, 0, nshot, nsrc, src_xyz, nrec, rec_xyz, 0, 0, work, L);
    if (st) return st;
    if (nshot == 0) return clear_header(L, work, work_bytes, s);
    if (!vel || (nsrc && !wavelet) || (nrec && !data)) return WAVE_ERR_ARG;
    if ((st = check_work(L, work, work_bytes))) return st;
    if ((st = setup(L, vel, s))) return st;
    const size_t fb = L.field() * sizeof(float);
    CK(cudaMemsetAsync(L.buf(0), 0, 2 * fb, s));
    const size_t nrow = L.hr.idx.size();
    if (nrow) CK(cudaMemsetAsync(L.slots_rec, 0, nrow * sizeof(float), s));
    int cur = 0;
    for (int n = 0; n + 1 < L.d.nt; ++n) {
        fwd_step(L, cur, 1 - cur, 1 - cur, n, wavelet, true, nullptr, nullptr, s);
        cur ^= 1;
    }
    if (nrec) {
        launch_finalize(L.tr.l, L.slots_rec, nshot, L.d.nt, data, s);
        launch_nan_scan(data, (long long)nshot * L.d.nt * nrec, L.err, s);
    }
    return queued();
}

wave_status_t wave_adjoint(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                           int nrec, const float* rec_xyz, const float* resid, float* src_out, void* work,
                           size_t work_bytes, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Layout L;
    wave_status_t st = plan(grid, 1, nshot, nsrc, src_xyz, nrec, rec_xyz, 0, 0, work, L);
    if (st) return st;
    if (nshot == 0) return clear_header(L, work, work_bytes, s);
    if (!vel || (nrec && !resid) || (nsrc && !src_out)) return WAVE_ERR_ARG;
    if ((st = check_work(L, work, work_bytes))) return st;
    if ((st = setup(L, vel, s))) return st;
    const size_t fb = L.field() * sizeof(float);
    CK(cudaMemsetAsync(L.buf(0), 0, 2 * fb, s));
    const size_t nrow = L.hs.idx.size();
    if (nrow) CK(cudaMemsetAsync(L.slots_src + (size_t)(L.d.nt - 1) * nrow, 0, nrow * sizeof(float), s));
    int cur = 0;
    for (int k = L.d.nt - 1; k >= 1; --k) {
        adj_step(L, cur, 1 - cur, k, resid, nullptr, true, -1, -1, s);
        cur ^= 1;
    }
    if (nsrc) {
        launch_finalize(L.ts.l, L.slots_src, nshot, L.d.nt, src_out, s);
        launch_nan_scan(src_out, (long long)nshot * L.d.nt * nsrc, L.err, s);
    }
    return queued();
}

}  // extern "C"

namespace {

// J' applied to a data-space vector, summed over shots: the residual is either
// given (resid) or formed on the fly as d_syn - d_obs (then the synthetic data
// and the misfit are produced as well).
wave_status_t gradient_impl(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                            const float* wavelet, int nrec, const float* rec_xyz, const float* d_obs,
                            const float* resid, float* grad, float* d_syn, double* misfit, int store, int nsnap,
                            int wrt, void* work, size_t work_bytes, cudaStream_t s)
{
    Layout L;
    wave_status_t st = plan(grid, 2, nshot, nsrc, src_xyz, nrec, rec_xyz, store, nsnap, work, L);
    if (st) return st;
    if (wrt != WAVE_WRT_SLOWNESS2 && wrt != WAVE_WRT_VELOCITY) return WAVE_ERR_ARG;
    const bool given = resid != nullptr;
    if (!vel || !grad || (nshot && nsrc && !wavelet) || (nshot && nrec && !given && !d_obs)) return WAVE_ERR_ARG;
    if ((st = check_work(L, work, work_bytes))) return st;
    const Dims& d = L.d;
    if (nshot == 0) {
        CK(cudaMemsetAsync(L.err, 0, sizeof(WsHeader), s));
        CK(cudaMemsetAsync(grad, 0, d.phys * sizeof(float), s));
        if (misfit) *misfit = 0.0;
        return WAVE_OK;
    }
    if ((st = setup(L, vel, s))) return st;
    const size_t field = L.field();
    const size_t fb = field * sizeof(float);
    // W0 W1 A0 A1 G Z are contiguous: clear them in one go.
    CK(cudaMemsetAsync(L.buf(0), 0, 6 * fb, s));
    const size_t nrow = L.hr.idx.size();
    if (nrow && !given) CK(cudaMemsetAsync(L.slots_rec, 0, nrow * sizeof(float), s));
    const long long ndata = (long long)nshot * d.nt * nrec;
    const int K = d.nt - 1;
    const float* amp_a = given ? resid : L.dsyn;
    const float* amp_b = given ? nullptr : d_obs;

    auto finalize_data = [&]() {
        if (given) return;
        if (nrec) {
            launch_finalize(L.tr.l, L.slots_rec, nshot, d.nt, L.dsyn, s);
            launch_misfit(L.dsyn, d_obs, ndata, L.part, kNumPartials, L.misfit, s);
        } else {
            cudaMemsetAsync(L.misfit, 0, sizeof(double), s);
        }
    };

    const int W0 = L.iW0, A0 = L.iA0;
    if (store != WAVE_STORE_CHECKPOINT) {
        if (L.st16) CK(cudaMemsetAsync(L.st16, 0, field * sizeof(__nv_bfloat16), s));
        if (L.iT0 >= 0) CK(cudaMemsetAsync(L.buf(L.iT0), 0, fb, s));
        int cur = 0;
        for (int n = 0; n < K; ++n) {
            __nv_bfloat16* r16 = L.st16 ? L.st16 + (size_t)(n + 1) * field : nullptr;
            float* r32 = L.iT0 >= 0 ? L.buf(L.iT0 + n + 1) : nullptr;
            fwd_step(L, W0 + cur, W0 + 1 - cur, W0 + 1 - cur, n, wavelet, !given, r16, r32, s);
            cur ^= 1;
        }
        finalize_data();
        int acur = 0;
        for (int k = K; k >= 1; --k) {
            if (L.st16) adj_step(L, A0 + acur, A0 + 1 - acur, k, amp_a, amp_b, false, -1, k, s);
            else adj_step(L, A0 + acur, A0 + 1 - acur, k, amp_a, amp_b, false, L.iT0 + k, -1, s);
            acur ^= 1;
        }
    } else if (K < 1) {
        finalize_data();
    } else {
        st = run_checkpointed(L, wavelet, amp_a, amp_b, !given, finalize_data, s);
        if (st) return st;
    }
    // A0 and A1 (contiguous) are free now: scratch for the reduction.
    launch_grad_reduce(d, L.buf(L.iG), gradient_accumulators(L.t, d.ndim, nshot), L.buf(A0), grad,
                       wrt == WAVE_WRT_VELOCITY ? vel : nullptr, s);
    launch_nan_scan(grad, d.phys, L.err, s);
    if (!given && d_syn && ndata)
        CK(cudaMemcpyAsync(d_syn, L.dsyn, ndata * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // the misfit lands in the caller's host double when the stream gets there
    // (a copy into pageable memory completes before cudaMemcpyAsync returns)
    if (misfit) CK(cudaMemcpyAsync(misfit, L.misfit, sizeof(double), cudaMemcpyDeviceToHost, s));
    return queued();
}

}  // namespace

extern "C" {

wave_status_t wave_gradient(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                            const float* wavelet, int nrec, const float* rec_xyz, const float* d_obs, float* grad,
                            float* d_syn, double* misfit, int store, int nsnap, int wrt, void* work,
                            size_t work_bytes, void* stream)
{
    return gradient_impl(grid, vel, nshot, nsrc, src_xyz, wavelet, nrec, rec_xyz, d_obs, nullptr, grad, d_syn,
                         misfit, store, nsnap, wrt, work, work_bytes, static_cast<cudaStream_t>(stream));
}

wave_status_t wave_jacobian_adjoint(const wave_grid_t* grid, const float* vel, int nshot, int nsrc,
                                    const float* src_xyz, const float* wavelet, int nrec, const float* rec_xyz,
                                    const float* resid, float* grad, int store, int nsnap, int wrt, void* work,
                                    size_t work_bytes, void* stream)
{
    if (nshot && nrec && !resid) return WAVE_ERR_ARG;
    static const float kNone = 0.0f;
    return gradient_impl(grid, vel, nshot, nsrc, src_xyz, wavelet, nrec, rec_xyz, nullptr, resid ? resid : &kNone,
                         grad, nullptr, nullptr, store, nsnap, wrt, work, work_bytes,
                         static_cast<cudaStream_t>(stream));
}

wave_status_t wave_born(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                        const float* wavelet, int nrec, const float* rec_xyz, const float* dm, float* data, void* work,
                        size_t work_bytes, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Layout L;
    wave_status_t st = plan(grid, 3, nshot, nsrc, src_xyz, nrec, rec_xyz, 0, 0, work, L);
    if (st) return st;
    if (nshot == 0) return clear_header(L, work, work_bytes, s);
    if (!vel || !dm || (nsrc && !wavelet) || (nrec && !data)) return WAVE_ERR_ARG;
    if ((st = check_work(L, work, work_bytes))) return st;
    L.t.vf = 0;  // the direct 2D kernel carries the scattering source
    if ((st = setup(L, vel, s))) return st;
    launch_prep_dm(L.d, dm, L.kap, L.dmv, s);
    const size_t fb = L.field() * sizeof(float);
    CK(cudaMemsetAsync(L.buf(0), 0, 5 * fb, s));
    const size_t nrow = L.hr.idx.size();
    if (nrow) CK(cudaMemsetAsync(L.slots_rec, 0, nrow * sizeof(float), s));
    int cur = 0, prev = 1, nxt = 2;  // background u^n, u^{n-1}, free
    int dcur = L.iA0, dprev = L.iA0 + 1;
    for (int n = 0; n + 1 < L.d.nt; ++n) {
        fwd_step(L, cur, prev, nxt, n, wavelet, false, nullptr, nullptr, s);  // u^{n+1}
        StepArgs a = base_args(L);
        a.u = L.buf(dcur);
        a.uprev = L.buf(dprev);
        a.unew = L.buf(dprev);
        a.u_buf = dcur;
        a.prev_buf = dprev;
        a.dmv = L.dmv;
        a.bs_a = L.buf(nxt);
        a.bs_b = L.buf(cur);
        a.bs_c = L.buf(prev);
        if (nrec > 0 && L.tr.l.ntap > 0) {
            a.gat = L.tr.l;
            a.slots = L.slots_rec;
            a.slot_row = n + 1;
        }
        launch_step(L.t, L.d.ndim, false, a, &L.maps, s);
        const int t = prev;
        prev = cur;
        cur = nxt;
        nxt = t;
        std::swap(dcur, dprev);
    }
    if (nrec) {
        launch_finalize(L.tr.l, L.slots_rec, nshot, L.d.nt, data, s);
        launch_nan_scan(data, (long long)nshot * L.d.nt * nrec, L.err, s);
    }
    return queued();
}

wave_status_t wave_ricker(float f0, float dt, int nt, float* out, void* stream)
{
    if (!(f0 > 0.0f) || !(dt > 0.0f) || nt < 0 || (nt && !out)) return WAVE_ERR_ARG;
    if (nt == 0) return WAVE_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_ricker(f0, dt, nt, out, s);
    CK(cudaGetLastError());
    return WAVE_OK;
}

wave_status_t wave_autotune(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                            const float* wavelet, int nrec, const float* rec_xyz, int steps, void* work,
                            size_t work_bytes, void* stream, int* best_fwd, int* best_adj)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (steps < 1 || nshot < 1) return WAVE_ERR_ARG;
    Layout L;
    wave_status_t st = plan(grid, 2, nshot, nsrc, src_xyz, nrec, rec_xyz, WAVE_STORE_CHECKPOINT, 1, work, L);
    if (st) return st;
    if (!vel || (nsrc && !wavelet)) return WAVE_ERR_ARG;
    if ((st = check_work(L, work, work_bytes))) return st;
    if ((st = setup(L, vel, s))) return st;
    if (L.d.ndim != 2) {
        // one 3D kernel: nothing to choose
        if (best_fwd) *best_fwd = -1;
        if (best_adj) *best_adj = -1;
        return finish(L, s);
    }
    const size_t fb = L.field() * sizeof(float);
    CK(cudaMemsetAsync(L.buf(0), 0, 6 * fb, s));
    const size_t nrow = L.hr.idx.size();
    if (nrow) CK(cudaMemsetAsync(L.slots_rec, 0, (size_t)L.d.nt * nrow * sizeof(float), s));
    CK(cudaMemsetAsync(L.dsyn, 0, (size_t)nshot * L.d.nt * nrec * sizeof(float), s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int nstep = std::max(1, std::min(steps, L.d.nt - 1));
    float best[2] = {1e30f, 1e30f};
    int pick[2] = {current_variant(0), current_variant(1)};
    for (int which = 0; which < 2; ++which) {
        for (int v = 0; v < variant_count(which); ++v) {
            if (which == 0) L.t.vf = v;
            else L.t.va = v;
            if (make_maps(L)) continue;
            auto run = [&](int n_steps) {
                for (int k = 0; k < n_steps; ++k) {
                    const int n = k % std::max(1, L.d.nt - 1);
                    if (which == 0) fwd_step(L, L.iW0 + (k & 1), L.iW0 + 1 - (k & 1), L.iW0 + 1 - (k & 1), n, wavelet,
                                             true, nullptr, nullptr, s);
                    else adj_step(L, L.iA0 + (k & 1), L.iA0 + 1 - (k & 1), std::max(1, n), L.dsyn, nullptr, false,
                                  L.iW0, -1, s);
                }
            };
            run(2);
            cudaEventRecord(e0, s);
            run(nstep);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                (void)cudaGetLastError();
                return WAVE_ERR_CUDA;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best[which]) {
                best[which] = ms;
                pick[which] = v;
            }
        }
        if (which == 0) L.t.vf = pick[0];
        else L.t.va = pick[1];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st = finish(L, s);
    if (st) return st;
    remember_tuning(L.d, nshot, pick[0], pick[1]);
    if (best_fwd) *best_fwd = pick[0];
    if (best_adj) *best_adj = pick[1];
    return WAVE_OK;
}

wave_status_t wave_set_variant(int which, int variant)
{
    return select_variant(which, variant) == 0 ? WAVE_OK : WAVE_ERR_ARG;
}

int wave_variant_count(int which) { return variant_count(which); }

wave_status_t wave_checkpoint_schedule(int nt, int nsnap, long long* fwd_steps, int* actions, int capacity,
                                       int* nactions)
{
    if (nt < 1 || nsnap < 0) return WAVE_ERR_ARG;
    const Schedule sch = make_schedule(nt, nsnap);
    if (fwd_steps) *fwd_steps = sch.fwd_steps;
    if (nactions) *nactions = (int)sch.actions.size();
    if (actions) {
        const int n = std::min<int>(capacity, (int)sch.actions.size());
        for (int i = 0; i < n; ++i) {
            const Action& a = sch.actions[i];
            actions[3 * i] = a.kind;
            actions[3 * i + 1] = a.kind == kAdvance || a.kind == kAdjointPair ? sch.state_of(a.a) : a.a;
            actions[3 * i + 2] = a.kind == kFinalize ? 0 : sch.state_of(a.b);
        }
    }
    return WAVE_OK;
}

}  // extern "C"
