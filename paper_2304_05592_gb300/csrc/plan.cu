// plan.cu -- host-side planning: padded geometry, tiling, interpolation tap
// tables grouped per tile, and the binomial checkpoint schedule.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace wave {

Dims make_dims(const wave_grid_t& g)
{
    Dims d;
    d.ndim = g.ndim;
    d.nx = g.nx;
    d.ny = g.ndim == 3 ? g.ny : 1;
    d.nz = g.nz;
    d.nb = g.nb;
    d.nt = g.nt;
    d.Nx = g.nx + 2 * g.nb;
    d.Ny = g.ndim == 3 ? g.ny + 2 * g.nb : 1;
    d.Nz = g.nz + 2 * g.nb;
    d.P = (d.Nx + 31) / 32 * 32;
    d.cell = (long long)d.Nz * d.Ny * d.P;
    d.phys = (long long)d.nx * d.ny * d.nz;
    d.h = g.h;
    d.dt = g.dt;
    d.vref = g.vref;
    return d;
}

// Variants picked by wave_autotune, per (padded grid, shot count).
namespace {
std::mutex g_tuned_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tuned;
}  // namespace

void remember_tuning(const Dims& d, int nshot, int vf, int va)
{
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    g_tuned[std::make_tuple(d.Nx, d.Nz, nshot)] = std::make_pair(vf, va);
}

Tiling choose_tiling(const Dims& d, int nshot)
{
    Tiling t;
    t.TX = kTX;
    t.vf = t.va = t.v3 = -1;
    if (d.ndim == 2) {
        t.TY = 1;
        t.TZc = kTZc2;
        t.vf = current_variant(0);
        t.va = current_variant(1);
        // an explicit wave_set_variant wins over a tuned choice
        std::lock_guard<std::mutex> lock(g_tuned_mu);
        auto it = g_tuned.find(std::make_tuple(d.Nx, d.Nz, nshot));
        if (it != g_tuned.end()) {
            if (!variant_forced(0)) t.vf = it->second.first;
            if (!variant_forced(1)) t.va = it->second.second;
        }
    } else {
        t.TY = 8;
        t.TZc = 4;  // divides every 3D variant's planes per CTA (32, 64, 76, 96)
        t.v3 = current_variant(2);
    }
    t.ncx = (d.Nx + t.TX - 1) / t.TX;
    t.ncy = (d.Ny + t.TY - 1) / t.TY;
    t.ncz = (d.Nz + t.TZc - 1) / t.TZc;
    return t;
}

int gradient_accumulators(const Tiling& t, int ndim, int nshot)
{
    if (ndim != 2) return nshot;
    const Variant2D v = variant_info(1, t.va);
    if (v.kind == 5) {
        const int ntz = (t.ncz * t.TZc + v.TZ - 1) / v.TZ;
        return persistent_slots(t.va, t.ncx, ntz, nshot);
    }
    return v.kind == 2 || v.kind == 4 || v.kind == 7 ? (nshot + v.G - 1) / v.G : nshot;
}

// Interpolation taps of one point: bilinear (2D) / trilinear (3D) weights on
// the padded grid, dropping taps of weight zero.
static bool point_taps(const Dims& d, const float* c, int* idx, float* w, int* n)
{
    const int nax = d.ndim;
    int nphys[3], npad[3];
    nphys[0] = d.nx;
    npad[0] = d.Nx;
    if (nax == 2) {
        nphys[1] = d.nz;
        npad[1] = d.Nz;
    } else {
        nphys[1] = d.ny;
        npad[1] = d.Ny;
        nphys[2] = d.nz;
        npad[2] = d.Nz;
    }
    int i0[3];
    double fr[3];
    const double h = d.h;
    for (int a = 0; a < nax; ++a) {
        const double x = c[a];
        if (!std::isfinite(x) || x < 0.0 || x > (nphys[a] - 1) * h) return false;
        const double f = x / h + d.nb;
        int i = (int)floor(f);
        if (i > npad[a] - 2) i = npad[a] - 2;
        i0[a] = i;
        fr[a] = f - i;
    }
    int k = 0;
    for (int corner = 0; corner < (1 << nax); ++corner) {
        double ww = 1.0;
        int ix = i0[0] + (corner & 1), iy = 0, iz;
        ww *= (corner & 1) ? fr[0] : 1.0 - fr[0];
        if (nax == 2) {
            iz = i0[1] + ((corner >> 1) & 1);
            ww *= ((corner >> 1) & 1) ? fr[1] : 1.0 - fr[1];
        } else {
            iy = i0[1] + ((corner >> 1) & 1);
            ww *= ((corner >> 1) & 1) ? fr[1] : 1.0 - fr[1];
            iz = i0[2] + ((corner >> 2) & 1);
            ww *= ((corner >> 2) & 1) ? fr[2] : 1.0 - fr[2];
        }
        if (ww == 0.0) continue;
        idx[k] = (int)(((long long)iz * d.Ny + iy) * d.P + ix);
        w[k] = (float)ww;
        ++k;
    }
    *n = k;
    return true;
}

wave_status_t build_taps(const Dims& d, const Tiling& t, int nshot, int npts, const float* xyz, HostTaps& out)
{
    out = HostTaps();
    out.npts = npts;
    const long long cps = t.cells_per_shot();
    const long long npts_all = (long long)nshot * npts;
    std::vector<int> cell_of;
    std::vector<int> idx_pt, ab_pt;
    std::vector<float> w_pt;
    out.pt_start.resize(npts_all + 1);
    cell_of.reserve(npts_all * 2);
    int tmp_idx[8];
    float tmp_w[8];
    for (int s = 0; s < nshot; ++s) {
        for (int p = 0; p < npts; ++p) {
            const long long pt = (long long)s * npts + p;
            out.pt_start[pt] = (int)idx_pt.size();
            int n = 0;
            if (!point_taps(d, xyz + pt * d.ndim, tmp_idx, tmp_w, &n)) return WAVE_ERR_GEOMETRY;
            for (int k = 0; k < n; ++k) {
                const int i = tmp_idx[k];
                const int x = i % d.P;
                const int r = i / d.P;
                const int y = r % d.Ny;
                const int z = r / d.Ny;
                // cells in (shot, cx, cy, cz) order with cz fastest
                const long long cell = (((long long)s * t.ncx + x / t.TX) * t.ncy + y / t.TY) * t.ncz + z / t.TZc;
                cell_of.push_back((int)cell);
                idx_pt.push_back(i);
                w_pt.push_back(tmp_w[k]);
                ab_pt.push_back((int)((long long)s * d.nt * npts + p));
            }
        }
    }
    out.pt_start[npts_all] = (int)idx_pt.size();
    const size_t ntap = idx_pt.size();
    // Stable counting sort of the taps by cell.
    out.cell_start.assign(nshot * cps + 1, 0);
    for (size_t j = 0; j < ntap; ++j) out.cell_start[cell_of[j] + 1]++;
    for (long long i = 0; i < nshot * cps; ++i) out.cell_start[i + 1] += out.cell_start[i];
    std::vector<int> fill(out.cell_start.begin(), out.cell_start.end() - 1);
    out.idx.resize(ntap);
    out.w.resize(ntap);
    out.ab.resize(ntap);
    out.slot.resize(ntap);
    std::vector<int> order(ntap);
    for (size_t j = 0; j < ntap; ++j) order[fill[cell_of[j]]++] = (int)j;
    // Inside a cell, taps of the same grid point become adjacent (stable by
    // point order), so one thread can own each injected point.
    for (long long c = 0; c < nshot * cps; ++c)
        std::stable_sort(order.begin() + out.cell_start[c], order.begin() + out.cell_start[c + 1],
                         [&](int x, int y) { return idx_pt[x] < idx_pt[y]; });
    for (size_t pos = 0; pos < ntap; ++pos) {
        const int j = order[pos];
        out.idx[pos] = idx_pt[j];
        out.w[pos] = w_pt[j];
        out.ab[pos] = ab_pt[j];
        out.slot[pos] = j;
    }
    return WAVE_OK;
}

// ---------------------------------------------------------------------------
// Binomial checkpointing (after Griewank & Walther's optimal reversal with a
// fixed number of snapshots), written over "macro positions": the state at
// position p, S_j(p) = (u^j, u^{j-1}), serves the adjoint steps j and j - 1.
// Unlike a reversal that needs the state *before* each step, every adjoint
// pair here needs the state *at* its own position, so a snapshot serves its
// position directly.  rev(a, b, s) runs the adjoint pairs of positions
// b, b-1, ..., a (a only if a > 0) with the state at a restorable and s free
// slots.  Cost model (macro advances):
//   T(0, s) = 0,  T(l, 0) = l (l + 1) / 2,
//   T(l, s) = min_{1<=m<=l}  m + T(l - m, s - 1) + T(m - 1, s).
// The split cost is convex in m and its first minimiser grows with l, so each
// row is filled with a pointer that only moves forward.  With s >= l this is
// a single sweep (m = 1 everywhere).
namespace {

struct CostTable {
    int L = 0, S = 0;
    std::vector<std::vector<long long>> T;
    std::vector<std::vector<int>> opt;
};

CostTable build_costs(int L, int S)
{
    CostTable c;
    c.L = L;
    c.S = S;
    c.T.assign(S + 1, std::vector<long long>(L + 1, 0));
    c.opt.assign(S + 1, std::vector<int>(L + 1, 0));
    for (int l = 0; l <= L; ++l) c.T[0][l] = (long long)l * (l + 1) / 2;
    for (int s = 1; s <= S; ++s) {
        int m = 1;
        for (int l = 1; l <= L; ++l) {
            if (m > l) m = l;
            auto f = [&](int mm) { return mm + c.T[s - 1][l - mm] + c.T[s][mm - 1]; };
            while (m + 1 <= l && f(m + 1) < f(m)) ++m;
            c.T[s][l] = f(m);
            c.opt[s][l] = m;
        }
    }
    return c;
}

struct Emitter {
    const CostTable& c;
    Schedule& sch;
    int at = 0;                   // macro position held by the working state
    std::vector<int> slot_of;     // slot holding the state of a macro position (-1: none)
    std::vector<int> free_slots;
    bool finalized = false;

    void ensure_at(int a)
    {
        if (at == a) return;
        const int slot = a == 0 ? -1 : slot_of[a];
        sch.actions.push_back({kRestore, slot, a});
        at = a;
    }
    void advance(int a, int b)
    {
        sch.actions.push_back({kAdvance, a, b});
        sch.advances += b - a;
        sch.fwd_steps += sch.state_of(b) - sch.state_of(a);
        at = b;
    }
    void adjoint_pair(int p)
    {
        if (!finalized) {
            sch.actions.push_back({kFinalize, 0, 0});
            finalized = true;
        }
        sch.actions.push_back({kAdjointPair, p, p});
    }
    void rev(int a, int b, int s)
    {
        const int l = b - a;
        if (l == 0) {
            if (a > 0) {
                ensure_at(a);
                adjoint_pair(a);
            }
            return;
        }
        if (s == 0) {
            for (int p = b; p >= a && p > 0; --p) {
                ensure_at(a);
                if (p > a) advance(a, p);
                adjoint_pair(p);
            }
            return;
        }
        const int m = c.opt[std::min(s, c.S)][l];
        const int cpos = a + m;
        ensure_at(a);
        advance(a, cpos);
        const int slot = free_slots.back();
        free_slots.pop_back();
        sch.actions.push_back({kSave, slot, cpos});
        slot_of[cpos] = slot;
        rev(cpos, b, s - 1);
        slot_of[cpos] = -1;
        free_slots.push_back(slot);
        rev(a, cpos - 1, s);
    }
};

}  // namespace

Schedule make_schedule(int nt, int nsnap)
{
    Schedule sch;
    sch.K = nt - 1;
    if (sch.K < 1) return sch;
    sch.jmin = (sch.K % 2 == 1) ? 1 : 2;
    sch.L = (sch.K - sch.jmin) / 2 + 1;
    const int S = std::max(0, std::min(nsnap, sch.L));
    sch.nsnap = S;
    static std::mutex mu;
    static std::map<std::pair<int, int>, CostTable> cache;
    std::lock_guard<std::mutex> lock(mu);  // held while the cached table is in use
    auto key = std::make_pair(sch.L, S);
    auto it = cache.find(key);
    if (it == cache.end()) {
        if (cache.size() > 16) cache.clear();
        it = cache.emplace(key, build_costs(sch.L, S)).first;
    }
    Emitter e{it->second, sch};
    e.slot_of.assign(sch.L + 1, -1);
    for (int i = S - 1; i >= 0; --i) e.free_slots.push_back(i);
    e.rev(0, sch.L, S);
    return sch;
}

}  // namespace wave
