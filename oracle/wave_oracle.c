/*
 * wave_oracle.c -- plain, slow FP64 CPU oracle for the acoustic FWI path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls this file;
 * only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (arxiv 2304.05592, "Wave-equation-based inversion",
 * Eq. eq-fwi):  F(m) = P_r A(m)^{-1} P_s^T with m the squared slowness, the
 * misfit 1/2 ||F(m) q - d||^2, its adjoint-state gradient J'(F(m)q - d) with
 * respect to m, and the pullback F' dy of the AD rule for F*q (the rrule of the
 * same section).  The paper does not fix the discretisation; this file writes
 * out the reading used throughout the project:
 *
 *   (M+E) u^{n+1} = (2M + dt^2 L) u^n - (M-E) u^{n-1} + dt^2 S q^n ,
 *       u^{-1} = u^0 = 0,  n = 0 .. nt-2,   d^n = R u^n  (n = 0 .. nt-1)
 *
 *   M = diag(m) on the padded grid (model extended into the sponge by edge
 *   replication), E = diag(eta dt / 2) with a quadratic sponge profile that
 *   does not depend on m, L = 8th-order centred Laplacian with zero values
 *   outside the padded grid, S = bilinear/trilinear injection with weights
 *   w / h^d, R = the same interpolation used for sampling (weights w).
 *
 * Every routine is a direct loop over that definition: no blocking, no fusion.
 * OpenMP only splits the outermost grid loop across threads.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OG_OK = 0, OG_ERR_ARG = 1, OG_ERR_CFL = 2, OG_ERR_GEOMETRY = 3, OG_ERR_OOM = 4 };

typedef struct {
    int ndim;       /* 2 or 3                                                */
    int nx, ny, nz; /* physical grid points; ny is ignored when ndim == 2    */
    int nb;         /* sponge cells added outside the physical grid, each side */
    int nt;         /* number of time samples                                */
    double h;       /* grid spacing (m), same on every axis                  */
    double dt;      /* time step (s)                                         */
    double vref;    /* sponge reference velocity (m/s); 0 disables damping   */
} og_grid;

/* 8th-order centred second-derivative weights (Taylor conditions, h = 1). */
static const double C8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

typedef struct {
    int Nx, Ny, Nz;
    long N;
} pdims;

static pdims padded(const og_grid* g)
{
    pdims d;
    d.Nx = g->nx + 2 * g->nb;
    d.Ny = (g->ndim == 3) ? g->ny + 2 * g->nb : 1;
    d.Nz = g->nz + 2 * g->nb;
    d.N = (long)d.Nx * d.Ny * d.Nz;
    return d;
}

static long at_index(const pdims* d, int ix, int iy, int iz)
{
    return ((long)iz * d->Ny + iy) * d->Nx + ix;
}

/* Value of a padded field, zero outside the padded grid (Dirichlet ghosts). */
static double value_or_zero(const pdims* d, const double* u, int ix, int iy, int iz)
{
    if (ix < 0 || ix >= d->Nx || iy < 0 || iy >= d->Ny || iz < 0 || iz >= d->Nz) return 0.0;
    return u[at_index(d, ix, iy, iz)];
}

static int check_grid(const og_grid* g)
{
    if (!g) return OG_ERR_ARG;
    if (g->ndim != 2 && g->ndim != 3) return OG_ERR_ARG;
    if (g->nx < 2 || g->nz < 2 || (g->ndim == 3 && g->ny < 2)) return OG_ERR_ARG;
    if (g->nb < 0 || g->nt < 1) return OG_ERR_ARG;
    if (!(g->h > 0.0) || !(g->dt > 0.0) || !(g->vref >= 0.0)) return OG_ERR_ARG;
    return OG_OK;
}

/* Largest stable Courant number of the leapfrog scheme: dt^2 v^2 ndim K / h^2 <= 4
 * with K the largest magnitude of the 1D symbol, reached at the Nyquist wavenumber. */
double og_courant_limit(int ndim)
{
    double k = -C8[0];
    for (int j = 1; j <= 4; ++j) k += 2.0 * fabs(C8[j]);
    return 2.0 / sqrt((double)ndim * k);
}

static int check_cfl(const og_grid* g, const double* vel, long nphys)
{
    double vmax = 0.0;
    for (long i = 0; i < nphys; ++i) {
        if (!(vel[i] > 0.0) || !isfinite(vel[i])) return OG_ERR_ARG;
        if (vel[i] > vmax) vmax = vel[i];
    }
    if (g->dt * vmax / g->h > og_courant_limit(g->ndim)) return OG_ERR_CFL;
    return OG_OK;
}

static long phys_count(const og_grid* g)
{
    return (long)g->nx * g->nz * (g->ndim == 3 ? g->ny : 1);
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Distance, in cells, from padded index i to the physical range [nb, nb+n-1]. */
static int sponge_depth(int i, int nb, int n)
{
    int a = nb - i, b = i - (nb + n - 1);
    int d = a > b ? a : b;
    return d > 0 ? d : 0;
}

/* m = 1/v^2 on the padded grid (edge replication into the sponge) and the
 * damping profile eta = gamma(d) / vref^2 (units s/m^2, the units of m per
 * second), gamma(d) = gamma0 (d/nb)^2 a damping rate, d the deepest per-axis
 * sponge depth in cells, gamma0 = 3 vref ln(1/R) / (2 nb h) with R = 1e-3.
 * Dividing by the frozen vref^2 (not by the local m) keeps eta independent of m. */
int og_model(const og_grid* g, const double* vel, double* m, double* eta)
{
    int st = check_grid(g);
    if (st) return st;
    pdims d = padded(g);
    double eta0 = (g->nb > 0 && g->vref > 0.0) ? 3.0 * log(1000.0) / (2.0 * g->nb * g->h * g->vref) : 0.0;
    for (int iz = 0; iz < d.Nz; ++iz)
        for (int iy = 0; iy < d.Ny; ++iy)
            for (int ix = 0; ix < d.Nx; ++ix) {
                long p = at_index(&d, ix, iy, iz);
                int jx = clampi(ix - g->nb, 0, g->nx - 1);
                int jz = clampi(iz - g->nb, 0, g->nz - 1);
                int jy = g->ndim == 3 ? clampi(iy - g->nb, 0, g->ny - 1) : 0;
                long q = ((long)jz * (g->ndim == 3 ? g->ny : 1) + jy) * g->nx + jx;
                double v = vel[q];
                if (m) m[p] = 1.0 / (v * v);
                if (eta) {
                    int dd = sponge_depth(ix, g->nb, g->nx);
                    int dz = sponge_depth(iz, g->nb, g->nz);
                    if (dz > dd) dd = dz;
                    if (g->ndim == 3) {
                        int dy = sponge_depth(iy, g->nb, g->ny);
                        if (dy > dd) dd = dy;
                    }
                    eta[p] = g->nb > 0 ? eta0 * ((double)dd / g->nb) * ((double)dd / g->nb) : 0.0;
                }
            }
    return OG_OK;
}

/* out = L u on the padded grid. */
int og_laplacian(const og_grid* g, const double* u, double* out)
{
    int st = check_grid(g);
    if (st) return st;
    pdims d = padded(g);
    double ih2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < d.Nz; ++iz)
        for (int iy = 0; iy < d.Ny; ++iy)
            for (int ix = 0; ix < d.Nx; ++ix) {
                long p = at_index(&d, ix, iy, iz);
                double s = g->ndim * C8[0] * u[p];
                for (int k = 1; k <= 4; ++k) {
                    s += C8[k] * (value_or_zero(&d, u, ix + k, iy, iz) + value_or_zero(&d, u, ix - k, iy, iz));
                    s += C8[k] * (value_or_zero(&d, u, ix, iy, iz + k) + value_or_zero(&d, u, ix, iy, iz - k));
                    if (g->ndim == 3)
                        s += C8[k] * (value_or_zero(&d, u, ix, iy + k, iz) + value_or_zero(&d, u, ix, iy - k, iz));
                }
                out[p] = s * ih2;
            }
    return OG_OK;
}

/* Interpolation taps of one point: bilinear (2D) or trilinear (3D) weights on
 * the padded grid.  Coordinates are metres from the first physical grid point,
 * ordered (x, z) in 2D and (x, y, z) in 3D.  Points outside the physical grid
 * are rejected. */
typedef struct {
    long idx[8];
    double w[8];
    int n;
} taps_t;

static int point_taps(const og_grid* g, const pdims* d, const double* c, taps_t* t)
{
    int nax = g->ndim;
    int n_ax[3], N_ax[3];
    n_ax[0] = g->nx;
    N_ax[0] = d->Nx;
    if (nax == 2) {
        n_ax[1] = g->nz;
        N_ax[1] = d->Nz;
    } else {
        n_ax[1] = g->ny;
        N_ax[1] = d->Ny;
        n_ax[2] = g->nz;
        N_ax[2] = d->Nz;
    }
    int i0[3];
    double fr[3];
    for (int a = 0; a < nax; ++a) {
        double x = c[a];
        if (!isfinite(x) || x < 0.0 || x > (n_ax[a] - 1) * g->h) return OG_ERR_GEOMETRY;
        double f = x / g->h + g->nb;
        int i = (int)floor(f);
        if (i > N_ax[a] - 2) i = N_ax[a] - 2;
        i0[a] = i;
        fr[a] = f - i;
    }
    int nc = 1 << nax;
    for (int corner = 0; corner < nc; ++corner) {
        int ix = i0[0] + (corner & 1);
        double w = (corner & 1) ? fr[0] : 1.0 - fr[0];
        int iy = 0, iz;
        if (nax == 2) {
            iz = i0[1] + ((corner >> 1) & 1);
            w *= ((corner >> 1) & 1) ? fr[1] : 1.0 - fr[1];
        } else {
            iy = i0[1] + ((corner >> 1) & 1);
            w *= ((corner >> 1) & 1) ? fr[1] : 1.0 - fr[1];
            iz = i0[2] + ((corner >> 2) & 1);
            w *= ((corner >> 2) & 1) ? fr[2] : 1.0 - fr[2];
        }
        t->idx[corner] = at_index(d, ix, iy, iz);
        t->w[corner] = w;
    }
    t->n = nc;
    return OG_OK;
}

static int build_taps(const og_grid* g, const pdims* d, int np, const double* xyz, taps_t** out)
{
    *out = NULL;
    if (np == 0) return OG_OK;
    taps_t* t = (taps_t*)calloc((size_t)np, sizeof(taps_t));
    if (!t) return OG_ERR_OOM;
    for (int i = 0; i < np; ++i) {
        int st = point_taps(g, d, xyz + (long)i * g->ndim, &t[i]);
        if (st) {
            free(t);
            return st;
        }
    }
    *out = t;
    return OG_OK;
}

/* R u: sample a padded field at the points. */
static void sample(const taps_t* t, int np, const double* u, double* out)
{
    for (int i = 0; i < np; ++i) {
        double s = 0.0;
        for (int k = 0; k < t[i].n; ++k) s += t[i].w[k] * u[t[i].idx[k]];
        out[i] = s;
    }
}

/* field += scale * R^T a (transposed interpolation). */
static void spread(const taps_t* t, int np, const double* a, double scale, double* field)
{
    for (int i = 0; i < np; ++i)
        for (int k = 0; k < t[i].n; ++k) field[t[i].idx[k]] += scale * t[i].w[k] * a[i];
}

/* One explicit step of (M+E) x_new = (2M + dt^2 L) x - (M-E) x_old + rhs_extra,
 * where rhs_extra has already been accumulated into x_new by the caller. */
static void leapfrog(const og_grid* g, const pdims* d, const double* m, const double* eta,
                     const double* x, const double* x_old, const double* lap, double* x_new)
{
    double dt2 = g->dt * g->dt;
    double hdt = 0.5 * g->dt;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < d->N; ++p) {
        double e = eta[p] * hdt;
        double rhs = 2.0 * m[p] * x[p] + dt2 * lap[p] - (m[p] - e) * x_old[p] + x_new[p];
        x_new[p] = rhs / (m[p] + e);
    }
}

static double hpow(const og_grid* g) { return g->ndim == 3 ? g->h * g->h * g->h : g->h * g->h; }

typedef struct {
    pdims d;
    double *m, *eta, *a, *b, *c, *lap;
    taps_t *src, *rec;
} og_work;

static void work_free(og_work* w)
{
    free(w->m);
    free(w->eta);
    free(w->a);
    free(w->b);
    free(w->c);
    free(w->lap);
    free(w->src);
    free(w->rec);
}

static int work_init(og_work* w, const og_grid* g, const double* vel, int nsrc, const double* src_xyz,
                     int nrec, const double* rec_xyz)
{
    memset(w, 0, sizeof(*w));
    int st = check_grid(g);
    if (st) return st;
    if (!vel || nsrc < 0 || nrec < 0 || (nsrc && !src_xyz) || (nrec && !rec_xyz)) return OG_ERR_ARG;
    st = check_cfl(g, vel, phys_count(g));
    if (st) return st;
    w->d = padded(g);
    size_t bytes = (size_t)w->d.N * sizeof(double);
    w->m = (double*)malloc(bytes);
    w->eta = (double*)malloc(bytes);
    w->a = (double*)calloc((size_t)w->d.N, sizeof(double));
    w->b = (double*)calloc((size_t)w->d.N, sizeof(double));
    w->c = (double*)calloc((size_t)w->d.N, sizeof(double));
    w->lap = (double*)malloc(bytes);
    if (!w->m || !w->eta || !w->a || !w->b || !w->c || !w->lap) {
        work_free(w);
        return OG_ERR_OOM;
    }
    og_model(g, vel, w->m, w->eta);
    st = build_taps(g, &w->d, nsrc, src_xyz, &w->src);
    if (!st) st = build_taps(g, &w->d, nrec, rec_xyz, &w->rec);
    if (st) work_free(w);
    return st;
}

/* Forward modelling d = F(m) q for one shot.
 * vel: physical velocity [nz][(ny)][nx]; wavelet: [nt][nsrc]; data out [nt][nrec];
 * field_out (optional): every u^n, [nt][N_padded]. */
int og_forward(const og_grid* g, const double* vel, int nsrc, const double* src_xyz, const double* wavelet,
               int nrec, const double* rec_xyz, double* data, double* field_out)
{
    og_work w;
    int st = work_init(&w, g, vel, nsrc, src_xyz, nrec, rec_xyz);
    if (st) return st;
    double *u_old = w.a, *u = w.b, *u_new = w.c;
    double src_scale = g->dt * g->dt / hpow(g);
    for (int n = 0; n < g->nt; ++n) {
        sample(w.rec, nrec, u, data + (long)n * nrec);
        if (field_out) memcpy(field_out + (long)n * w.d.N, u, (size_t)w.d.N * sizeof(double));
        if (n == g->nt - 1) break;
        og_laplacian(g, u, w.lap);
        memset(u_new, 0, (size_t)w.d.N * sizeof(double));
        spread(w.src, nsrc, wavelet + (long)n * nsrc, src_scale, u_new);
        leapfrog(g, &w.d, w.m, w.eta, u, u_old, w.lap, u_new);
        double* t = u_old;
        u_old = u;
        u = u_new;
        u_new = t;
    }
    work_free(&w);
    return OG_OK;
}

/* Adjoint in q (the pullback F' dy): from a data residual r [nt][nrec] compute
 * (F^T r)^n = dt^2 S^T mu^{n+1}, n = 0..nt-2, and 0 at n = nt-1, where
 * (M+E) mu^k = (2M + dt^2 L) mu^{k+1} - (M-E) mu^{k+2} + R^T r^k, k = nt-1..1,
 * mu^{nt} = mu^{nt+1} = 0.  field_out (optional) receives mu^k at row k
 * (row 0 is left zero). */
int og_adjoint(const og_grid* g, const double* vel, int nsrc, const double* src_xyz, int nrec,
               const double* rec_xyz, const double* resid, double* src_out, double* field_out)
{
    og_work w;
    int st = work_init(&w, g, vel, nsrc, src_xyz, nrec, rec_xyz);
    if (st) return st;
    double *mu2 = w.a, *mu1 = w.b, *mu0 = w.c; /* mu^{k+2}, mu^{k+1}, mu^k */
    double src_scale = g->dt * g->dt / hpow(g);
    for (int i = 0; i < nsrc; ++i) src_out[(long)(g->nt - 1) * nsrc + i] = 0.0;
    if (field_out) memset(field_out, 0, (size_t)g->nt * w.d.N * sizeof(double));
    for (int k = g->nt - 1; k >= 1; --k) {
        og_laplacian(g, mu1, w.lap);
        memset(mu0, 0, (size_t)w.d.N * sizeof(double));
        spread(w.rec, nrec, resid + (long)k * nrec, 1.0, mu0);
        leapfrog(g, &w.d, w.m, w.eta, mu1, mu2, w.lap, mu0);
        sample(w.src, nsrc, mu0, src_out + (long)(k - 1) * nsrc);
        for (int i = 0; i < nsrc; ++i) src_out[(long)(k - 1) * nsrc + i] *= src_scale;
        if (field_out) memcpy(field_out + (long)k * w.d.N, mu0, (size_t)w.d.N * sizeof(double));
        double* t = mu2;
        mu2 = mu1;
        mu1 = mu0;
        mu0 = t;
    }
    work_free(&w);
    return OG_OK;
}

/* Adjoint of the edge-replicating extension: sum padded values onto the
 * physical cell they were copied from. */
static void extend_adjoint(const og_grid* g, const pdims* d, const double* gpad, double* gphys)
{
    memset(gphys, 0, (size_t)phys_count(g) * sizeof(double));
    int nyp = g->ndim == 3 ? g->ny : 1;
    for (int iz = 0; iz < d->Nz; ++iz)
        for (int iy = 0; iy < d->Ny; ++iy)
            for (int ix = 0; ix < d->Nx; ++ix) {
                int jx = clampi(ix - g->nb, 0, g->nx - 1);
                int jz = clampi(iz - g->nb, 0, g->nz - 1);
                int jy = g->ndim == 3 ? clampi(iy - g->nb, 0, g->ny - 1) : 0;
                gphys[((long)jz * nyp + jy) * g->nx + jx] += gpad[at_index(d, ix, iy, iz)];
            }
}

/* FWI gradient of Phi(m) = 1/2 sum_n ||R u^n - dobs^n||^2 for one shot, with
 * respect to the physical squared slowness:
 *   grad_pad = - sum_{n=0}^{nt-2} mu^{n+1} .* (u^{n+1} - 2 u^n + u^{n-1}),
 *   grad     = Extend^T grad_pad,
 * mu from the adjoint recursion driven by the residual r = R u - dobs.
 * The forward wavefield is kept in full (plain storage). */
int og_gradient(const og_grid* g, const double* vel, int nsrc, const double* src_xyz, const double* wavelet,
                int nrec, const double* rec_xyz, const double* dobs, double* grad, double* misfit,
                double* resid_out)
{
    int st = check_grid(g);
    if (st) return st;
    pdims d = padded(g);
    long nd = (long)g->nt * nrec;
    double* U = (double*)malloc((size_t)g->nt * d.N * sizeof(double));
    double* dsyn = (double*)malloc((size_t)(nd ? nd : 1) * sizeof(double));
    if (!U || !dsyn) {
        free(U);
        free(dsyn);
        return OG_ERR_OOM;
    }
    st = og_forward(g, vel, nsrc, src_xyz, wavelet, nrec, rec_xyz, dsyn, U);
    if (st) {
        free(U);
        free(dsyn);
        return st;
    }
    double phi = 0.0;
    for (long i = 0; i < nd; ++i) {
        dsyn[i] -= dobs[i]; /* now the residual */
        phi += 0.5 * dsyn[i] * dsyn[i];
    }
    if (misfit) *misfit = phi;
    if (resid_out) memcpy(resid_out, dsyn, (size_t)nd * sizeof(double));

    og_work w;
    st = work_init(&w, g, vel, nsrc, src_xyz, nrec, rec_xyz);
    if (st) {
        free(U);
        free(dsyn);
        return st;
    }
    double* gpad = (double*)calloc((size_t)d.N, sizeof(double));
    if (!gpad) {
        work_free(&w);
        free(U);
        free(dsyn);
        return OG_ERR_OOM;
    }
    double *mu2 = w.a, *mu1 = w.b, *mu0 = w.c;
    for (int k = g->nt - 1; k >= 1; --k) {
        og_laplacian(g, mu1, w.lap);
        memset(mu0, 0, (size_t)d.N * sizeof(double));
        spread(w.rec, nrec, dsyn + (long)k * nrec, 1.0, mu0);
        leapfrog(g, &d, w.m, w.eta, mu1, mu2, w.lap, mu0);
        /* mu0 = mu^k pairs with forward step n = k-1: u^k - 2 u^{k-1} + u^{k-2} */
        const double* up = U + (long)k * d.N;
        const double* uc = U + (long)(k - 1) * d.N;
        const double* um = k >= 2 ? U + (long)(k - 2) * d.N : NULL;
        for (long p = 0; p < d.N; ++p) {
            double utt = up[p] - 2.0 * uc[p] + (um ? um[p] : 0.0);
            gpad[p] -= mu0[p] * utt;
        }
        double* t = mu2;
        mu2 = mu1;
        mu1 = mu0;
        mu0 = t;
    }
    extend_adjoint(g, &d, gpad, grad);
    free(gpad);
    work_free(&w);
    free(U);
    free(dsyn);
    return OG_OK;
}

/* Born modelling (Jacobian J of d = F(m) q applied to dm, physical grid):
 * (M+E) du^{n+1} = (2M + dt^2 L) du^n - (M-E) du^{n-1} - Extend(dm) .* (u^{n+1} - 2u^n + u^{n-1}),
 * dd^n = R du^n. */
int og_born(const og_grid* g, const double* vel, int nsrc, const double* src_xyz, const double* wavelet,
            int nrec, const double* rec_xyz, const double* dm, double* dd)
{
    og_work w;
    int st = work_init(&w, g, vel, nsrc, src_xyz, nrec, rec_xyz);
    if (st) return st;
    pdims d = w.d;
    double* big = (double*)calloc((size_t)4 * d.N, sizeof(double));
    if (!big) {
        work_free(&w);
        return OG_ERR_OOM;
    }
    double *e_old = big, *e = big + d.N, *e_new = big + 2 * d.N, *dmp = big + 3 * d.N;
    /* Extend(dm): edge replication, same map as the model. */
    {
        int nyp = g->ndim == 3 ? g->ny : 1;
        for (int iz = 0; iz < d.Nz; ++iz)
            for (int iy = 0; iy < d.Ny; ++iy)
                for (int ix = 0; ix < d.Nx; ++ix) {
                    int jx = clampi(ix - g->nb, 0, g->nx - 1);
                    int jz = clampi(iz - g->nb, 0, g->nz - 1);
                    int jy = g->ndim == 3 ? clampi(iy - g->nb, 0, g->ny - 1) : 0;
                    dmp[at_index(&d, ix, iy, iz)] = dm[((long)jz * nyp + jy) * g->nx + jx];
                }
    }
    double *u_old = w.a, *u = w.b, *u_new = w.c;
    double src_scale = g->dt * g->dt / hpow(g);
    for (int n = 0; n < g->nt; ++n) {
        sample(w.rec, nrec, e, dd + (long)n * nrec);
        if (n == g->nt - 1) break;
        /* background step n -> n+1 */
        og_laplacian(g, u, w.lap);
        memset(u_new, 0, (size_t)d.N * sizeof(double));
        spread(w.src, nsrc, wavelet + (long)n * nsrc, src_scale, u_new);
        leapfrog(g, &d, w.m, w.eta, u, u_old, w.lap, u_new);
        /* linearised step with the secondary source */
        og_laplacian(g, e, w.lap);
        for (long p = 0; p < d.N; ++p) e_new[p] = -dmp[p] * (u_new[p] - 2.0 * u[p] + u_old[p]);
        leapfrog(g, &d, w.m, w.eta, e, e_old, w.lap, e_new);
        double* t = u_old;
        u_old = u;
        u = u_new;
        u_new = t;
        t = e_old;
        e_old = e;
        e = e_new;
        e_new = t;
    }
    free(big);
    work_free(&w);
    return OG_OK;
}

/* Ricker wavelet with peak frequency f, delayed by t0 = 1/f, sampled at
 * t_n = n dt:  q(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0. */
void og_ricker(double f, double dt, int nt, double* q)
{
    double t0 = 1.0 / f;
    for (int n = 0; n < nt; ++n) {
        double a = M_PI * f * (n * dt - t0);
        a *= a;
        q[n] = (1.0 - 2.0 * a) * exp(-a);
    }
}

long og_padded_points(const og_grid* g)
{
    if (check_grid(g)) return -1;
    return padded(g).N;
}

int og_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of later calls (n >= 1); used to time the oracle on one core and on all. */
void og_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
