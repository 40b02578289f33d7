"""Seeded synthetic inputs: velocity models and acquisition geometry.

This module holds no arithmetic of the wave solver.  It only draws inputs
(velocity models in m/s, source/receiver coordinates in metres, grid settings)
that both the CUDA library and the CPU oracle consume.  Every generator takes a
seed and uses ``numpy.random.default_rng``.

The paper runs on a Compass-derived model and on Sleipner-derived plumes that
are not available here; these stand-ins reproduce the *shape* of those
workloads (layered backgrounds, Gaussian-random lateral heterogeneity,
surface or crosswell acquisition, plume-shaped velocity drops).

Conventions: 2D arrays are [nz][nx], 3D arrays [nz][ny][nx] (x fastest);
coordinates are (x, z) in 2D and (x, y, z) in 3D, in metres from the first
physical grid point.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    ndim: int
    nx: int
    nz: int
    h: float
    dt: float
    nt: int
    nb: int
    f0: float                 # Ricker peak frequency (Hz)
    vel: np.ndarray           # float32 physical velocity
    src: np.ndarray           # float32 [nshot][nsrc][ndim]
    rec: np.ndarray           # float32 [nshot][nrec][ndim]
    ny: int = 1
    vref: float = 0.0         # sponge reference velocity (frozen, m/s)
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nshot(self) -> int:
        return int(self.src.shape[0])

    @property
    def padded_points(self) -> int:
        p = 2 * self.nb
        n = (self.nx + p) * (self.nz + p)
        return n * (self.ny + p) if self.ndim == 3 else n

    def with_shots(self, idx) -> "Problem":
        idx = np.atleast_1d(np.asarray(idx))
        return Problem(self.ndim, self.nx, self.nz, self.h, self.dt, self.nt, self.nb, self.f0,
                       self.vel, self.src[idx].copy(), self.rec[idx].copy(), self.ny, self.vref,
                       self.name, dict(self.extra))

    def with_nt(self, nt: int) -> "Problem":
        return Problem(self.ndim, self.nx, self.nz, self.h, self.dt, int(nt), self.nb, self.f0,
                       self.vel, self.src, self.rec, self.ny, self.vref, self.name, dict(self.extra))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def two_layer(nx: int, nz: int, h: float, v_top: float, v_bottom: float, z_interface: float) -> np.ndarray:
    """Velocity switching from v_top to v_bottom at the first row with z >= z_interface."""
    z = np.arange(nz) * h
    v = np.where(z >= z_interface - 1e-9, v_bottom, v_top)
    return _f32(np.repeat(v[:, None], nx, axis=1))


def gaussian_random_field(shape, sigma_cells: float, rng) -> np.ndarray:
    """White noise smoothed by a Gaussian kernel (std sigma_cells), scaled to unit std."""
    from scipy.ndimage import gaussian_filter

    w = rng.standard_normal(shape)
    s = gaussian_filter(w, sigma=sigma_cells, mode="reflect")
    return s / s.std()


def config1(seed: int = 1) -> Problem:
    """201 x 201 at 10 m, two layers 1500/2500 m/s (interface at z = 1 km),
    dt = 0.8 ms, nt = 1000, 40-cell sponge, 15 Hz Ricker at (1000, 20) m,
    201 receivers at z = 20 m every 10 m."""
    nx = nz = 201
    h = 10.0
    vel = two_layer(nx, nz, h, 1500.0, 2500.0, 1000.0)
    src = _f32([[[1000.0, 20.0]]])
    rec = _f32(np.stack([np.arange(nx) * h, np.full(nx, 20.0)], axis=1)[None])
    return Problem(2, nx, nz, h, 0.8e-3, 1000, 40, 15.0, vel, src, rec, vref=2500.0, name="config1")


def layered_gaussian(nx: int, nz: int, h: float, vmin: float, vmax: float, std: float,
                     corr_m: float, seed: int) -> np.ndarray:
    """Linear-in-depth background vmin -> vmax with a Gaussian-random relative
    perturbation of the given std and correlation length corr_m."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz) * h
    bg = vmin + (vmax - vmin) * z / z[-1]
    pert = gaussian_random_field((nz, nx), corr_m / h, rng)
    v = bg[:, None] * (1.0 + std * pert)
    return _f32(v)


def config2(seed: int = 2, nshot: int = 32, nt: int = 4000) -> Problem:
    """512 (x) x 256 (z) at 6.25 m, background 1500 -> 3500 m/s plus 5 %
    Gaussian-random perturbation (100 m correlation), 32 sources every 100 m at
    z = 12.5 m, 512 receivers at z = 12.5 m, 20 Hz Ricker, dt = 0.5 ms, 2 s."""
    nx, nz, h = 512, 256, 6.25
    vel = layered_gaussian(nx, nz, h, 1500.0, 3500.0, 0.05, 100.0, seed)
    xs = 50.0 + 100.0 * np.arange(nshot)
    src = _f32(np.stack([xs, np.full(nshot, 12.5)], axis=1)[:, None, :])
    rx = np.arange(nx) * h
    rec1 = np.stack([rx, np.full(nx, 12.5)], axis=1)
    rec = _f32(np.repeat(rec1[None], nshot, axis=0))
    vref = float(vel.max())
    return Problem(2, nx, nz, h, 0.5e-3, nt, 40, 20.0, vel, src, rec, vref=vref, name="config2")


def layered_3d(nx: int, ny: int, nz: int, h: float, nlayers: int, vmin: float, vmax: float,
               seed: int) -> np.ndarray:
    """Flat layers with seeded thicknesses (vmin at the top, vmax at the bottom)
    plus one seeded ellipsoidal anomaly of +/-10 %."""
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.uniform(0.1, 0.95, nlayers - 1)) * nz * h
    vlay = np.linspace(vmin, vmax, nlayers)
    z = np.arange(nz) * h
    vz = vlay[np.searchsorted(cuts, z, side="right")]
    v = np.broadcast_to(vz[:, None, None], (nz, ny, nx)).astype(np.float64).copy()
    c = rng.uniform([0.3, 0.3, 0.4], [0.7, 0.7, 0.7]) * np.array([nx, ny, nz]) * h
    ax = rng.uniform(0.08, 0.2, 3) * np.array([nx, ny, nz]) * h
    amp = rng.choice([-0.1, 0.1])
    X = np.arange(nx) * h
    Y = np.arange(ny) * h
    r2 = (((X[None, None, :] - c[0]) / ax[0]) ** 2 + ((Y[None, :, None] - c[1]) / ax[1]) ** 2
          + ((z[:, None, None] - c[2]) / ax[2]) ** 2)
    v[r2 <= 1.0] *= 1.0 + amp
    return _f32(v)


def config3(seed: int = 3, nt: int = 2000, n: tuple = (400, 400, 300)) -> Problem:
    """400 x 400 x 300 at 10 m, six layers 1500 -> 4000 m/s with an ellipsoidal
    anomaly, 15 Hz Ricker at the surface centre, receivers on the full
    400 x 400 surface grid at z = 10 m, dt = 1 ms, nt = 2000."""
    nx, ny, nz = n
    h = 10.0
    vel = layered_3d(nx, ny, nz, h, 6, 1500.0, 4000.0, seed)
    src = _f32([[[(nx // 2) * h, (ny // 2) * h, 10.0]]])
    gx, gy = np.meshgrid(np.arange(nx) * h, np.arange(ny) * h, indexing="xy")
    rec = _f32(np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 10.0)], axis=1)[None])
    vref = float(vel.max())
    return Problem(3, nx, nz, h, 1.0e-3, nt, 40, 15.0, vel, src, rec, ny=ny, vref=vref, name="config3")


def random_layers(nx: int, nz: int, h: float, rng, nlayer_range=(2, 5), vmin=1500.0, vmax=3500.0) -> np.ndarray:
    """Random flat layers with increasing velocity (config-1-style models)."""
    nl = int(rng.integers(nlayer_range[0], nlayer_range[1] + 1))
    cuts = np.sort(rng.uniform(0.15, 0.9, nl - 1)) * nz * h
    vl = np.sort(rng.uniform(vmin, vmax, nl))
    z = np.arange(nz) * h
    vz = vl[np.searchsorted(cuts, z, side="right")]
    return _f32(np.repeat(vz[:, None], nx, axis=1))


def small_2d(seed: int = 0, nx: int = 67, nz: int = 45, h: float = 10.0, nt: int = 300, nb: int = 12,
             nshot: int = 3, nrec: int = 23, off_grid: bool = True, f0: float = 12.0) -> Problem:
    """Small layered+random 2D problem with off-grid sources/receivers, sized so
    the oracle runs in well under a second and the CUDA tiles are ragged."""
    rng = np.random.default_rng(seed)
    vel = random_layers(nx, nz, h, rng, vmin=1500.0, vmax=3000.0)
    vel = _f32(vel * (1.0 + 0.03 * gaussian_random_field((nz, nx), 3.0, rng)))
    Lx, Lz = (nx - 1) * h, (nz - 1) * h
    src = np.zeros((nshot, 1, 2))
    src[:, 0, 0] = rng.uniform(0.1, 0.9, nshot) * Lx
    src[:, 0, 1] = rng.uniform(0.05, 0.3, nshot) * Lz
    rec = np.zeros((nshot, nrec, 2))
    for s in range(nshot):
        rec[s, :, 0] = np.sort(rng.uniform(0.0, Lx, nrec))
        rec[s, :, 1] = rng.uniform(0.0, 0.5, nrec) * Lz
    if not off_grid:
        src = np.round(src / h) * h
        rec = np.round(rec / h) * h
    vmax = float(vel.max())
    dt = float(np.float32(0.4 * 0.5547 * h / vmax))
    return Problem(2, nx, nz, h, dt, nt, nb, f0, vel, _f32(src), _f32(rec), vref=vmax, name="small2d")


def small_3d(seed: int = 0, nx: int = 37, ny: int = 29, nz: int = 23, h: float = 10.0, nt: int = 120,
             nb: int = 8, nshot: int = 2, nrec: int = 17, f0: float = 15.0) -> Problem:
    """Small layered 3D problem with off-grid sources/receivers."""
    rng = np.random.default_rng(seed)
    vel = layered_3d(nx, ny, nz, h, 3, 1500.0, 2800.0, seed)
    L = np.array([(nx - 1) * h, (ny - 1) * h, (nz - 1) * h])
    src = np.zeros((nshot, 1, 3))
    src[:, 0, :] = rng.uniform([0.2, 0.2, 0.1], [0.8, 0.8, 0.4], (nshot, 3)) * L
    rec = rng.uniform([0.0, 0.0, 0.0], [1.0, 1.0, 0.3], (nshot, nrec, 3)) * L
    vmax = float(vel.max())
    dt = float(np.float32(0.4 * 0.4529 * h / vmax))
    return Problem(3, nx, nz, h, dt, nt, nb, f0, vel, _f32(src), _f32(rec), ny=ny, vref=vmax, name="small3d")


def uneven_batch(seed: int = 4, nshot: int = 64, scale: float = 1.0) -> list[Problem]:
    """64 independent 2D shots with seeded sizes nx in [256, 768], nz in
    [128, 384], h in [6.25, 12.5], nt in [1500, 4000], dt = 0.4 x the stability
    limit (rounded down to 0.05 ms), random layered models, one source near the
    surface and a receiver at every surface grid point.  ``scale`` shrinks the
    grid sizes and nt for tests."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nshot):
        nx = max(24, int(rng.integers(256, 769) * scale))
        nz = max(16, int(rng.integers(128, 385) * scale))
        h = float(rng.choice([6.25, 7.5, 10.0, 12.5]))
        nt = max(40, int(rng.integers(1500, 4001) * scale))
        vel = random_layers(nx, nz, h, rng)
        vmax = float(vel.max())
        dt = float(np.float32(np.floor(0.4 * 0.5547 * h / vmax / 5e-5) * 5e-5))
        sx = float(rng.uniform(0.1, 0.9) * (nx - 1) * h)
        src = _f32([[[sx, 2 * h]]])
        rec = _f32(np.stack([np.arange(nx) * h, np.full(nx, 2 * h)], axis=1)[None])
        f0 = float(rng.uniform(8.0, 15.0))
        out.append(Problem(2, nx, nz, h, dt, nt, 40 if scale >= 1.0 else 10, f0, vel, src, rec,
                           vref=vmax, name=f"uneven{s}"))
    return out


def observed_noise(shape, scale: float, seed: int) -> np.ndarray:
    """Seeded Gaussian noise array (float32) used as a stand-in observed record."""
    rng = np.random.default_rng(seed)
    return _f32(scale * rng.standard_normal(shape))


# --- plume-shaped time-lapse perturbations --------------------------------------

def patchy_velocity(sw, vp, rho, phi, k_min=36.6e9, k_brine=2.735e9, k_co2=0.125e9, rho_brine=1000.0,
                    rho_co2=700.0):
    """P-wave velocity after a CO2 saturation sw under patchy mixing: the rock
    physics model R of arxiv 2304.05592 (section "Putting it all together",
    after Avseth, Mukerji and Mavko 2010).  The brine-saturated moduli come from
    vp and vs = vp / sqrt(3); Gassmann's relation gives the bulk modulus of the
    rock fully saturated with CO2; the patchy mixture averages the two
    P-wave moduli harmonically with weights 1 - sw and sw; density changes by
    phi sw (rho_co2 - rho_brine).  Returns (vp_new, rho_new)."""
    sw, vp, rho = np.asarray(sw, float), np.asarray(vp, float), np.asarray(rho, float)
    mu = rho * vp ** 2 / 3.0                       # shear modulus (vs^2 = vp^2 / 3)
    k_sat = rho * vp ** 2 - 4.0 / 3.0 * mu         # brine-saturated bulk modulus
    # Gassmann: K_sat/(K_min - K_sat) - K_fl/(phi (K_min - K_fl)) is the same
    # for every pore fluid; swap brine for CO2
    a = k_sat / (k_min - k_sat) - k_brine / (phi * (k_min - k_brine)) + k_co2 / (phi * (k_min - k_co2))
    k_co2_sat = k_min * a / (1.0 + a)
    m1, m2 = k_sat + 4.0 / 3.0 * mu, k_co2_sat + 4.0 / 3.0 * mu
    m_mix = 1.0 / ((1.0 - sw) / m1 + sw / m2)      # P-wave modulus of the patchy mixture
    rho_new = rho + phi * sw * (rho_co2 - rho_brine)
    return np.sqrt(m_mix / rho_new), rho_new


def plume_saturation(nz: int, nx: int, rng, z_cap: int, z_bot: int) -> np.ndarray:
    """CO2 saturation in [0, 1] on [nz][nx]: an inverted cone rising from an
    injection point at the reservoir bottom (row z_bot) to the seal (row z_cap),
    spreading under the seal, plus one to three thin lateral lobes (stacked
    high-permeability streaks); edges are smoothed over a few cells."""
    z, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    xi = rng.uniform(0.3, 0.7) * nx
    height = z_bot - z_cap
    w0 = rng.uniform(0.01, 0.03) * nx
    slope = rng.uniform(0.4, 1.2)
    half = w0 + np.clip(z_bot - z, 0.0, None) * slope   # cone half-width, wider upwards
    inside = (z >= z_cap) & (z <= z_bot)
    d = np.where(inside, np.abs(x - xi) - half, np.inf)
    s = 1.0 / (1.0 + np.exp(np.clip(d / 2.0, -50, 50)))
    # spreading under the seal
    t_cap = rng.uniform(0.08, 0.2) * height
    w_cap = half.max() * rng.uniform(1.1, 1.6)
    cap = (z >= z_cap) & (z <= z_cap + t_cap)
    s = np.maximum(s, np.where(cap, 1.0 / (1.0 + np.exp(np.clip((np.abs(x - xi) - w_cap) / 2.0, -50, 50))), 0.0))
    for _ in range(int(rng.integers(1, 4))):
        zl = rng.uniform(z_cap + 0.3 * height, z_bot - 0.1 * height)
        tl = rng.uniform(0.03, 0.08) * height
        wl = half.max() * rng.uniform(1.0, 2.0)
        xl = xi + rng.uniform(-0.3, 0.3) * wl
        lobe = (np.abs(z - zl) <= tl) & inside
        s = np.maximum(s, np.where(lobe, 1.0 / (1.0 + np.exp(np.clip((np.abs(x - xl) - wl) / 2.0, -50, 50))), 0.0))
    return np.where(inside, s, 0.0) * rng.uniform(0.6, 1.0)


def plume_model(seed: int, nx: int = 512, nz: int = 256, h: float = 10.0):
    """Baseline model and plume perturbation (both float32 [nz][nx], m/s).

    Baseline: 3-5 flat layers 1500-3500 m/s with a thin fast seal (2-4 % of
    the depth) and a reservoir layer (2.8-3.3 km/s) below it.  Perturbation: the patchy
    velocity drop of a plume-shaped saturation in the reservoir (porosity
    0.25, density from Gardner's relation rho = 310 vp^0.25), rescaled so that
    its largest relative drop is 2-8 %."""
    rng = np.random.default_rng(seed)
    base = random_layers(nx, nz, h, rng, nlayer_range=(3, 5)).astype(float)
    z_cap = int(rng.uniform(0.45, 0.6) * nz)
    t_seal = max(2, int(rng.uniform(0.02, 0.04) * nz))
    z_res = z_cap + t_seal
    z_bot = min(nz - 4, z_res + int(rng.uniform(0.15, 0.25) * nz))
    # with vs = vp / sqrt(3) the CO2-saturated modulus stays positive for vp above ~2.7 km/s
    v_res = rng.uniform(2800.0, 3300.0)
    base[z_cap:z_res] = min(v_res * 1.25, 4000.0)
    base[z_res:z_bot + 1] = v_res
    sw = plume_saturation(nz, nx, rng, z_res, z_bot)
    rho = 310.0 * base ** 0.25
    vp_new, _ = patchy_velocity(sw, base, rho, 0.25)
    dv = np.minimum(vp_new - base, 0.0)  # drops only (removes 1e-13 rounding where sw ~ 0)
    if not np.all(np.isfinite(dv)):
        raise ValueError("patchy substitution left the valid range")
    drop = float(np.max(-dv / base))
    if drop > 0:
        dv *= rng.uniform(0.02, 0.08) / drop
    return _f32(base), _f32(dv)


def plume_acquisition(nx: int = 512, nz: int = 256, h: float = 10.0, nshot: int = 8, nt: int = 2000,
                      dt: float = 0.8e-3, f0: float = 15.0, nb: int = 40, vref: float = 4000.0) -> Problem:
    """Surface acquisition over the plume models: nshot sources at 20 m depth,
    evenly spread, a receiver at every surface grid point (20 m depth); the
    velocity field of the returned Problem is a placeholder (set per model)."""
    Lx = (nx - 1) * h
    src = np.zeros((nshot, 1, 2))
    src[:, 0, 0] = np.linspace(0.06, 0.94, nshot) * Lx
    src[:, 0, 1] = 2 * h
    rec = np.stack([np.arange(nx) * h, np.full(nx, 2 * h)], axis=1)
    rec = np.repeat(rec[None], nshot, axis=0)
    vel = np.full((nz, nx), 2000.0, np.float32)
    return Problem(2, nx, nz, h, dt, nt, nb, f0, vel, _f32(src), _f32(rec), vref=vref, name="plume")
