"""Seeded synthetic inputs shaped like the gCMCRT workloads.

This module builds *inputs only*: spherical grids (longitude x latitude x
pressure level), per-cell temperature, pressure, density and wind, and the
opacity tables a job reads (grey/Rayleigh/cloud parameters, a correlated-k
table, a Doppler cross-section table).  It holds none of the Monte Carlo
method's arithmetic: no cell-table preparation, no sampling, no ray marching.
Both the CUDA path and the CPU oracle read what this module returns.

The paper post-processes GCM outputs (Sect. 9-13) that are not available
here, so every field below is an analytic, seeded stand-in with the sizes and
structure of the paper's cases:

* radial grid: N_r cells between N_r + 1 log-uniform pressure edges, with edge
  heights from the hypsometric relation dz = (k_B T / (mu m_u g)) ln(p_lo/p_hi)
  using the horizontally averaged layer temperature, bottom radius R0 = 1 R_J;
  the cell density is the hydrostatic layer mean rho = dp / (g dz), so a
  cell's vertical optical depth is kappa dp / g exactly (the paper uses a
  height grid, Sect. 6, and takes T, p, rho per cell from the GCM, Sect. 7);
* temperature: day/night blend T_h = T_n + (T_d - T_n) max(0, cos(lon - 15 deg) cos(lat))
  with a Guillot-like vertical profile (closed form in `guillot_T`);
* correlated-k table: k(b, g, T, p) = k_med(b) (T/1500)^aT (p/1 bar)^ap exp(sigma_ln * Phi^-1(g)),
  k_med log-uniform over 4 dex, sigma_ln = 2, 8 Gauss-Legendre g-ordinates;
* cross-section table: 5000 pseudo-Voigt lines (Thompson, Cox & Hastings 1987
  FWHM and mixing parameter), Doppler width from T for mass 18 u, Lorentz width
  proportional to p (296/T)^0.5, on a log-uniform lambda grid at R = 1e5;
* wind: 5 km/s cos^2(lat) eastward jet plus a 3 km/s day-to-night flow along
  great circles from the substellar point, proportional to sin(angular distance).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

K_B = 1.380649e-23          # J/K
M_U = 1.66053906660e-27     # kg
H_PLANCK = 6.62607015e-34   # J s
C_LIGHT = 2.99792458e8      # m/s
R_JUP = 7.1492e7            # m
BAR = 1.0e5                 # Pa

MODE_ALBEDO = 0
MODE_EMISSION = 1
MODE_TRANSMISSION = 2

OPAC_ALBEDO = 0       # per-lambda grey absorption + Rayleigh + per-cell cloud profile
OPAC_KTABLE = 1       # correlated-k table k[band][g][T][p]
OPAC_XSEC = 2         # high-resolution cross-section table sigma[lambda][T][p]


@dataclasses.dataclass
class Grid:
    nlon: int
    nlat: int
    nr: int
    r_edges: np.ndarray      # float64 [nr+1], m, r_edges[0] = R0 (bottom)
    lat_edges: np.ndarray    # float64 [nlat+1], rad, -pi/2 .. pi/2
    lon_edges: np.ndarray    # float64 [nlon+1], rad, span 2 pi
    T: np.ndarray            # float32 [ncell], K,  flattened [k][j][i] (lon fastest)
    p: np.ndarray            # float32 [ncell], Pa
    rho: np.ndarray          # float32 [ncell], kg/m^3
    wind: Optional[np.ndarray] = None   # float32 [3][ncell] (u east, v north, w up), m/s

    @property
    def ncell(self) -> int:
        return self.nlon * self.nlat * self.nr

    @property
    def R0(self) -> float:
        return float(self.r_edges[0])

    @property
    def R_toa(self) -> float:
        return float(self.r_edges[-1])


@dataclasses.dataclass
class AlbedoOpacity:
    """alpha_ext = rho (kabs + kray) + acld * qcld ; scattering from Rayleigh and cloud."""
    kabs: np.ndarray         # float64 [nlam], m^2/kg, grey gas absorption per wavelength
    kray: np.ndarray         # float64 [nlam], m^2/kg, Rayleigh scattering per wavelength
    qcld: np.ndarray         # float64 [nlam], cloud extinction scale per wavelength
    wcld: np.ndarray         # float64 [nlam], cloud single-scattering albedo
    gcld: np.ndarray         # float64 [nlam], cloud HG asymmetry factor
    acld: Optional[np.ndarray] = None   # float32 [ncell], m^-1 cloud extinction profile
    kind: int = OPAC_ALBEDO

    @property
    def nlam(self) -> int:
        return len(self.kray)


@dataclasses.dataclass
class KTable:
    lam: np.ndarray          # float64 [nb] band-centre wavelength, m
    wg: np.ndarray           # float64 [ng] g-ordinate weights (sum 1)
    gpts: np.ndarray         # float64 [ng] g-ordinates in (0,1)
    Tg: np.ndarray           # float64 [nT] K, increasing
    pg: np.ndarray           # float64 [np] Pa, increasing
    k: np.ndarray            # float32 [nb][ng][nT][np] m^2/kg
    kind: int = OPAC_KTABLE


@dataclasses.dataclass
class XsecTable:
    lam: np.ndarray          # float64 [nl] table wavelengths, m, increasing
    Tg: np.ndarray           # float64 [nT]
    pg: np.ndarray           # float64 [np]
    sigma: np.ndarray        # float32 [nl][nT][np] mass cross-section, m^2/kg
    view_theta: float = 0.5 * math.pi   # viewing polar angle (colatitude) of the observer
    view_phi: float = math.pi           # viewing longitude of the observer
    omega_rot: float = 0.0              # planetary rotation rate, rad/s
    kind: int = OPAC_XSEC


@dataclasses.dataclass
class Options:
    survival: int = 1            # 1 survival biasing (W <- W omega), 0 analog absorb/scatter
    w_rr: float = 1.0e-3         # Russian roulette when W < w_rr * W_launch
    p_surv: float = 0.1          # roulette survival probability
    tau_peel_cut: float = 50.0   # stop a peel-off / chord march beyond this optical depth
    tau_vert_max: float = 30.0   # emission: only cells with vertical tau above them < this emit
    beta_emis: float = 0.5       # emission: hybrid biasing fraction of the uniform-in-cell pdf
    scatter_emission: int = 0    # emission: follow packets after the launch peel-off
    max_steps: int = 1 << 22     # per-packet cap on cell segments
    hg_iso_eps: float = 1.0e-4   # |g| below this samples isotropically
    cloud_phase: int = 0         # 0 Henyey-Greenstein clouds, 1 two-term HG (g1 = g, g2 = -g/2, a = 1 - g2^2)
    surface_albedo: float = 0.0  # Lambertian lower boundary (0: black)
    trans_scatter: int = 0       # transmission on scattering opacities: packets scatter after their chord
    ld_law: int = 0              # stellar limb darkening: 0 none, 1 linear, 2 quadratic, 3 square-root,
                                 # 4 logarithmic, 5 power-2, 6 four-coefficient
    ld_coef: tuple = (0.0, 0.0, 0.0, 0.0)
    star_radius: float = 0.0     # m
    star_dist: float = 0.0       # m, planet-star distance
    transit_xy: tuple = (0.0, 0.0)   # planet centre on the stellar disk along the launch basis (e1, e2), m
    g_bias: int = 0              # emission band jobs (per-packet g): 0 q = p, 1 uniform, 2 composite
    g_beta: float = 0.5          # composite: q = (1 - g_beta) p + g_beta / N_g
    forced_first: int = 0        # forced scattering: 1 the first flight, 2 every flight
    cont_abs: int = 0            # continuous absorption
    path_bias: int = 0           # biased flights: 0 forced, 1 path length stretching, 2 hybrid


@dataclasses.dataclass
class Source:
    star: np.ndarray                 # float64 [3] unit vector from planet centre towards the star
    obs: np.ndarray                  # float64 [n_obs][3] unit vectors towards the observer(s)
    opts: Options = dataclasses.field(default_factory=Options)


@dataclasses.dataclass
class Job:
    lam_idx: int
    g_idx: int                       # g-ordinate (emission) or phase / observer index (albedo)
    n_packets: int
    key: int                         # 32-bit job key (Philox counter word 3)
    obs_idx: int = -1                # albedo: which observer of the source this job tallies (-1: all)


@dataclasses.dataclass
class Workload:
    name: str
    mode: int
    grid: Grid
    opac: object
    source: Source
    jobs: list
    seed: int
    notes: dict = dataclasses.field(default_factory=dict)

    @property
    def total_packets(self) -> int:
        return int(sum(j.n_packets for j in self.jobs))


# --------------------------------------------------------------------------- grids

def pressure_edges(p_top_bar: float, p_bot_bar: float, nr: int) -> np.ndarray:
    """N_r + 1 log-uniform pressure edges in Pa, index 0 at the bottom."""
    return np.logspace(math.log10(p_bot_bar), math.log10(p_top_bar), nr + 1) * BAR


def lat_lon_edges(nlon: int, nlat: int):
    lat = np.linspace(-0.5 * math.pi, 0.5 * math.pi, nlat + 1)
    lon = np.linspace(-math.pi, math.pi, nlon + 1)
    return lat, lon


def cell_centres(nlon, nlat, lat_edges, lon_edges):
    latc = 0.5 * (lat_edges[:-1] + lat_edges[1:])
    lonc = 0.5 * (lon_edges[:-1] + lon_edges[1:])
    LAT, LON = np.meshgrid(latc, lonc, indexing="ij")   # [nlat][nlon]
    return LAT, LON


def guillot_T(T_h, p_pa, gamma=0.5, T_int=400.0, p_ref=0.1 * BAR):
    """Guillot (2010)-like profile with tau = p / p_ref:
    T^4 = 3/4 T_int^4 (2/3 + tau) + 3/4 T_h^4 [2/3 + 1/(gamma sqrt3) + (gamma/sqrt3 - 1/(gamma sqrt3)) exp(-gamma tau sqrt3)]."""
    tau = p_pa / p_ref
    s3 = math.sqrt(3.0)
    irr = 2.0 / 3.0 + 1.0 / (gamma * s3) + (gamma / s3 - 1.0 / (gamma * s3)) * np.exp(-gamma * tau * s3)
    T4 = 0.75 * T_int ** 4 * (2.0 / 3.0 + tau) + 0.75 * T_h ** 4 * irr
    return T4 ** 0.25


def hotjupiter_T(nlon, nlat, nr, lat_edges, lon_edges, p_cell, T_day=2200.0, T_night=1000.0,
                 hotspot_deg=15.0):
    LAT, LON = cell_centres(nlon, nlat, lat_edges, lon_edges)
    m = np.maximum(0.0, np.cos(LON - math.radians(hotspot_deg)) * np.cos(LAT))
    T_h = T_night + (T_day - T_night) * m                     # [nlat][nlon]
    T = guillot_T(T_h[None, :, :], p_cell[:, None, None])     # [nr][nlat][nlon]
    return T, m


def build_grid(nlon, nlat, nr, p_top_bar, p_bot_bar, T_cells, mu=2.3, grav=10.0, R0=R_JUP,
               lat_edges=None, lon_edges=None, wind=None):
    """Hypsometric radial grid from the area-weighted mean layer temperature."""
    if lat_edges is None or lon_edges is None:
        lat_edges, lon_edges = lat_lon_edges(nlon, nlat)
    pe = pressure_edges(p_top_bar, p_bot_bar, nr)
    T3 = np.asarray(T_cells, dtype=np.float64).reshape(nr, nlat, nlon)
    area = (np.sin(lat_edges[1:]) - np.sin(lat_edges[:-1]))[:, None] * np.diff(lon_edges)[None, :]
    Tmean = (T3 * area[None]).sum(axis=(1, 2)) / area.sum()
    H = K_B * Tmean / (mu * M_U * grav)
    dz = H * np.log(pe[:-1] / pe[1:])
    r_edges = R0 + np.concatenate([[0.0], np.cumsum(dz)])
    p_cell = np.sqrt(pe[:-1] * pe[1:])
    rho_layer = (pe[:-1] - pe[1:]) / (grav * dz)
    ncell = nlon * nlat * nr
    p = np.broadcast_to(p_cell[:, None, None], (nr, nlat, nlon)).reshape(ncell)
    rho = np.broadcast_to(rho_layer[:, None, None], (nr, nlat, nlon)).reshape(ncell)
    return Grid(nlon=nlon, nlat=nlat, nr=nr, r_edges=r_edges.astype(np.float64),
                lat_edges=np.asarray(lat_edges, np.float64), lon_edges=np.asarray(lon_edges, np.float64),
                T=T3.reshape(ncell).astype(np.float32), p=p.astype(np.float32),
                rho=rho.astype(np.float32), wind=wind)


def uniform_grid(nlon, nlat, nr, R0, R_toa, rho=1.0, T=1000.0, p=1.0e4, lat_edges=None, lon_edges=None,
                 r_edges=None):
    """Homogeneous test grid: constant rho, T, p (used for analytic cases)."""
    if lat_edges is None or lon_edges is None:
        lat_edges, lon_edges = lat_lon_edges(nlon, nlat)
    if r_edges is None:
        r_edges = np.linspace(R0, R_toa, nr + 1)
    ncell = nlon * nlat * nr
    return Grid(nlon=nlon, nlat=nlat, nr=nr, r_edges=np.asarray(r_edges, np.float64),
                lat_edges=np.asarray(lat_edges, np.float64), lon_edges=np.asarray(lon_edges, np.float64),
                T=np.full(ncell, T, np.float32), p=np.full(ncell, p, np.float32),
                rho=np.full(ncell, rho, np.float32))


def phase_dirs(phases_deg):
    a = np.radians(np.asarray(phases_deg, dtype=np.float64))
    return np.stack([np.cos(a), np.sin(a), np.zeros_like(a)], axis=1)


# --------------------------------------------------------------------------- configurations

def config1_albedo(n_packets=100_000, seed=1, nlon=32, nlat=16, nr=20, omega=0.5, tau_vert=10.0,
                   survival=1):
    """Albedo, plain: 32 x 16 x 20 cells, 1e-5..100 bar, isothermal 1500 K, mu = 2.3, g = 10,
    grey extinction with vertical tau = 10 at the bottom, uniform Rayleigh scattering with
    omega = 0.5, star and observer at phase 0, one wavelength."""
    grav = 10.0
    p_top, p_bot = 1e-5, 100.0
    T = np.full(nlon * nlat * nr, 1500.0)
    grid = build_grid(nlon, nlat, nr, p_top, p_bot, T, grav=grav)
    kext = tau_vert * grav / ((p_bot - p_top) * BAR)        # = 1.0000001e-5 m^2/kg
    opac = AlbedoOpacity(kabs=np.array([(1 - omega) * kext]), kray=np.array([omega * kext]),
                         qcld=np.zeros(1), wcld=np.zeros(1), gcld=np.zeros(1), acld=None)
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[1.0, 0.0, 0.0]]),
                 opts=Options(survival=survival))
    jobs = [Job(lam_idx=0, g_idx=0, n_packets=int(n_packets), key=0)]
    return Workload("albedo_32x16x20_1e5", MODE_ALBEDO, grid, opac, src, jobs, seed,
                    notes=dict(kext=kext, grav=grav))


def hotjupiter_grid(nlon=128, nlat=64, nr=50, p_top=1e-6, p_bot=100.0, wind=False, grav=10.0):
    lat_e, lon_e = lat_lon_edges(nlon, nlat)
    pe = pressure_edges(p_top, p_bot, nr)
    p_cell = np.sqrt(pe[:-1] * pe[1:])
    T3, m = hotjupiter_T(nlon, nlat, nr, lat_e, lon_e, p_cell)
    W = wind_field(nlon, nlat, nr, lat_e, lon_e) if wind else None
    return build_grid(nlon, nlat, nr, p_top, p_bot, T3, grav=grav, lat_edges=lat_e, lon_edges=lon_e, wind=W), m


def make_ktable(rng, nb=30, ng=8, nT=20, npr=15, lam_lo=1e-6, lam_hi=5e-6, sigma_ln=2.0, aT=1.0, ap=0.3,
                split=None):
    """Synthetic correlated-k table: Gauss-Legendre g-ordinates on [0, 1], or with split = (n1, n2, gs)
    a split quadrature of n1 points on [0, gs] and n2 on [gs, 1] (e.g. 8 + 8 with gs = 0.9)."""
    from scipy.special import ndtri
    lam = np.geomspace(lam_lo, lam_hi, nb)
    if split is None:
        x, w = np.polynomial.legendre.leggauss(ng)
        gpts = 0.5 * (x + 1.0)
        wg = 0.5 * w
    else:
        n1, n2, gs = split
        x1, w1 = np.polynomial.legendre.leggauss(n1)
        x2, w2 = np.polynomial.legendre.leggauss(n2)
        gpts = np.concatenate([0.5 * gs * (x1 + 1.0), gs + 0.5 * (1.0 - gs) * (x2 + 1.0)])
        wg = np.concatenate([0.5 * gs * w1, 0.5 * (1.0 - gs) * w2])
        ng = n1 + n2
    Tg = np.geomspace(500.0, 3000.0, nT)
    pg = np.geomspace(1e-6 * BAR, 100.0 * BAR, npr)
    kmed = 10.0 ** rng.uniform(-5.0, -1.0, nb)
    k = (kmed[:, None, None, None]
         * (Tg[None, None, :, None] / 1500.0) ** aT
         * (pg[None, None, None, :] / BAR) ** ap
         * np.exp(sigma_ln * ndtri(gpts))[None, :, None, None])
    return KTable(lam=lam, wg=wg, gpts=gpts, Tg=Tg, pg=pg, k=k.astype(np.float32))


def config2_emission(n_packets=1_000_000, seed=2, nlon=128, nlat=64, nr=50, nb=30, ng=8,
                     bands=None, gpoints=None, obs=None, split=None, per_packet_g=False, g_bias=0, g_beta=0.5):
    """Emission: 128 x 64 x 50 hot-Jupiter grid (1e-6..100 bar), correlated-k 30 bands x 8
    g-ordinates, scattering off, observer at the substellar direction, 1e6 packets per (band, g).
    per_packet_g: one job per band whose packets draw their g-ordinate (g_bias, g_beta; split gives
    a split quadrature, e.g. (8, 8, 0.9))."""
    rng = np.random.default_rng(seed)
    grid, _ = hotjupiter_grid(nlon, nlat, nr)
    kt = make_ktable(rng, nb=nb, ng=ng, split=split)
    ng = len(kt.wg)
    if obs is None:
        obs = np.array([[1.0, 0.0, 0.0]])
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.asarray(obs, np.float64),
                 opts=Options(scatter_emission=0, g_bias=g_bias, g_beta=g_beta))
    bands = range(nb) if bands is None else bands
    gpoints = range(ng) if gpoints is None else gpoints
    if per_packet_g:
        jobs = [Job(lam_idx=b, g_idx=-1, n_packets=int(n_packets), key=(b << 8) | 0xFF) for b in bands]
    else:
        jobs = [Job(lam_idx=b, g_idx=g, n_packets=int(n_packets), key=(b << 8) | g) for b in bands for g in gpoints]
    return Workload(f"emission_{nlon}x{nlat}x{nr}_{nb}bx{ng}g", MODE_EMISSION, grid, kt, src, jobs, seed)


def cloud_profile(grid: Grid, m_day, tau_cld=5.0, p_peak=0.1 * BAR, width_dex=0.5, day_thin=0.6):
    """Log-normal cloud deck: layer tau proportional to exp(-(log10(p/p_peak))^2 / (2 w^2)),
    column tau = tau_cld (thinned by (1 - day_thin * m) towards the hot spot)."""
    nr, nlat, nlon = grid.nr, grid.nlat, grid.nlon
    p_layer = grid.p.reshape(nr, nlat, nlon)[:, 0, 0].astype(np.float64)
    gk = np.exp(-(np.log10(p_layer / p_peak)) ** 2 / (2.0 * width_dex ** 2))
    dtau = tau_cld * gk / gk.sum()
    dz = np.diff(grid.r_edges)
    a = (dtau / dz)[:, None, None] * (1.0 - day_thin * m_day)[None, :, :]
    return np.broadcast_to(a, (nr, nlat, nlon)).reshape(grid.ncell).astype(np.float32)


def config3_phase_curve(seed=3, nlon=128, nlat=64, nr=50, nlam=40, nphase=24, n_lo=10_000, n_hi=1_000_000,
                        lam_lo=0.3e-6, lam_hi=1.0e-6):
    """Batched albedo phase curve: C2's grid + Rayleigh gas + log-normal cloud deck (peak 0.1 bar,
    0.5 dex, omega = 0.9, HG g = 0.6); 24 phase angles x 40 wavelengths, packets per job uniform in
    [1e4, 1e6]."""
    rng = np.random.default_rng(seed)
    grid, m = hotjupiter_grid(nlon, nlat, nr)
    lam = np.geomspace(lam_lo, lam_hi, nlam)
    kray = 3.1e-5 * (lam / 0.5e-6) ** -4
    kabs = 5.0e-5 * 10.0 ** (0.5 * np.sin(12.0 * np.log(lam / lam_lo)))
    opac = AlbedoOpacity(kabs=kabs, kray=kray, qcld=np.ones(nlam), wcld=np.full(nlam, 0.9),
                         gcld=np.full(nlam, 0.6), acld=cloud_profile(grid, m))
    phases = np.arange(nphase) * (360.0 / nphase)
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=phase_dirs(phases), opts=Options())
    npk = rng.integers(n_lo, n_hi + 1, size=(nlam, nphase))
    jobs = [Job(lam_idx=l, g_idx=ph, n_packets=int(npk[l, ph]), key=(l << 8) | ph, obs_idx=ph)
            for l in range(nlam) for ph in range(nphase)]
    return Workload(f"phasecurve_{nlon}x{nlat}x{nr}_{nlam}lx{nphase}ph", MODE_ALBEDO, grid, opac, src, jobs,
                    seed, notes=dict(phases_deg=phases.tolist()))


def config7_emission_hires(n_packets=100_000, seed=7, nlon=96, nlat=48, nr=60, n_lam=9532, lam_subset=None,
                           n_lines=5000, p_top=1e-6, p_bot=100.0, rot_period_days=3.5):
    """High-resolution emission (Sect. 7): C2's day-night temperature structure and C4's winds on the
    96 x 48 x 60 grid, sigma(lambda, T, p) at R = 1e5 over 1.0-1.1 um with per-cell Doppler shifts
    towards an observer over the dayside (+x), n_packets per wavelength."""
    rng = np.random.default_rng(seed)
    grid, _ = hotjupiter_grid(nlon, nlat, nr, p_top=p_top, p_bot=p_bot, wind=True)
    xs, margin = make_xsec_table(rng, n_lines=n_lines, n_lam=n_lam)
    xs.omega_rot = 2.0 * math.pi / (rot_period_days * 86400.0)
    xs.view_theta = 0.5 * math.pi      # observer on the +x axis: colatitude 90 deg, longitude 0
    xs.view_phi = 0.0
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[1.0, 0.0, 0.0]]), opts=Options(scatter_emission=0))
    lams = range(n_lam) if lam_subset is None else lam_subset
    jobs = [Job(lam_idx=margin + l, g_idx=0, n_packets=int(n_packets), key=l) for l in lams]
    return Workload(f"emission_hires_{nlon}x{nlat}x{nr}_{n_lam}l", MODE_EMISSION, grid, xs, src, jobs, seed,
                    notes=dict(margin=margin))


R_SUN = 6.957e8
AU = 1.495978707e11


def config6_transit_scatter(seed=6, nlon=128, nlat=64, nr=50, nlam=40, n_packets=200_000, lam_lo=0.3e-6,
                            lam_hi=1.0e-6):
    """Optical transmission spectrum with multiple scattering (Sect. 5.1): the phase-curve atmosphere
    (Rayleigh gas + cloud deck, omega 0.9, two-term HG g = 0.6) seen in transit, quadratic stellar limb
    darkening (Sun-like star at 0.05 AU, transit impact parameter 0.3), n_packets chords per wavelength."""
    grid, m = hotjupiter_grid(nlon, nlat, nr)
    lam = np.geomspace(lam_lo, lam_hi, nlam)
    kray = 3.1e-5 * (lam / 0.5e-6) ** -4
    kabs = 5.0e-5 * 10.0 ** (0.5 * np.sin(12.0 * np.log(lam / lam_lo)))
    opac = AlbedoOpacity(kabs=kabs, kray=kray, qcld=np.ones(nlam), wcld=np.full(nlam, 0.9),
                         gcld=np.full(nlam, 0.6), acld=cloud_profile(grid, m))
    opts = Options(trans_scatter=1, cloud_phase=1, ld_law=2, ld_coef=(0.45, 0.2, 0.0, 0.0), star_radius=R_SUN,
                   star_dist=0.05 * AU, transit_xy=(0.0, 0.3 * R_SUN))
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]), opts=opts)
    jobs = [Job(lam_idx=l, g_idx=0, n_packets=int(n_packets), key=l) for l in range(nlam)]
    return Workload(f"transit_scatter_{nlon}x{nlat}x{nr}_{nlam}l", MODE_TRANSMISSION, grid, opac, src, jobs, seed)


def wind_field(nlon, nlat, nr, lat_edges, lon_edges, u_jet=5000.0, v_dn=3000.0):
    """(u east, v north, w up) in m/s: cos^2(lat) eastward jet + day->night great-circle flow
    |v| = v_dn sin(angular distance from the substellar point at lon 0, lat 0)."""
    LAT, LON = cell_centres(nlon, nlat, lat_edges, lon_edges)
    n = np.stack([np.cos(LAT) * np.cos(LON), np.cos(LAT) * np.sin(LON), np.sin(LAT)], axis=-1)
    s = np.array([1.0, 0.0, 0.0])
    tang = s[None, None, :] - (n @ s)[..., None] * n          # points towards the substellar point
    vdn = -v_dn * tang
    east = np.stack([-np.sin(LON), np.cos(LON), np.zeros_like(LON)], axis=-1)
    north = np.stack([-np.sin(LAT) * np.cos(LON), -np.sin(LAT) * np.sin(LON), np.cos(LAT)], axis=-1)
    u = u_jet * np.cos(LAT) ** 2 + (vdn * east).sum(-1)
    v = (vdn * north).sum(-1)
    w = np.zeros_like(u)
    W = np.stack([u, v, w], axis=0)                             # [3][nlat][nlon]
    W = np.broadcast_to(W[:, None, :, :], (3, nr, nlat, nlon)).reshape(3, nr * nlat * nlon)
    return np.ascontiguousarray(W, dtype=np.float32)


def pseudo_voigt_fwhm_eta(fG, fL):
    """Thompson, Cox & Hastings (1987) pseudo-Voigt total FWHM and Lorentz fraction."""
    f = (fG ** 5 + 2.69269 * fG ** 4 * fL + 2.42843 * fG ** 3 * fL ** 2 + 4.47163 * fG ** 2 * fL ** 3
         + 0.07842 * fG * fL ** 4 + fL ** 5) ** 0.2
    x = fL / f
    eta = 1.36603 * x - 0.47719 * x ** 2 + 0.11116 * x ** 3
    return f, eta


def make_xsec_table(rng, n_lines=5000, R=1.0e5, lam0=1.0e-6, n_lam=9532, margin=8, nT=20, npr=15,
                    p_top=1e-6, p_bot=100.0, sigma_cont=3.0e-5, s_max=1.5e-2, mass_u=18.0):
    """sigma(lambda, T, p) in m^2/kg on lambda_i = lam0 exp((i - margin)/R), i = 0 .. n_lam + 2 margin - 1.
    Lines are deposited on the index grid and convolved (FFT) with a unit-area pseudo-Voigt profile."""
    nl = n_lam + 2 * margin
    lam = lam0 * np.exp((np.arange(nl) - margin) / R)
    Tg = np.geomspace(500.0, 3000.0, nT)
    pg = np.geomspace(p_top * BAR, p_bot * BAR, npr)
    centres = rng.uniform(margin, margin + n_lam, n_lines)          # in index units
    strength = s_max * 10.0 ** rng.uniform(-6.0, 0.0, n_lines)
    pad = 4096
    nfft = 1 << int(math.ceil(math.log2(nl + 2 * pad)))
    stick = np.zeros(nfft)
    i0 = np.floor(centres).astype(np.int64)
    fr = centres - i0
    np.add.at(stick, i0 + pad, strength * (1.0 - fr))
    np.add.at(stick, i0 + 1 + pad, strength * fr)
    S = np.fft.rfft(stick)
    off = np.arange(nfft)
    off = np.where(off < nfft // 2, off, off - nfft).astype(np.float64)
    sigma = np.empty((nl, nT, npr), dtype=np.float64)
    m_kg = mass_u * M_U
    for a, T in enumerate(Tg):
        fG = R * math.sqrt(8.0 * K_B * T * math.log(2.0) / m_kg) / C_LIGHT      # FWHM in index units
        for b, p in enumerate(pg):
            fL = 2.0 * 0.05 * (p / 101325.0) * math.sqrt(296.0 / T) * 1.0e-4 * R   # 0.05 cm^-1/atm HWHM at 1e4 cm^-1
            f, eta = pseudo_voigt_fwhm_eta(fG, fL)
            g = math.sqrt(4.0 * math.log(2.0) / math.pi) / f * np.exp(-4.0 * math.log(2.0) * off ** 2 / f ** 2)
            lor = (f / (2.0 * math.pi)) / (off ** 2 + 0.25 * f ** 2)
            kern = eta * lor + (1.0 - eta) * g
            kern /= kern.sum()
            spec = np.fft.irfft(S * np.fft.rfft(kern), nfft)[pad:pad + nl]
            sigma[:, a, b] = sigma_cont + np.maximum(spec, 0.0)
    return XsecTable(lam=lam, Tg=Tg, pg=pg, sigma=sigma.astype(np.float32)), margin


def config4_transmission(n_packets=10_000, seed=4, nlon=96, nlat=48, nr=60, n_lam=9532, lam_subset=None,
                         n_lines=5000, p_top=1e-6, p_bot=100.0, rot_period_days=3.5):
    """High-resolution transmission: 96 x 48 x 60 grid with winds, sigma(lambda, T, p) at R = 1e5 over
    1.0-1.1 um, per-cell Doppler shift, 1e4 limb chords per wavelength."""
    rng = np.random.default_rng(seed)
    grid, _ = hotjupiter_grid(nlon, nlat, nr, p_top=p_top, p_bot=p_bot, wind=True)
    xs, margin = make_xsec_table(rng, n_lines=n_lines, n_lam=n_lam)
    xs.omega_rot = 2.0 * math.pi / (rot_period_days * 86400.0)
    xs.view_theta = 0.5 * math.pi      # observer on the -x axis: colatitude 90 deg, longitude 180 deg
    xs.view_phi = math.pi
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]), opts=Options())
    lams = range(n_lam) if lam_subset is None else lam_subset
    jobs = [Job(lam_idx=margin + l, g_idx=0, n_packets=int(n_packets), key=l) for l in lams]
    return Workload(f"transmission_{nlon}x{nlat}x{nr}_{n_lam}l", MODE_TRANSMISSION, grid, xs, src, jobs, seed,
                    notes=dict(margin=margin))


# --------------------------------------------------------------------------- serving stream

@dataclasses.dataclass
class Scene:
    """One resident planet model of the serving workload: a grid and the three modes' inputs."""
    grid: Grid
    albedo: AlbedoOpacity
    ktable: KTable
    xsec: XsecTable
    margin: int                      # first usable index of the cross-section wavelength grid
    src_albedo: Source
    src_emission: Source
    src_transmission: Source


@dataclasses.dataclass
class Request:
    mode: int
    scene: int
    lam_idx: int
    g_idx: int
    obs_idx: int
    n_packets: int
    key: int


@dataclasses.dataclass
class ServingWorkload:
    name: str
    scenes: list
    requests: list
    seed: int


SERVING_GRIDS = ((32, 16, 20), (64, 32, 40), (128, 64, 50), (256, 128, 100))


def config5_serving(n_requests=10_000, seed=5, grids=SERVING_GRIDS, n_lo=1.0e4, n_hi=1.0e7, nlam_alb=8,
                    nphase=4, nb=8, ng=4, n_lam_x=64, n_lines=300):
    """Serving: a stream of spectrum requests mixing albedo, emission and transmission (1/3 each), on
    grids drawn uniformly from 32x16x20 .. 256x128x100 (each a hot-Jupiter model with winds, a Rayleigh
    + cloud albedo opacity over nlam_alb wavelengths and nphase observer phases, an nb x ng k-table and
    an n_lam_x-point Doppler cross-section table), packets per request log-uniform in [n_lo, n_hi].
    Each request is one (mode, wavelength / band, g or phase) job.  Arrival times are drawn by the
    caller (Poisson at a chosen rate)."""
    rng = np.random.default_rng(seed)
    scenes = []
    for (nlon, nlat, nr) in grids:
        grid, m = hotjupiter_grid(nlon, nlat, nr, wind=True)
        lam = np.geomspace(0.3e-6, 1.0e-6, nlam_alb)
        alb = AlbedoOpacity(kabs=5.0e-5 * 10.0 ** (0.5 * np.sin(12.0 * np.log(lam / 0.3e-6))),
                            kray=3.1e-5 * (lam / 0.5e-6) ** -4, qcld=np.ones(nlam_alb),
                            wcld=np.full(nlam_alb, 0.9), gcld=np.full(nlam_alb, 0.6), acld=cloud_profile(grid, m))
        kt = make_ktable(rng, nb=nb, ng=ng)
        xs, margin = make_xsec_table(rng, n_lines=n_lines, n_lam=n_lam_x)
        xs.omega_rot = 2.0 * math.pi / (3.5 * 86400.0)
        xs.view_theta = 0.5 * math.pi
        xs.view_phi = math.pi
        phases = np.arange(nphase) * (180.0 / nphase)
        scenes.append(Scene(
            grid=grid, albedo=alb, ktable=kt, xsec=xs, margin=margin,
            src_albedo=Source(star=np.array([1.0, 0.0, 0.0]), obs=phase_dirs(phases), opts=Options()),
            src_emission=Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[1.0, 0.0, 0.0]]),
                                opts=Options(scatter_emission=0)),
            src_transmission=Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]),
                                    opts=Options())))
    modes = rng.integers(0, 3, n_requests)
    sc = rng.integers(0, len(grids), n_requests)
    npk = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_requests)).astype(np.int64)
    reqs = []
    for q in range(n_requests):
        mode = int(modes[q])
        if mode == MODE_ALBEDO:
            lam, g, obs = int(rng.integers(nlam_alb)), int(rng.integers(nphase)), -1
            obs = g
        elif mode == MODE_EMISSION:
            lam, g, obs = int(rng.integers(nb)), int(rng.integers(ng)), -1
        else:
            lam, g, obs = int(scenes[sc[q]].margin + rng.integers(n_lam_x)), 0, -1
        reqs.append(Request(mode=mode, scene=int(sc[q]), lam_idx=lam, g_idx=g, obs_idx=obs,
                            n_packets=int(max(npk[q], 1)), key=q))
    return ServingWorkload(f"serving_{n_requests}req", scenes, reqs, seed)


# --------------------------------------------------------------------------- small analytic cases

def uniform_absorber_sphere(alpha=2.0e-6, R0=R_JUP, H_atm=5.0e6, nlon=4, nlat=4, nr=4, n_packets=20000,
                            seed=11):
    """Pure-absorber shell R0..R0+H with constant alpha (rho = 1, kappa = alpha): chord tau(b) =
    2 alpha sqrt(R_toa^2 - b^2) for b >= R0."""
    grid = uniform_grid(nlon, nlat, nr, R0, R0 + H_atm, rho=1.0)
    xs_lam = np.array([1.0e-6, 1.1e-6])
    xs = XsecTable(lam=xs_lam, Tg=np.array([500.0, 3000.0]), pg=np.array([1.0, 1.0e7]),
                   sigma=np.full((2, 2, 2), alpha, np.float32), omega_rot=0.0)
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]), opts=Options())
    jobs = [Job(lam_idx=0, g_idx=0, n_packets=n_packets, key=0)]
    return Workload("uniform_absorber", MODE_TRANSMISSION, grid, xs, src, jobs, seed)


def uniform_scattering_sphere(alpha=8.0e-9, omega=1.0e-3, g=0.5, R0=R_JUP, H_atm=R_JUP, nlon=4, nlat=4, nr=4,
                              n_packets=20000, seed=14, trans_scatter=1, survival=1, ld_law=0,
                              ld_coef=(0.0, 0.0, 0.0, 0.0), star_radius=0.0, star_dist=0.0, transit_xy=(0.0, 0.0)):
    """Transmission through a uniform shell R0..R0+H of extinction alpha, single-scattering albedo omega
    and HG asymmetry g, all in one cloud component (P_gas = 0): chord tau(b) = 2 alpha sqrt(R_toa^2 - b^2).
    The default thick shell (R_toa = 2 R0) has chord optical depths up to ~2."""
    grid = uniform_grid(nlon, nlat, nr, R0, R0 + H_atm, rho=1.0)
    opac = AlbedoOpacity(kabs=np.array([0.0]), kray=np.array([0.0]), qcld=np.ones(1), wcld=np.array([omega]),
                         gcld=np.array([g]), acld=np.full(grid.ncell, alpha, np.float32))
    opts = Options(survival=survival, trans_scatter=trans_scatter, ld_law=ld_law, ld_coef=tuple(ld_coef),
                   star_radius=star_radius, star_dist=star_dist, transit_xy=tuple(transit_xy))
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]), opts=opts)
    jobs = [Job(lam_idx=0, g_idx=0, n_packets=n_packets, key=0)]
    return Workload("uniform_scatterer", MODE_TRANSMISSION, grid, opac, src, jobs, seed)


def slab_sphere_albedo(omega=0.5, tau=20.0, phase="iso", g=0.0, n_packets=100_000, seed=12, thin=1.0e-4,
                       nlon=8, nlat=8, survival=1, surface_albedo=0.0, obs=None, forced_first=0, cont_abs=0,
                       path_bias=0):
    """Homogeneous one-layer atmosphere of thickness thin * R0 and vertical optical depth tau on a
    black (or Lambertian, surface_albedo) sphere: locally a plane-parallel slab.  phase = 'iso'
    (HG with g = 0), 'hg', 'tthg' (two-term HG of asymmetry g) or 'rayleigh'."""
    R0 = R_JUP
    H = thin * R0
    grid = uniform_grid(nlon, nlat, 1, R0, R0 + H, rho=1.0)
    kext = tau / H
    if phase == "rayleigh":
        opac = AlbedoOpacity(kabs=np.array([(1 - omega) * kext]), kray=np.array([omega * kext]),
                             qcld=np.zeros(1), wcld=np.zeros(1), gcld=np.zeros(1))
    else:
        opac = AlbedoOpacity(kabs=np.array([0.0]), kray=np.array([0.0]), qcld=np.ones(1),
                             wcld=np.array([omega]), gcld=np.array([g if phase in ("hg", "tthg") else 0.0]),
                             acld=np.full(grid.ncell, kext, np.float32))
    src = Source(star=np.array([1.0, 0.0, 0.0]),
                 obs=np.array([[1.0, 0.0, 0.0]]) if obs is None else np.atleast_2d(np.asarray(obs, np.float64)),
                 opts=Options(survival=survival, w_rr=1e-4, cloud_phase=1 if phase == "tthg" else 0,
                              surface_albedo=surface_albedo, forced_first=forced_first, cont_abs=cont_abs,
                              path_bias=path_bias))
    jobs = [Job(lam_idx=0, g_idx=0, n_packets=n_packets, key=0)]
    return Workload(f"slab_{phase}_w{omega}_t{tau}", MODE_ALBEDO, grid, opac, src, jobs, seed)


def isothermal_emitter(tau=2.0, T=1500.0, thin=1.0e-4, nlon=8, nlat=8, nr=4, n_packets=100_000, seed=13,
                       lam=2.0e-6, taus=None, wg=None, g_bias=0, g_beta=0.5):
    """Isothermal, uniform-kappa shell with scattering off: escaping intensity B (1 - exp(-tau/mu)).
    taus, wg: a band of g-ordinates with vertical optical depths taus and weights wg, run as one
    job with per-packet g sampling."""
    R0 = R_JUP
    H = thin * R0
    grid = uniform_grid(nlon, nlat, nr, R0, R0 + H, rho=1.0, T=T, p=1.0e4)
    taus = np.array([tau]) if taus is None else np.asarray(taus, np.float64)
    wg = np.array([1.0]) if wg is None else np.asarray(wg, np.float64)
    kap = taus / H
    kt = KTable(lam=np.array([lam]), wg=wg, gpts=(np.arange(len(taus)) + 0.5) / len(taus),
                Tg=np.array([500.0, 3000.0]), pg=np.array([1.0, 1.0e7]),
                k=np.broadcast_to(kap[None, :, None, None], (1, len(taus), 2, 2)).astype(np.float32))
    src = Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[1.0, 0.0, 0.0]]),
                 opts=Options(scatter_emission=0, g_bias=g_bias, g_beta=g_beta))
    jobs = [Job(lam_idx=0, g_idx=0 if len(taus) == 1 else -1, n_packets=n_packets, key=0)]
    return Workload("isothermal_emitter", MODE_EMISSION, grid, kt, src, jobs, seed)
