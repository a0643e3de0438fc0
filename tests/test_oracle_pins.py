"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published known-answer
vectors, closed-form CDFs and integrals, brute-force enumeration of ray/surface crossings,
an independent adding-doubling plane-parallel solver (itself pinned to Chandrasekhar's
H-function, single-scattering closed forms and flux conservation), and exact ledger closure.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import refsolvers as R
from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------ RNG

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


# ------------------------------------------------------------------ samplers and phase functions (Sect. 3)

def rayleigh_cdf(mu):
    # integral of p(mu) = 3/8 (1 + mu^2) from -1: (mu^3 + 3 mu + 4) / 8
    return (mu ** 3 + 3.0 * mu + 4.0) / 8.0


def hg_cdf(mu, g):
    return (1.0 - g * g) / (2.0 * g) * (1.0 / np.sqrt(1.0 + g * g - 2.0 * g * mu) - 1.0 / (1.0 + g))


def test_rayleigh_sampler_is_inverse_cdf():
    z = np.linspace(1e-6, 1 - 1e-6, 2001)
    mu = np.array([O.sample_rayleigh(v) for v in z])
    assert np.all(np.diff(mu) > 0)
    assert np.max(np.abs(rayleigh_cdf(mu) - z)) < 1e-12
    assert abs(O.sample_rayleigh(0.5)) < 1e-15


def test_rayleigh_sampler_ks():
    rng = np.random.default_rng(5)
    mu = np.array([O.sample_rayleigh(v) for v in rng.random(40000)])
    assert stats.kstest(mu, rayleigh_cdf).pvalue > 1e-3


@pytest.mark.parametrize("g", [-0.7, -0.1, 0.3, 0.6, 0.9])
def test_hg_sampler_is_inverse_cdf(g):
    z = np.linspace(1e-6, 1 - 1e-6, 2001)
    mu = np.array([O.sample_hg(g, v) for v in z])
    assert np.all(np.diff(mu) >= 0)
    assert np.max(np.abs(hg_cdf(mu, g) - z)) < 1e-9


def test_hg_sampler_small_g_is_isotropic():
    for v in (0.1, 0.5, 0.93):
        assert O.sample_hg(0.0, v) == 2 * v - 1
        assert O.sample_hg(5e-5, v) == 2 * v - 1


@pytest.mark.parametrize("pgas,g", [(1.0, 0.0), (0.0, 0.6), (0.0, 0.9), (0.3, 0.6), (0.0, -0.4)])
def test_theta_is_normalised_over_the_sphere(pgas, g):
    x, w = np.polynomial.legendre.leggauss(400)
    tot = 2.0 * math.pi * sum(wi * O.theta(xi, pgas, g) for xi, wi in zip(x, w))
    assert abs(tot - 1.0) < 1e-8
    # HG mean cosine is g
    if pgas == 0.0:
        mean = 2.0 * math.pi * sum(wi * xi * O.theta(xi, 0.0, g) for xi, wi in zip(x, w))
        assert abs(mean - g) < 1e-6


def test_turn_keeps_unit_length_and_polar_angle():
    rng = np.random.default_rng(7)
    for _ in range(500):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        mu = rng.uniform(-1, 1)
        psi = rng.uniform(0, 2 * math.pi)
        n = O.turn(d, mu, psi)
        assert abs(np.linalg.norm(n) - 1) < 1e-12
        assert abs(n @ d - mu) < 1e-12
    # azimuth uniform: the mean of the turned directions over psi is mu d
    d = np.array([0.3, -0.5, 0.81])
    d /= np.linalg.norm(d)
    m = np.mean([O.turn(d, 0.2, p) for p in np.linspace(0, 2 * math.pi, 4000, endpoint=False)], axis=0)
    assert np.linalg.norm(m - 0.2 * d) < 1e-10


def test_planck_integrates_to_sigma_T4_over_pi():
    T = 1500.0
    lam = np.geomspace(1e-8, 1e-2, 200001)
    B = np.array([O.planck(l, T) for l in lam])
    tot = np.trapezoid(B * lam, np.log(lam))
    sigma_sb = 5.670374419e-8
    assert abs(tot / (sigma_sb * T ** 4 / math.pi) - 1) < 1e-4


# ------------------------------------------------------------------ geometry: brute-force enumeration

def _grids():
    fat_r = np.array([1.0, 1.2, 1.45, 1.7, 2.0])
    g1 = S.uniform_grid(4, 4, 4, 1.0, 2.0, r_edges=fat_r)
    g2 = S.uniform_grid(8, 6, 5, S.R_JUP, S.R_JUP + 1.0e7)
    lat3 = np.array([-math.pi / 2, -0.9, -0.2, 0.0, 0.35, 1.1, math.pi / 2])
    lon3 = np.linspace(0.3, 0.3 + 2 * math.pi, 6)
    g3 = S.uniform_grid(5, 6, 4, 1.0, 1.5, lat_edges=lat3, lon_edges=lon3)
    # degenerate grids: two longitude cells (both edges lie in the plane y = 0, so only the half-plane
    # test tells them apart), one longitude cell, one latitude band
    g4 = S.uniform_grid(2, 3, 3, 1.0, 2.0)
    g5 = S.uniform_grid(1, 1, 2, 1.0, 2.0)
    g6 = S.uniform_grid(3, 1, 2, 1.0, 2.0)
    return [g1, g2, g3, g4, g5, g6]


def _random_interior_point(rng, g):
    r = rng.uniform(g.r_edges[0] * 1.0001, g.r_edges[-1] * 0.9999)
    sl = rng.uniform(-0.999, 0.999)
    ph = rng.uniform(0, 2 * math.pi)
    cl = math.sqrt(1 - sl * sl)
    return np.array([r * cl * math.cos(ph), r * cl * math.sin(ph), r * sl])


def _flat(g, x):
    i, j, k = R._locate(g, x)
    return (k * g.nlat + j) * g.nlon + i


def _compare(g, o, d):
    alpha = np.ones(g.ncell)
    cells, lens, st = O.trace_ray(g, alpha, o, d, _flat(g, o))
    ref = R.brute_segments(g, o, d)
    assert st in (1, 2)
    assert len(ref) == len(cells), (o, d, len(ref), len(cells))
    scale = g.r_edges[-1]
    for (rc, rl), c, l in zip(ref, cells, lens):
        assert rc == c
        assert abs(rl - l) <= 1e-12 * scale + 1e-10 * rl


@pytest.mark.parametrize("gi", [0, 1, 2, 3, 4, 5])
def test_march_matches_brute_force_random_rays(gi):
    g = _grids()[gi]
    rng = np.random.default_rng(100 + gi)
    for _ in range(600):
        o = _random_interior_point(rng, g)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        _compare(g, o, d)


def test_march_matches_brute_force_special_rays():
    g = _grids()[0]
    rng = np.random.default_rng(9)
    rays = []
    # near-polar passes
    for _ in range(50):
        o = np.array([rng.uniform(-0.05, 0.05), rng.uniform(-0.05, 0.05), rng.uniform(1.25, 1.9)])
        o *= rng.uniform(1.05, 1.1) / np.linalg.norm(o) * np.linalg.norm(o)
        d = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-0.2, 0.2)])
        rays.append((o, d / np.linalg.norm(d)))
    # grazing shells: closest approach just above an inner shell
    for k in (1, 2, 3):
        for eps in (1e-3, 1e-6, 1e-9):
            p = g.r_edges[k] * (1 + eps)
            ph = rng.uniform(0, 2 * math.pi)
            c = np.array([p * math.cos(ph), p * math.sin(ph), 0.1])
            c *= p / np.linalg.norm(c)
            t = np.cross(c, [0.0, 0.0, 1.0])
            t /= np.linalg.norm(t)
            rays.append((c - 0.3 * t, t))
    # equator-plane crossings and horizontal rays
    for _ in range(50):
        o = _random_interior_point(rng, g)
        d = np.array([rng.normal(), rng.normal(), -np.sign(o[2]) * abs(rng.normal())])
        rays.append((o, d / np.linalg.norm(d)))
        rays.append((o, np.array([o[1], -o[0], 0.0]) / math.hypot(o[0], o[1])))
    for o, d in rays:
        if not (g.r_edges[0] < np.linalg.norm(o) < g.r_edges[-1]):
            continue
        _compare(g, o, d)


# ------------------------------------------------------------------ transmission (Sect. 5.1)

ALPHA32 = float(np.float32(2.0e-6))     # the table stores the uniform cross-section in FP32

def test_chord_tau_of_uniform_absorber_matches_closed_form():
    wl = S.uniform_absorber_sphere(n_packets=4000)
    job = wl.jobs[0]
    r = O.run(wl, job, per_packet=True)
    g = wl.grid
    key = [wl.seed & 0xFFFFFFFF, wl.seed >> 32]
    for n in range(job.n_packets):
        w = O.philox([n, 0, 0, job.key], key)
        u = ((w[0] >> 8) + 0.5) / 2 ** 24
        b = g.R0 + u * (g.R_toa - g.R0)
        tau = 2.0 * ALPHA32 * math.sqrt(g.R_toa ** 2 - b * b)
        if tau <= wl.source.opts.tau_peel_cut:
            # FP64 conditioning of R^2 - b^2 near grazing: path-length error ~ 1e-12 R_TOA
            assert abs(r["pk_tau"][n] - tau) <= 1e-12 * tau + ALPHA32 * 1e-12 * g.R_toa


def test_transmission_integral_within_3_sigma():
    wl = S.uniform_absorber_sphere(n_packets=200_000)
    job = wl.jobs[0]
    r = O.run(wl, job, per_packet=True, nthreads=8)
    g = wl.grid
    f = r["pk_f"][:, 0] * (g.R_toa - g.R0) * g.R_toa
    est = 2.0 * f.mean()
    sig = 2.0 * f.std() / math.sqrt(len(f))
    exact = R.transmission_integral_uniform(ALPHA32, g.R0, g.R_toa)
    assert abs(est - exact) < 3 * sig


# ------------------------------------------------------------------ energy ledger

@pytest.mark.parametrize("survival", [1, 0])
def test_energy_ledger_closes(survival):
    wl = S.config1_albedo(n_packets=20000, nlon=8, nlat=6, nr=10, survival=survival)
    r = O.run(wl, wl.jobs[0], nthreads=4)
    L = r["ledger"]
    lhs = L[0] + L[4]
    rhs = L[1] + L[2] + L[3] + L[5] + L[6] + L[7]
    assert L[6] == 0 and L[7] == 0
    assert abs(lhs - rhs) <= 1e-12 * lhs
    if survival == 0:
        assert L[4] == 0 and L[5] == 0


# ------------------------------------------------------------------ albedo vs plane-parallel solutions (Sect. 5.2, 9)

AD_CASES = [
    ("iso", [1.0], 0.5, 20.0),
    ("iso", [1.0], 1.0, 2.0),
    ("iso", [1.0], 0.9, 0.5),
    ("rayleigh", [1.0, 0.0, 0.5], 1.0, 2.0),
    ("rayleigh", [1.0, 0.0, 0.5], 0.5, 20.0),
]


@pytest.mark.parametrize("phase,beta,omega,tau", AD_CASES)
def test_geometric_albedo_matches_adding_doubling(phase, beta, omega, tau):
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase=phase, n_packets=100_000)
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = math.pi * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.AddingDoubling(beta, omega, tau, n=40).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-5 * ref, (est, ref, sig)


@pytest.mark.parametrize("phase,beta,omega,tau", [AD_CASES[2], AD_CASES[4]])
def test_analog_scattering_matches_adding_doubling(phase, beta, omega, tau):
    """Analog mode (scatter with probability omega, else absorb) has the same expectation."""
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase=phase, n_packets=200_000, survival=0)
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = math.pi * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.AddingDoubling(beta, omega, tau, n=40).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-5 * ref, (est, ref, sig)
    assert r["ledger"][4] == 0 and r["ledger"][2] > 0


def test_frequent_roulette_matches_adding_doubling():
    """Russian roulette at W < 0.5 W_launch with survival probability 0.5 (so after nearly every second
    scattering) leaves the expectation unchanged: survivors carry W / p_surv."""
    phase, beta, omega, tau = AD_CASES[0]
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase=phase, n_packets=200_000)
    wl.source.opts.w_rr, wl.source.opts.p_surv = 0.5, 0.5
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = math.pi * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.AddingDoubling(beta, omega, tau, n=40).geometric_albedo()
    L = r["ledger"]
    assert L[4] > 0.05 * L[0] and L[5] > 0.05 * L[0]
    assert abs(est - ref) < 3 * sig + 1e-5 * ref, (est, ref, sig)


def test_adding_doubling_pins():
    # semi-infinite isotropic: H-function
    for om in (0.5, 0.9):
        ad = R.AddingDoubling([1.0], om, 2000.0).geometric_albedo()
        assert abs(ad / R.ag_isotropic_semi_infinite(om) - 1) < 1e-6
    # single scattering: A_g -> omega P(-1) / 8
    for beta, P1 in (([1.0], 1.0), ([1.0, 0.0, 0.5], 1.5)):
        ad = R.AddingDoubling(beta, 1e-4, 100.0).geometric_albedo()
        assert abs(ad / (1e-4 * P1 / 8) - 1) < 3e-4
    # conservative slab: reflected + transmitted flux = 1
    for beta in ([1.0], [1.0, 0.0, 0.5]):
        ad = R.AddingDoubling(beta, 1.0, 3.0)
        assert np.max(np.abs(ad.plane_albedo() + ad.flux_transmission() - 1)) < 2e-6


@pytest.mark.parametrize("phase,g,p_back", [("hg", 0.6, (1 - 0.6) / (1 + 0.6) ** 2), ("iso", 0.0, 1.0),
                                             ("rayleigh", 0.0, 1.5)])
def test_single_scattering_albedo(phase, g, p_back):
    """Semi-infinite, weakly scattering: A_g = omega P(mu = -1) / 8 to first order in omega (omega/8
    isotropic, 3 omega/16 Rayleigh, omega (1 - g)/(8 (1 + g)^2) HG)."""
    om = 1e-3
    wl = S.slab_sphere_albedo(omega=om, tau=30.0, phase=phase, g=g, n_packets=100_000)
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = math.pi * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = om * p_back / 8
    # higher orders contribute O(omega) relative
    assert abs(est - ref) < 3 * sig + 2 * om * ref, (est, ref, sig)


def test_semi_infinite_isotropic_albedo_matches_h_function():
    """A thick isotropic layer (tau = 60) against Chandrasekhar's H-function:
    A_g = (omega/4) int_0^1 H(mu)^2 mu dmu."""
    om = 0.9
    wl = S.slab_sphere_albedo(omega=om, tau=60.0, phase="iso", n_packets=200_000)
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = math.pi * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.ag_isotropic_semi_infinite(om)
    assert abs(est - ref) < 3 * sig + 1e-4 * ref, (est, ref, sig)


# ------------------------------------------------------------------ emission (Sect. 5.3)

def test_isothermal_shell_emission_matches_closed_form():
    tau = 2.0
    wl = S.isothermal_emitter(tau=tau, n_packets=100_000)
    job = wl.jobs[0]
    cells = O.prep_cells(wl, job)
    r = O.run(wl, job, cells=cells, per_packet=True, nthreads=8)
    scale = cells["L_tot"]
    f = scale * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    B = O.planck(wl.opac.lam[0], float(wl.grid.T[0]))
    Rm = 0.5 * (wl.grid.R0 + wl.grid.R_toa)
    ref = R.emission_shell_Lp(B, tau, Rm)
    assert abs(est - ref) < 3 * sig + 2e-4 * ref, (est, ref, sig)


def test_thick_transparent_shell_emission_is_occulted_by_the_core():
    """An optically thin isothermal shell R0..2R0 held in one cell emits uniformly per volume; towards a
    distant observer the black core hides the points in its cylindrical shadow, of volume
    2 pi/3 [R_TOA^3 - (R_TOA^2 - R0^2)^(3/2) - R0^3].  The visible fraction pins the launch position
    (uniform in r^3, sin(lat) and lon) and the occultation of peel-offs by the lower boundary."""
    wl = S.isothermal_emitter(tau=1e-6, thin=1.0, nlon=1, nlat=1, nr=1, n_packets=200_000)
    g = wl.grid
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = 4 * math.pi * r["pk_f"][:, 0]          # W e^-tau with W = 1 for a single emitting cell
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    R0, Rt = g.R0, g.R_toa
    v_shadow = 2 * math.pi / 3 * (Rt ** 3 - (Rt ** 2 - R0 ** 2) ** 1.5 - R0 ** 3)
    ref = 1.0 - v_shadow / (4 * math.pi / 3 * (Rt ** 3 - R0 ** 3))
    # e^-tau of the longest path is 1 - 4e-6
    assert abs(est - ref) < 3 * sig + 4e-6, (est, ref, sig)


def test_emission_tables():
    wl = S.config2_emission(n_packets=1000, nlon=16, nlat=8, nr=12, nb=3, ng=2)
    g = wl.grid
    c = O.prep_emission(g, wl.opac, 1, 1, wl.source.opts)
    # volumes: sum of L / (4 pi alpha B) over all cells is the shell volume
    B = np.array([O.planck(wl.opac.lam[1], t) for t in g.T.astype(np.float64)])
    V = c["L"] / (4 * math.pi * c["alpha"] * B)
    assert abs(V.sum() / (4 * math.pi / 3 * (g.R_toa ** 3 - g.R0 ** 3)) - 1) < 1e-12
    # pdf: monotone cdf summing to 1, E_q[W] = 1
    q = np.diff(np.concatenate([[0.0], c["cdf"]]))
    assert np.all(q >= 0) and abs(c["cdf_total"] - 1) < 1e-12
    assert abs(np.sum(q * c["wcell"]) - 1) < 1e-12
    # tau_vert cut recomputed from alpha
    a = c["alpha"].reshape(g.nr, g.nlat, g.nlon)
    dz = np.diff(g.r_edges)
    above = np.cumsum((a * dz[:, None, None])[::-1], axis=0)[::-1] - a * dz[:, None, None]
    incl = (above < wl.source.opts.tau_vert_max).reshape(-1)
    assert np.array_equal(incl, q > 0) or np.array_equal(incl & (q > 0), q > 0)
    assert c["n_incl"] == int(incl.sum())


# ------------------------------------------------------------------ Doppler (Sect. 7)

def test_doppler_zero_wind_is_unshifted_and_rotation_matches_vector_form():
    wl = S.config4_transmission(nlon=12, nlat=6, nr=5, n_lam=200, n_lines=100, lam_subset=[50])
    g, xs = wl.grid, wl.opac
    li = wl.jobs[0].lam_idx
    c = O.prep_xsec(g, xs, li)
    # zero wind and no rotation: alpha is the table at the rest wavelength exactly
    g0 = S.Grid(**{**g.__dict__, "wind": np.zeros_like(g.wind)})
    xs0 = S.XsecTable(lam=xs.lam, Tg=xs.Tg, pg=xs.pg, sigma=xs.sigma, view_theta=xs.view_theta,
                      view_phi=xs.view_phi, omega_rot=0.0)
    c0 = O.prep_xsec(g0, xs0, li)
    assert np.all(c0["vlos"] == 0)
    g0b = S.Grid(**{**g.__dict__, "wind": None})
    assert np.array_equal(O.prep_xsec(g0b, xs0, li)["alpha"], c0["alpha"])
    # solid-body rotation only: v_LOS = -(Omega x r) . n_obs with n_obs the unit vector to the observer
    xsr = S.XsecTable(lam=xs.lam, Tg=xs.Tg, pg=xs.pg, sigma=xs.sigma, view_theta=xs.view_theta,
                      view_phi=xs.view_phi, omega_rot=xs.omega_rot)
    cr = O.prep_xsec(g0, xsr, li)
    n_obs = np.array([math.sin(xs.view_theta) * math.cos(xs.view_phi),
                      math.sin(xs.view_theta) * math.sin(xs.view_phi), math.cos(xs.view_theta)])
    LAT, LON = S.cell_centres(g.nlon, g.nlat, g.lat_edges, g.lon_edges)
    rmid = 0.5 * (g.r_edges[:-1] + g.r_edges[1:])
    pos = np.stack([np.cos(LAT) * np.cos(LON), np.cos(LAT) * np.sin(LON), np.sin(LAT)], -1)
    vel = np.cross(np.array([0, 0, xs.omega_rot]), pos[None] * rmid[:, None, None, None])
    ref = -(vel @ n_obs).reshape(-1)
    assert np.max(np.abs(cr["vlos"] - ref)) < 1e-9 * np.max(np.abs(ref))
    # wind components: v_LOS = -(u e_east + v e_north + w e_up) . n_obs
    u, v, w = (g.wind[k].astype(np.float64).reshape(g.nr, g.nlat, g.nlon) for k in range(3))
    east = np.stack([-np.sin(LON), np.cos(LON), 0 * LON], -1)
    north = np.stack([-np.sin(LAT) * np.cos(LON), -np.sin(LAT) * np.sin(LON), np.cos(LAT)], -1)
    vec = u[..., None] * east + v[..., None] * north + w[..., None] * pos[None]
    refw = -(vec @ n_obs).reshape(-1) + ref
    assert np.max(np.abs(c["vlos"] - refw)) < 1e-9 * np.max(np.abs(refw))


def test_power_law_opacity_is_interpolated_exactly():
    """k(T, p) = k0 (T/T0)^a (p/p0)^b is linear in (ln T, ln p), so the bilinear interpolation of ln k in
    (ln T, ln p) (Sect. 7) returns it exactly between the table nodes, to the FP32 rounding of the table
    (an interpolation linear in T or p would be off by up to percents).  Both the k-table and the
    cross-section path."""
    g, _ = S.hotjupiter_grid(16, 8, 12)
    Tg, pg = np.geomspace(500.0, 3000.0, 4), np.geomspace(1e-1, 1e7, 5)
    law = lambda T, p: 1e-3 * (T / 1500.0) ** 1.3 * (p / 1e5) ** 0.45  # noqa: E731
    k = law(Tg[:, None], pg[None, :])
    ref = g.rho.astype(np.float64) * law(g.T.astype(np.float64), g.p.astype(np.float64))
    kt = S.KTable(lam=np.array([2e-6]), wg=np.array([1.0]), gpts=np.array([0.5]), Tg=Tg, pg=pg,
                  k=k[None, None].astype(np.float32))
    np.testing.assert_allclose(O.prep_emission(g, kt, 0, 0, S.Options())["alpha"], ref, rtol=1e-6)
    xs = S.XsecTable(lam=np.array([1.0e-6, 1.1e-6]), Tg=Tg, pg=pg,
                     sigma=np.broadcast_to(k, (2,) + k.shape).astype(np.float32))
    np.testing.assert_allclose(O.prep_xsec(g, xs, 0)["alpha"], ref, rtol=1e-6)


def test_uniform_translation_shifts_the_spectrum_by_whole_bins():
    """A planet moving bodily away from the observer at v sees every line at lambda / (1 - v/c) (Sect. 7).
    On a table uniform in ln(lambda) with step 1/R, v = c (1 - e^(-k/R)) moves the opacity spectrum of
    every cell by exactly k table bins, whatever the interpolation between bins."""
    Rres, k, n = 1.0e5, 3, 160
    lam = 1.0e-6 * np.exp(np.arange(n) / Rres)
    line = 1.0e-3 * (1.0 + 200.0 * np.exp(-0.5 * ((np.arange(n) - 80.0) / 6.0) ** 2))
    sigma = np.broadcast_to(line[:, None, None], (n, 2, 2)).astype(np.float32)
    xs = S.XsecTable(lam=lam, Tg=np.array([500.0, 3000.0]), pg=np.array([1.0, 1.0e7]), sigma=sigma)
    g = S.uniform_grid(6, 4, 2, S.R_JUP, 1.1 * S.R_JUP)
    v = 2.99792458e8 * -math.expm1(-k / Rres)
    n_obs = np.array([math.sin(xs.view_theta) * math.cos(xs.view_phi),
                      math.sin(xs.view_theta) * math.sin(xs.view_phi), math.cos(xs.view_theta)])
    V = -v * n_obs                       # recession from the observer at speed v
    LAT, LON = S.cell_centres(g.nlon, g.nlat, g.lat_edges, g.lon_edges)
    east = np.stack([-np.sin(LON), np.cos(LON), 0 * LON], -1)
    north = np.stack([-np.sin(LAT) * np.cos(LON), -np.sin(LAT) * np.sin(LON), np.cos(LAT)], -1)
    up = np.stack([np.cos(LAT) * np.cos(LON), np.cos(LAT) * np.sin(LON), np.sin(LAT)], -1)
    comp = [np.broadcast_to(e @ V, (g.nr, g.nlat, g.nlon)).reshape(-1) for e in (east, north, up)]
    moving = S.Grid(**{**g.__dict__, "wind": np.stack(comp).astype(np.float32)})
    still = [O.prep_xsec(g, xs, i)["alpha"] for i in range(n)]
    for i in range(k, n):
        c = O.prep_xsec(moving, xs, i)
        assert np.allclose(c["vlos"], v, rtol=1e-6, atol=0)
        np.testing.assert_allclose(c["alpha"], still[i - k], rtol=1e-6)
    # the line centre moves by lambda_c v / c to first order
    assert abs(lam[80 + k] - lam[80] - lam[80] * v / 2.99792458e8) < 1e-4 * lam[80] * v / 2.99792458e8


def test_step_cap_books_exactly_the_packets_it_cuts():
    """Per-packet step cap (not in the paper; the design's reading of it): the weight booked as step-capped
    is that of the packets whose peel-off needs more cell steps than the cap allows, found by running the
    same packets without a cap; a packet whose ray ends on exactly its last allowed step is not booked,
    and every other packet keeps its uncapped contribution."""
    wl = S.config2_emission(n_packets=4000, nlon=16, nlat=8, nr=12, nb=2, ng=2, bands=[1], gpoints=[1])
    job = wl.jobs[0]
    cells = O.prep_cells(wl, job)
    free = O.run(wl, job, cells=cells, per_packet=True, n_trace=4000, max_trace=400)
    cap = int(np.median(free["pk_steps"]))
    wl.source.opts.max_steps = cap
    capped = O.run(wl, job, cells=cells, per_packet=True)
    first = np.array([c[c >= 0][0] for c in (free["tr_cell"][q, :free["tr_n"][q]] for q in range(4000))])
    W = np.asarray(cells["wcell"])[first]                 # launch weight of each packet (one g-ordinate)
    cut = free["pk_steps"] > cap
    assert cut.any() and (free["pk_steps"] == cap).any()
    assert capped["ledger"][6] == pytest.approx(W[cut].sum(), rel=1e-12)
    np.testing.assert_array_equal(capped["pk_steps"], np.minimum(free["pk_steps"], cap))
    np.testing.assert_array_equal(capped["pk_f"][~cut], free["pk_f"][~cut])
    assert np.all(capped["pk_f"][cut] == 0.0)
