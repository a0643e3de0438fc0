"""The seeded synthetic inputs follow their stated recipes (sizes, value ranges and structure of the
paper's workloads). These check the generators only: no method arithmetic is involved."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2110_15640_gb300 import synth as S


def _log_uniform_edges(g, p_top, p_bot):
    """Pressure at the grid's edges from its hydrostatic layer densities: p_top + sum over the layers
    above of rho g dz."""
    dz = np.diff(g.r_edges)
    rho = g.rho.reshape(g.nr, g.nlat, g.nlon)[:, 0, 0].astype(np.float64)
    dp = rho * 10.0 * dz
    return p_top * S.BAR + np.concatenate([np.cumsum(dp[::-1])[::-1], [0.0]])


def test_albedo_32x16x20_recipe():
    wl = S.config1_albedo()
    g = wl.grid
    assert (g.nlon, g.nlat, g.nr) == (32, 16, 20) and g.R0 == S.R_JUP
    # isothermal 1500 K, mu = 2.3, g = 10: scale height 542.3 km, 1e-5..100 bar is ln(1e7) scale heights
    H = S.K_B * 1500.0 / (2.3 * S.M_U * 10.0)
    assert abs(H - 542.3e3) < 0.1e3
    assert abs((g.R_toa - g.R0) / (H * math.log(1e7)) - 1) < 1e-12
    assert np.all(g.T == 1500.0)
    # the layer densities are hydrostatic: the edges come back log-uniform in pressure
    pe = _log_uniform_edges(g, 1e-5, 100.0)
    np.testing.assert_allclose(pe, np.logspace(2, -5, 21) * S.BAR, rtol=2e-6)
    # grey extinction with vertical tau = 10 over the column, half of it Rayleigh scattering
    k = wl.opac.kabs[0] + wl.opac.kray[0]
    assert abs(k / 1.0000001e-5 - 1) < 1e-12
    assert wl.opac.kabs[0] == wl.opac.kray[0]
    col = k * np.sum(g.rho.reshape(g.nr, g.nlat, g.nlon)[:, 0, 0].astype(np.float64) * np.diff(g.r_edges))
    assert abs(col - 10.0) < 1e-5
    assert np.array_equal(wl.source.star, wl.source.obs[0])       # phase 0
    assert len(wl.jobs) == 1 and wl.jobs[0].n_packets == 100_000


def test_emission_128x64x50_recipe():
    wl = S.config2_emission()
    g, kt = wl.grid, wl.opac
    assert (g.nlon, g.nlat, g.nr) == (128, 64, 50)
    np.testing.assert_allclose(_log_uniform_edges(g, 1e-6, 100.0), np.logspace(2, -6, 51) * S.BAR, rtol=2e-6)
    # day-night temperature: the hottest column sits at the 15 deg hot spot on the equator, and the
    # night side's columns all share one profile
    T = g.T.reshape(g.nr, g.nlat, g.nlon).astype(np.float64)
    LAT, LON = S.cell_centres(g.nlon, g.nlat, g.lat_edges, g.lon_edges)
    j, i = np.unravel_index(np.argmax(T[g.nr // 2]), LAT.shape)
    assert abs(math.degrees(LON[j, i]) - 15.0) <= 360.0 / g.nlon and abs(math.degrees(LAT[j, i])) <= 180.0 / g.nlat
    night = np.cos(LON - math.radians(15.0)) * np.cos(LAT) <= 0
    assert np.ptp(T[:, night], axis=1).max() == 0.0
    # the Guillot-like profile with gamma = 0.5 cools the top to 0.92 T_h and the internal heat
    # (T_int = 400 K) warms the 100 bar level above T_h
    assert 0.9 * 1000.0 <= T.min() <= 1000.0 and 2200.0 <= T.max() <= 1.25 * 2200.0
    # 30 bands log-spaced over 1-5 um, 8 Gauss-Legendre g-ordinates on [0, 1], k increasing with g
    assert len(kt.lam) == 30 and abs(kt.lam[0] - 1e-6) < 1e-18 and abs(kt.lam[-1] - 5e-6) < 1e-18
    np.testing.assert_allclose(np.diff(np.log(kt.lam)), math.log(5.0) / 29, rtol=1e-12)
    assert len(kt.wg) == 8 and abs(kt.wg.sum() - 1) < 1e-14 and np.all((kt.gpts > 0) & (kt.gpts < 1))
    assert np.all(np.diff(kt.k.astype(np.float64), axis=1) > 0)
    # 240 jobs of 1e6 packets with distinct Philox job keys
    assert len(wl.jobs) == 240 and all(j.n_packets == 1_000_000 for j in wl.jobs)
    assert len({j.key for j in wl.jobs}) == 240


def test_phase_curve_recipe():
    wl = S.config3_phase_curve()
    assert len(wl.jobs) == 960
    # 24 observer phases 0..345 deg in 15 deg steps, each job tallies one of them
    ang = np.degrees(np.arctan2(wl.source.obs[:, 1], wl.source.obs[:, 0])) % 360.0
    np.testing.assert_allclose(ang, np.arange(24) * 15.0, atol=1e-9)
    assert sorted({j.obs_idx for j in wl.jobs}) == list(range(24))
    n = np.array([j.n_packets for j in wl.jobs])
    assert n.min() >= 10_000 and n.max() <= 1_000_000
    assert stats.kstest((n - 1e4) / (1e6 - 1e4), "uniform").pvalue > 1e-3
    assert len({j.key for j in wl.jobs}) == 960
    # the cloud deck peaks near 0.1 bar and has a column optical depth of at most 5
    g = wl.grid
    a = wl.opac.acld.reshape(g.nr, g.nlat, g.nlon).astype(np.float64)
    dz = np.diff(g.r_edges)
    col = (a * dz[:, None, None]).sum(0)
    assert col.max() <= 5.0 * (1 + 1e-6) and col.min() > 0
    p_peak = g.p.reshape(g.nr, g.nlat, g.nlon)[np.argmax(a[:, 0, 0] * dz), 0, 0]
    assert abs(math.log10(p_peak / (0.1 * S.BAR))) < 0.2
    assert np.all(wl.opac.wcld == 0.9) and np.all(wl.opac.gcld == 0.6)


def test_transmission_96x48x60_recipe():
    wl = S.config4_transmission()
    g, xs, m = wl.grid, wl.opac, wl.notes["margin"]
    assert (g.nlon, g.nlat, g.nr) == (96, 48, 60)
    assert len(wl.jobs) == 9532 and all(j.n_packets == 10_000 for j in wl.jobs)
    lam = np.array([xs.lam[j.lam_idx] for j in wl.jobs])
    np.testing.assert_allclose(lam, 1.0e-6 * np.exp(np.arange(9532) / 1.0e5), rtol=1e-14)
    assert xs.sigma.shape == (9532 + 2 * m, 20, 15) and np.all(xs.sigma > 0)
    assert abs(xs.Tg[0] - 500.0) < 1e-9 and abs(xs.Tg[-1] - 3000.0) < 1e-9
    # winds: a cos^2(lat) jet of 5 km/s and a 3 km/s day-night flow, no vertical motion
    u, v, w = (c.astype(np.float64) for c in g.wind)
    assert np.all(w == 0) and np.sqrt(u ** 2 + v ** 2).max() <= 8000.0
    # rotation period 3.5 days; observer opposite the star
    assert abs(2 * math.pi / xs.omega_rot / 86400.0 - 3.5) < 1e-12
    assert np.array_equal(wl.source.obs[0], -wl.source.star)


def test_serving_stream_recipe():
    sw = S.config5_serving(n_requests=10_000)
    assert [(s.grid.nlon, s.grid.nlat, s.grid.nr) for s in sw.scenes] == list(S.SERVING_GRIDS)
    modes = np.array([r.mode for r in sw.requests])
    scenes = np.array([r.scene for r in sw.requests])
    for k in range(3):
        assert abs((modes == k).mean() - 1 / 3) < 4 * math.sqrt(2 / 9 / len(modes))
    for k in range(4):
        assert abs((scenes == k).mean() - 1 / 4) < 4 * math.sqrt(3 / 16 / len(scenes))
    n = np.array([r.n_packets for r in sw.requests], np.float64)
    x = (np.log(n) - math.log(1e4)) / (math.log(1e7) - math.log(1e4))
    assert x.min() >= -1e-9 and x.max() <= 1 + 1e-9
    # log-uniform (the integer truncation moves ln n by less than 1e-4)
    assert stats.kstest(x, "uniform").pvalue > 1e-3
    assert len({r.key for r in sw.requests}) == len(sw.requests)


@pytest.mark.parametrize("builder", [S.config1_albedo, S.config3_phase_curve])
def test_generators_are_seeded(builder):
    a, b = builder(), builder()
    assert np.array_equal(a.grid.T, b.grid.T) and np.array_equal(a.grid.rho, b.grid.rho)
    assert [j.n_packets for j in a.jobs] == [j.n_packets for j in b.jobs]


def test_transit_scatter_recipe():
    wl = S.config6_transit_scatter()
    g, op = wl.grid, wl.source.opts
    assert (g.nlon, g.nlat, g.nr) == (128, 64, 50) and wl.mode == S.MODE_TRANSMISSION
    assert len(wl.jobs) == 40 and all(j.n_packets == 200_000 for j in wl.jobs)
    # quadratic limb darkening of a Sun-like star at 0.05 AU, transit impact parameter 0.3
    assert op.trans_scatter == 1 and op.cloud_phase == 1 and op.ld_law == 2 and tuple(op.ld_coef[:2]) == (0.45, 0.2)
    assert op.star_radius == S.R_SUN and abs(op.star_dist / S.AU - 0.05) < 1e-15
    assert abs(math.hypot(*op.transit_xy) / S.R_SUN - 0.3) < 1e-12
    assert np.array_equal(wl.source.obs[0], -wl.source.star)


def test_emission_hires_recipe():
    wl = S.config7_emission_hires(lam_subset=range(0, 9532, 10))
    g, xs, m = wl.grid, wl.opac, wl.notes["margin"]
    assert (g.nlon, g.nlat, g.nr) == (96, 48, 60) and wl.mode == S.MODE_EMISSION and g.wind is not None
    assert len(wl.jobs) == 954 and all(j.n_packets == 100_000 for j in wl.jobs)
    lam = np.array([xs.lam[j.lam_idx] for j in wl.jobs])
    np.testing.assert_allclose(lam, 1.0e-6 * np.exp(np.arange(0, 9532, 10) / 1.0e5), rtol=1e-14)
    # the observer looks at the dayside (+x): colatitude 90 deg, longitude 0
    assert xs.view_theta == 0.5 * math.pi and xs.view_phi == 0.0
    assert np.array_equal(wl.source.obs[0], [1.0, 0.0, 0.0]) and wl.source.opts.scatter_emission == 0
    assert m == 8
