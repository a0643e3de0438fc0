"""Pins of the oracle's transmission with multiple scattering and stellar limb darkening (Sect. 5.1),
against closed forms and quadratures written from the geometry, not from the oracle:

* each limb-darkening law equals 1 at the disk centre, and its disk normalisation 2 int mu I dmu
  equals the law's closed-form integral;
* on a uniform shell, the chord column is (1/(R_t - R0)) int (b/R_t)(1 - e^-tau(b)) db with
  tau(b) = 2 alpha sqrt(R_t^2 - b^2); with limb darkening the integrand carries the azimuthal mean of
  I(mu) over the chord's ring on the stellar disk (central and grazing transits);
* the scattered column's first order: a packet launched at b scatters first at optical depth t
  (pdf e^-t) and peels off forwards through the rest of its chord, so
  E[f b/R_t | b] = omega Theta(0 deg) tau(b) e^-tau(b) (b/R_t), up to terms of order omega^2;
  HG g = 0.5 makes forward and backward Theta differ 27-fold and the thick shell (R_t = 2 R0) makes
  b/R_t range over [0.5, 1], so a wrong peel direction or a missing b/R_t fails;
* the ledger closes under survival biasing and analog scattering;
* the stellar solid angle Omega_star against its small-disk series pi x^2 (1 + x^2/4 + x^4/8);
* an opaque planet small against the star: depth (R_TOA/R_star)^2 I(mu_c)/n_LD; scattered light
  lowers the effective blocked area;
* the transit post-scale: no scattering and no limb darkening give R0^2 + 2 I_p."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S

LAWS = [
    (1, [0.6, 0, 0, 0], lambda c: 1 - c[0] / 3),
    (2, [0.4, 0.25, 0, 0], lambda c: 1 - c[0] / 3 - c[1] / 6),
    (3, [0.3, 0.35, 0, 0], lambda c: 1 - c[0] / 3 - c[1] / 5),
    (4, [0.5, 0.2, 0, 0], lambda c: 1 - c[0] / 3 + 2 * c[1] / 9),
    (5, [0.7, 0.6, 0, 0], lambda c: 1 - c[0] * c[1] / (c[1] + 2)),
    (6, [0.5, -0.2, 0.4, -0.1], lambda c: 1 - sum(c[k - 1] * k / (k + 4) for k in range(1, 5))),
]


@pytest.mark.parametrize("law,coef,norm", LAWS)
def test_limb_darkening_laws(law, coef, norm):
    assert abs(O.limb(law, coef, 1.0) - 1.0) < 1e-15
    n = integrate.quad(lambda m: 2 * m * O.limb(law, coef, m), 0, 1, epsabs=1e-13, epsrel=1e-12)[0]
    assert abs(n - norm(coef)) < 1e-9
    assert O.limb(0, coef, 0.3) == 1.0


def _shell(wl):
    g = wl.grid
    alpha = float(np.float32(wl.opac.acld[0]))
    return g.R0, g.R_toa, alpha


def _mc(wl, col):
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = r["pk_f"][:, col]
    return f.mean(), f.std() / math.sqrt(len(f)), r


def test_chord_column_uniform_shell_no_ld():
    wl = S.uniform_scattering_sphere(omega=0.0, n_packets=400_000)
    R0, Rt, a = _shell(wl)
    tau = lambda b: 2 * a * math.sqrt(max(Rt * Rt - b * b, 0.0))  # noqa: E731
    ref = integrate.quad(lambda b: (b / Rt) * (1 - math.exp(-tau(b))), R0, Rt, epsrel=1e-12)[0] / (Rt - R0)
    est, sig, r = _mc(wl, 0)
    assert abs(est - ref) < 3 * sig, (est, ref, sig)
    assert np.all(r["pk_f"][:, 1] == 0.0)          # omega = 0: no scattered light


def _ring_mean_ld(b, law, coef, Rs, tx, ty):
    def I(psi):
        X, Y = tx + b * math.cos(psi), ty + b * math.sin(psi)
        q = (X * X + Y * Y) / (Rs * Rs)
        return O.limb(law, coef, math.sqrt(1 - q)) if q < 1 else 0.0
    # the ring crosses the stellar limb where t . (cos psi, sin psi) = (Rs^2 - b^2 - |t|^2) / (2 b):
    # integrate between those angles, where I has its kink and its square-root edge
    r, p0 = math.hypot(tx, ty), math.atan2(ty, tx)
    cuts = []
    if r > 0:
        k = (Rs * Rs - b * b - r * r) / (2 * b * r)
        if -1 < k < 1:
            a = math.acos(k)
            cuts = sorted((p0 + s * a) % (2 * math.pi) for s in (-1, 1))
    edges = [0.0] + cuts + [2 * math.pi]
    tot = sum(integrate.quad(I, lo, hi, epsrel=1e-10, limit=200)[0] for lo, hi in zip(edges, edges[1:]) if hi > lo)
    return tot / (2 * math.pi)


@pytest.mark.parametrize("where", ["central", "grazing"])
def test_chord_column_with_limb_darkening(where):
    Rs = 5.0 * S.R_JUP
    txy = (0.0, 0.0) if where == "central" else (0.3 * Rs, 0.75 * Rs)   # grazing: part of the ring is off the star
    law, coef = 2, [0.4, 0.25, 0.0, 0.0]
    wl = S.uniform_scattering_sphere(omega=0.0, n_packets=400_000, ld_law=law, ld_coef=coef, star_radius=Rs,
                                     transit_xy=txy)
    R0, Rt, a = _shell(wl)
    tau = lambda b: 2 * a * math.sqrt(max(Rt * Rt - b * b, 0.0))  # noqa: E731
    ref = integrate.quad(lambda b: (b / Rt) * (1 - math.exp(-tau(b))) * _ring_mean_ld(b, law, coef, Rs, *txy),
                         R0, Rt, epsrel=1e-7, limit=200)[0] / (Rt - R0)
    est, sig, r = _mc(wl, 0)
    assert abs(est - ref) < 3 * sig, (est, ref, sig)
    if where == "grazing":
        assert (r["pk_f"][:, 0] == 0).mean() > 0.01     # chords off the stellar disk carry nothing
        assert r["ledger"][0] < 0.99 * wl.jobs[0].n_packets


def test_scattered_column_first_order():
    omega, g = 1.0e-3, 0.5
    wl = S.uniform_scattering_sphere(omega=omega, g=g, n_packets=1_000_000)
    R0, Rt, a = _shell(wl)
    theta_fwd = (1 - g * g) / (1 - g) ** 3 / (4 * math.pi)
    tau = lambda b: 2 * a * math.sqrt(max(Rt * Rt - b * b, 0.0))  # noqa: E731
    ref = integrate.quad(lambda b: (b / Rt) * omega * theta_fwd * tau(b) * math.exp(-tau(b)), R0, Rt,
                         epsrel=1e-12)[0] / (Rt - R0)
    est, sig, r = _mc(wl, 1)
    # second and higher orders carry another factor omega (survival biasing) times a probability < 1
    assert abs(est - ref) < 3 * sig + omega * ref, (est, ref, sig)
    assert abs(est - ref) < 0.01 * ref


@pytest.mark.parametrize("survival", [1, 0])
def test_ledger_closes_transmission_scattering(survival):
    wl = S.uniform_scattering_sphere(omega=0.8, n_packets=20_000, survival=survival, ld_law=2,
                                     ld_coef=[0.4, 0.25], star_radius=5 * S.R_JUP, transit_xy=(0.0, 2 * S.R_JUP))
    L = O.run(wl, wl.jobs[0], nthreads=4)["ledger"]
    assert L[1] > 0 and L[2] > 0
    assert abs((L[0] + L[4]) - (L[1] + L[2] + L[3] + L[5] + L[6] + L[7])) <= 1e-12 * L[0]


@pytest.mark.parametrize("x", [0.1, 0.01])
def test_stellar_solid_angle_small_disk_series(x):
    """Omega_star of a stellar disk of angular radius asin(x), x = R_star / d, against its series
    pi x^2 (1 + x^2/4 + x^4/8): the first term is the disk area over d^2."""
    wl = S.uniform_scattering_sphere(n_packets=10, star_radius=x * 1.0e9, star_dist=1.0e9)
    r = O.run(wl, wl.jobs[0])
    om = O.transit(wl, r["tally"], 10)["omega_star"]
    ref = math.pi * x * x * (1 + x * x / 4 + x ** 4 / 8)
    assert abs(om / ref - 1) < 1e-7, (om, ref)


def test_opaque_small_planet_depth_with_limb_darkening():
    """An opaque atmosphere blocks the disk of radius R_TOA.  Small against the star (R_TOA = R_star/100),
    it hides the intensity at its centre, so the depth is (R_TOA/R_star)^2 I(mu_c)/n_LD, with
    mu_c = sqrt(1 - rho_c^2/R_star^2) at the planet's sky position rho_c and n_LD = 1 - c1/3 - c2/6 for
    the quadratic law (the variation of I across the planet enters at order (R_TOA/R_star)^2)."""
    c1, c2 = 0.4, 0.25
    wl = S.uniform_scattering_sphere(alpha=1e-3, omega=0.0, trans_scatter=0, n_packets=100_000, ld_law=2,
                                     ld_coef=(c1, c2, 0.0, 0.0))
    g = wl.grid
    Rs = 100.0 * g.R_toa
    wl.source.opts.star_radius = Rs
    wl.source.opts.transit_xy = (0.6 * Rs, 0.0)
    n = wl.jobs[0].n_packets
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    t = O.transit(wl, r["tally"], n)
    mu_c = math.sqrt(1 - 0.6 ** 2)
    ref = (g.R_toa / Rs) ** 2 * (1 - c1 * (1 - mu_c) - c2 * (1 - mu_c) ** 2) / (1 - c1 / 3 - c2 / 6)
    f = r["pk_f"][:, 0]
    sig = 2 * (g.R_toa - g.R0) * g.R_toa * f.std() / math.sqrt(n) / (Rs ** 2 * t["n_ld"])
    assert abs(t["depth"] - ref) < 3 * sig + 2e-4 * ref, (t["depth"], ref, sig)


def test_scattered_light_lowers_the_transit_area():
    """Light the atmosphere scatters towards the observer adds to the starlight seen through the limb,
    so with a stellar disk of non-zero solid angle the effective blocked area falls below the chords'."""
    wl = S.uniform_scattering_sphere(omega=0.9, g=0.8, n_packets=50_000, star_radius=S.R_SUN, star_dist=0.05 * S.AU)
    n = wl.jobs[0].n_packets
    r = O.run(wl, wl.jobs[0], nthreads=8)
    t = O.transit(wl, r["tally"], n)
    assert t["I_p_scattered"] > 0 and t["omega_star"] > 0
    assert t["area_over_pi"] < wl.grid.R0 ** 2 + 2 * t["I_p_direct"]


def test_transit_postscale_reduces_to_area():
    wl = S.uniform_scattering_sphere(omega=0.0, trans_scatter=0, n_packets=1000)
    r = O.run(wl, wl.jobs[0], nthreads=4)
    t = O.transit(wl, r["tally"], 1000)
    ref = O.postscale(wl, wl.jobs[0], r["tally"][0], 1000)
    assert t["I_p_scattered"] == 0.0 and t["w_core"] == 1.0 and t["n_ld"] == 1.0
    assert abs(t["area_over_pi"] / ref["area_over_pi"] - 1) < 1e-15
