"""Pins of the oracle's two-term Henyey-Greenstein clouds and Lambertian lower boundary (Sect. 3),
against closed forms and an independent plane-parallel solver:

* a Lambert sphere of albedo A_s with no atmosphere has geometric albedo A_g = (2/3) A_s and phase law
  Phi(alpha) = [sin alpha + (pi - alpha) cos alpha] / pi;
* the two-term HG function with the paper's defaults (g1 = g, g2 = -g/2, a = 1 - g2^2) is normalised,
  has mean cosine a g1 + (1 - a) g2, and its sampler follows its CDF (KS test);
* a homogeneous TTHG slab on a black sphere has the geometric albedo of the adding-doubling solver fed
  the TTHG Legendre moments beta_l = (2l + 1)(a g1^l + (1 - a) g2^l);
* through a purely absorbing layer over a white Lambert sphere the escaping fraction is (2 E3(tau))^2,
  which pins the cosine-weighted direction of the reflected light;
* the energy ledger closes with a reflecting surface (survival biasing and analog)."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import refsolvers as R
from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S


def _lambert_phase(alpha):
    return (math.sin(alpha) + (math.pi - alpha) * math.cos(alpha)) / math.pi


def test_lambert_sphere_albedo_and_phase_law():
    As = 0.6
    alphas = [0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4]
    obs = [[math.cos(a), math.sin(a), 0.0] for a in alphas]
    wl = S.slab_sphere_albedo(omega=1.0, tau=0.0, phase="iso", n_packets=400_000, surface_albedo=As, obs=obs)
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    for o, a in enumerate(alphas):
        f = math.pi * r["pk_f"][:, o]
        est, sig = f.mean(), f.std() / math.sqrt(len(f))
        ref = 2.0 / 3.0 * As * _lambert_phase(a)
        assert abs(est - ref) < 3 * sig + 1e-9, (a, est, ref, sig)


def _tthg_params(g):
    g2 = -0.5 * g
    return g, g2, 1.0 - g2 * g2


@pytest.mark.parametrize("g", [0.0, 0.3, 0.8])
def test_tthg_normalisation_and_mean_cosine(g):
    g1, g2, a = _tthg_params(g)
    norm = integrate.quad(lambda m: O.phase_tthg(m, g), -1, 1, epsabs=1e-12)[0] / 2
    mean = integrate.quad(lambda m: m * O.phase_tthg(m, g), -1, 1, epsabs=1e-12)[0] / 2
    assert abs(norm - 1) < 1e-8
    assert abs(mean - (a * g1 + (1 - a) * g2)) < 1e-8
    # the mixture of the expected phase function: Theta = (P_gas P_Ray + (1 - P_gas) P_TTHG) / (4 pi)
    for mu, pg in ((0.3, 0.25), (-0.7, 0.0)):
        ref = (pg * 0.75 * (1 + mu * mu) + (1 - pg) * O.phase_tthg(mu, g)) / (4 * math.pi)
        assert abs(O.theta_kind(mu, pg, g, 1) / ref - 1) < 1e-14


def test_tthg_sampler_follows_its_cdf():
    g = 0.6
    rng = np.random.default_rng(7)
    zc, z = rng.random(20000), rng.random(20000)
    mus = np.array([O.sample_cloud(g, a, b, 1) for a, b in zip(zc, z)])
    cdf = lambda m: integrate.quad(lambda t: O.phase_tthg(t, g), -1, m, epsabs=1e-12)[0] / 2  # noqa: E731
    grid = np.linspace(-1, 1, 401)
    table = np.array([cdf(m) for m in grid])
    p = stats.kstest(mus, lambda m: np.interp(m, grid, table)).pvalue
    assert p > 1e-3, p


@pytest.mark.parametrize("omega,tau", [(0.9, 2.0), (1.0, 1.0)])
def test_tthg_slab_matches_adding_doubling(omega, tau):
    g = 0.5
    g1, g2, a = _tthg_params(g)
    beta = [(2 * l + 1) * (a * g1 ** l + (1 - a) * g2 ** l) for l in range(48)]
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase="tthg", g=g, n_packets=150_000)
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = math.pi * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.AddingDoubling(beta, omega, tau, n=48).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-4 * ref, (est, ref, sig)


@pytest.mark.parametrize("tau", [0.2, 0.5])
def test_lambert_reflection_through_absorbing_layer(tau):
    """A purely absorbing thin layer of vertical depth tau over a white Lambert sphere: starlight over the
    disk reaches the surface with mean transmission 2 E3(tau) (incidence cosines have density 2 mu), and
    the cosine-weighted reflected light leaves with the same 2 E3(tau), so the escaping fraction of the
    incident power is (2 E3(tau))^2 (an isotropic reflection would give 2 E3(tau) E2(tau))."""
    from scipy.special import expn
    wl = S.slab_sphere_albedo(omega=0.0, tau=tau, phase="iso", n_packets=200_000, surface_albedo=1.0)
    L = O.run(wl, wl.jobs[0], nthreads=8)["ledger"]
    est = L[1] / L[0]
    sig = math.sqrt(est * (1 - est) / wl.jobs[0].n_packets)
    ref = (2 * expn(3, tau)) ** 2
    assert abs(est - ref) < 3 * sig + 1e-3 * ref, (est, ref, sig)


@pytest.mark.parametrize("survival", [1, 0])
def test_ledger_closes_with_surface(survival):
    wl = S.slab_sphere_albedo(omega=0.8, tau=1.0, phase="tthg", g=0.4, n_packets=20_000, survival=survival,
                              surface_albedo=0.5)
    L = O.run(wl, wl.jobs[0], nthreads=4)["ledger"]
    assert L[3] > 0 and L[1] > 0
    assert abs((L[0] + L[4]) - (L[1] + L[2] + L[3] + L[5] + L[6] + L[7])) <= 1e-12 * L[0]
