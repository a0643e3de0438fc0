"""Pins of the oracle's forced scattering (Sect. 4.2: on the first flight, or on every flight) and
continuous absorption (Sect. 4.1):

* both leave the expectation unchanged: a homogeneous slab's geometric albedo with either or both
  options meets the adding-doubling value within 3 sigma (Rayleigh and isotropic, thin and thick);
* forced first scattering lowers the variance of an optically thin slab (every packet scatters);
* continuous absorption at omega = 1 is survival biasing exactly: the same packets, steps and f;
* transmission with multiple scattering: the scattered column is unchanged by forcing (3 sigma), and a
  reflecting surface, where the first flight is not forced, still gives the unforced expectation;
* the energy ledger closes under both options, with survival biasing and analog scattering."""
import math

import numpy as np
import pytest

import refsolvers as R
from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S


def _ag(wl):
    r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    f = math.pi * r["pk_f"][:, 0]
    return f.mean(), f.std() / math.sqrt(len(f)), r


@pytest.mark.parametrize("ff,ca", [(1, 0), (0, 1), (1, 1), (2, 0), (2, 1)])
@pytest.mark.parametrize("phase,beta,omega,tau", [("rayleigh", [1.0, 0.0, 0.5], 0.6, 0.3),
                                                  ("iso", [1.0], 0.9, 2.0)])
def test_slab_albedo_unchanged(ff, ca, phase, beta, omega, tau):
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase=phase, n_packets=200_000, forced_first=ff, cont_abs=ca)
    est, sig, _ = _ag(wl)
    ref = R.AddingDoubling(beta, omega, tau, n=40).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-4 * ref, (est, ref, sig)


def test_forcing_lowers_variance_of_thin_slab():
    kw = dict(omega=0.6, tau=0.1, phase="rayleigh", n_packets=100_000)
    _, s0, _ = _ag(S.slab_sphere_albedo(**kw))
    _, s1, _ = _ag(S.slab_sphere_albedo(forced_first=1, **kw))
    assert s1 < 0.4 * s0, (s1, s0)


def test_forcing_every_flight_lowers_variance_further():
    kw = dict(omega=0.95, tau=0.2, phase="iso", n_packets=100_000)
    _, s1, _ = _ag(S.slab_sphere_albedo(forced_first=1, **kw))
    _, s2, r = _ag(S.slab_sphere_albedo(forced_first=2, **kw))
    assert s2 < s1, (s2, s1)
    L = r["ledger"]
    assert L[1] > 0 and abs((L[0] + L[4]) - (L[1] + L[2] + L[3] + L[5] + L[6] + L[7])) <= 1e-12 * L[0]


def test_continuous_absorption_at_omega_one_is_survival_biasing():
    kw = dict(omega=1.0, tau=2.0, phase="rayleigh", n_packets=20_000)
    a = O.run(*(lambda w: (w, w.jobs[0]))(S.slab_sphere_albedo(**kw)), per_packet=True, nthreads=4)
    b = O.run(*(lambda w: (w, w.jobs[0]))(S.slab_sphere_albedo(cont_abs=1, **kw)), per_packet=True, nthreads=4)
    np.testing.assert_array_equal(a["pk_steps"], b["pk_steps"])
    np.testing.assert_allclose(b["pk_f"], a["pk_f"], rtol=1e-13, atol=0)


def test_transmission_scattered_column_unchanged_by_forcing():
    res = []
    for ff in (0, 1):
        wl = S.uniform_scattering_sphere(omega=0.5, g=0.5, n_packets=400_000)
        wl.source.opts.forced_first = ff
        r = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
        f = r["pk_f"][:, 1]
        res.append((f.mean(), f.var() / len(f)))
    (m0, v0), (m1, v1) = res
    assert abs(m1 - m0) < 3 * math.sqrt(v0 + v1), (m0, m1)


def test_reflecting_surface_with_forcing():
    res = []
    for ff in (0, 1):
        wl = S.slab_sphere_albedo(omega=0.8, tau=0.5, phase="rayleigh", n_packets=300_000, surface_albedo=0.4,
                                  forced_first=ff)
        est, sig, _ = _ag(wl)
        res.append((est, sig))
    (m0, s0), (m1, s1) = res
    assert abs(m1 - m0) < 3 * math.hypot(s0, s1), (m0, m1)


@pytest.mark.parametrize("survival", [1, 0])
def test_ledger_closes(survival):
    for wl in (S.slab_sphere_albedo(omega=0.7, tau=1.0, phase="hg", g=0.5, n_packets=20_000, survival=survival,
                                    forced_first=1, cont_abs=1, surface_albedo=0.3),
               S.uniform_scattering_sphere(omega=0.7, n_packets=20_000, survival=survival)):
        wl.source.opts.forced_first = 1
        wl.source.opts.cont_abs = 1
        L = O.run(wl, wl.jobs[0], nthreads=4)["ledger"]
        assert abs((L[0] + L[4]) - (L[1] + L[2] + L[3] + L[5] + L[6] + L[7])) <= 1e-12 * L[0]


@pytest.mark.parametrize("ff,pb", [(1, 1), (1, 2), (2, 1), (2, 2)])
@pytest.mark.parametrize("phase,beta,omega,tau", [("rayleigh", [1.0, 0.0, 0.5], 0.6, 0.3),
                                                  ("iso", [1.0], 0.9, 3.0)])
def test_slab_albedo_unchanged_by_path_biasing(ff, pb, phase, beta, omega, tau):
    """Path length stretching (composite of the natural and the stretched exponential) and the hybrid
    (forced, composite of the truncated exponential and the uniform in tau) leave the albedo unchanged."""
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase=phase, n_packets=200_000, forced_first=ff, path_bias=pb)
    est, sig, _ = _ag(wl)
    ref = R.AddingDoubling(beta, omega, tau, n=40).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-4 * ref, (est, ref, sig)


def test_hybrid_lowers_variance_of_thin_slab():
    kw = dict(omega=0.6, tau=0.1, phase="rayleigh", n_packets=100_000)
    _, s0, _ = _ag(S.slab_sphere_albedo(**kw))
    _, s2, _ = _ag(S.slab_sphere_albedo(forced_first=1, path_bias=2, **kw))
    assert s2 < 0.5 * s0, (s2, s0)


@pytest.mark.parametrize("pb", [1, 2])
@pytest.mark.parametrize("survival", [1, 0])
def test_ledger_closes_with_path_biasing(pb, survival):
    """The p/q reweights of biased flights are booked with the roulette's gain and loss."""
    wl = S.slab_sphere_albedo(omega=0.9, tau=3.0, phase="rayleigh", n_packets=20_000, forced_first=2, path_bias=pb,
                              survival=survival, cont_abs=1)
    L = O.run(wl, wl.jobs[0], nthreads=4)["ledger"]
    assert L[4] > 0 and L[5] > 0
    assert abs((L[0] + L[4]) - (L[1] + L[2] + L[3] + L[5] + L[6] + L[7])) <= 1e-12 * (L[0] + L[4])
