"""Pins of the oracle's host post-scale (S9, Sect. 5) against facts that do not go through its formulas:

* albedo: a Lambert sphere of albedo A_s under a transparent shell as thick as its radius has the
  geometric albedo (2/3) A_s referenced to the sphere, and a quarter of that referenced to the top of
  the shell (the incident flux is normalised over the disk of radius R_TOA, Sect. 5.2);
* emission: an optically thick isothermal shell radiates as a black body, so the disk-averaged
  intensity I_p is B_lambda(T) and the flux F_p is pi B_lambda(T) (Sect. 5.3);
* transmission: an opaque atmosphere blocks the whole disk of radius R_TOA, and a uniform absorber
  blocks R0^2 plus the closed-form chord integral (Sect. 5.1).

The post-scale is linear in the tally sum, so the Monte Carlo sigma of each observable is the sigma of
the tally sum times the post-scale's own slope."""
import math

import numpy as np

import refsolvers as R
from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S


def _estimate(wl, key, col=0, nthreads=8, cells=None):
    job = wl.jobs[0]
    cells = O.prep_cells(wl, job) if cells is None else cells
    r = O.run(wl, job, cells=cells, per_packet=True, nthreads=nthreads)
    n = job.n_packets
    f = r["pk_f"][:, col]
    got = O.postscale(wl, job, r["tally"][col], n, cells=cells)[key]
    slope = O.postscale(wl, job, 1.0, n, cells=cells)[key] - O.postscale(wl, job, 0.0, n, cells=cells)[key]
    sig = abs(slope) * f.std() * math.sqrt(n)
    return float(np.asarray(got).reshape(-1)[0]), float(sig), r


def test_albedo_lambert_sphere_under_transparent_shell():
    As = 0.8
    wl = S.slab_sphere_albedo(omega=1.0, tau=0.0, phase="iso", thin=1.0, n_packets=400_000, surface_albedo=As)
    g = wl.grid
    assert abs(g.R_toa / g.R0 - 2.0) < 1e-12
    a_r0, s_r0, _ = _estimate(wl, "A_g_R0")
    a_toa, s_toa, _ = _estimate(wl, "A_g_toa")
    assert abs(a_r0 - 2.0 / 3.0 * As) < 3 * s_r0, (a_r0, s_r0)
    assert abs(a_toa - 2.0 / 3.0 * As / 4.0) < 3 * s_toa, (a_toa, s_toa)


def test_emission_thick_isothermal_shell_is_a_black_body():
    T, lam, tau = 1500.0, 2.0e-6, 8.0
    wl = S.isothermal_emitter(tau=tau, T=T, lam=lam, n_packets=200_000)
    B = O.planck(lam, T)
    # limb-to-centre: the thin shell's mean radius and its residual transparency 2 E3(tau) shift I_p by
    # about 1e-4 relative, far below the Monte Carlo error
    ip, sig, _ = _estimate(wl, "I_p")
    assert abs(ip - B) < 3 * sig + 2e-4 * B, (ip / B, sig / B)
    fp, sfp, _ = _estimate(wl, "F_p")
    assert abs(fp - math.pi * B) < 3 * sfp + 2e-4 * math.pi * B, (fp / (math.pi * B), sfp)


def test_transmission_opaque_atmosphere_blocks_the_toa_disk():
    # alpha = 1e-3 per metre: a chord has tau ~ 1e3 or more (tens within metres of the top), so 1 - e^-tau
    # is 1 to 1e-12 for every chord
    wl = S.uniform_absorber_sphere(alpha=1.0e-3, n_packets=50_000)
    g = wl.grid
    area, sig, r = _estimate(wl, "area_over_pi")
    assert np.all(np.exp(-r["pk_tau"]) < 1e-12)
    assert abs(area - g.R_toa ** 2) < 3 * sig + 1e-12 * g.R_toa ** 2, (area / g.R_toa ** 2, sig)


def test_transmission_uniform_absorber_area():
    wl = S.uniform_absorber_sphere(n_packets=200_000)
    g = wl.grid
    area, sig, _ = _estimate(wl, "area_over_pi")
    alpha = float(np.float32(2.0e-6))     # the table stores the uniform cross-section in FP32
    ref = g.R0 ** 2 + R.transmission_integral_uniform(alpha, g.R0, g.R_toa)
    assert abs(area - ref) < 3 * sig, ((area - ref) / sig)
