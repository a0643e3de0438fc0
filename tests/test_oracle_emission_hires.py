"""Pins of the oracle's emission on cross-section opacities (high resolution with Doppler shifts, Sect. 7):

* with no winds and no rotation the Doppler shift is zero and each cell's extinction is the table value
  at the job's wavelength, bilinear in (ln T, ln p) of ln sigma, exactly the k-table interpolation: the
  cell tables (alpha, L, cumulative pdf, launch weights) equal those of a one-g k-table built from the
  same sigma slice;
* an isothermal shell of constant sigma meets the closed form of the escaping emission;
* with winds the tables follow the Doppler-shifted extinction (a shifted line moves the luminosity)."""
import dataclasses
import math

import numpy as np

import refsolvers as R
from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S


def test_no_doppler_equals_ktable_slice():
    wl = S.config7_emission_hires(nlon=16, nlat=8, nr=12, n_lam=120, lam_subset=[40], n_lines=60, n_packets=1000)
    grid = dataclasses.replace(wl.grid, wind=None)
    xs = dataclasses.replace(wl.opac, omega_rot=0.0)
    job = wl.jobs[0]
    l = job.lam_idx
    kt = S.KTable(lam=np.array([xs.lam[l]]), wg=np.array([1.0]), gpts=np.array([0.5]), Tg=xs.Tg, pg=xs.pg,
                  k=np.ascontiguousarray(xs.sigma[l][None, None]).astype(np.float32))
    cx = O.prep_emission_xsec(grid, xs, l, wl.source.opts)
    ck = O.prep_emission(grid, kt, 0, 0, wl.source.opts)
    for k in ("alpha", "L", "cdf", "wcell"):
        np.testing.assert_allclose(cx[k], ck[k], rtol=1e-12, atol=0)
    assert abs(cx["L_tot"] / ck["L_tot"] - 1) < 1e-12 and cx["n_incl"] == ck["n_incl"]


def test_isothermal_constant_sigma_closed_form():
    tau, T, lam = 2.0, 1500.0, 1.05e-6
    ref_wl = S.isothermal_emitter(tau=tau, T=T, lam=lam, n_packets=400_000)
    H = ref_wl.grid.R_toa - ref_wl.grid.R0
    xs = S.XsecTable(lam=np.array([1.0e-6, lam, 1.1e-6]), Tg=np.array([500.0, 3000.0]), pg=np.array([1.0, 1.0e7]),
                     sigma=np.full((3, 2, 2), tau / H, np.float32), omega_rot=0.0)
    wl = dataclasses.replace(ref_wl, opac=xs, jobs=[S.Job(lam_idx=1, g_idx=0, n_packets=400_000, key=0)])
    cells = O.prep_cells(wl, wl.jobs[0])
    r = O.run(wl, wl.jobs[0], cells=cells, per_packet=True, nthreads=8)
    f = cells["L_tot"] * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    B = O.planck(lam, T)
    ref = R.emission_shell_Lp(B, tau, 0.5 * (wl.grid.R0 + wl.grid.R_toa))
    assert abs(est - ref) < 3 * sig + 2e-4 * ref, (est, ref, sig)


def test_winds_shift_the_extinction():
    wl = S.config7_emission_hires(nlon=16, nlat=8, nr=12, n_lam=120, lam_subset=[40], n_lines=60, n_packets=1000)
    still = dataclasses.replace(wl.opac, omega_rot=0.0)
    c_w = O.prep_emission_xsec(wl.grid, wl.opac, wl.jobs[0].lam_idx, wl.source.opts)
    c_0 = O.prep_emission_xsec(dataclasses.replace(wl.grid, wind=None), still, wl.jobs[0].lam_idx, wl.source.opts)
    # the extinction is each cell's table value at its own shifted wavelength
    a_w = O.prep_xsec(wl.grid, wl.opac, wl.jobs[0].lam_idx)["alpha"]
    np.testing.assert_array_equal(c_w["alpha"], a_w)
    assert np.max(np.abs(c_w["alpha"] / c_0["alpha"] - 1)) > 1e-3
