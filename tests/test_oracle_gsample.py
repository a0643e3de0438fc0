"""Pins of the oracle's per-packet g-ordinate sampling in emission (Sect. 4.7):

* the g table: q sums to 1, sum_g q W = sum_g p = 1, uniform q = 1/N_g, composite q >= beta/N_g
  (so an 8 + 8 split quadrature's low-weight high-g block keeps at least beta/2 of the packets);
* an isothermal shell whose band has three g-ordinates of different opacity: the band job's L_p
  equals sum_g w_g times the closed form at each tau_g, for every bias (unbiased, uniform, composite);
* on a 3D hot-Jupiter grid with an 8 + 8 split k-table, the band job agrees with the sum over g of
  w_g times the per-g (stratified) jobs."""
import math

import numpy as np
import pytest

import refsolvers as R
from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S


@pytest.mark.parametrize("bias", [0, 1, 2])
def test_g_table_identities(bias):
    kt = S.make_ktable(np.random.default_rng(3), nb=1, split=(8, 8, 0.9))
    L = np.random.default_rng(4).uniform(0.1, 10.0, 16)
    gt = O.g_table(kt.wg, L, bias, 0.5)
    assert abs(gt["q"].sum() - 1) < 1e-14 and abs(gt["qcdf"][-1] - 1) < 1e-14
    assert abs(np.sum(gt["q"] * gt["W"]) - 1) < 1e-14
    p = kt.wg * L / np.sum(kt.wg * L)
    np.testing.assert_allclose(gt["p"], p, rtol=1e-14)
    if bias == 1:
        np.testing.assert_allclose(gt["q"], 1 / 16, rtol=1e-15)
    if bias == 2:
        assert np.all(gt["q"] >= 0.5 / 16 * (1 - 1e-15))
        assert gt["q"][8:].sum() >= 0.25 - 1e-15
    assert abs(gt["L_band"] - np.sum(kt.wg * L)) < 1e-12 * gt["L_band"]


@pytest.mark.parametrize("bias", [0, 1, 2])
def test_isothermal_band_matches_weighted_closed_form(bias):
    taus, wg = [0.1, 1.0, 5.0], [0.5, 0.3, 0.2]
    wl = S.isothermal_emitter(taus=taus, wg=wg, n_packets=600_000, g_bias=bias)
    job = wl.jobs[0]
    cells = O.prep_cells(wl, job)
    r = O.run(wl, job, cells=cells, per_packet=True, nthreads=8)
    f = cells["L_tot"] * r["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    B = O.planck(wl.opac.lam[0], float(wl.grid.T[0]))
    Rm = 0.5 * (wl.grid.R0 + wl.grid.R_toa)
    ref = sum(w * R.emission_shell_Lp(B, t, Rm) for w, t in zip(wg, taus))
    assert abs(est - ref) < 3 * sig + 2e-4 * ref, (est, ref, sig)


@pytest.mark.parametrize("bias", [0, 2])
def test_band_job_matches_sum_over_g_jobs(bias):
    kw = dict(nlon=16, nlat=8, nr=12, nb=2, bands=[1], split=(4, 4, 0.9))
    wb = S.config2_emission(n_packets=400_000, per_packet_g=True, g_bias=bias, **kw)
    wg = S.config2_emission(n_packets=100_000, **kw)
    band = wb.jobs[0]
    cb = O.prep_cells(wb, band)
    rb = O.run(wb, band, cells=cb, per_packet=True, nthreads=8)
    fb = cb["L_tot"] * rb["pk_f"][:, 0]
    est, var = fb.mean(), fb.var() / len(fb)
    ref = 0.0
    for job in wg.jobs:
        c = O.prep_cells(wg, job)
        r = O.run(wg, job, cells=c, per_packet=True, nthreads=8)
        f = c["L_tot"] * r["pk_f"][:, 0]
        w = wg.opac.wg[job.g_idx]
        ref += w * f.mean()
        var += w * w * f.var() / len(f)
    assert abs(est - ref) < 3 * math.sqrt(var), (est, ref, math.sqrt(var))
