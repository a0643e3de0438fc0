"""Transmission with multiple scattering and stellar limb darkening (Sect. 5.1) on the GPU, against
the FP64 oracle:

* FP64 path: per-packet parity (identical cell sequences, steps, both tally columns) on the cloudy
  phase-curve atmosphere seen in transit (two-term HG clouds, a reflecting surface), with quadratic
  limb darkening on a grazing transit where some chords miss the stellar disk; survival and analog;
* FP32 path: the same packets within the FP32 bars of the other tests; the scattered column's
  first-order closed form on a uniform shell;
* the host transit post-scale against the oracle's, for every limb-darkening law;
* argument checks."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S

pytestmark = pytest.mark.gpu

R_STAR = 7.0e8


@pytest.fixture(scope="module")
def G():
    from paper_2110_15640_gb300 import build, gcmc
    build.build()
    ctx = gcmc.Context(0)
    yield ctx
    ctx.close()


def cloudy_transit(n, survival=1, ld_law=2, As=0.3):
    """The phase-curve atmosphere (Rayleigh gas + cloud deck) on a 12x6x10 grid in transit geometry:
    star +x, observer -x, multiple scattering, TTHG clouds, a Lambertian surface, quadratic limb
    darkening on a grazing transit (planet centre at 0.95 R_star: part of the annulus is off the disk)."""
    wl = S.config3_phase_curve(nlon=12, nlat=6, nr=10, nlam=2, nphase=1, n_lo=n, n_hi=n)
    opts = dataclasses.replace(wl.source.opts, survival=survival, trans_scatter=1, cloud_phase=1, surface_albedo=As,
                               ld_law=ld_law, ld_coef=(0.4, 0.25, 0.0, 0.0), star_radius=R_STAR, star_dist=10 * R_STAR,
                               transit_xy=(0.0, 0.95 * R_STAR))
    src = S.Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]), opts=opts)
    return dataclasses.replace(wl, name="cloudy_transit", mode=S.MODE_TRANSMISSION, source=src,
                               jobs=[S.Job(lam_idx=1, g_idx=0, n_packets=n, key=5)])


def _load(ctx, wl, prec):
    from paper_2110_15640_gb300 import gcmc
    return gcmc.load_workload(ctx, wl, prec)


@pytest.mark.parametrize("survival", [1, 0])
def test_fp64_per_packet_parity_transit(G, survival):
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy_transit(3000, survival=survival)
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    ntr, mtr = 300, 6000
    ref = O.run(wl, job, per_packet=True, n_trace=ntr, max_trace=mtr, nthreads=8)
    f_o = ref["pk_f"]
    assert f_o.shape[1] == 2 and (f_o[:, 1] > 0).sum() > 100 and (f_o[:, 0] == 0).sum() > 100
    got = G.run_debug(jobs[0], n_trace=ntr, max_trace=mtr, n_obs=2)
    same = 0
    for q in range(ntr):
        no, ng = ref["tr_n"][q], got["tr_n"][q]
        if no == ng and np.array_equal(ref["tr_cell"][q, :no], got["tr_cell"][q, :ng]):
            lo, lg = ref["tr_len"][q, :no], got["tr_len"][q, :ng]
            same += int(np.all(np.abs(lo - lg) <= 1e-9 * np.abs(lo) + 1e-9))
    assert same >= ntr - 1, f"{same}/{ntr} identical traces"
    np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
    # a peel-off through optical depth tau carries the march's rounding of tau as the relative error
    # tau dtau of e^-tau: slant paths at the limb reach tau ~ 45 (f ~ 1e-20), so below 1e-12 of the
    # largest value the bar is 1e-8
    big = f_o >= 1e-12 * f_o.max()
    np.testing.assert_allclose(got["pk_f"][big], f_o[big], rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(got["pk_f"], f_o, rtol=1e-8, atol=1e-300)
    np.testing.assert_allclose(got["tally"][:2], ref["tally"], rtol=1e-12, atol=job.n_packets * 2.0 ** -33)
    st = got["stats"]
    assert st.steps == ref["steps"]
    np.testing.assert_allclose(list(st.ledger), ref["ledger"], rtol=1e-12, atol=64 * job.n_packets * 2.0 ** -33)


def test_fp32_transit_matches_oracle(G):
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy_transit(20000)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    ref = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
    got = G.run_debug(jobs[0], n_obs=2)
    close = np.abs(got["pk_f"] - ref["pk_f"]) <= 1e-3 * np.abs(ref["pk_f"]) + 1e-300
    trel = np.abs(got["tally"][:2] / ref["tally"] - 1)
    print(f"FP32 transit: close {close.mean():.5f}; tally rel {trel}")
    assert close.mean() >= 0.99
    assert np.all(trel < 1e-4)


def test_fp32_scattered_column_first_order(G):
    """Uniform thick shell, omega = 1e-3, HG g = 0.5: the scattered column against its first-order
    closed form omega Theta(0) tau e^-tau (b / R_t), averaged over b in [R0, R_t]."""
    from paper_2110_15640_gb300 import gcmc
    omega, g = 1.0e-3, 0.5
    wl = S.uniform_scattering_sphere(omega=omega, g=g, n_packets=4_000_000)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    t, st = G.run_packets(jobs[0])
    R0, Rt = wl.grid.R0, wl.grid.R_toa
    a = float(np.float32(wl.opac.acld[0]))
    theta_fwd = (1 - g * g) / (1 - g) ** 3 / (4 * math.pi)
    tau = lambda b: 2 * a * math.sqrt(max(Rt * Rt - b * b, 0.0))  # noqa: E731
    ref1 = integrate.quad(lambda b: (b / Rt) * omega * theta_fwd * tau(b) * math.exp(-tau(b)), R0, Rt,
                          epsrel=1e-12)[0] / (Rt - R0)
    ref0 = integrate.quad(lambda b: (b / Rt) * (1 - math.exp(-tau(b))), R0, Rt, epsrel=1e-12)[0] / (Rt - R0)
    N = jobs[0].n_packets
    # per-packet spread measured on the oracle's smaller run of the same workload
    r = O.run(wl, wl.jobs[0], n_run=200_000, per_packet=True, nthreads=8)
    s1 = r["pk_f"][:, 1].std() / math.sqrt(N)
    s0 = r["pk_f"][:, 0].std() / math.sqrt(N)
    assert abs(t[1] / N - ref1) < 3 * s1 + omega * ref1, (t[1] / N, ref1, s1)
    assert abs(t[0] / N - ref0) < 3 * s0, (t[0] / N, ref0, s0)


@pytest.mark.parametrize("law,coef", [(0, [0, 0, 0, 0]), (1, [0.6, 0, 0, 0]), (2, [0.4, 0.25, 0, 0]),
                                      (3, [0.3, 0.35, 0, 0]), (4, [0.5, 0.2, 0, 0]), (5, [0.7, 0.6, 0, 0]),
                                      (6, [0.5, -0.2, 0.4, -0.1]), (2, [1.2, 0.5, 0, 0])])
def test_transit_postscale_matches_oracle(G, law, coef):
    wl = cloudy_transit(1000)
    wl.source.opts = dataclasses.replace(wl.source.opts, ld_law=law, ld_coef=tuple(coef))
    gid = G.upload_grid(wl.grid)
    sid = G.set_source(gid, wl.source)
    tally = np.array([123.456, 7.89])
    got = G.transit(gid, sid, tally, 1000)
    ref = O.transit(wl, tally, 1000)
    ref["area"] = ref["area_over_pi"]
    for k in ("I_p_direct", "I_p_scattered", "omega_star", "I_p", "w_core", "area", "depth"):
        assert abs(got[k] - ref[k]) <= 1e-9 * abs(ref[k]) + 1e-300, (k, got[k], ref[k])
    # a law that goes negative near the limb (the last case) is integrated numerically
    assert abs(got["n_ld"] - ref["n_ld"]) < 1e-8


def test_transit_argument_checks(G):
    from paper_2110_15640_gb300 import gcmc
    wl = S.uniform_absorber_sphere(n_packets=100)
    wl.source.opts = dataclasses.replace(wl.source.opts, trans_scatter=1)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    with pytest.raises(gcmc.GcmcError):        # multiple scattering needs scattering opacities
        G.run_packets(jobs[0])
    for bad in (dict(ld_law=2, star_radius=0.0), dict(ld_law=9, star_radius=1.0),
                dict(star_radius=2.0, star_dist=1.0)):
        src = dataclasses.replace(wl.source, opts=dataclasses.replace(wl.source.opts, **bad))
        with pytest.raises(gcmc.GcmcError):
            G.set_source(gid, src)


def test_debug_output_columns(G):
    """A transit job with multiple scattering tallies two columns: the library reports them, the
    per-packet form fills that many by default, and a one-column pk_f is refused before any work."""
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy_transit(500)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    assert G.job_columns(jobs[0]) == 2
    got = G.run_debug(jobs[0])
    assert got["pk_f"].shape == (500, 2)
    wide = G.run_debug(jobs[0], n_obs=5)
    np.testing.assert_array_equal(wide["pk_f"][:, :2], got["pk_f"])
    assert not wide["pk_f"][:, 2:].any()
    with pytest.raises(gcmc.GcmcError) as e:
        G.run_debug(jobs[0], n_obs=1)
    assert e.value.status == gcmc.ERR_ARG
    G.run_packets(jobs[0])   # the context is still usable


def test_transit_kernel_variants_equal_bitwise(G):
    """The optional-physics scattering kernel (multiple scattering, TTHG clouds, a surface, limb darkening)
    in its variant for 5 resident blocks per SM gives the uncapped variant's tallies bit for bit (the
    same code; only the register budget differs), and both agree with the plain form, which runs the
    kernel compiled with every optional feature (other code, so other roundings), to the FP32 tally bar."""
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy_transit(20000)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    tp, sp = G.run_packets(jobs[0])
    out = {}
    for shape in ((128, 5), (128, 0), (256, 0)):
        tv, sv = G.run_batch(jobs, cfg=gcmc.gcmc_launch_cfg(shape[0], shape[1], 512, 16, 8, 0))
        out[shape] = (tv[0][:2].copy(), sv[0].steps)
    rel = {k: np.abs(v[0] / tp[:2] - 1) for k, v in out.items()}
    print("plain", tp[:2], sp.steps, {k: (v[0], v[1], rel[k]) for k, v in out.items()})
    assert np.array_equal(out[(128, 5)][0], out[(128, 0)][0]) and out[(128, 5)][1] == out[(128, 0)][1]
    assert np.array_equal(out[(256, 0)][0], out[(128, 0)][0])
    for k in out:
        assert np.all(rel[k] < 1e-4), (k, rel[k])
