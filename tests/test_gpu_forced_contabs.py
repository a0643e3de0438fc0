"""Forced scattering (first flight or every flight) and continuous absorption (Sect. 4.1, 4.2) on the GPU,
against the FP64 oracle:

* FP64 path: per-packet parity (cell sequences, steps, f, ledger) on the cloudy 3D atmosphere over a
  reflecting surface (first flights that end on it are not forced) and on the cloudy atmosphere in
  transit with multiple scattering; survival biasing and analog;
* FP32 path: the same packets within the FP32 bars of the other tests;
* a slab's geometric albedo with both options against adding-doubling (FP64 path)."""
import dataclasses
import math

import numpy as np
import pytest

import refsolvers as R
from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2110_15640_gb300 import build, gcmc
    build.build()
    ctx = gcmc.Context(0)
    yield ctx
    ctx.close()


def cloudy(n, survival=1, transit=False, ff=1, pb=0):
    """The phase-curve atmosphere on a 12x6x10 grid, gas absorption cut 1000x and Rayleigh 10x, two-term HG
    clouds, forced first scattering and continuous absorption; either over a Lambertian surface (A_s =
    0.5, four phase observers) or seen in transit with multiple scattering."""
    wl = S.config3_phase_curve(nlon=12, nlat=6, nr=10, nlam=2, nphase=4, n_lo=n, n_hi=n)
    opac = dataclasses.replace(wl.opac, kabs=wl.opac.kabs * 1e-3, kray=wl.opac.kray * 0.1)
    opts = dataclasses.replace(wl.source.opts, cloud_phase=1, survival=survival, forced_first=ff, cont_abs=1,
                               path_bias=pb)
    if transit:
        opts = dataclasses.replace(opts, trans_scatter=1)
        src = S.Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]), opts=opts)
        return dataclasses.replace(wl, name="forced_transit", mode=S.MODE_TRANSMISSION, opac=opac, source=src,
                                   jobs=[S.Job(lam_idx=1, g_idx=0, n_packets=n, key=9)])
    opts = dataclasses.replace(opts, surface_albedo=0.5)
    return dataclasses.replace(wl, name="forced_surface", opac=opac, source=dataclasses.replace(wl.source, opts=opts),
                               jobs=[S.Job(lam_idx=1, g_idx=0, n_packets=n, key=77)])


def _load(ctx, wl, prec):
    from paper_2110_15640_gb300 import gcmc
    return gcmc.load_workload(ctx, wl, prec)


@pytest.mark.parametrize("transit,survival,ff,pb", [(False, 1, 1, 0), (False, 0, 1, 0), (True, 1, 1, 0), (True, 0, 1, 0),
                                                    (False, 1, 2, 0), (True, 0, 2, 0), (False, 1, 1, 1), (True, 0, 2, 1),
                                                    (False, 0, 2, 2), (True, 1, 1, 2)])
def test_fp64_per_packet_parity(G, survival, transit, ff, pb):
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy(3000, survival, transit, ff, pb)
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    ncol = O.tally_cols(wl, job)
    ntr, mtr = 300, 8000
    ref = O.run(wl, job, per_packet=True, n_trace=ntr, max_trace=mtr, nthreads=8)
    got = G.run_debug(jobs[0], n_trace=ntr, max_trace=mtr, n_obs=ncol)
    same = 0
    for q in range(ntr):
        no, ng = ref["tr_n"][q], got["tr_n"][q]
        if no == ng and np.array_equal(ref["tr_cell"][q, :no], got["tr_cell"][q, :ng]):
            lo, lg = ref["tr_len"][q, :no], got["tr_len"][q, :ng]
            # every-flight forcing keeps packets scattering for hundreds of events: the two sides' FP64
            # positions drift apart by ~1e-13 relative (~1e-5 m), negligible against 1e5 m cells
            same += int(np.all(np.abs(lo - lg) <= 1e-9 * np.abs(lo) + 1e-5))
    assert same >= ntr - 1, f"{same}/{ntr} identical traces"
    np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
    # f carries e^-tau of its peel-off and, with continuous absorption, e^-tau_abs of every flight before
    # it: the march's FP64 rounding of those depths enters as tau times itself, so contributions far
    # below the largest are compared against it (1e-14 of the largest), the rest to 1e-10
    f_o = ref["pk_f"]
    np.testing.assert_allclose(got["pk_f"], f_o, rtol=1e-10, atol=1e-14 * f_o.max())
    st = got["stats"]
    assert st.steps == ref["steps"]
    np.testing.assert_allclose(list(st.ledger), ref["ledger"], rtol=1e-12, atol=64 * job.n_packets * 2.0 ** -33)
    L = ref["ledger"]
    assert L[2] > 0 and abs((L[0] + L[4]) - (L[1] + L[2] + L[3] + L[5] + L[6] + L[7])) <= 1e-12 * L[0]


@pytest.mark.parametrize("transit,ff,pb", [(False, 1, 0), (True, 1, 0), (False, 2, 0), (False, 2, 1), (True, 1, 2)])
def test_fp32_matches_oracle(G, transit, ff, pb):
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy(20000, 1, transit, ff, pb)
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    ncol = O.tally_cols(wl, job)
    ref = O.run(wl, job, per_packet=True, nthreads=8)
    got = G.run_debug(jobs[0], n_obs=ncol)
    # every forced packet scatters, so most peel off through deep slant paths; their FP32 error is
    # tau times the FP32 rounding of tau, and they are compared against the largest contribution
    f_o = ref["pk_f"]
    close = np.abs(got["pk_f"] - f_o) <= 1e-3 * np.abs(f_o) + 1e-6 * f_o.max()
    trel = np.abs(got["tally"][:ncol] / ref["tally"] - 1)
    print(f"FP32 forced + continuous absorption ({'transit' if transit else 'surface'}): close {close.mean():.5f};"
          f" tally rel {trel}")
    assert close.mean() >= 0.99
    assert np.all(trel < 1e-4)


def test_fp64_slab_with_both_options_vs_adding_doubling(G):
    from paper_2110_15640_gb300 import gcmc
    wl = S.slab_sphere_albedo(omega=0.6, tau=0.3, phase="rayleigh", n_packets=400_000, forced_first=1, cont_abs=1)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    got = G.run_debug(jobs[0])
    f = math.pi * got["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.AddingDoubling([1.0, 0.0, 0.5], 0.6, 0.3, n=40).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-5 * ref, (est, ref, sig)


@pytest.mark.parametrize("transit", [False, True])
def test_kernel_variants_equal_bitwise(G, transit):
    """The kernel built with continuous absorption, in its variant for 5 resident blocks per SM, gives the
    uncapped variant's tallies bit for bit (the same code; only the register budget differs)."""
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy(20000, transit=transit, ff=2, pb=2)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    out = {}
    for shape in ((128, 5), (128, 0), (256, 0)):
        tv, sv = G.run_batch(jobs, cfg=gcmc.gcmc_launch_cfg(shape[0], shape[1], 512, 16, 8, 0))
        out[shape] = (tv[0].copy(), sv[0].steps, list(sv[0].ledger))
    ref = out[(128, 0)]
    for shape, v in out.items():
        assert np.array_equal(v[0], ref[0]) and v[1] == ref[1] and v[2] == ref[2], shape
