"""Two-term HG clouds and a Lambertian lower boundary (Sect. 3) on the GPU, against the FP64 oracle.

* FP64 path: per-packet parity (identical cell sequences, steps, peel-off sums) on a 3D cloudy
  grid thin enough that a sixth of the weight reaches the reflecting surface, with observers on
  both sides of the terminator (surface peel-offs skip observers below the local horizon);
  survival biasing and analog.
* FP32 path: the same packets within the FP32 bars of the other albedo tests; the Lambert sphere's
  closed forms (A_g = 2/3 A_s, phase law); ledger closure with a surface.
* A homogeneous TTHG slab against adding-doubling with the TTHG Legendre moments (FP64 path)."""
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


def cloudy_surface(n, survival=1, As=0.5):
    """The phase-curve atmosphere (Rayleigh gas + cloud deck, omega 0.9, g 0.6) on a 12x6x10 grid with
    the gas absorption cut 1000x and Rayleigh 10x, TTHG clouds, a Lambertian surface of albedo As,
    one job peeling off towards all four phase observers (0, 90, 180, 270 deg)."""
    wl = S.config3_phase_curve(nlon=12, nlat=6, nr=10, nlam=2, nphase=4, n_lo=n, n_hi=n)
    opac = dataclasses.replace(wl.opac, kabs=wl.opac.kabs * 1e-3, kray=wl.opac.kray * 0.1)
    opts = dataclasses.replace(wl.source.opts, cloud_phase=1, surface_albedo=As, survival=survival)
    return dataclasses.replace(wl, name=f"cloudy_surface_As{As}", opac=opac,
                               source=dataclasses.replace(wl.source, opts=opts),
                               jobs=[S.Job(lam_idx=1, g_idx=0, n_packets=n, key=77)])


def _load(ctx, wl, prec):
    from paper_2110_15640_gb300 import gcmc
    return gcmc.load_workload(ctx, wl, prec)


@pytest.mark.parametrize("survival", [1, 0])
def test_fp64_per_packet_parity_tthg_surface(G, survival):
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy_surface(3000, survival=survival)
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    nobs = len(O.job_observers(wl, job))
    assert nobs == 4
    ntr, mtr = 300, 6000
    ref = O.run(wl, job, per_packet=True, n_trace=ntr, max_trace=mtr, nthreads=8)
    assert ref["ledger"][3] > 0.05 * ref["ledger"][0]          # the surface is reached
    got = G.run_debug(jobs[0], n_trace=ntr, max_trace=mtr, n_obs=nobs)
    same = 0
    for q in range(ntr):
        no, ng = ref["tr_n"][q], got["tr_n"][q]
        if no == ng and np.array_equal(ref["tr_cell"][q, :no], got["tr_cell"][q, :ng]):
            lo, lg = ref["tr_len"][q, :no], got["tr_len"][q, :ng]
            same += int(np.all(np.abs(lo - lg) <= 1e-9 * np.abs(lo) + 1e-9))
    assert same >= ntr - 1, f"{same}/{ntr} identical traces"
    np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
    np.testing.assert_allclose(got["pk_f"], ref["pk_f"], rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(got["tally"][:nobs], ref["tally"], rtol=1e-12, atol=job.n_packets * 2.0 ** -33)
    st = got["stats"]
    assert st.steps == ref["steps"]
    np.testing.assert_allclose(list(st.ledger), ref["ledger"], rtol=1e-12, atol=64 * job.n_packets * 2.0 ** -33)


def test_fp32_parity_tthg_surface(G):
    """FP32 march against the FP64 oracle on identical packets: per-packet peel-off sums within 1e-3
    relative for >= 99% of packets and observers, each observer's tally within 1e-4."""
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy_surface(20000)
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    ref = O.run(wl, job, per_packet=True, nthreads=8)
    got = G.run_debug(jobs[0], n_obs=4)
    f_o, f_g = ref["pk_f"], got["pk_f"]
    close = np.abs(f_g - f_o) <= 1e-3 * np.abs(f_o) + 1e-300
    trel = np.abs(got["tally"][:4] / ref["tally"] - 1)
    print(f"FP32 TTHG + surface: close {close.mean():.5f}; tally rel {trel}")
    assert close.mean() >= 0.99
    assert np.all(trel < 1e-4)


def _lambert_phase(alpha):
    return (math.sin(alpha) + (math.pi - alpha) * math.cos(alpha)) / math.pi


def test_fp32_lambert_sphere_closed_form(G):
    from paper_2110_15640_gb300 import gcmc
    As = 0.6
    alphas = [0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4]
    obs = [[math.cos(a), math.sin(a), 0.0] for a in alphas]
    wl = S.slab_sphere_albedo(omega=1.0, tau=0.0, phase="iso", n_packets=1_000_000, surface_albedo=As, obs=obs)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    got = G.run_debug(jobs[0], n_obs=4)
    for o, a in enumerate(alphas):
        f = math.pi * got["pk_f"][:, o]
        est, sig = f.mean(), f.std() / math.sqrt(len(f))
        ref = 2.0 / 3.0 * As * _lambert_phase(a)
        assert abs(est - ref) < 3 * sig + 1e-9, (a, est, ref, sig)


def test_fp64_tthg_slab_vs_adding_doubling(G):
    from paper_2110_15640_gb300 import gcmc
    g, omega, tau = 0.5, 0.9, 2.0
    g2 = -0.5 * g
    a = 1 - g2 * g2
    beta = [(2 * l + 1) * (a * g ** l + (1 - a) * g2 ** l) for l in range(48)]
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase="tthg", g=g, n_packets=200_000)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    got = G.run_debug(jobs[0])
    f = math.pi * got["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.AddingDoubling(beta, omega, tau, n=48).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-4 * ref, (est, ref, sig)


def test_ledger_closes_with_surface(G):
    from paper_2110_15640_gb300 import gcmc
    for surv in (1, 0):
        wl = cloudy_surface(50000, survival=surv)
        gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
        t, st = G.run_packets(jobs[0])
        L = list(st.ledger)
        assert L[3] > 0 and st.packets == 50000
        lhs = L[0] + L[4]
        rhs = L[1] + L[2] + L[3] + L[5] + L[6] + L[7]
        assert abs(lhs - rhs) < 64 * 50000 * 2.0 ** -33 + 1e-6 * lhs


def test_source_validation(G):
    from paper_2110_15640_gb300 import gcmc
    wl = cloudy_surface(100)
    gid = G.upload_grid(wl.grid)
    for bad in (dict(surface_albedo=1.5), dict(surface_albedo=-0.1), dict(cloud_phase=7)):
        src = dataclasses.replace(wl.source, opts=dataclasses.replace(wl.source.opts, **bad))
        with pytest.raises(gcmc.GcmcError):
            G.set_source(gid, src)
