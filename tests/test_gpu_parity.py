"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded
inputs and the same Philox streams.

Tolerances
* FP64 path: identical cell sequences for every traced packet, per-segment path lengths within 1e-9
  relative (plus 1e-9 m absolute for corner cuts), per-packet f within 1e-10 relative, tallies within
  1e-9.
* FP32 path (FP32 march, FP64 tallies): positions at planetary radius carry ~ulp(7e7 m) = 8 m, so
  per-segment lengths differ from the FP64 oracle by metres (measured and reported); the tally
  bar is 1e-5 relative on identical packet sets; per-packet f within 1e-3 relative for >= 99%
  of packets (a packet whose launch or interaction lands within metres of a face may take a
  different cell sequence).
"""
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


def _load(ctx, wl, prec):
    from paper_2110_15640_gb300 import gcmc
    return gcmc.load_workload(ctx, wl, prec)


def _fp(name):
    from paper_2110_15640_gb300 import gcmc
    return getattr(gcmc, name)


def small_albedo(n=3000, survival=1):
    return S.config1_albedo(n_packets=n, nlon=8, nlat=6, nr=10, survival=survival)


def small_emission(n=4000):
    return S.config2_emission(n_packets=n, nlon=16, nlat=8, nr=12, nb=2, ng=2, bands=[1], gpoints=[1])


def small_transmission(n=3000):
    return S.config4_transmission(n_packets=n, nlon=12, nlat=6, nr=8, n_lam=60, n_lines=40, lam_subset=[20])


def _trace_compare(tr_o, tr_g, n_o, n_g, rel, absl):
    """returns (number of packets with identical cell sequences, max relative length error on those)"""
    same = 0
    worst = 0.0
    for q in range(len(n_o)):
        a, b = n_o[q], n_g[q]
        if a == b and np.array_equal(tr_o["cell"][q, :a], tr_g["cell"][q, :b]):
            same += 1
            lo, lg = tr_o["len"][q, :a], tr_g["len"][q, :b]
            err = np.abs(lo - lg) / (np.abs(lo) * rel + absl + 1e-300)
            worst = max(worst, float(err.max(initial=0.0)))
    return same, worst


# ------------------------------------------------------------------ RNG

def test_philox_matches_oracle_and_curand(G):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(2000, 2), dtype=np.uint64).astype(np.uint32)
    mine, cur = G.selftest_philox(ctr, key)
    assert np.array_equal(mine, cur)
    for q in range(0, 2000, 97):
        assert O.philox(ctr[q], key[q]) == [int(x) for x in mine[q]]


# ------------------------------------------------------------------ S1 cell tables

def test_cell_tables_albedo(G):
    wl = S.config3_phase_curve(nlon=16, nlat=8, nr=12, nlam=3, nphase=2)
    gid, oid, sid, jobs = _load(G, wl, _fp("FP64"))
    for j, job in zip(wl.jobs[:3], jobs[:3]):
        ref = O.prep_cells(wl, j)
        got = G.prep_cells(job, wl.grid.ncell)
        for k in ("alpha", "omega", "g", "pgas"):
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-15, atol=0)


def test_cell_tables_emission(G):
    """Emission cell tables against the oracle.  FP64 runs follow the definitions term by term (1e-13).
    FP32 runs compute alpha = rho k_ab exp(wT d1 + wp d2 + wT wp d3) in FP32 from the k-table node
    records: expf (<= 2 ulp), FP32 weights and differences (<= 1 ulp of an O(1) argument) and three
    roundings bound alpha, L_i, the pdf and the FP32 weights to ~5e-7 relative; 2e-6 is asserted."""
    wl = S.config2_emission(n_packets=1000, nlon=16, nlat=8, nr=12, nb=3, ng=3)
    for prec in ("FP64", "FP32"):
        gid, oid, sid, jobs = _load(G, wl, _fp(prec))
        rt = 1e-13 if prec == "FP64" else 2e-6
        for j, job in list(zip(wl.jobs, jobs))[::4]:
            ref = O.prep_cells(wl, j)
            got = G.prep_cells(job, wl.grid.ncell)
            st = got["stats"]
            np.testing.assert_allclose(got["lum"], ref["L"], rtol=rt)
            np.testing.assert_allclose(got["cdf"], ref["cdf"], rtol=max(rt, 1e-12), atol=1e-15)
            # monotone, and exactly flat over the cells the tau_vert cut excludes
            dq = np.diff(np.concatenate([[0.0], got["cdf"]]))
            q_ref = np.diff(np.concatenate([[0.0], ref["cdf"]]))
            assert np.all(dq >= 0)
            assert np.array_equal(dq == 0, q_ref == 0)
            np.testing.assert_allclose(got["wcell"], ref["wcell"], rtol=max(rt, 1e-12))
            assert st.n_emit_cells == ref["n_incl"]
            assert abs(st.l_tot / ref["L_tot"] - 1) < rt
            np.testing.assert_allclose(got["alpha"], ref["alpha"], rtol=rt)


def test_cell_tables_transmission(G):
    wl = S.config4_transmission(nlon=12, nlat=6, nr=8, n_lam=80, n_lines=60, lam_subset=[0, 17, 79])
    for prec, rt in (("FP64", 1e-12), ("FP32", 2e-5)):
        gid, oid, sid, jobs = _load(G, wl, _fp(prec))
        for j, job in zip(wl.jobs, jobs):
            ref = O.prep_cells(wl, j)
            got = G.prep_cells(job, wl.grid.ncell)
            np.testing.assert_allclose(got["alpha"], ref["alpha"], rtol=rt)


# ------------------------------------------------------------------ packets: FP64 path

@pytest.mark.parametrize("maker", [small_albedo, small_emission, small_transmission])
def test_fp64_per_packet_parity(G, maker):
    wl = maker()
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, _fp("FP64"))
    nobs = len(O.job_observers(wl, job))
    ntr, mtr = 300, 4000
    ref = O.run(wl, job, per_packet=True, n_trace=ntr, max_trace=mtr, nthreads=8)
    got = G.run_debug(jobs[0], n_trace=ntr, max_trace=mtr, n_obs=nobs)
    # identical segment lists
    same, worst = _trace_compare({"cell": ref["tr_cell"], "len": ref["tr_len"]},
                                 {"cell": got["tr_cell"], "len": got["tr_len"]}, ref["tr_n"], got["tr_n"], 1e-9, 1e-9)
    assert same == ntr, f"{same}/{ntr} identical traces"
    assert worst <= 1.0, worst
    np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
    np.testing.assert_allclose(got["pk_f"], ref["pk_f"], rtol=1e-10, atol=1e-300)
    # tallies are 64-bit fixed point with 2^-32 resolution: each packet's f is rounded by <= 2^-33
    np.testing.assert_allclose(got["tally"][:nobs], ref["tally"], rtol=1e-12, atol=job.n_packets * 2.0 ** -33)
    st = got["stats"]
    assert st.steps == ref["steps"]
    np.testing.assert_allclose(list(st.ledger), ref["ledger"], rtol=1e-12, atol=64 * job.n_packets * 2.0 ** -33)


# ------------------------------------------------------------------ packets: FP32 path

@pytest.mark.parametrize("maker", [small_albedo, small_emission, small_transmission])
def test_fp32_parity(G, maker):
    """FP32 march against the FP64 oracle on identical packets.  Emission and transmission compare
    each packet's optical depth (what the march computes): |dtau| <= 1e-4 tau + 1e-5 for >= 99% of
    packets; albedo compares each packet's peel-off sum f: |df| <= 1e-3 |f| for >= 99%.  The tally
    of the job is within 1e-5 relative of the oracle's."""
    wl = maker(n=20000)
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, _fp("FP32"))
    nobs = len(O.job_observers(wl, job))
    ref = O.run(wl, job, per_packet=True, nthreads=8)
    got = G.run_debug(jobs[0], n_obs=nobs)
    if wl.mode == 0:
        f_o, f_g = ref["pk_f"][:, 0], got["pk_f"][:, 0]
        close = np.abs(f_g - f_o) <= 1e-3 * np.abs(f_o) + 1e-300
        err = np.abs(f_g - f_o) / np.maximum(np.abs(f_o), 1e-300)
    else:
        t_o, t_g = ref["pk_tau"], got["pk_tau"]
        close = np.abs(t_g - t_o) <= 1e-4 * t_o + 1e-5
        err = np.abs(t_g - t_o) / np.maximum(t_o, 1e-300)
    trel = abs(got["tally"][0] / ref["tally"][0] - 1)
    print(f"FP32 {wl.name}: per-packet rel err median {np.median(err):.2e} p99 {np.quantile(err, 0.99):.2e} "
          f"close {close.mean():.5f}; tally rel {trel:.2e}")
    assert close.mean() >= 0.99
    assert trel < 1e-5


# ------------------------------------------------------------------ batched form equals the plain form

def test_batched_equals_plain_bitwise(G):
    wl = S.config3_phase_curve(nlon=16, nlat=8, nr=12, nlam=2, nphase=3, n_lo=700, n_hi=3000)
    gid, oid, sid, jobs = _load(G, wl, _fp("FP32"))
    tb, sb = G.run_batch(jobs)
    for q, job in enumerate(jobs):
        tp, sp = G.run_packets(job)
        assert tp[0] == tb[q][0]
        assert sp.steps == sb[q].steps and sp.packets == sb[q].packets == job.n_packets
    # independent of the work-item size and refill interval, and of the kernel variant the blocks per SM
    # select (scattering kernels compiled for 5 and 6 resident 128-thread blocks)
    from paper_2110_15640_gb300 import gcmc
    tc, _ = G.run_batch(jobs, cfg=gcmc.gcmc_launch_cfg(64, 0, 96, 3, 7, 0))
    assert np.array_equal(tc, tb)
    for bps in (5, 6, 8):
        tv, _ = G.run_batch(jobs, cfg=gcmc.gcmc_launch_cfg(128, bps, 512, 16, 8, 0))
        assert np.array_equal(tv, tb), bps


def test_batched_variants_equal_plain_bitwise_emission(G):
    """Absorber-only kernels compiled for 6 and 8 resident blocks per SM, and the uncapped one, give the
    plain form's tallies bit for bit."""
    from paper_2110_15640_gb300 import gcmc
    wl = small_emission(n=20000)
    gid, oid, sid, jobs = _load(G, wl, _fp("FP32"))
    tp, sp = G.run_packets(jobs[0])
    for shape in ((128, 0), (128, 6), (128, 8), (256, 0)):
        tv, sv = G.run_batch(jobs, cfg=gcmc.gcmc_launch_cfg(shape[0], shape[1], 512, 24, 16, 0))
        assert np.array_equal(tv[0], tp), shape
        assert sv[0].steps == sp.steps


def test_async_submit_poll_matches_batch(G):
    wl = small_emission(n=5000)
    gid, oid, sid, jobs = _load(G, wl, _fp("FP32"))
    tb, _ = G.run_batch(jobs)
    t = G.submit(jobs)
    res = None
    for _ in range(100000):
        res = G.poll(t, len(jobs))
        if res is not None:
            break
    assert res is not None
    assert np.array_equal(res[0], tb)


# ------------------------------------------------------------------ edge cases

def test_edge_cases(G):
    from paper_2110_15640_gb300 import gcmc
    wl = small_albedo(n=257)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    # zero packets
    j0 = gcmc.Context.job(gid, oid, sid, 0, 0, 0, 0, 1, 0)
    t, st = G.run_packets(j0)
    assert t[0] == 0 and st.packets == 0
    # ragged count (not a multiple of the block or the warp)
    ref = O.run(wl, wl.jobs[0])
    t, st = G.run_packets(jobs[0])
    assert st.packets == 257 and abs(t[0] / ref["tally"][0] - 1) < 1e-9
    # invalid arguments are rejected
    bad = gcmc.Context.job(gid, oid, sid, 1, 0, 0, 10, 1, 0)   # emission mode with albedo opacity
    with pytest.raises(gcmc.GcmcError) as e:
        G.run_packets(bad)
    assert e.value.status == gcmc.ERR_ARG
    g2 = S.uniform_grid(4, 4, 3, 1.0, 2.0)
    g2.T[5] = float("nan")
    with pytest.raises(gcmc.GcmcError) as e:
        G.upload_grid(g2)
    assert e.value.status == gcmc.ERR_NAN
    g3 = S.uniform_grid(4, 4, 3, 1.0, 2.0)
    g3.lon_edges = g3.lon_edges * 0.5
    with pytest.raises(gcmc.GcmcError) as e:
        G.upload_grid(g3)
    assert e.value.status == gcmc.ERR_ARG


def test_degenerate_grids(G):
    """one longitude cell, one latitude band, one radial layer; two longitude cells, whose edges both lie
    in the plane y = 0"""
    from paper_2110_15640_gb300 import gcmc
    for nlon, nlat, nr in ((1, 4, 3), (6, 1, 3), (1, 1, 1), (2, 3, 3), (2, 1, 2)):
        wl = S.slab_sphere_albedo(omega=0.7, tau=3.0, n_packets=2000, nlon=nlon, nlat=nlat)
        if nr != 1:
            wl.grid = S.uniform_grid(nlon, nlat, nr, wl.grid.R0, wl.grid.R_toa, rho=1.0)
            wl.opac.acld = np.full(wl.grid.ncell, float(wl.opac.acld[0]), np.float32)
        gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
        ref = O.run(wl, wl.jobs[0], per_packet=True)
        got = G.run_debug(jobs[0])
        np.testing.assert_allclose(got["pk_f"][:, 0], ref["pk_f"][:, 0], rtol=1e-9, atol=1e-300)


# ------------------------------------------------------------------ analytic cases on the GPU (FP32 path)

def test_gpu_transmission_integral_3sigma(G):
    from paper_2110_15640_gb300 import gcmc
    wl = S.uniform_absorber_sphere(n_packets=400_000)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    got = G.run_debug(jobs[0])
    g = wl.grid
    f = got["pk_f"][:, 0] * (g.R_toa - g.R0) * g.R_toa
    est, sig = 2 * f.mean(), 2 * f.std() / math.sqrt(len(f))
    exact = R.transmission_integral_uniform(float(np.float32(2e-6)), g.R0, g.R_toa)
    assert abs(est - exact) < 3 * sig
    obs = G.postscale(gid, gcmc.TRANSMISSION, got["tally"][0], jobs[0].n_packets)
    assert abs(2 * obs["I_p"] / est - 1) < 1e-6


@pytest.mark.parametrize("phase,beta,omega,tau", [("iso", [1.0], 1.0, 2.0), ("rayleigh", [1.0, 0.0, 0.5], 0.5, 20.0)])
def test_gpu_albedo_vs_adding_doubling(G, phase, beta, omega, tau):
    """Thin homogeneous layer (1e-4 R0) on a black sphere against the plane-parallel adding-doubling
    albedo, on the FP64 path: in FP32 a 7 km layer at 7e7 m is resolved only to ~1e-3 of its depth."""
    from paper_2110_15640_gb300 import gcmc
    wl = S.slab_sphere_albedo(omega=omega, tau=tau, phase=phase, n_packets=200_000)
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    got = G.run_debug(jobs[0])
    f = math.pi * got["pk_f"][:, 0]
    est, sig = f.mean(), f.std() / math.sqrt(len(f))
    ref = R.AddingDoubling(beta, omega, tau, n=40).geometric_albedo()
    assert abs(est - ref) < 3 * sig + 1e-5 * ref
    obs = G.postscale(gid, gcmc.ALBEDO, got["tally"][0], jobs[0].n_packets)
    assert abs(obs["A_g"] / est - 1) < 1e-6


def test_gpu_fp32_albedo_config1_matches_oracle(G):
    """Config-1 geometry (20 layers over 16 scale heights) in FP32: geometric albedo within 1e-5 of
    the FP64 oracle on the same 1e5 packets."""
    from paper_2110_15640_gb300 import gcmc
    wl = S.config1_albedo()
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    t, st = G.run_packets(jobs[0])
    ref = O.run(wl, wl.jobs[0], nthreads=8)
    assert abs(t[0] / ref["tally"][0] - 1) < 1e-5
    assert st.packets == 100_000


def test_gpu_ledger_closes(G):
    from paper_2110_15640_gb300 import gcmc
    for surv in (1, 0):
        wl = small_albedo(n=50000, survival=surv)
        gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
        t, st = G.run_packets(jobs[0])
        L = list(st.ledger)
        lhs = L[0] + L[4]
        rhs = L[1] + L[2] + L[3] + L[5] + L[6] + L[7]
        # fixed-point rounding: <= 2^-33 per ledger entry, a handful of entries per packet
        assert abs(lhs - rhs) < 64 * 50000 * 2.0 ** -33 + 1e-6 * lhs


def test_heavy_roulette_per_packet_parity(G):
    """Roulette at W < 0.5 W_launch with survival probability 0.5 (after nearly every second scattering
    under survival biasing): FP64 per-packet f, steps and the ledger against the oracle."""
    from paper_2110_15640_gb300 import gcmc
    for surv in (1,):
        wl = S.slab_sphere_albedo(omega=0.5, tau=20.0, phase="iso", n_packets=3000, survival=surv)
        wl.source.opts.w_rr, wl.source.opts.p_surv = 0.5, 0.5
        gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
        ref = O.run(wl, wl.jobs[0], per_packet=True, nthreads=8)
        got = G.run_debug(jobs[0])
        np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
        # deep in a tau = 20 layer 7 km thick at 7e7 m, f carries e^-tau_obs of slant paths whose FP64
        # lengths agree to the module's 1e-9; with tau_obs <= 50 (the cut) f agrees to 5e-8 (measured on
        # a GB300: 8.6e-10 at most, identical steps)
        np.testing.assert_allclose(got["pk_f"][:, 0], ref["pk_f"][:, 0], rtol=5e-8, atol=1e-300)
        L = ref["ledger"]
        np.testing.assert_allclose(list(got["stats"].ledger), L, rtol=1e-12, atol=64 * 3000 * 2.0 ** -33)
        assert L[5] > 0.01 * L[0]


@pytest.mark.parametrize("maker,cap", [(small_albedo, 9), (small_emission, 6), (small_transmission, 4)])
def test_step_cap_per_packet_parity(G, maker, cap):
    """A per-packet step cap small enough to stop most packets: the cap ends a packet's ray before the
    step that would exceed it (the oracle's march rule), in the middle of a ray or at the start of the
    next one (a peel-off after a flight).  FP64 per-packet steps and f, the capped weight of the ledger,
    and the batched kernel (whose lanes are refilled) equal to the plain one."""
    from paper_2110_15640_gb300 import gcmc
    wl = maker(n=3000)
    wl.source.opts.max_steps = cap
    job = wl.jobs[0]
    nobs = len(O.job_observers(wl, job))
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP64)
    ref = O.run(wl, job, per_packet=True, nthreads=8)
    got = G.run_debug(jobs[0], n_obs=nobs)
    np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
    assert np.mean(ref["pk_steps"] == cap) > 0.3            # the cap does stop packets
    np.testing.assert_allclose(got["pk_f"], ref["pk_f"], rtol=1e-10, atol=1e-300)
    L = ref["ledger"]
    assert L[6] > 0
    np.testing.assert_allclose(list(got["stats"].ledger), L, rtol=1e-12, atol=64 * job.n_packets * 2.0 ** -33)
    tp, sp = G.run_packets(jobs[0])
    tb, sb = G.run_batch(jobs, cfg=gcmc.gcmc_launch_cfg(64, 0, 96, 3, 7, 0))
    assert np.array_equal(tp, tb[0]) and sp.steps == sb[0].steps == ref["steps"]
    assert list(sp.ledger) == list(sb[0].ledger)


# ------------------------------------------------------------------ full-size grid, sampled packets

def test_full_size_emission_sampled_packets(G):
    from paper_2110_15640_gb300 import gcmc
    wl = S.config2_emission(n_packets=1_000_000, bands=[7], gpoints=[5])
    job = wl.jobs[0]
    for prec in ("FP64", "FP32"):
        gid, oid, sid, jobs = _load(G, wl, getattr(gcmc, prec))
        cells = O.prep_cells(wl, job)
        for p0 in (0, 333_333, 999_000):
            ref = O.run(wl, job, cells=cells, packet0=p0, n_run=1000, per_packet=True, nthreads=8)
            got = G.run_debug(jobs[0], packet0=p0, n_run=1000)
            if prec == "FP64":
                np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
                np.testing.assert_allclose(got["pk_f"], ref["pk_f"], rtol=1e-10, atol=1e-300)
            else:
                rel = np.abs(got["pk_f"][:, 0] - ref["pk_f"][:, 0]) / np.maximum(ref["pk_f"][:, 0], 1e-300)
                assert np.mean(rel < 1e-3) >= 0.99


def test_full_size_emission_batch_sampled_jobs(G):
    """The emission batch at full size (128 x 64 x 50 cells, 30 bands x 8 g-ordinates, 10^6 packets per
    job) through the persistent batched kernel: every 12th job's tally against the oracle's on the same
    packets, and the whole batch's tallies independent of the launch parameters."""
    import os
    from paper_2110_15640_gb300 import gcmc
    wl = S.config2_emission()
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    tb, sb = G.run_batch(jobs)
    tc, _ = G.run_batch(jobs, cfg=gcmc.gcmc_launch_cfg(256, 8, 128, 8, 16, 0))
    assert np.array_equal(tb, tc)
    rels = []
    for q in range(0, len(jobs), 12):
        job = wl.jobs[q]
        ref = O.run(wl, job, nthreads=min(16, os.cpu_count() or 1))
        assert sb[q].packets == job.n_packets
        rels.append(abs(tb[q][0] / ref["tally"][0] - 1))
        # FP32 cell sequences differ from the FP64 oracle's for packets within metres of a face
        assert abs(sb[q].steps / ref["steps"] - 1) < 1e-4
    print(f"full-size emission batch: FP32 tally vs oracle, max rel {max(rels):.2e}, mean {np.mean(rels):.2e}")
    # the module's FP32 tally bar (measured on a GB300: max 2.9e-6, mean 1.7e-6 over the 20 jobs)
    assert max(rels) < 1e-5


@pytest.mark.parametrize("name", ["phase_curve", "transmission"])
def test_full_size_batches_sampled_jobs(G, name):
    """The phase-curve batch (128 x 64 x 50 cells, 40 wavelengths x 24 phases, 10^4..10^6 packets per
    job) and the high-resolution transmission batch (96 x 48 x 60 cells, 9532 wavelengths x 10^4
    chords) at full size through the persistent batched kernel: evenly spaced jobs' FP32 tallies
    against the oracle's on the same packets.

    Multiple scattering: a packet whose FP32 cell sequence leaves the oracle's (launch or interaction
    within metres of a face) continues on another path, so its contribution is an independent draw
    of the same distribution, and the tally difference is sampling noise of those few packets.  The
    bar is a tenth of the job's Monte Carlo standard error (measured on a GB300: at most 0.009 of it;
    at most 9.6e-5 relative).  Chords do not scatter: the module's FP32 tally bar, 1e-5 relative."""
    import os
    from paper_2110_15640_gb300 import gcmc
    scat = name == "phase_curve"
    wl = S.config3_phase_curve() if scat else S.config4_transmission()
    n_sample = 8 if scat else 20
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    tb, sb = G.run_batch(jobs)
    rels, srels, zs = [], [], []
    for q in [(k * len(jobs)) // n_sample for k in range(n_sample)]:
        job = wl.jobs[q]
        ref = O.run(wl, job, nthreads=min(16, os.cpu_count() or 1), per_packet=scat)
        assert sb[q].packets == job.n_packets
        d = tb[q][0] - ref["tally"][0]
        rels.append(abs(d / ref["tally"][0]))
        srels.append(abs(sb[q].steps / ref["steps"] - 1))
        if scat:
            f = ref["pk_f"][:, 0]
            zs.append(abs(d) / (f.std() * math.sqrt(len(f))))
    print(f"full-size {name} batch: FP32 tally vs oracle, max rel {max(rels):.2e}, mean {np.mean(rels):.2e};"
          f" steps max rel {max(srels):.2e}" + (f"; max |diff| / MC sigma {max(zs):.3f}" if scat else ""))
    if scat:
        assert max(zs) < 0.1
    else:
        assert max(rels) < 1e-5
    assert max(srels) < 1e-3


def test_full_size_phase_curve_split_by_packet(G):
    """The full-size phase curve (128 x 64 x 50 cells, cloud deck, multiple scattering) in FP32 against
    the FP64 oracle, split by packet.  On four jobs spread over the 960, the first 200,000 packets are
    traced on both sides (windows of 10,000): packets whose cell sequences agree with the oracle's must
    give the same sum of peel-off contributions within 1e-5 relative (the tally bar on identical
    packets); the packets whose FP32 sequence left the oracle's (a launch or interaction within metres of
    a face, then an independent path) are reported against the Monte Carlo standard error of their own
    sum, and their difference must stay below 3 of it."""
    import os
    from paper_2110_15640_gb300 import gcmc
    wl = S.config3_phase_curve()
    gid, oid, sid, jobs = _load(G, wl, gcmc.FP32)
    nth = min(16, os.cpu_count() or 1)
    win, n_max, mtr = 10000, 200_000, 4000
    for q in [(k * len(jobs)) // 4 for k in range(4)]:
        job = wl.jobs[q]
        cells = O.prep_cells(wl, job)
        n_run = min(n_max, job.n_packets)
        sa_o = sa_g = sd_o = sd_g = 0.0
        var_d, n_same = 0.0, 0
        for p0 in range(0, n_run, win):
            n = min(win, n_run - p0)
            ref = O.run(wl, job, cells=cells, packet0=p0, n_run=n, per_packet=True, n_trace=n, max_trace=mtr,
                        nthreads=nth)
            got = G.run_debug(jobs[q], packet0=p0, n_run=n, n_trace=n, max_trace=mtr, n_obs=1)
            # a packet whose trace fills the buffer (thousands of segments) cannot be compared cell by cell:
            # it goes with the diverged remainder
            same = np.array([ref["tr_n"][k] == got["tr_n"][k] and ref["tr_n"][k] < mtr and
                             np.array_equal(ref["tr_cell"][k, :ref["tr_n"][k]], got["tr_cell"][k, :got["tr_n"][k]])
                             for k in range(n)])
            fo, fg = ref["pk_f"][:, 0], got["pk_f"][:, 0]
            sa_o += fo[same].sum()
            sa_g += fg[same].sum()
            sd_o += fo[~same].sum()
            sd_g += fg[~same].sum()
            var_d += float(((fo[~same] ** 2).sum() + (fg[~same] ** 2).sum()))
            n_same += int(same.sum())
        rel = abs(sa_g / sa_o - 1)
        z = abs(sd_g - sd_o) / math.sqrt(var_d) if var_d > 0 else 0.0
        print(f"phase curve job {q}: {n_same}/{n_run} packets with identical FP32 cell sequences, their tally "
              f"rel {rel:.2e}; diverged remainder {n_run - n_same} packets, |diff| / sigma {z:.2f}")
        assert rel < 1e-5
        assert z < 3.0


@pytest.mark.parametrize("grid,ng", [((16, 8, 12), 8), ((31, 15, 21), 4)])
def test_emission_pdf_sweep_equals_per_block_scan(G, grid, ng):
    """A batch of enough emission jobs to fill the GPU builds each job's fixed-point cumulative pdf in one
    sweep per job; a single job (the plain form) with the per-block pdf and scan.  The pdf is integers,
    so the two give the same launch cells, and tallies, steps, L_tot and the pdf total agree bit for bit.
    Grids of one tile (1,536 cells) and of two tiles and a ragged tail (9,765 cells: the running total
    carried across tiles, the last thread's four cells straddling the end)."""
    nlon, nlat, nr = grid
    wl = S.config2_emission(n_packets=3000, nlon=nlon, nlat=nlat, nr=nr, nb=30, ng=ng)
    gid, oid, sid, jobs = _load(G, wl, _fp("FP32"))
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert 3 * len(jobs) >= 2 * nsm            # the batch takes the one-sweep-per-job path
    tb, sb = G.run_batch(jobs)
    for q in range(0, len(jobs), 37):
        tp, sp = G.run_packets(jobs[q])
        assert np.array_equal(tp, tb[q]), q
        assert sp.steps == sb[q].steps and sp.l_tot == sb[q].l_tot and sp.cdf_total == sb[q].cdf_total, q


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
@pytest.mark.parametrize("obs", [(1.0, 0.0, 0.0), (0.6, 0.0, 0.8)])
def test_peel_off_parity_in_and_out_of_the_equatorial_plane(G, obs, prec):
    """Emission peel-offs towards an observer in the equatorial plane (rays parallel to it: the closed-form
    latitude exit) and out of it (dz != 0: the general cone solver), on packets 18,000-19,999 of 20,000,
    which start high in the atmosphere and cross cones and half-planes (in the 300 traced: ~30 and ~390
    in the plane, ~90 and ~100 out of it).  FP64: traces identical to the oracle's, f within 1e-10; FP32:
    optical depths within the FP32 per-packet bar for >= 99% of packets, their f sum within 1e-5."""
    from paper_2110_15640_gb300 import gcmc
    wl = S.config2_emission(n_packets=20000, nlon=16, nlat=8, nr=12, nb=2, ng=2, bands=[1], gpoints=[1],
                            obs=np.array([obs]))
    job = wl.jobs[0]
    gid, oid, sid, jobs = _load(G, wl, getattr(gcmc, prec))
    p0, n = 18000, 2000
    if prec == "FP64":
        ntr, mtr = 300, 4000
        ref = O.run(wl, job, packet0=p0, n_run=n, per_packet=True, n_trace=ntr, max_trace=mtr, nthreads=8)
        got = G.run_debug(jobs[0], packet0=p0, n_run=n, n_trace=ntr, max_trace=mtr, n_obs=1)
        same, worst = _trace_compare({"cell": ref["tr_cell"], "len": ref["tr_len"]},
                                     {"cell": got["tr_cell"], "len": got["tr_len"]}, ref["tr_n"], got["tr_n"],
                                     1e-9, 1e-9)
        assert same == ntr, f"{same}/{ntr} identical traces"
        assert worst <= 1.0, worst
        np.testing.assert_array_equal(got["pk_steps"], ref["pk_steps"])
        np.testing.assert_allclose(got["pk_f"], ref["pk_f"], rtol=1e-10, atol=1e-300)
    else:
        ref = O.run(wl, job, packet0=p0, n_run=n, per_packet=True, nthreads=8)
        got = G.run_debug(jobs[0], packet0=p0, n_run=n, n_obs=1)
        t_o, t_g = ref["pk_tau"], got["pk_tau"]
        close = np.abs(t_g - t_o) <= 1e-4 * t_o + 1e-5
        frel = abs(got["pk_f"][:, 0].sum() / ref["pk_f"][:, 0].sum() - 1)
        print(f"FP32 observer {obs}: close {close.mean():.5f}; f sum rel {frel:.2e}")
        assert close.mean() >= 0.99
        assert frel < 1e-5
