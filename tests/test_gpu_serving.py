"""The continuous-batching server (gcmc_server_*) on the GPU.

Requests of the three modes on two resident grids are submitted while others run, with few
completion slots and a small HBM budget so that admission, publication to the running kernel and
slot reuse all happen many times.  Every request's tallies and step counts must be bit-identical to
the same request served alone: its packets draw their random numbers from (seed, packet, event,
job key) and tallies are 64-bit fixed point, so nothing in the mix can change them.  The served
results also agree with the batched form (a different kernel) to FP32 rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2110_15640_gb300 import build, gcmc, synth
    build.build()
    sw = synth.config5_serving(n_requests=60, grids=((16, 8, 10), (32, 16, 20)), n_lo=1.0e3, n_hi=4.0e4,
                               n_lam_x=16, n_lines=50)
    ctx = gcmc.Context(0)
    jobs = gcmc.load_serving(ctx, sw)
    yield gcmc, sw, ctx, jobs
    ctx.close()


def _drain(sv, want, got, timeout_s=120.0):
    import time
    t0 = time.perf_counter()
    while len(got) < want:
        for t in sv.progress():
            got[t] = sv.result(t)
        assert time.perf_counter() - t0 < timeout_s, "served jobs did not complete"


def test_served_results_identical_alone_and_in_mix(setup):
    gcmc, sw, ctx, jobs = setup
    sv = gcmc.Server(ctx, max_jobs=6, hbm_budget=24 << 20, idle_us=500)
    try:
        tickets, got, peak_admitted = [], {}, 0
        for q, j in enumerate(jobs):                 # staggered: submissions interleave with progress
            tickets.append(sv.submit(j))
            if q % 3 == 2:
                for t in sv.progress():
                    got[t] = sv.result(t)
                peak_admitted = max(peak_admitted, sv.query().admitted)
        _drain(sv, len(jobs), got)
        st = sv.query()
        assert st.completed == len(jobs) and st.pending == 0 and st.admitted == 0 and st.bytes_in_use == 0
        assert peak_admitted > 1                     # jobs overlapped on the device
        for q, j in enumerate(jobs):
            alone = sv.run_all([j])[0]
            mixed = got[tickets[q]]
            assert np.array_equal(alone[0], mixed[0]), (q, alone[0], mixed[0])
            assert alone[1].steps == mixed[1].steps and alone[1].packets == mixed[1].packets == j.n_packets
            assert list(alone[1].ledger) == list(mixed[1].ledger)
    finally:
        sv.close()


def test_served_results_match_batched_form(setup):
    gcmc, sw, ctx, jobs = setup
    sv = gcmc.Server(ctx, max_jobs=64)
    try:
        served = sv.run_all(jobs[:24])
    finally:
        sv.close()
    same = 0
    for j, (tal, st) in zip(jobs[:24], served):
        ref, rst = ctx.run_batch([j])
        same += int(np.array_equal(tal, ref[0]) and st.steps == rst[0].steps)
        # the same packets through another kernel instantiation: equal up to FP32 rounding of a
        # path (a packet whose march rounds differently moves its own contribution only)
        np.testing.assert_allclose(tal[0], ref[0][0], rtol=1e-3, atol=j.n_packets * 2.0 ** -32)
        assert abs(st.steps - rst[0].steps) <= max(2, 1e-3 * rst[0].steps)
    print(f"served == batched bit for bit in {same} of 24 jobs")


def test_job_larger_than_budget_runs_alone(setup):
    gcmc, sw, ctx, jobs = setup
    sv = gcmc.Server(ctx, hbm_budget=1)           # every job exceeds it: admitted one at a time
    try:
        out = sv.run_all(jobs[:4])
        assert all(st.packets == j.n_packets for j, (_, st) in zip(jobs[:4], out))
    finally:
        sv.close()


def test_server_rejects_bad_jobs(setup):
    gcmc, sw, ctx, jobs = setup
    sv = gcmc.Server(ctx)
    try:
        bad = gcmc.gcmc_job.from_buffer_copy(jobs[0])
        bad.n_packets = 0
        with pytest.raises(gcmc.GcmcError):
            sv.submit(bad)
    finally:
        sv.close()


def test_served_optional_physics(setup):
    """Jobs with the optional physics (two-term HG clouds over a Lambertian surface, forced first scattering
    with continuous absorption, transmission with multiple scattering and limb darkening) through the
    server: bit-identical alone and in a mix, and equal to the batched form up to FP32 rounding."""
    import dataclasses
    from paper_2110_15640_gb300 import synth
    gcmc, sw, ctx, _ = setup
    wl = synth.config3_phase_curve(nlon=12, nlat=6, nr=10, nlam=2, nphase=4, n_lo=20000, n_hi=20000)
    opac = dataclasses.replace(wl.opac, kabs=wl.opac.kabs * 1e-3, kray=wl.opac.kray * 0.1)
    base = dataclasses.replace(wl.source.opts, cloud_phase=1)
    variants = [dataclasses.replace(base, surface_albedo=0.5),
                dataclasses.replace(base, forced_first=1, cont_abs=1)]
    gid = ctx.upload_grid(wl.grid)
    oid = ctx.upload_opacity(gid, opac)
    jobs = []
    for k, op in enumerate(variants):
        sid = ctx.set_source(gid, dataclasses.replace(wl.source, opts=op))
        jobs.append(gcmc.Context.job(gid, oid, sid, gcmc.ALBEDO, 1, 0, 20000, 3, 40 + k))
    tr_opts = dataclasses.replace(base, trans_scatter=1, ld_law=2, ld_coef=(0.4, 0.25, 0.0, 0.0), star_radius=7.0e8,
                                  star_dist=7.0e9, transit_xy=(0.0, 3.0e8))
    sid_t = ctx.set_source(gid, synth.Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]),
                                             opts=tr_opts))
    jobs.append(gcmc.Context.job(gid, oid, sid_t, gcmc.TRANSMISSION, 1, 0, 20000, 3, 50))
    sv = gcmc.Server(ctx, max_jobs=4)
    try:
        mixed = sv.run_all(jobs)
        for q, j in enumerate(jobs):
            alone = sv.run_all([j])[0]
            assert np.array_equal(alone[0], mixed[q][0]) and alone[1].steps == mixed[q][1].steps
        # plain requests, then these while the plain kernel runs: the server switches kernel variants (the
        # plain kernel drains before one with the optional physics starts), and every request still
        # equals itself served alone, bit for bit
        import time
        plain = list(setup[3][:4])
        t0 = time.perf_counter()
        while sv.query().kernel_running and time.perf_counter() - t0 < 10.0:   # the last kernel leaves when idle
            sv.progress()
            time.sleep(0.01)
        n0 = sv.query().kernel_launches
        tickets = [sv.submit(j) for j in plain]
        got = {}
        t0 = time.perf_counter()
        while not sv.query().kernel_running and len(got) < len(tickets) and time.perf_counter() - t0 < 10.0:
            for t in sv.progress():
                got[t] = sv.result(t)
        tickets += [sv.submit(j) for j in jobs]      # held until the plain kernel has drained
        _drain(sv, len(tickets), got)
        assert sv.query().kernel_launches >= n0 + 2
        for t, j in zip(tickets, plain + jobs):
            alone = sv.run_all([j])[0]
            assert np.array_equal(alone[0], got[t][0]) and alone[1].steps == got[t][1].steps
    finally:
        sv.close()
    tb, sb = ctx.run_batch(jobs)
    for q, j in enumerate(jobs):
        np.testing.assert_allclose(mixed[q][0][:2], tb[q][:2], rtol=1e-3, atol=j.n_packets * 2.0 ** -32)
        assert abs(mixed[q][1].steps - sb[q].steps) <= max(2, 1e-3 * sb[q].steps)
