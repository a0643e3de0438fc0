"""Captured batches (gcmc_graph_*): a batch captured into a CUDA graph and replayed gives tallies
bit-identical to the batched call, on every replay (fixed-point sums, counter-based random numbers)."""
import numpy as np
import pytest

from paper_2110_15640_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_graph_replays_match_run_batch():
    import torch
    from paper_2110_15640_gb300 import build, gcmc
    build.build()
    stream = torch.cuda.Stream()
    ctx = gcmc.Context(0, stream=stream)
    try:
        wl = S.config2_emission(n_packets=20_000, nlon=16, nlat=8, nr=12, nb=2, ng=3)
        _, _, _, jobs = gcmc.load_workload(ctx, wl, gcmc.FP32)
        cfg = gcmc.gcmc_launch_cfg(128, 0, 256, 4, 8, 0)
        ref, rst = ctx.run_batch(jobs, cfg=cfg)
        g = ctx.graph(jobs, cfg)
        try:
            dev = torch.zeros((len(jobs), gcmc.MAX_OBS), dtype=torch.float64, device="cuda")
            for _ in range(3):
                g.launch(dev)
                tal, sts = g.read()
                assert np.array_equal(tal, ref)
                assert [s.steps for s in sts] == [s.steps for s in rst]
            torch.cuda.synchronize()
            assert np.array_equal(dev.cpu().numpy(), ref)
        finally:
            g.close()
        # albedo (scattering kernel) as well
        wa = S.config3_phase_curve(nlon=12, nlat=6, nr=10, nlam=2, nphase=2, n_lo=5000, n_hi=5000)
        _, _, _, ja = gcmc.load_workload(ctx, wa, gcmc.FP32)
        ra, _ = ctx.run_batch(ja, cfg=cfg)
        ga = ctx.graph(ja, cfg)
        try:
            ga.launch()
            assert np.array_equal(ga.read()[0], ra)
        finally:
            ga.close()
    finally:
        ctx.close()


def test_graph_with_optional_physics_and_band_jobs():
    """Batches whose jobs need the optional kernel code (a band job; forced first scattering with
    continuous absorption over a reflecting surface; transmission with multiple scattering and limb
    darkening) replay from a CUDA graph with the batched call's bits."""
    import dataclasses
    import torch
    from paper_2110_15640_gb300 import build, gcmc
    build.build()
    stream = torch.cuda.Stream()
    ctx = gcmc.Context(0, stream=stream)
    try:
        wb = S.config2_emission(n_packets=20_000, nlon=16, nlat=8, nr=12, nb=2, bands=[1], split=(2, 2, 0.9),
                                per_packet_g=True, g_bias=2)
        _, _, _, jb = gcmc.load_workload(ctx, wb, gcmc.FP32)
        wl = S.config3_phase_curve(nlon=12, nlat=6, nr=10, nlam=2, nphase=2, n_lo=10_000, n_hi=10_000)
        opac = dataclasses.replace(wl.opac, kabs=wl.opac.kabs * 1e-3, kray=wl.opac.kray * 0.1)
        gid = ctx.upload_grid(wl.grid)
        oid = ctx.upload_opacity(gid, opac)
        op = dataclasses.replace(wl.source.opts, cloud_phase=1, surface_albedo=0.5, forced_first=1, cont_abs=1)
        sid = ctx.set_source(gid, dataclasses.replace(wl.source, opts=op))
        top = dataclasses.replace(wl.source.opts, trans_scatter=1, ld_law=2, ld_coef=(0.4, 0.25, 0.0, 0.0),
                                  star_radius=7.0e8, star_dist=7.0e9)
        sid_t = ctx.set_source(gid, S.Source(star=np.array([1.0, 0.0, 0.0]), obs=np.array([[-1.0, 0.0, 0.0]]),
                                             opts=top))
        jobs = jb + [gcmc.Context.job(gid, oid, sid, gcmc.ALBEDO, 1, 0, 10_000, 3, 7),
                     gcmc.Context.job(gid, oid, sid_t, gcmc.TRANSMISSION, 0, 0, 10_000, 3, 8)]
        ref, rst = ctx.run_batch(jobs)
        g = ctx.graph(jobs)
        try:
            for _ in range(2):
                g.launch()
                tal, sts = g.read()
                assert np.array_equal(tal, ref)
                assert [s.steps for s in sts] == [s.steps for s in rst]
        finally:
            g.close()
    finally:
        ctx.close()
