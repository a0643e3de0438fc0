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
