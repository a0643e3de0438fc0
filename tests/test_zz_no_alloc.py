"""The allocation-free entry point gcmc_emission_pdf_noalloc against the library's own emission
cell-table entry point (gcmc_prep_cells), through the C ABI, on two calls in a row.

Some callers cannot call cudaMalloc: code that must not trigger the implicit device-wide
synchronisation of cudaMalloc/cudaFree, or hosts that give a library only memory they allocated
themselves.  The variant uses a fixed scratch array in the library's device memory instead; this
test checks it gives the same cumulative pdf, launch weights and totals as the allocating path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_pdf_matches_prep_cells_twice():
    import torch
    from paper_2110_15640_gb300 import build, gcmc, synth
    build.build()
    ctx = gcmc.Context(0)
    try:
        wl = synth.config2_emission(n_packets=1000, bands=[3], gpoints=[5])      # 128 x 64 x 50 cells
        _, _, _, jobs = gcmc.load_workload(ctx, wl, gcmc.FP64)   # FP64 tables, as the entry point computes
        n = wl.grid.ncell
        ref = ctx.prep_cells(jobs[0], n)
        st = ref["stats"]
        # input in the library's convention: L_i, negative for the cells the tau_vert cut excludes
        # (those are exactly the cells with zero pdf, as the hybrid pdf has a uniform part)
        q = np.diff(np.concatenate([[0.0], ref["cdf"]]))
        lum = torch.tensor(np.where(q > 0, ref["lum"], -1.0), dtype=torch.float64, device="cuda")
        beta = wl.source.opts.beta_emis
        for call in range(2):
            cdf = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            wcell = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            tot = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            rc = gcmc.emission_pdf_noalloc(lum, n, beta, cdf, wcell, tot)
            assert rc == gcmc.OK
            torch.cuda.synchronize()
            np.testing.assert_allclose(cdf.cpu().numpy(), ref["cdf"], rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(wcell.cpu().numpy(), ref["wcell"], rtol=1e-12)
            t = tot.cpu().numpy()
            assert abs(t[0] / st.l_tot - 1) < 1e-12
            assert int(t[1]) == st.n_emit_cells
            assert abs(t[2] / st.cdf_total - 1) < 1e-12
        # sizes above the compiled maximum are refused before any work is queued
        assert gcmc.emission_pdf_noalloc(lum, gcmc.NOALLOC_MAX_CELLS + 1, beta, cdf, wcell, tot) == gcmc.ERR_RANGE
    finally:
        ctx.close()
