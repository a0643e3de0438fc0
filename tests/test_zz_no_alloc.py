"""The allocation-free entry point gcmc_emission_pdf_noalloc through the C ABI, on two calls in a row:
against the library's own emission cell-table entry point (gcmc_prep_cells) and against the FP64
oracle's cell tables.

Some callers cannot call cudaMalloc: code that must not trigger the implicit device-wide
synchronisation of cudaMalloc/cudaFree, or hosts that give a library only memory they allocated
themselves.  The variant uses a fixed scratch array in the library's device memory instead; this
test checks it gives the same cumulative pdf, launch weights and totals as the allocating path and
the oracle, and that it writes nothing outside the caller's arrays (each array is the head of a
larger NaN-filled guard buffer whose tail must stay NaN)."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

GUARD = 64   # doubles of NaN after each output array


def _guarded(torch, n):
    buf = torch.full((n + GUARD,), float("nan"), dtype=torch.float64, device="cuda")
    return buf, buf[:n]


def _lum_input(lum, cdf):
    """the entry point's input convention: L_i, negative for the cells the tau_vert cut excludes
    (exactly the cells with zero pdf, as the hybrid pdf has a uniform part)"""
    q = np.diff(np.concatenate([[0.0], cdf]))
    return np.where(q > 0, lum, -1.0)


def test_noalloc_pdf_matches_prep_cells_and_oracle_twice():
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
        orc = O.prep_cells(wl, wl.jobs[0])
        beta = wl.source.opts.beta_emis
        cases = [("library", _lum_input(ref["lum"], ref["cdf"]), ref["cdf"], ref["wcell"],
                  (st.l_tot, st.n_emit_cells, st.cdf_total), 1e-12),
                 ("oracle", _lum_input(orc["L"], orc["cdf"]), orc["cdf"], orc["wcell"],
                  (orc["L_tot"], orc["n_incl"], orc["cdf_total"]), 1e-12)]
        for name, lum_h, cdf_r, w_r, tot_r, rt in cases:
            lum = torch.tensor(lum_h, dtype=torch.float64, device="cuda")
            for call in range(2):
                cbuf, cdf = _guarded(torch, n)
                wbuf, wcell = _guarded(torch, n)
                tbuf, tot = _guarded(torch, 3)
                rc = gcmc.emission_pdf_noalloc(lum, n, beta, cdf, wcell, tot)
                assert rc == gcmc.OK, (name, call, rc)
                torch.cuda.synchronize()
                np.testing.assert_allclose(cdf.cpu().numpy(), cdf_r, rtol=rt, atol=1e-15)
                np.testing.assert_allclose(wcell.cpu().numpy(), w_r, rtol=rt)
                t = tot.cpu().numpy()
                assert abs(t[0] / tot_r[0] - 1) < rt
                assert int(t[1]) == tot_r[1]
                assert abs(t[2] / tot_r[2] - 1) < rt
                for b in (cbuf, wbuf, tbuf):
                    assert torch.isnan(b[-GUARD:]).all(), f"{name}: write past an output array"
        # in place: the luminosities replaced by the cumulative pdf
        buf, inplace = _guarded(torch, n)
        inplace.copy_(torch.tensor(cases[0][1], dtype=torch.float64, device="cuda"))
        wbuf, wcell = _guarded(torch, n)
        tbuf, tot = _guarded(torch, 3)
        assert gcmc.emission_pdf_noalloc(inplace, n, beta, inplace, wcell, tot) == gcmc.OK
        torch.cuda.synchronize()
        np.testing.assert_allclose(inplace.cpu().numpy(), ref["cdf"], rtol=1e-12, atol=1e-15)
        assert torch.isnan(buf[-GUARD:]).all()
        # refused before any work is queued: sizes above the compiled maximum, overlapping arrays
        assert gcmc.emission_pdf_noalloc(lum, gcmc.NOALLOC_MAX_CELLS + 1, beta, cdf, wcell, tot) == gcmc.ERR_RANGE
        assert gcmc.emission_pdf_noalloc(lum, n, beta, cbuf[1:n + 1], cbuf[:n], tot) == gcmc.ERR_ARG
    finally:
        ctx.close()
