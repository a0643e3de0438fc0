"""Contribution functions (Sect. 6) on the GPU against the oracle, through the C ABI.

The per-cell counters receive the same fixed-point contribution as the tally, so over cells and both
kinds (thermal, scattered) they add up to the tally; on the FP64 path every packet's contributions
match the oracle's, so the per-cell sums agree to the fixed-point quantum."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2110_15640_gb300 import build, gcmc
    build.build()
    c = gcmc.Context(0)
    yield c
    c.close()


CASES = {
    "albedo": lambda: S.config1_albedo(n_packets=20_000, nlon=8, nlat=6, nr=10),
    "emission": lambda: S.config2_emission(n_packets=20_000, nlon=16, nlat=8, nr=12, nb=2, ng=2, bands=[1],
                                           gpoints=[1]),
    "phase": lambda: S.config3_phase_curve(nlon=12, nlat=6, nr=10, nlam=2, nphase=2, n_lo=20_000, n_hi=20_000),
}


@pytest.mark.parametrize("case", list(CASES))
def test_contrib_fp64_matches_oracle(ctx, case):
    from paper_2110_15640_gb300 import gcmc
    wl = CASES[case]()
    _, _, _, jobs = gcmc.load_workload(ctx, wl, gcmc.FP64)
    nobs = len(O.job_observers(wl, wl.jobs[0]))
    tal, cf, st = ctx.run_contrib(jobs[0], wl.grid.ncell, nobs)
    ref = O.run(wl, wl.jobs[0], cf=True, nthreads=8)
    # each contribution is rounded to 2^-32 once; a packet contributes at most a few hundred times
    quantum = st.packets * 256 * 2.0 ** -33
    np.testing.assert_allclose(cf, ref["cf"], rtol=1e-9, atol=quantum)
    for o in range(nobs):
        assert abs(cf[:, o].sum() - tal[o]) <= 1e-12 * abs(tal[o])
    kinds = cf.reshape(2, -1).sum(axis=1)
    if wl.mode == gcmc.EMISSION:
        assert kinds[1] == 0.0 and kinds[0] > 0.0
    else:
        assert kinds[0] == 0.0 and kinds[1] > 0.0


def test_contrib_fp32_closure_and_agreement(ctx):
    from paper_2110_15640_gb300 import gcmc
    wl = CASES["emission"]()
    _, _, _, jobs = gcmc.load_workload(ctx, wl, gcmc.FP32)
    tal, cf, st = ctx.run_contrib(jobs[0], wl.grid.ncell, 1)
    assert abs(cf.sum() - tal[0]) <= 1e-12 * tal[0]          # integer sums of the same contributions
    ref = O.run(wl, wl.jobs[0], cf=True, nthreads=8)
    # FP32 marches: per-packet optical depths within ~1e-4, so cell shares agree to ~1e-4
    share, share_ref = cf[0, 0] / cf.sum(), ref["cf"][0, 0] / ref["cf"].sum()
    big = share_ref > 1e-3 * share_ref.max()
    np.testing.assert_allclose(share[big], share_ref[big], rtol=2e-3, atol=1e-7)
    # the tally of the contribution run equals the batched run's
    tb, _ = ctx.run_batch([jobs[0]])
    assert tb[0][0] == tal[0]


def test_contrib_refuses_transmission(ctx):
    from paper_2110_15640_gb300 import gcmc
    wl = S.config4_transmission(n_packets=100, nlon=12, nlat=6, nr=8, n_lam=60, n_lines=40, lam_subset=[20])
    _, _, _, jobs = gcmc.load_workload(ctx, wl, gcmc.FP32)
    with pytest.raises(gcmc.GcmcError):
        ctx.run_contrib(jobs[0], wl.grid.ncell, 1)
