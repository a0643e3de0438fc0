"""S9 on the GPU path: the library's host post-scale (gcmc_postscale) against the oracle's
(oracle.postscale) for all three modes (Sect. 5.1 transmission <I_p> and area, Sect. 5.2 geometric
albedo, Sect. 5.3 emission L_p, I_p, F_p).

Two comparisons per mode:
* the post-scale alone: both applied to the oracle's own tally, N and L_tot, so they must agree to
  FP64 rounding of a few products (1e-14 relative);
* the whole path: a job run on the FP64 CUDA path, its tally and L_tot post-scaled by the library,
  against the oracle's full run of the same packets.  The FP64 tally is a sum of per-packet f, each
  rounded to the 2^-32 fixed-point quantum (at most 2^-33 per packet), and L_tot agrees to 1e-13
  (the cell-table parity test), so each observable agrees to 1e-12 + N 2^-33 / tally relative."""
import pytest

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


def _cases():
    return [
        ("albedo", S.config1_albedo(n_packets=3000, nlon=8, nlat=6, nr=10)),
        ("emission", S.config2_emission(n_packets=4000, nlon=16, nlat=8, nr=12, nb=2, ng=2, bands=[1],
                                        gpoints=[1])),
        ("transmission", S.config4_transmission(n_packets=3000, nlon=12, nlat=6, nr=8, n_lam=60, n_lines=40,
                                                lam_subset=[20])),
    ]


# the library's observable field for each of the oracle's keys
_KEYS = {0: {"S": "S", "A_g_toa": "A_g", "A_g_R0": "A_g_R0"},
         1: {"L_p": "L_p", "I_p": "I_p", "F_p": "F_p"},
         2: {"I_p": "I_p", "area_over_pi": "area"}}


def _close(a, b, rt):
    return abs(a - b) <= rt * max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("name,wl", _cases(), ids=[c[0] for c in _cases()])
def test_postscale_matches_oracle(G, name, wl):
    from paper_2110_15640_gb300 import gcmc
    job = wl.jobs[0]
    gid, oid, sid, jobs = gcmc.load_workload(G, wl, gcmc.FP64)
    cells = O.prep_cells(wl, job)
    ref = O.run(wl, job, cells=cells, nthreads=8)
    n = job.n_packets
    l_tot_o = cells.get("L_tot", 0.0)
    want = O.postscale(wl, job, ref["tally"][0], n, cells=cells)
    # the post-scale alone, on the oracle's tally and L_tot
    got = G.postscale(gid, wl.mode, ref["tally"][0], n, l_tot_o)
    for ko, kg in _KEYS[wl.mode].items():
        assert _close(got[kg], float(want[ko]), 1e-14), (name, ko, got[kg], want[ko])
    # the whole FP64 path: GPU tally and L_tot through the library's post-scale
    t, st = G.run_packets(jobs[0])
    got2 = G.postscale(gid, wl.mode, t[0], n, st.l_tot)
    rt = 1e-12 + n * 2.0 ** -33 / abs(ref["tally"][0])
    for ko, kg in _KEYS[wl.mode].items():
        assert _close(got2[kg], float(want[ko]), rt), (name, ko, got2[kg], want[ko], rt)
    if wl.mode == 1:
        assert abs(st.l_tot / l_tot_o - 1) < 1e-13
