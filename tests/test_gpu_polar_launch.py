"""GPU regression: an emission packet launched with the largest launch uniform in the north pole band.

The FP32 launch samples c = 1 - |sin(lat)| linearly in a latitude band (Sect. 5.3's emission launch
point, uniform in volume within its cell).  Its largest uniform, 1 - 2^-25, rounds to 1 in FP32; at the
top of the north pole band that gave c = 0, or a hair below 0 through the rounding of the band edge, so
cos(lat) was not a number (or the point sat on the polar axis, where the longitude is undefined).  On
the 64 x 32 x 40 grid the edge rounds so that c < 0.  This test finds, by brute force over Philox
counters, a packet whose launch word gives that uniform, makes it the last packet of an emission job
(so its stratified target falls in the last cell of the pdf, which lies in the north pole band), and
runs it through every kernel form: its peel-off must match the FP64 oracle's packet and no job may
report a tally out of range.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S

pytestmark = pytest.mark.gpu

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)


def philox_words(n, event, key, seed):
    """Philox4x32-10 (Salmon et al. 2011) of the counters (n lo, n hi, event, key) under the 64-bit seed,
    vectorised over packet indices n (uint64 array); returns the four output words."""
    c0 = n & MASK
    c1 = n >> np.uint64(32)
    c2 = np.full_like(n, event)
    c3 = np.full_like(n, key)
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    for r in range(10):
        if r:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0), p1 & MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1), p0 & MASK)
    return c0, c1, c2, c3


def first_top_packet(seed, key, word, block=1 << 22, limit=1 << 28):
    """first packet index whose launch draw (event 0) has all top 24 bits of `word` set"""
    for start in range(0, limit, block):
        n = np.arange(start, start + block, dtype=np.uint64)
        w = philox_words(n, 0, key, seed)[word]
        hit = np.nonzero((w >> np.uint64(8)) == np.uint64(0xFFFFFF))[0]
        if hit.size:
            return int(n[hit[0]])
    raise AssertionError("no packet with the largest uniform below the search limit")


@pytest.fixture(scope="module")
def G():
    from paper_2110_15640_gb300 import build, gcmc
    build.build()
    ctx = gcmc.Context(0)
    yield ctx
    ctx.close()


def test_top_uniform_in_north_pole_band(G):
    from paper_2110_15640_gb300 import gcmc
    probe = S.config2_emission(n_packets=1, nlon=64, nlat=32, nr=40, nb=2, ng=2, bands=[1], gpoints=[1])
    seed, key = int(probe.seed), int(probe.jobs[0].key)
    n = first_top_packet(seed, key, word=2)        # word 2: the sin(lat) uniform of the launch
    w = O.philox([n & 0xFFFFFFFF, n >> 32, 0, key], [seed & 0xFFFFFFFF, seed >> 32])
    assert w[2] >> 8 == 0xFFFFFF                   # the search's Philox agrees with the oracle's

    wl = S.config2_emission(n_packets=n + 1, nlon=64, nlat=32, nr=40, nb=2, ng=2, bands=[1], gpoints=[1])
    job = wl.jobs[0]
    g = wl.grid
    ref = O.run(wl, job, packet0=n, n_run=1, per_packet=True, n_trace=1, max_trace=4000)
    cells_o = ref["tr_cell"][0, :ref["tr_n"][0]]
    first = cells_o[cells_o >= 0][0]
    assert (first // g.nlon) % g.nlat == g.nlat - 1     # launched in the north pole band

    gid, oid, sid, jobs = gcmc.load_workload(G, wl, gcmc.FP32)
    got = G.run_debug(jobs[0], packet0=n, n_run=1, n_trace=1, max_trace=4000)
    cells_g = got["tr_cell"][0, :got["tr_n"][0]]
    f_o, f_g = ref["pk_f"][0, 0], got["pk_f"][0, 0]
    print(f"packet {n}: oracle {len(cells_o)} segments f {f_o:.6e}; FP32 {len(cells_g)} segments f {f_g:.6e}")
    assert np.isfinite(got["pk_tau"][0]) and np.isfinite(f_g)
    assert np.array_equal(cells_g, cells_o)
    assert abs(f_g - f_o) <= 1e-3 * abs(f_o)
    assert got["stats"].flags == 0

    # the whole job through the plain and the batched kernels (fresh lane state, refilled lanes)
    tp, sp = G.run_packets(jobs[0])
    tb, sb = G.run_batch(jobs)
    assert sp.flags == 0 and sb[0].flags == 0
    assert sp.packets == sb[0].packets == n + 1
    assert tp[0] == tb[0][0] and np.isfinite(tp[0])
