"""Where the FP32 march leaves the FP64 oracle's cell sequence, and why.

The FP32 path rounds positions to FP32: at the planet's radius (~7e7 m) one unit in the last place
is 8 m, so a launch or interaction point carries a few metres of rounding, and optical depths are
accumulated in FP32.  A packet can then take another cell sequence than the oracle's only where its
ray passes within metres of a face (or, after scatterings, where the rounding has accumulated).  This
test runs 20,000 packets of each workload through the FP32 CUDA path (through the C ABI) and the oracle
on the same Philox streams, compares the per-packet segment lists, and checks every packet that leaves
the per-packet bar or whose cell sequence differs:

* Divergent packets.  At the first differing segment, the oracle's ray (its positions are logged)
  and the GPU's leave the last common cell C at along-ray positions s_o and s_g; between them one side
  places the ray in C, the other in the neighbour X beyond the face F between them.  Where the oracle's
  ray went beyond F, the depth it reached beyond F over that interval (a grazing dip below a shell is
  shallow however long); where the GPU's went beyond F, how close the oracle's ray came to F.  On packets
  that have not scattered (emission peel-offs, limb chords) that distance must lie within a rounding bound
  (normal to F): DELTA_X = 64 m (8 FP32 ulps at the planetary radius) for shells and
  half-planes; for cones DELTA_X plus the resolution of FP32 sin(latitude) (EPS32 / cos(latitude) radians:
  90 m at latitude 87 degrees).  On packets that have scattered, the FP32 ray may have drifted by the
  accumulated length differences D of the flights before it (interaction points are placed from FP32
  optical depths), so the bound grows by D; or the interval holds no more optical depth than the FP32
  accumulation error of the flight.
* Packets outside the per-packet bar with identical cell sequences (their optical depths differ by more
  than 1e-4 relative because segment lengths differ: mostly peel-offs past the cut-off depth, where a
  segment holds tens of optical depths, and rays that cross a latitude cone or a shell at a grazing
  angle, where a crossing moves along the ray by up to kilometres for metres of rounding).  Following
  each ray along the oracle's line by the GPU's own segment lengths, every crossing point must lie
  within that bound of the face it crosses, measured normal to that face (plus D after scatterings).

The measured fractions of identical cell sequences are printed: on a GB300 they were 0.99995 (emission
16 x 8 x 12), 0.99995 (emission 128 x 64 x 50), 1.0 (transmission), 0.99985 (albedo) and 0.99845
(transit with multiple scattering).  The asserted floors are 0.9999 for packets that do not scatter and
0.998 for packets that do."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S

pytestmark = pytest.mark.gpu

N = 20000
MAX_TRACE = 1500
DELTA_X = 64.0          # m: 8 FP32 ulps at 7e7 m (a launch point carries several roundings of its coordinates)
EPS32 = 2.0 ** -24


def _face_bound(face):
    """How far from a face the FP32 march can place its crossing: DELTA_X of position rounding, and for a
    latitude cone the resolution of FP32 sin(latitude) (of the edge and of the ray): an error of EPS32 in a
    sine is an angle of EPS32 / cos(latitude), which near the poles is far more than an ulp of position
    (1.2e-6 rad, 90 m at R_J, at latitude 87 degrees)"""
    if face[0] == "lat":
        return DELTA_X + 4.0 * EPS32 * 8.0e7 / max(abs(math.cos(face[1])), 1e-3)
    return DELTA_X


@pytest.fixture(scope="module")
def G():
    from paper_2110_15640_gb300 import build, gcmc
    build.build()
    ctx = gcmc.Context(0)
    yield ctx
    ctx.close()


# ------------------------------------------------------------------ geometry of the oracle's logged rays

def _ijk(grid, c):
    return c % grid.nlon, (c // grid.nlon) % grid.nlat, c // (grid.nlon * grid.nlat)


def _face(grid, c, x):
    """the face between cell c and its neighbour x: ('r', radius), ('lat', latitude) or ('lon', longitude)"""
    ic, jc, kc = _ijk(grid, c)
    ix, jx, kx = _ijk(grid, x)
    if kx != kc:
        return ("r", grid.r_edges[max(kc, kx)])
    if jx != jc:
        return ("lat", grid.lat_edges[max(jc, jx)])
    return ("lon", grid.lon_edges[ic + 1] if (ic + 1) % grid.nlon == ix else grid.lon_edges[ic])


def _dist(face, P):
    """normal distance of points P [..., 3] from a face"""
    kind, v = face
    if kind == "r":
        return np.abs(np.linalg.norm(P, axis=-1) - v)
    if kind == "lat":
        lat = np.arctan2(P[..., 2], np.hypot(P[..., 0], P[..., 1]))
        return np.linalg.norm(P, axis=-1) * np.abs(np.sin(lat - v))
    return np.abs(-math.sin(v) * P[..., 0] + math.cos(v) * P[..., 1])


def _depth(grid, c, x, face, P):
    """signed distance of points P beyond face F (between cell c and its neighbour x), positive on x's side"""
    kind, v = face
    ic, jc, kc = _ijk(grid, c)
    ix, jx, kx = _ijk(grid, x)
    if kind == "r":
        d = np.linalg.norm(P, axis=-1) - v
        return -d if kx < kc else d
    if kind == "lat":
        lat = np.arctan2(P[..., 2], np.hypot(P[..., 0], P[..., 1]))
        d = np.linalg.norm(P, axis=-1) * np.sin(lat - v)
        return d if jx > jc else -d
    d = -math.sin(v) * P[..., 0] + math.cos(v) * P[..., 1]
    return d if (ic + 1) % grid.nlon == ix else -d


def _rays(cells):
    """(start, end) index ranges of the rays of a trace (a ray starts at a marker < 0)"""
    starts = [q for q, c in enumerate(cells) if c < 0] + [len(cells)]
    return list(zip(starts[:-1], starts[1:]))


def _divergence(grid, alpha, co, lo, po, cg, lg, multi):
    """returns (ok, info) for a packet whose cell sequences differ"""
    no, ng = len(co), len(cg)
    m = next((q for q in range(min(no, ng)) if co[q] != cg[q]), min(no, ng))
    st = max(q for q in range(m) if co[q] < 0)
    if m == st + 1:       # the two sides disagree on a ray's first cell (cannot happen after a match)
        return False, dict(m=m, kind="start")
    # drift: length differences of the flights (rays of kind -1 or -4) before this ray, and of this ray's
    # segments before the divergence
    D = 0.0
    for a, b in _rays(co[:st]):
        if co[a] in (-1, -4):
            D += float(np.abs(lo[a + 1:b] - lg[a + 1:b]).sum())
    D += float(np.abs(lo[st + 1:m - 1] - lg[st + 1:m - 1]).sum())
    C = int(co[m - 1])
    P0 = po[st]
    d = (po[st + 1] - P0) / np.linalg.norm(po[st + 1] - P0)
    so, sg = float(lo[st + 1:m].sum()), float(lg[st + 1:m].sum())
    A = int(co[m]) if m < no else -9
    B = int(cg[m]) if m < ng else -9
    X = A if so <= sg else B
    s = np.linspace(min(so, sg), max(so, sg), 65)
    P = P0[None, :] + s[:, None] * d[None, :]
    if X >= 0:
        face = _face(grid, C, X)
        dep = _depth(grid, C, X, face, P)
        if so <= sg:
            # the oracle's ray went beyond F into X while the GPU's stayed in C: how deep beyond F it went
            # (a grazing dip below a shell is shallow however long the dip)
            dist = float(max(dep.max(), 0.0))
        else:
            # the GPU's ray went beyond F while the oracle's stayed in C: how close the oracle's ray came to F
            dist = float(max(-dep.max(), 0.0))
    else:   # that side's ray ended there: at a boundary shell, or (interaction, cut-off) inside C
        r_end = float(np.linalg.norm(P0 + min(so, sg) * d))
        face = ("r", grid.r_edges[-1] if abs(r_end - grid.r_edges[-1]) < abs(r_end - grid.r_edges[0]) else grid.r_edges[0])
        dist = float(_dist(face, P).max())
    fb = _face_bound(face)
    dtau = float(alpha[C]) * abs(so - sg)
    tau_ray = float(np.dot(alpha[np.maximum(co[st + 1:m], 0)], lo[st + 1:m]))
    info = dict(m=int(m), face=face[0], dist=dist, bound=fb, drift=D, dtau=dtau, tau=tau_ray)
    if not multi:
        return dist <= fb, info
    # optical depth the FP32 flight may be off by at C: the optical depth of its length differences so far,
    # C's share of the drift, the FP32 accumulation (one rounding per step) and -ln of the FP32 draw
    dl = np.abs(lo[st + 1:m - 1] - lg[st + 1:m - 1])
    tau_bound = (float(np.dot(alpha[co[st + 1:m - 1]], dl)) + float(alpha[C]) * (fb + D)
                 + (m - st) * 2.0 ** -22 * max(tau_ray, 1.0) + 1e-6)
    info["tau_bound"] = tau_bound
    return dist <= fb + D or dtau <= tau_bound, info


def _cell_faces(grid, c):
    """the six faces of cell c (the poles and a single longitude cell have no face there)"""
    i, j, k = _ijk(grid, c)
    f = [("r", grid.r_edges[k]), ("r", grid.r_edges[k + 1])]
    if j > 0:
        f.append(("lat", grid.lat_edges[j]))
    if j + 1 < grid.nlat:
        f.append(("lat", grid.lat_edges[j + 1]))
    if grid.nlon > 1:
        f += [("lon", grid.lon_edges[i]), ("lon", grid.lon_edges[i + 1])]
    return f


def _crossings_on_faces(grid, co, lo, po, lg, multi):
    """Identical cell sequences: where the GPU's FP32 march crosses each face.  Every ray is followed along
    the oracle's line (its logged start point and direction) by the GPU's own cumulative segment lengths;
    each crossing point found that way must lie within the face's rounding bound (_face_bound) of the face
    it crosses, measured normal to the face.  (Along the ray, a crossing at a grazing angle can move by kilometres for metres of position
    or coefficient rounding; normal to the face it cannot.)  After scatterings the ray's start may have
    drifted by the length differences D of the flights before it: the bound is the face's + D.  Segments that
    end in an interaction (their length follows the sampled optical depth) are skipped.  Returns the worst
    ratio of distance to bound."""
    worst, drift = 0.0, 0.0
    for a, b in _rays(co):
        d_ray = drift if multi else 0.0
        if co[a] in (-1, -4):
            drift += float(np.abs(lo[a + 1:b] - lg[a + 1:b]).sum())
        if b - a < 2:
            continue
        P0 = po[a]
        d = po[b - 1] - P0
        if np.linalg.norm(d) == 0.0:
            continue
        d = d / np.linalg.norm(d)
        sg = 0.0
        for q in range(a + 1, b):
            sg += float(lg[q])
            if q + 1 < b:
                face = _face(grid, int(co[q]), int(co[q + 1]))
            else:
                # the ray's last segment: ends on a face of its cell (escape, bottom, a cut-off after the crossing)
                # or inside it (an interaction)
                faces = _cell_faces(grid, int(co[q]))
                dd = [float(_dist(f, po[q])) for f in faces]
                if min(dd) > 1e-3:
                    continue
                face = faces[int(np.argmin(dd))]
            worst = max(worst, float(_dist(face, P0 + sg * d)) / (_face_bound(face) + d_ray))
    return worst


CASES = [
    ("albedo_8x6x10", lambda: S.config1_albedo(n_packets=N, nlon=8, nlat=6, nr=10), True),
    ("emission_16x8x12", lambda: S.config2_emission(n_packets=N, nlon=16, nlat=8, nr=12, nb=2, ng=2, bands=[1],
                                                     gpoints=[1]), False),
    ("transmission_12x6x8", lambda: S.config4_transmission(n_packets=N, nlon=12, nlat=6, nr=8, n_lam=60, n_lines=40,
                                                           lam_subset=[20]), False),
    ("emission_128x64x50", lambda: S.config2_emission(n_packets=1_000_000, bands=[7], gpoints=[5]), False),
    ("transit_scatter_32x16x20", lambda: S.config6_transit_scatter(nlon=32, nlat=16, nr=20, nlam=1, n_packets=N), True),
]


@pytest.mark.parametrize("name,maker,multi", CASES, ids=[c[0] for c in CASES])
def test_fp32_divergences_are_rounding(G, name, maker, multi):
    from paper_2110_15640_gb300 import gcmc
    wl = maker()
    job = wl.jobs[0]
    _, _, _, jobs = gcmc.load_workload(G, wl, gcmc.FP32)
    cells = O.prep_cells(wl, job)
    alpha = np.asarray(cells["alpha"], np.float64)
    ncol = O.tally_cols(wl, job)
    ref = O.run(wl, job, cells=cells, n_run=N, per_packet=True, n_trace=N, max_trace=MAX_TRACE, nthreads=16)
    got = G.run_debug(jobs[0], n_run=N, n_trace=N, max_trace=MAX_TRACE, n_obs=ncol)
    assert int(ref["tr_n"].max()) < MAX_TRACE and int(got["tr_n"].max()) < MAX_TRACE
    # the per-packet bar of the FP32 parity test
    if wl.mode == 0:
        f_o, f_g = ref["pk_f"][:, 0], got["pk_f"][:, 0]
        outside = np.abs(f_g - f_o) > 1e-3 * np.abs(f_o) + 1e-300
    else:
        t_o, t_g = ref["pk_tau"], got["pk_tau"]
        outside = np.abs(t_g - t_o) > 1e-4 * t_o + 1e-5
    same = np.array([ref["tr_n"][q] == got["tr_n"][q] and
                     np.array_equal(ref["tr_cell"][q, :ref["tr_n"][q]], got["tr_cell"][q, :got["tr_n"][q]])
                     for q in range(N)])
    bad, infos, worst_len, n_same_out = [], [], 0.0, 0
    for q in np.nonzero(~same | outside)[0]:
        one = O.run(wl, job, cells=cells, packet0=int(q), n_run=1, n_trace=1, max_trace=MAX_TRACE, trace_pos=True)
        n1 = int(one["tr_n"][0])
        co, lo, po = one["tr_cell"][0, :n1], one["tr_len"][0, :n1], one["tr_pos"][0, :n1]
        ng = int(got["tr_n"][q])
        cg, lg = got["tr_cell"][q, :ng], got["tr_len"][q, :ng]
        if same[q]:
            w = _crossings_on_faces(wl.grid, co, lo, po, lg, multi)
            worst_len = max(worst_len, w)
            n_same_out += 1
            if w > 1.0:
                bad.append((int(q), "crossing off its face", w))
        else:
            ok, info = _divergence(wl.grid, alpha, co, lo, po, cg, lg, multi)
            infos.append(info)
            if not ok:
                bad.append((int(q), info))
    frac = float(same.mean())
    print(f"FP32 {name}: identical cell sequences {frac:.5f} ({int((~same).sum())} of {N} differ); "
          f"outside the per-packet bar {int(outside.sum())} ({n_same_out} with identical cells: worst crossing "
          f"distance / bound {worst_len:.3f}); divergences "
          + "; ".join(f"{i['face']} d={i.get('dist', float('nan')):.1f} m drift={i.get('drift', 0):.1f} m" for i in infos[:8]))
    assert not bad, bad[:5]
    assert frac >= (0.998 if multi else 0.9999)
