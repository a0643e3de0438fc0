"""Pins of the oracle's contribution functions (Sect. 6: CF = f(cell) / sum f, with separate thermal
and scattering counters), against what the geometry and the method fix:

* closure: the per-cell sums add up to the job's tally (every peel-off contribution is attributed to
  exactly one cell);
* the sums do not depend on the thread count (contributions are merged in packet order);
* an optically thin isothermal shell seen from +x: every visible cell emits the same luminosity per
  unit volume and its light escapes unattenuated, so the thermal CF per unit volume is uniform on the
  visible hemisphere; cells whose line of sight to +x runs into the black planet contribute nothing;
* single scattering in an optically thin shell lit and seen from +x: the scattering rate per unit
  volume is alpha F wherever the parallel beam reaches, so the scattered CF per unit volume is uniform
  on the lit hemisphere and zero where the planet blocks both the beam and the line of sight."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_15640_gb300 import synth as S


def _cell_geometry(grid):
    lat, lon, r = grid.lat_edges, grid.lon_edges, grid.r_edges
    latc = 0.5 * (lat[:-1] + lat[1:])
    lonc = 0.5 * (lon[:-1] + lon[1:])
    xdir = np.cos(latc)[:, None] * np.cos(lonc)[None, :]                  # [nlat][nlon]
    vol = ((r[1:] ** 3 - r[:-1] ** 3) / 3.0)[:, None, None] * \
        (np.sin(lat[1:]) - np.sin(lat[:-1]))[None, :, None] * np.diff(lon)[None, None, :]
    x = np.broadcast_to(xdir[None], (grid.nr, grid.nlat, grid.nlon)).reshape(-1)
    return x, vol.reshape(-1)


def test_cf_closure_and_thread_independence():
    wl = S.config1_albedo(n_packets=3000, nlon=8, nlat=6, nr=10)
    a = O.run(wl, wl.jobs[0], cf=True, nthreads=1)
    b = O.run(wl, wl.jobs[0], cf=True, nthreads=5)
    assert np.array_equal(a["cf"], b["cf"])
    assert abs(a["cf"].sum() / a["tally"][0] - 1) < 1e-12
    assert a["cf"][0].sum() == 0.0                        # albedo: every contribution is a scattering
    we = S.config2_emission(n_packets=2000, nlon=12, nlat=6, nr=8, nb=2, ng=2)
    e = O.run(we, we.jobs[1], cf=True, nthreads=3)
    assert abs(e["cf"][0].sum() / e["tally"][0] - 1) < 1e-12
    assert e["cf"][1].sum() == 0.0                        # no scattering after emission


def test_cf_thermal_thin_shell_uniform_per_volume():
    wl = S.isothermal_emitter(tau=2e-3, nlon=12, nlat=8, nr=2, n_packets=200_000)
    r = O.run(wl, wl.jobs[0], cf=True, nthreads=8)
    x, vol = _cell_geometry(wl.grid)
    th = r["cf"][0, 0]
    lit, dark = x > 0.45, x < -0.45          # whole cells on either side of the terminator
    per_vol = th[lit] / vol[lit]
    assert np.max(np.abs(per_vol / per_vol.mean() - 1)) < 0.02
    assert np.all(th[dark] == 0.0)


def test_cf_scattered_thin_shell_uniform_per_volume():
    wl = S.slab_sphere_albedo(omega=1.0, tau=2e-3, phase="iso", n_packets=12_000_000, nlon=12, nlat=8)
    r = O.run(wl, wl.jobs[0], cf=True, nthreads=8)
    x, vol = _cell_geometry(wl.grid)
    sc = r["cf"][1, 0]
    lit, dark = x > 0.45, x < -0.45          # whole cells on either side of the terminator
    per_vol = sc[lit] / vol[lit]
    # ~2e3 scatterings per lit cell (most packets cross the thin shell without interacting):
    # 4.5 sigma of the Monte Carlo noise is ~10%
    assert np.max(np.abs(per_vol / per_vol.mean() - 1)) < 0.10
    assert abs(np.mean(per_vol / per_vol.mean()) - 1) < 1e-12
    assert np.all(sc[dark] == 0.0)
