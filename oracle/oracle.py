"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU
baseline are the only callers.  Nothing in the product package imports this module.

Also holds the oracle's own host post-scale (Sect. 5 of the paper): geometric albedo
A_g = pi S, phase function Phi = S(alpha)/S(0), emission L_p = (L_tot/N) sum f,
I_p = L_p / (pi R_TOA^2), F_p = pi I_p, and the transmission integral
<I_p> = (R_TOA - R0)/N sum W (1 - e^-tau) b with (R_p/R_star)^2 R_star^2 = R0^2 + 2 <I_p>.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAX_OBS = 32
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C11, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Grid_c(C.Structure):
    _fields_ = [("nlon", C.c_int32), ("nlat", C.c_int32), ("nr", C.c_int32), ("pad", C.c_int32),
                ("r_edges", C.POINTER(C.c_double)), ("lat_edges", C.POINTER(C.c_double)),
                ("lon_edges", C.POINTER(C.c_double))]


class Cells_c(C.Structure):
    _fields_ = [("alpha", C.POINTER(C.c_double)), ("omega", C.POINTER(C.c_double)),
                ("g", C.POINTER(C.c_double)), ("pgas", C.POINTER(C.c_double)),
                ("cdf", C.POINTER(C.c_double)), ("wcell", C.POINTER(C.c_double)),
                ("cdf_total", C.c_double), ("pad", C.c_double),
                ("ng", C.c_int32), ("pad2", C.c_int32), ("g_qcdf", C.POINTER(C.c_double)),
                ("g_w", C.POINTER(C.c_double)), ("g_cdftot", C.POINTER(C.c_double))]


class Source_c(C.Structure):
    _fields_ = [("star", C.c_double * 3), ("n_obs", C.c_int32), ("survival", C.c_int32),
                ("obs", (C.c_double * 3) * MAX_OBS),
                ("w_rr", C.c_double), ("p_surv", C.c_double), ("tau_peel_cut", C.c_double),
                ("tau_vert_max", C.c_double), ("beta_emis", C.c_double), ("hg_iso_eps", C.c_double),
                ("scatter_emission", C.c_int32), ("pad", C.c_int32), ("max_steps", C.c_int64),
                ("cloud_phase", C.c_int32), ("pad2", C.c_int32), ("surface_albedo", C.c_double),
                ("trans_scatter", C.c_int32), ("ld_law", C.c_int32), ("ld_coef", C.c_double * 4),
                ("star_radius", C.c_double), ("star_dist", C.c_double), ("transit_xy", C.c_double * 2),
                ("g_bias", C.c_int32), ("pad3", C.c_int32), ("g_beta", C.c_double),
                ("forced_first", C.c_int32), ("cont_abs", C.c_int32), ("path_bias", C.c_int32), ("pad4", C.c_int32)]


class Run_c(C.Structure):
    _fields_ = [("mode", C.c_int32), ("job_key", C.c_uint32), ("seed", C.c_uint64),
                ("n_packets", C.c_int64), ("packet0", C.c_int64), ("n_run", C.c_int64),
                ("nthreads", C.c_int32), ("n_trace", C.c_int32), ("max_trace", C.c_int32), ("pad", C.c_int32),
                ("tally", C.POINTER(C.c_double)), ("ledger", C.POINTER(C.c_double)),
                ("steps", C.POINTER(C.c_int64)), ("pk_f", C.POINTER(C.c_double)),
                ("pk_steps", C.POINTER(C.c_int64)), ("pk_tau", C.POINTER(C.c_double)),
                ("tr_cell", C.POINTER(C.c_int32)), ("tr_len", C.POINTER(C.c_double)),
                ("tr_n", C.POINTER(C.c_int32)), ("cf", C.POINTER(C.c_double)), ("tr_pos", C.POINTER(C.c_double))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            D, P = C.c_double, C.POINTER
            _lib.orc_philox.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            for name in ("orc_sample_iso", "orc_sample_rayleigh", "orc_phase_rayleigh"):
                getattr(_lib, name).argtypes = [D]
                getattr(_lib, name).restype = D
            _lib.orc_sample_hg.argtypes = [D, D, D]
            _lib.orc_sample_hg.restype = D
            _lib.orc_phase_hg.argtypes = [D, D]
            _lib.orc_phase_hg.restype = D
            _lib.orc_theta.argtypes = [D, D, D]
            _lib.orc_theta.restype = D
            _lib.orc_phase_tthg.argtypes = [D, D]
            _lib.orc_phase_tthg.restype = D
            _lib.orc_theta_kind.argtypes = [D, D, D, C.c_int]
            _lib.orc_theta_kind.restype = D
            _lib.orc_sample_cloud.argtypes = [D, D, D, D, C.c_int]
            _lib.orc_sample_cloud.restype = D
            _lib.orc_limb.argtypes = [C.c_int, P(D), D]
            _lib.orc_limb.restype = D
            _lib.orc_planck.argtypes = [D, D]
            _lib.orc_planck.restype = D
            _lib.orc_turn.argtypes = [P(D), D, D, P(D)]
            _lib.orc_trace_ray.argtypes = [P(Grid_c), P(D), P(D), P(D), C.c_int32, C.c_int32, C.c_int32,
                                           P(C.c_int32), P(D), P(C.c_int32)]
            _lib.orc_trace_ray.restype = C.c_int
            _lib.orc_prep_albedo.argtypes = [C.c_int64, P(D), P(D), D, D, D, D, D, P(D), P(D), P(D), P(D)]
            _lib.orc_prep_emission.argtypes = [P(Grid_c), P(D), P(D), P(D), P(C.c_float), C.c_int, C.c_int,
                                               P(D), P(D), D, D, D, P(D), P(D), P(D), P(D), P(D), P(D),
                                               P(C.c_int64)]
            _lib.orc_emission_tables.argtypes = [P(Grid_c), P(D), P(D), D, D, D, P(D), P(D), P(D), P(D), P(D),
                                                 P(C.c_int64)]
            _lib.orc_prep_xsec.argtypes = [P(Grid_c), P(D), P(D), P(D), P(D), P(C.c_float), C.c_int, C.c_int,
                                           C.c_int, P(D), P(D), P(D), D, D, D, D, P(D), P(D)]
            _lib.orc_run.argtypes = [P(Grid_c), P(Cells_c), P(Source_c), P(Run_c)]
            _lib.orc_run.restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _GridHandle:
    """Keeps the FP64 arrays alive while C holds pointers to them."""

    def __init__(self, grid):
        self.r = _f64(grid.r_edges)
        self.lat = _f64(grid.lat_edges)
        self.lon = _f64(grid.lon_edges)
        self.c = Grid_c(grid.nlon, grid.nlat, grid.nr, 0, _dp(self.r), _dp(self.lat), _dp(self.lon))


# ------------------------------------------------------------------ primitives

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (C.c_uint32 * 4)()
    lib().orc_philox(c, k, out)
    return [int(x) for x in out]


def sample_rayleigh(z):
    return lib().orc_sample_rayleigh(float(z))


def sample_hg(g, z, eps=1e-4):
    return lib().orc_sample_hg(float(g), float(z), float(eps))


def phase_hg(mu, g):
    return lib().orc_phase_hg(float(mu), float(g))


def phase_rayleigh(mu):
    return lib().orc_phase_rayleigh(float(mu))


def theta(mu, pgas, g):
    return lib().orc_theta(float(mu), float(pgas), float(g))


def phase_tthg(mu, g):
    return lib().orc_phase_tthg(float(mu), float(g))


def theta_kind(mu, pgas, g, kind):
    return lib().orc_theta_kind(float(mu), float(pgas), float(g), int(kind))


def sample_cloud(g, zc, z, kind, eps=1e-4):
    return lib().orc_sample_cloud(float(g), float(zc), float(z), float(eps), int(kind))


def limb(law, coef, mu):
    c = (C.c_double * 4)(*[float(v) for v in (list(coef) + [0.0] * 4)[:4]])
    return lib().orc_limb(int(law), c, float(mu))


def planck(lam, T):
    return lib().orc_planck(float(lam), float(T))


def turn(d, mu, psi):
    d = (C.c_double * 3)(*map(float, d))
    out = (C.c_double * 3)()
    lib().orc_turn(d, float(mu), float(psi), out)
    return np.array(list(out))


def trace_ray(grid, alpha, o, d, cell_flat, entry=-1, max_seg=100000):
    G = _GridHandle(grid)
    a = _f64(alpha)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    cells = np.zeros(max_seg, np.int32)
    lens = np.zeros(max_seg, np.float64)
    st = C.c_int32(0)
    n = lib().orc_trace_ray(C.byref(G.c), _dp(a), _dp(o), _dp(d), int(cell_flat), int(entry), int(max_seg),
                            cells.ctypes.data_as(C.POINTER(C.c_int32)), _dp(lens), C.byref(st))
    return cells[:n].copy(), lens[:n].copy(), int(st.value)


# ------------------------------------------------------------------ S1 cell tables

def prep_albedo(grid, opac, lam_idx):
    n = grid.ncell
    rho = _f64(grid.rho)
    acld = _f64(opac.acld) if opac.acld is not None else None
    out = {k: np.zeros(n) for k in ("alpha", "omega", "g", "pgas")}
    lib().orc_prep_albedo(n, _dp(rho), _dp(acld), float(opac.kabs[lam_idx]), float(opac.kray[lam_idx]),
                          float(opac.qcld[lam_idx]), float(opac.wcld[lam_idx]), float(opac.gcld[lam_idx]),
                          _dp(out["alpha"]), _dp(out["omega"]), _dp(out["g"]), _dp(out["pgas"]))
    return out


def prep_emission(grid, kt, band, gidx, opts):
    n = grid.ncell
    G = _GridHandle(grid)
    T, p, rho = _f64(grid.T), _f64(grid.p), _f64(grid.rho)
    sl = np.ascontiguousarray(kt.k[band, gidx], dtype=np.float32)
    Tg, pg = _f64(kt.Tg), _f64(kt.pg)
    out = {k: np.zeros(n) for k in ("alpha", "L", "cdf", "wcell")}
    Ltot, ctot, ninc = C.c_double(), C.c_double(), C.c_int64()
    lib().orc_prep_emission(C.byref(G.c), _dp(T), _dp(p), _dp(rho), sl.ctypes.data_as(C.POINTER(C.c_float)),
                            len(Tg), len(pg), _dp(Tg), _dp(pg), float(kt.lam[band]), float(opts.tau_vert_max),
                            float(opts.beta_emis), _dp(out["alpha"]), _dp(out["L"]), _dp(out["cdf"]),
                            _dp(out["wcell"]), C.byref(Ltot), C.byref(ctot), C.byref(ninc))
    out.update(L_tot=Ltot.value, cdf_total=ctot.value, n_incl=ninc.value)
    return out


def prep_emission_xsec(grid, xs, lam_idx, opts):
    """Emission cell tables on cross-section opacities (high resolution, Sect. 7): alpha from the
    Doppler-shifted cross-sections of each cell, then the same tau_vert cut, luminosities and hybrid pdf
    as with k-tables, with B at the job's rest wavelength."""
    n = grid.ncell
    G = _GridHandle(grid)
    alpha = _f64(prep_xsec(grid, xs, lam_idx)["alpha"])
    T = _f64(grid.T)
    out = {k: np.zeros(n) for k in ("L", "cdf", "wcell")}
    Ltot, ctot, ninc = C.c_double(), C.c_double(), C.c_int64()
    lib().orc_emission_tables(C.byref(G.c), _dp(T), _dp(alpha), float(xs.lam[lam_idx]), float(opts.tau_vert_max),
                              float(opts.beta_emis), _dp(out["L"]), _dp(out["cdf"]), _dp(out["wcell"]),
                              C.byref(Ltot), C.byref(ctot), C.byref(ninc))
    out.update(alpha=alpha, L_tot=Ltot.value, cdf_total=ctot.value, n_incl=ninc.value)
    return out


def prep_xsec(grid, xs, lam_idx):
    n = grid.ncell
    G = _GridHandle(grid)
    T, p, rho = _f64(grid.T), _f64(grid.p), _f64(grid.rho)
    wind = _f64(grid.wind.reshape(-1)) if grid.wind is not None else None
    sig = np.ascontiguousarray(xs.sigma, dtype=np.float32)
    lamg, Tg, pg = _f64(xs.lam), _f64(xs.Tg), _f64(xs.pg)
    alpha = np.zeros(n)
    vlos = np.zeros(n)
    lib().orc_prep_xsec(C.byref(G.c), _dp(T), _dp(p), _dp(rho), _dp(wind), sig.ctypes.data_as(C.POINTER(C.c_float)),
                        len(lamg), len(Tg), len(pg), _dp(lamg), _dp(Tg), _dp(pg), float(xs.lam[lam_idx]),
                        float(xs.view_theta), float(xs.view_phi), float(xs.omega_rot), _dp(alpha), _dp(vlos))
    return {"alpha": alpha, "vlos": vlos}


def prep_cells(wl, job):
    """S1 for one job of a workload (dispatch on the opacity kind)."""
    if wl.mode == 0:
        return prep_albedo(wl.grid, wl.opac, job.lam_idx)
    if wl.mode == 1:
        if not hasattr(wl.opac, "wg"):
            return prep_emission_xsec(wl.grid, wl.opac, job.lam_idx, wl.source.opts)
        if job.g_idx < 0:
            return prep_band(wl, job)
        return prep_emission(wl.grid, wl.opac, job.lam_idx, job.g_idx, wl.source.opts)
    if hasattr(wl.opac, "kray"):
        # transmission through scattering opacities (gas + clouds at the job's wavelength)
        return prep_albedo(wl.grid, wl.opac, job.lam_idx)
    return prep_xsec(wl.grid, wl.opac, job.lam_idx)


def g_table(wg, L_g, bias=0, beta=0.5):
    """Per-packet g-ordinate sampling (Sect. 4.7) of an emission band: unbiased p(g) = w_g L_g / sum w L;
    the sampling pdf q(g) = p(g) (bias 0), 1/N_g (bias 1, uniform) or (1 - beta) p(g) + beta / N_g
    (bias 2, composite); each packet of ordinate g carries W_g = p(g) / q(g)."""
    wg = np.asarray(wg, np.float64)
    L_g = np.asarray(L_g, np.float64)
    ng = len(wg)
    wl_ = wg * L_g
    p = wl_ / wl_.sum()
    if bias == 0:
        q = p.copy()
    elif bias == 1:
        q = np.full(ng, 1.0 / ng)
    else:
        q = (1.0 - beta) * p + beta / ng
    W = np.where(q > 0, p / np.where(q > 0, q, 1.0), 0.0)
    return {"p": p, "q": q, "W": W, "qcdf": np.cumsum(q), "L_band": float(wl_.sum())}


def prep_band(wl, job):
    """S1 of an emission band job with per-packet g sampling: every g-ordinate's cell tables and the
    g table; tables are concatenated [g][ncell]."""
    op = wl.source.opts
    ng = len(wl.opac.wg)
    per = [prep_emission(wl.grid, wl.opac, job.lam_idx, g, op) for g in range(ng)]
    gt = g_table(wl.opac.wg, [c["L_tot"] for c in per], int(getattr(op, "g_bias", 0)),
                 float(getattr(op, "g_beta", 0.5)))
    out = {k: np.concatenate([c[k] for c in per]) for k in ("alpha", "L", "cdf", "wcell")}
    out.update(per_g=per, gtab=gt, L_tot=gt["L_band"], cdf_total=1.0,
               cdf_tot_g=np.array([c["cdf_total"] for c in per]))
    return out


# ------------------------------------------------------------------ packets

def _source_struct(src, obs):
    s = Source_c()
    for i in range(3):
        s.star[i] = float(src.star[i])
    obs = np.atleast_2d(np.asarray(obs, np.float64))
    if len(obs) > MAX_OBS:
        raise ValueError("too many observer directions")
    s.n_obs = len(obs)
    for o in range(len(obs)):
        for i in range(3):
            s.obs[o][i] = float(obs[o][i])
    op = src.opts
    s.survival = int(op.survival)
    s.w_rr, s.p_surv, s.tau_peel_cut = float(op.w_rr), float(op.p_surv), float(op.tau_peel_cut)
    s.tau_vert_max, s.beta_emis, s.hg_iso_eps = float(op.tau_vert_max), float(op.beta_emis), float(op.hg_iso_eps)
    s.scatter_emission = int(op.scatter_emission)
    s.max_steps = int(op.max_steps)
    s.cloud_phase = int(getattr(op, "cloud_phase", 0))
    s.surface_albedo = float(getattr(op, "surface_albedo", 0.0))
    s.trans_scatter = int(getattr(op, "trans_scatter", 0))
    s.ld_law = int(getattr(op, "ld_law", 0))
    for i, v in enumerate((list(getattr(op, "ld_coef", ())) + [0.0] * 4)[:4]):
        s.ld_coef[i] = float(v)
    s.star_radius = float(getattr(op, "star_radius", 0.0))
    s.star_dist = float(getattr(op, "star_dist", 0.0))
    for i, v in enumerate(getattr(op, "transit_xy", (0.0, 0.0))):
        s.transit_xy[i] = float(v)
    s.forced_first = int(getattr(op, "forced_first", 0))
    s.cont_abs = int(getattr(op, "cont_abs", 0))
    s.path_bias = int(getattr(op, "path_bias", 0))
    return s, len(obs)


def tally_cols(wl, job):
    """Tally columns of a job: one per observer (albedo, emission); transmission: the chord column,
    plus the scattered-light column when packets scatter after their chord."""
    if wl.mode == 2:
        return 2 if int(getattr(wl.source.opts, "trans_scatter", 0)) else 1
    return len(job_observers(wl, job))


def job_observers(wl, job):
    obs = np.atleast_2d(wl.source.obs)
    if getattr(job, "obs_idx", -1) >= 0:
        return obs[job.obs_idx:job.obs_idx + 1]
    return obs


def run(wl, job, cells=None, packet0=0, n_run=None, nthreads=1, per_packet=False, n_trace=0, max_trace=0, cf=False,
        trace_pos=False):
    """Run packets of one job through the oracle; returns tallies, ledger, step count and
    (optionally) per-packet f, steps, tau and segment traces, and the contribution-function sums
    (Sect. 6): cf[kind][obs][cell] = sum of the peel-off contributions f leaving from the cell,
    kind 0 thermal (emission launch), 1 scattered.  trace_pos adds tr_pos [n_trace][max_trace][3]: the
    end point of each traced segment, and at a march start (cell < 0) the point it starts from."""
    if cells is None:
        cells = prep_cells(wl, job)
    G = _GridHandle(wl.grid)
    keep = {k: _f64(cells.get(k)) for k in ("alpha", "omega", "g", "pgas", "cdf", "wcell")}
    gt = cells.get("gtab")
    if gt is not None:
        keep.update(qcdf=_f64(gt["qcdf"]), gw=_f64(gt["W"]), gct=_f64(cells["cdf_tot_g"]))
    cc = Cells_c(_dp(keep["alpha"]), _dp(keep["omega"]), _dp(keep["g"]), _dp(keep["pgas"]), _dp(keep["cdf"]),
                 _dp(keep["wcell"]), float(cells.get("cdf_total", 0.0)), 0.0,
                 len(gt["qcdf"]) if gt is not None else 0, 0, _dp(keep.get("qcdf")), _dp(keep.get("gw")),
                 _dp(keep.get("gct")))
    obs = job_observers(wl, job)
    sc, nobs = _source_struct(wl.source, obs)
    ncol = tally_cols(wl, job)
    n_run = job.n_packets - packet0 if n_run is None else int(n_run)
    tally = np.zeros(ncol)
    ledger = np.zeros(8)
    steps = np.zeros(1, np.int64)
    pk_f = np.zeros((n_run, ncol)) if per_packet else None
    pk_steps = np.zeros(n_run, np.int64) if per_packet else None
    pk_tau = np.zeros(n_run) if per_packet else None
    n_trace = min(int(n_trace), n_run)
    tr_cell = np.zeros((n_trace, max_trace), np.int32) if n_trace else None
    tr_len = np.zeros((n_trace, max_trace)) if n_trace else None
    tr_n = np.zeros(n_trace, np.int32) if n_trace else None
    tr_pos = np.zeros((n_trace, max_trace, 3)) if n_trace and trace_pos else None
    cfa = np.zeros((2, nobs, wl.grid.ncell)) if cf else None
    ip = lambda a, t: a.ctypes.data_as(C.POINTER(t)) if a is not None else None  # noqa: E731
    ra = Run_c(int(wl.mode), int(job.key) & 0xFFFFFFFF, int(wl.seed), int(job.n_packets), int(packet0), n_run,
               int(nthreads), n_trace, int(max_trace), 0, _dp(tally), _dp(ledger), ip(steps, C.c_int64),
               _dp(pk_f), ip(pk_steps, C.c_int64), _dp(pk_tau), ip(tr_cell, C.c_int32), _dp(tr_len),
               ip(tr_n, C.c_int32), _dp(cfa), _dp(tr_pos))
    rc = lib().orc_run(C.byref(G.c), C.byref(cc), C.byref(sc), C.byref(ra))
    if rc != 0:
        raise RuntimeError(f"oracle run failed: {rc}")
    out = dict(tally=tally, ledger=ledger, steps=int(steps[0]), n_run=n_run, cells=cells)
    if per_packet:
        out.update(pk_f=pk_f, pk_steps=pk_steps, pk_tau=pk_tau)
    if n_trace:
        out.update(tr_cell=tr_cell, tr_len=tr_len, tr_n=tr_n)
        if tr_pos is not None:
            out["tr_pos"] = tr_pos
    if cf:
        out["cf"] = cfa
    return out


# ------------------------------------------------------------------ S9 host post-scale (Sect. 5)

def postscale(wl, job, tally_sum, n_packets, cells=None):
    """Observables from one job's tally sum (sum over packets of f)."""
    g = wl.grid
    if wl.mode == 0:
        S = np.asarray(tally_sum) / n_packets
        return {"S": S, "A_g_toa": math.pi * S, "A_g_R0": math.pi * S * (g.R_toa / g.R0) ** 2}
    if wl.mode == 1:
        Ltot = cells["L_tot"]
        Lp = Ltot / n_packets * np.asarray(tally_sum)
        Ip = Lp / (math.pi * g.R_toa ** 2)
        return {"L_p": Lp, "I_p": Ip, "F_p": math.pi * Ip}
    Ip = (g.R_toa - g.R0) / n_packets * g.R_toa * np.asarray(tally_sum)
    return {"I_p": Ip, "area_over_pi": g.R0 ** 2 + 2.0 * Ip}

def transit(wl, tally, n_packets):
    """Transit observables (Sect. 5.1) from a transmission job's tally columns (chord, scattered).

    I_p = (R_TOA - R0)/N R_TOA (T_chord - Omega_star T_scat): the scattered light is the packets' power
    per steradian towards the observer, relative to the stellar intensity times the solid angle
    Omega_star of the stellar disk seen from the planet.  With limb darkening the planet's opaque
    core blocks the intensity at the planet centre, and the depth divides by the disk-averaged
    intensity 2 int_0^1 mu I(mu)/I(1) dmu."""
    from scipy import integrate
    g, op = wl.grid, wl.source.opts
    k = (g.R_toa - g.R0) / n_packets * g.R_toa
    t = np.atleast_1d(np.asarray(tally, np.float64))
    I_dir = k * t[0]
    I_sca = k * t[1] if len(t) > 1 else 0.0
    Rs, a = float(getattr(op, "star_radius", 0.0)), float(getattr(op, "star_dist", 0.0))
    omega_star = 2.0 * math.pi * (1.0 - math.sqrt(1.0 - (Rs / a) ** 2)) if a > Rs > 0 else 0.0
    I_p = I_dir - omega_star * I_sca
    law, coef = int(getattr(op, "ld_law", 0)), list(getattr(op, "ld_coef", (0.0,) * 4))
    if law:
        q = (op.transit_xy[0] ** 2 + op.transit_xy[1] ** 2) / Rs ** 2
        w_core = limb(law, coef, math.sqrt(1.0 - q)) if q < 1.0 else 0.0
        n_ld = integrate.quad(lambda m: 2.0 * m * limb(law, coef, m), 0.0, 1.0, epsabs=1e-13, epsrel=1e-12)[0]
    else:
        w_core, n_ld = 1.0, 1.0
    area = w_core * g.R0 ** 2 + 2.0 * I_p
    return {"I_p_direct": I_dir, "I_p_scattered": I_sca, "omega_star": omega_star, "I_p": I_p,
            "w_core": w_core, "n_ld": n_ld, "area_over_pi": area,
            "depth": area / (Rs ** 2 * n_ld) if Rs > 0 else float("nan")}
