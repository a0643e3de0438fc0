"""Python binding of libgcmc (include/gcmc.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays / torch tensors
into the C descriptors and back.  Importing it loads libgcmc.so from this package directory and
raises if the library has not been built (build with `python -m paper_2110_15640_gb300.build`).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgcmc.so")
MAX_OBS = 8

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STEP_CAP, ERR_TIMEOUT, ERR_NOT_READY, ERR_NAN, ERR_RANGE = 0, -1, -2, -3, -4, -5, -6, -7, -8
ALBEDO, EMISSION, TRANSMISSION = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
FP32, FP64 = 0, 1
OPAC_ALBEDO, OPAC_KTABLE, OPAC_XSEC = 0, 1, 2

PD = C.POINTER(C.c_double)
PF = C.POINTER(C.c_float)


class gcmc_grid_desc(C.Structure):
    _fields_ = [("nlon", C.c_int32), ("nlat", C.c_int32), ("nr", C.c_int32), ("memory", C.c_int32),
                ("r_edges", C.c_void_p), ("lat_edges", C.c_void_p), ("lon_edges", C.c_void_p),
                ("T", C.c_void_p), ("p", C.c_void_p), ("rho", C.c_void_p), ("wind", C.c_void_p)]


class gcmc_opacity_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("memory", C.c_int32), ("nlam", C.c_int32),
                ("kabs", C.c_void_p), ("kray", C.c_void_p), ("qcld", C.c_void_p), ("wcld", C.c_void_p),
                ("gcld", C.c_void_p), ("acld", C.c_void_p),
                ("nb", C.c_int32), ("ng", C.c_int32), ("nT", C.c_int32), ("np", C.c_int32),
                ("lam", C.c_void_p), ("Tg", C.c_void_p), ("pg", C.c_void_p), ("k", C.c_void_p),
                ("nl", C.c_int32), ("pad", C.c_int32), ("xlam", C.c_void_p), ("sigma", C.c_void_p),
                ("view_theta", C.c_double), ("view_phi", C.c_double), ("omega_rot", C.c_double),
                ("gw", C.c_void_p)]


class gcmc_source_desc(C.Structure):
    _fields_ = [("star", C.c_double * 3), ("n_obs", C.c_int32), ("survival", C.c_int32),
                ("obs", (C.c_double * 3) * MAX_OBS), ("w_rr", C.c_double), ("p_surv", C.c_double),
                ("tau_peel_cut", C.c_double), ("tau_vert_max", C.c_double), ("beta_emis", C.c_double),
                ("hg_iso_eps", C.c_double), ("scatter_emission", C.c_int32), ("precision", C.c_int32),
                ("max_steps", C.c_int64), ("cloud_phase", C.c_int32), ("pad2", C.c_int32),
                ("surface_albedo", C.c_double), ("trans_scatter", C.c_int32), ("ld_law", C.c_int32),
                ("ld_coef", C.c_double * 4), ("star_radius", C.c_double), ("star_dist", C.c_double),
                ("transit_xy", C.c_double * 2), ("g_bias", C.c_int32), ("pad3", C.c_int32),
                ("g_beta", C.c_double), ("forced_first", C.c_int32), ("cont_abs", C.c_int32),
                ("path_bias", C.c_int32), ("pad4", C.c_int32)]


class gcmc_stats(C.Structure):
    _fields_ = [("packets", C.c_int64), ("steps", C.c_int64), ("ledger", C.c_double * 8), ("l_tot", C.c_double),
                ("cdf_total", C.c_double), ("n_emit_cells", C.c_int64), ("flags", C.c_int64)]


class gcmc_job(C.Structure):
    _fields_ = [("grid_id", C.c_int32), ("opac_id", C.c_int32), ("source_id", C.c_int32), ("mode", C.c_int32),
                ("lam_idx", C.c_int32), ("g_idx", C.c_int32), ("obs_idx", C.c_int32), ("job_key", C.c_uint32),
                ("n_packets", C.c_int64), ("seed", C.c_uint64)]


class gcmc_launch_cfg(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("chunk", C.c_int32), ("interval", C.c_int32),
                ("refill_min", C.c_int32), ("pad", C.c_int32)]


class gcmc_server_cfg(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("chunk", C.c_int32), ("interval", C.c_int32),
                ("refill_min", C.c_int32), ("max_jobs", C.c_int32), ("hbm_budget", C.c_uint64),
                ("idle_us", C.c_int32), ("pad", C.c_int32)]


class gcmc_server_stats(C.Structure):
    _fields_ = [("pending", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("bytes_in_use", C.c_uint64), ("kernel_launches", C.c_int64), ("kernel_running", C.c_int32),
                ("grid_blocks", C.c_int32)]


class gcmc_observables(C.Structure):
    _fields_ = [("S", C.c_double), ("A_g", C.c_double), ("A_g_R0", C.c_double), ("L_p", C.c_double),
                ("I_p", C.c_double), ("F_p", C.c_double), ("area", C.c_double)]


class gcmc_transit_obs(C.Structure):
    _fields_ = [("I_p_direct", C.c_double), ("I_p_scattered", C.c_double), ("omega_star", C.c_double),
                ("I_p", C.c_double), ("w_core", C.c_double), ("n_ld", C.c_double), ("area", C.c_double),
                ("depth", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgcmc.so is not built ({LIB_PATH}); run `python -m paper_2110_15640_gb300.build`")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        sig = {
            "gcmc_create": ([C.c_int, P(C.c_void_p)], C.c_int),
            "gcmc_destroy": ([C.c_void_p], C.c_int),
            "gcmc_set_stream": ([C.c_void_p, C.c_void_p], C.c_int),
            "gcmc_set_allocator": ([C.c_void_p, ALLOC_FN, FREE_FN, C.c_void_p], C.c_int),
            "gcmc_last_error": ([C.c_void_p], C.c_char_p),
            "gcmc_upload_grid": ([C.c_void_p, P(gcmc_grid_desc), P(C.c_int)], C.c_int),
            "gcmc_upload_opacity": ([C.c_void_p, C.c_int, P(gcmc_opacity_desc), P(C.c_int)], C.c_int),
            "gcmc_set_source": ([C.c_void_p, C.c_int, P(gcmc_source_desc), P(C.c_int)], C.c_int),
            "gcmc_run_packets": ([C.c_void_p, P(gcmc_job), C.c_void_p, C.c_int, P(gcmc_stats)], C.c_int),
            "gcmc_run_batch": ([C.c_void_p, P(gcmc_job), C.c_int, P(gcmc_launch_cfg), C.c_void_p, C.c_int,
                                P(gcmc_stats)], C.c_int),
            "gcmc_submit": ([C.c_void_p, P(gcmc_job), C.c_int, P(gcmc_launch_cfg), P(C.c_uint64)], C.c_int),
            "gcmc_run_contrib": ([C.c_void_p, P(gcmc_job), C.c_void_p, C.c_void_p, P(gcmc_stats)], C.c_int),
            "gcmc_graph_create": ([C.c_void_p, P(gcmc_job), C.c_int, P(gcmc_launch_cfg), P(C.c_void_p)], C.c_int),
            "gcmc_graph_launch": ([C.c_void_p, C.c_void_p], C.c_int),
            "gcmc_graph_read": ([C.c_void_p, C.c_void_p, P(gcmc_stats)], C.c_int),
            "gcmc_graph_destroy": ([C.c_void_p], C.c_int),
            "gcmc_poll": ([C.c_void_p, C.c_uint64, C.c_void_p, P(gcmc_stats)], C.c_int),
            "gcmc_job_columns": ([C.c_void_p, P(gcmc_job), P(C.c_int32)], C.c_int),
            "gcmc_run_packets_debug": ([C.c_void_p, P(gcmc_job), C.c_int64, C.c_int64, C.c_void_p, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, P(gcmc_stats)], C.c_int),
            "gcmc_prep_cells": ([C.c_void_p, P(gcmc_job)] + [C.c_void_p] * 7 + [P(gcmc_stats)], C.c_int),
            "gcmc_postscale": ([C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int64, C.c_double,
                                P(gcmc_observables)], C.c_int),
            "gcmc_transit": ([C.c_void_p, C.c_int, C.c_int, P(C.c_double), C.c_int64, P(gcmc_transit_obs)], C.c_int),
            "gcmc_selftest_philox": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
            "gcmc_version": ([], C.c_char_p),
            "gcmc_release_grid": ([C.c_void_p, C.c_int], C.c_int),
            "gcmc_release_opacity": ([C.c_void_p, C.c_int], C.c_int),
            "gcmc_set_profiling": ([C.c_void_p, C.c_int], C.c_int),
            "gcmc_get_profile": ([C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_int64)], C.c_int),
            "gcmc_kernel_launches": ([], C.c_int64),
            "gcmc_gather_bench": ([C.c_void_p, C.c_int64, C.c_int, C.c_int64, P(C.c_double)], C.c_int),
            "gcmc_emission_pdf_noalloc": ([C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p], C.c_int),
            "gcmc_server_create": ([C.c_void_p, P(gcmc_server_cfg), P(C.c_void_p)], C.c_int),
            "gcmc_server_submit": ([C.c_void_p, P(gcmc_job), P(C.c_uint64)], C.c_int),
            "gcmc_server_progress": ([C.c_void_p, P(C.c_uint64), C.c_int, P(C.c_int)], C.c_int),
            "gcmc_server_result": ([C.c_void_p, C.c_uint64, C.c_void_p, P(gcmc_stats)], C.c_int),
            "gcmc_server_query": ([C.c_void_p, P(gcmc_server_stats)], C.c_int),
            "gcmc_server_times": ([C.c_void_p, C.c_uint64, P(C.c_double)], C.c_int),
            "gcmc_server_destroy": ([C.c_void_p, C.c_double], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


EXPORTED = ["gcmc_create", "gcmc_destroy", "gcmc_set_stream", "gcmc_set_allocator", "gcmc_last_error",
            "gcmc_upload_grid", "gcmc_upload_opacity", "gcmc_set_source", "gcmc_run_packets", "gcmc_run_batch",
            "gcmc_submit", "gcmc_poll", "gcmc_run_contrib", "gcmc_graph_create", "gcmc_graph_launch",
            "gcmc_graph_read", "gcmc_graph_destroy", "gcmc_job_columns", "gcmc_run_packets_debug", "gcmc_prep_cells",
            "gcmc_postscale",
            "gcmc_selftest_philox", "gcmc_version", "gcmc_release_grid", "gcmc_release_opacity",
            "gcmc_set_profiling", "gcmc_get_profile", "gcmc_kernel_launches", "gcmc_gather_bench",
            "gcmc_emission_pdf_noalloc", "gcmc_server_create", "gcmc_server_submit", "gcmc_server_progress",
            "gcmc_server_result", "gcmc_server_query", "gcmc_server_destroy", "gcmc_server_times",
            "gcmc_transit"]
NOALLOC_MAX_CELLS = 4194304


class GcmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gcmc status {status}: {msg}")
        self.status = status


def _ptr(a):
    """Pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


class Context:
    """One libgcmc context on one device.  Keeps the host arrays of descriptors alive during calls."""

    def __init__(self, device=0, stream=None, torch_allocator=False):
        self.h = C.c_void_p()
        self._check(lib().gcmc_create(int(device), C.byref(self.h)), "gcmc_create")
        self._keep = []
        if torch_allocator:
            import torch

            dev = int(device)

            def _alloc(n, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), dev)
                except Exception:  # noqa: BLE001 - the C side reports GCMC_ERR_OOM on NULL
                    return None

            def _free(p, user):
                torch.cuda.caching_allocator_delete(p)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            self._check(lib().gcmc_set_allocator(self.h, self._cb[0], self._cb[1], None), "gcmc_set_allocator")
        if stream is not None:
            self.set_stream(stream)

    # -------------------------------------------------------------- plumbing
    def _check(self, st, what):
        if st != OK:
            msg = lib().gcmc_last_error(self.h).decode() if self.h else ""
            raise GcmcError(st, f"{what}: {msg}")

    def close(self):
        if self.h:
            lib().gcmc_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        self._check(lib().gcmc_set_stream(self.h, C.c_void_p(int(handle) if handle else 0)), "gcmc_set_stream")

    # -------------------------------------------------------------- uploads
    def upload_grid(self, grid, device_arrays=None, memory=MEM_DEVICE):
        """grid: synth.Grid (host arrays).  device_arrays: optional dict of arrays (torch tensors) for
        T, p, rho, wind, r_edges, lat_edges, lon_edges living in `memory` (device or pinned host)."""
        if device_arrays is not None:
            a = device_arrays
            mem = memory
        else:
            a = dict(r_edges=_host(grid.r_edges, np.float64), lat_edges=_host(grid.lat_edges, np.float64),
                     lon_edges=_host(grid.lon_edges, np.float64), T=_host(grid.T, np.float32),
                     p=_host(grid.p, np.float32), rho=_host(grid.rho, np.float32),
                     wind=_host(None if grid.wind is None else grid.wind.reshape(-1), np.float32))
            mem = MEM_HOST
        d = gcmc_grid_desc(grid.nlon, grid.nlat, grid.nr, mem, _ptr(a["r_edges"]), _ptr(a["lat_edges"]),
                           _ptr(a["lon_edges"]), _ptr(a["T"]), _ptr(a["p"]), _ptr(a["rho"]), _ptr(a.get("wind")))
        gid = C.c_int()
        self._check(lib().gcmc_upload_grid(self.h, C.byref(d), C.byref(gid)), "gcmc_upload_grid")
        return gid.value

    def upload_opacity(self, grid_id, opac, device_arrays=None, memory=MEM_DEVICE):
        d = gcmc_opacity_desc()
        keep = {}
        kind = opac.kind
        d.kind = kind
        if device_arrays is not None:
            keep = device_arrays
            d.memory = memory
        else:
            d.memory = MEM_HOST
            if kind == OPAC_ALBEDO:
                keep = dict(kabs=_host(opac.kabs, np.float64), kray=_host(opac.kray, np.float64),
                            qcld=_host(opac.qcld, np.float64), wcld=_host(opac.wcld, np.float64),
                            gcld=_host(opac.gcld, np.float64), acld=_host(opac.acld, np.float32))
            elif kind == OPAC_KTABLE:
                keep = dict(lam=_host(opac.lam, np.float64), Tg=_host(opac.Tg, np.float64),
                            pg=_host(opac.pg, np.float64), k=_host(opac.k, np.float32),
                            gw=_host(opac.wg, np.float64))
            else:
                keep = dict(xlam=_host(opac.lam, np.float64), Tg=_host(opac.Tg, np.float64),
                            pg=_host(opac.pg, np.float64), sigma=_host(opac.sigma, np.float32))
        if kind == OPAC_ALBEDO:
            d.nlam = len(opac.kray)
            for f in ("kabs", "kray", "qcld", "wcld", "gcld", "acld"):
                setattr(d, f, _ptr(keep.get(f)))
        elif kind == OPAC_KTABLE:
            d.nb, d.ng, d.nT, d.np = opac.k.shape
            for f in ("lam", "Tg", "pg", "k", "gw"):
                setattr(d, f, _ptr(keep.get(f)))
        else:
            d.nl, d.nT, d.np = opac.sigma.shape
            for f in ("xlam", "Tg", "pg", "sigma"):
                setattr(d, f, _ptr(keep.get(f)))
            d.view_theta, d.view_phi, d.omega_rot = opac.view_theta, opac.view_phi, opac.omega_rot
        oid = C.c_int()
        self._check(lib().gcmc_upload_opacity(self.h, int(grid_id), C.byref(d), C.byref(oid)), "gcmc_upload_opacity")
        return oid.value

    def set_sources(self, grid_id, source, precision=FP32):
        """Sources holding every observer of `source`, MAX_OBS per source (a source of the C ABI holds
        at most MAX_OBS directions); returns the source ids.  Observer o is entry o % MAX_OBS of
        source o // MAX_OBS."""
        import copy
        obs = np.atleast_2d(np.asarray(source.obs, np.float64))
        sids = []
        for o0 in range(0, len(obs), MAX_OBS):
            part = copy.copy(source)
            part.obs = obs[o0:o0 + MAX_OBS]
            sids.append(self.set_source(grid_id, part, precision))
        return sids

    def set_source(self, grid_id, source, precision=FP32):
        d = gcmc_source_desc()
        for i in range(3):
            d.star[i] = float(source.star[i])
        obs = np.atleast_2d(np.asarray(source.obs, np.float64))
        d.n_obs = len(obs)
        for o in range(len(obs)):
            for i in range(3):
                d.obs[o][i] = float(obs[o][i])
        op = source.opts
        d.survival = int(op.survival)
        d.w_rr, d.p_surv, d.tau_peel_cut = float(op.w_rr), float(op.p_surv), float(op.tau_peel_cut)
        d.tau_vert_max, d.beta_emis, d.hg_iso_eps = float(op.tau_vert_max), float(op.beta_emis), float(op.hg_iso_eps)
        d.scatter_emission = int(op.scatter_emission)
        d.precision = int(precision)
        d.max_steps = int(op.max_steps)
        d.cloud_phase = int(op.cloud_phase)
        d.surface_albedo = float(op.surface_albedo)
        d.trans_scatter = int(op.trans_scatter)
        d.ld_law = int(op.ld_law)
        for i, v in enumerate((list(op.ld_coef) + [0.0] * 4)[:4]):
            d.ld_coef[i] = float(v)
        d.star_radius, d.star_dist = float(op.star_radius), float(op.star_dist)
        d.transit_xy[0], d.transit_xy[1] = (float(v) for v in op.transit_xy)
        d.g_bias, d.g_beta = int(op.g_bias), float(op.g_beta)
        d.forced_first, d.cont_abs, d.path_bias = int(op.forced_first), int(op.cont_abs), int(op.path_bias)
        sid = C.c_int()
        self._check(lib().gcmc_set_source(self.h, int(grid_id), C.byref(d), C.byref(sid)), "gcmc_set_source")
        return sid.value

    # -------------------------------------------------------------- runs
    @staticmethod
    def job(grid_id, opac_id, source_id, mode, lam_idx, g_idx, n_packets, seed, key, obs_idx=-1):
        return gcmc_job(int(grid_id), int(opac_id), int(source_id), int(mode), int(lam_idx), int(g_idx),
                        int(obs_idx), int(key) & 0xFFFFFFFF, int(n_packets), int(seed))

    def run_packets(self, job, tallies=None):
        """Plain form.  tallies: optional torch CUDA tensor [MAX_OBS] float64 (device output)."""
        st = gcmc_stats()
        if tallies is not None:
            self._check(lib().gcmc_run_packets(self.h, C.byref(job), _ptr(tallies), MEM_DEVICE, None),
                        "gcmc_run_packets")
            return tallies, None
        out = np.zeros(MAX_OBS)
        self._check(lib().gcmc_run_packets(self.h, C.byref(job), _ptr(out), MEM_HOST, C.byref(st)), "gcmc_run_packets")
        return out, st

    def run_batch(self, jobs, cfg=None, tallies=None, stats=True):
        arr = (gcmc_job * len(jobs))(*jobs)
        cfgp = C.byref(cfg) if cfg is not None else None
        sts = (gcmc_stats * len(jobs))() if stats else None
        if tallies is not None:
            self._check(lib().gcmc_run_batch(self.h, arr, len(jobs), cfgp, _ptr(tallies), MEM_DEVICE, sts),
                        "gcmc_run_batch")
            return tallies, sts
        out = np.zeros((len(jobs), MAX_OBS))
        self._check(lib().gcmc_run_batch(self.h, arr, len(jobs), cfgp, _ptr(out), MEM_HOST, sts), "gcmc_run_batch")
        return out, sts

    def run_contrib(self, job, ncell, n_obs=1):
        """One albedo or emission job with contribution functions: (tallies [MAX_OBS],
        cf [2][n_obs][ncell] sums of f by the cell each peel-off leaves from (thermal, scattered),
        gcmc_stats).  The contribution function of a cell is cf / tally."""
        out = np.zeros(MAX_OBS)
        cf = np.zeros((2, n_obs, ncell))
        st = gcmc_stats()
        self._check(lib().gcmc_run_contrib(self.h, C.byref(job), _ptr(out), _ptr(cf), C.byref(st)), "gcmc_run_contrib")
        return out, cf, st

    def graph(self, jobs, cfg=None):
        """A captured batch (gcmc_graph_*): Graph.launch(tallies=None) replays it on the context's stream."""
        return Graph(self, jobs, cfg)

    def submit(self, jobs, cfg=None):
        arr = (gcmc_job * len(jobs))(*jobs)
        t = C.c_uint64()
        self._check(lib().gcmc_submit(self.h, arr, len(jobs), C.byref(cfg) if cfg is not None else None, C.byref(t)),
                    "gcmc_submit")
        return t.value

    def poll(self, ticket, n_jobs):
        out = np.zeros((n_jobs, MAX_OBS))
        sts = (gcmc_stats * n_jobs)()
        st = lib().gcmc_poll(self.h, C.c_uint64(ticket), _ptr(out), sts)
        if st == ERR_NOT_READY:
            return None
        self._check(st, "gcmc_poll")
        return out, sts

    def job_columns(self, job):
        n = C.c_int32(0)
        self._check(lib().gcmc_job_columns(self.h, C.byref(job), C.byref(n)), "gcmc_job_columns")
        return n.value

    def run_debug(self, job, packet0=0, n_run=None, n_trace=0, max_trace=0, n_obs=None):
        """per-packet results; pk_f has n_obs columns (default: the job's tally columns; fewer are refused)"""
        n_run = job.n_packets - packet0 if n_run is None else int(n_run)
        n_obs = self.job_columns(job) if n_obs is None else int(n_obs)
        pk_f = np.zeros((n_run, n_obs))
        pk_steps = np.zeros(n_run, np.int64)
        pk_tau = np.zeros(n_run)
        n_trace = min(int(n_trace), n_run)
        tr_cell = np.zeros((max(n_trace, 1), max(max_trace, 1)), np.int32)
        tr_len = np.zeros((max(n_trace, 1), max(max_trace, 1)))
        tr_n = np.zeros(max(n_trace, 1), np.int32)
        tally = np.zeros(MAX_OBS)
        st = gcmc_stats()
        self._check(lib().gcmc_run_packets_debug(self.h, C.byref(job), int(packet0), n_run, _ptr(pk_f), n_obs,
                                                 _ptr(pk_steps), _ptr(pk_tau), n_trace, int(max_trace),
                                                 _ptr(tr_cell), _ptr(tr_len), _ptr(tr_n), _ptr(tally), C.byref(st)),
                    "gcmc_run_packets_debug")
        out = dict(pk_f=pk_f, pk_steps=pk_steps, pk_tau=pk_tau, tally=tally, stats=st)
        if n_trace:
            out.update(tr_cell=tr_cell[:n_trace], tr_len=tr_len[:n_trace], tr_n=tr_n[:n_trace])
        return out

    def prep_cells(self, job, ncell):
        out = {k: np.zeros(ncell) for k in ("alpha", "omega", "g", "pgas", "lum", "cdf", "wcell")}
        st = gcmc_stats()
        self._check(lib().gcmc_prep_cells(self.h, C.byref(job), *[_ptr(out[k]) for k in
                                                                   ("alpha", "omega", "g", "pgas", "lum", "cdf", "wcell")],
                                          C.byref(st)), "gcmc_prep_cells")
        out["stats"] = st
        return out

    def postscale(self, grid_id, mode, tally, n_packets, l_tot=0.0):
        o = gcmc_observables()
        self._check(lib().gcmc_postscale(self.h, int(grid_id), int(mode), float(tally), int(n_packets), float(l_tot),
                                         C.byref(o)), "gcmc_postscale")
        return {f: getattr(o, f) for f, _ in gcmc_observables._fields_}

    def transit(self, grid_id, source_id, tally, n_packets):
        """Transit observables of a transmission job from its tally columns (chord, scattered)."""
        t = (C.c_double * 2)(*[float(v) for v in (list(np.atleast_1d(tally)) + [0.0, 0.0])[:2]])
        o = gcmc_transit_obs()
        self._check(lib().gcmc_transit(self.h, int(grid_id), int(source_id), t, int(n_packets), C.byref(o)),
                    "gcmc_transit")
        return {f: getattr(o, f) for f, _ in gcmc_transit_obs._fields_}

    def release_grid(self, grid_id):
        self._check(lib().gcmc_release_grid(self.h, int(grid_id)), "gcmc_release_grid")

    def release_opacity(self, opac_id):
        self._check(lib().gcmc_release_opacity(self.h, int(opac_id)), "gcmc_release_opacity")

    def set_profiling(self, on=True):
        self._check(lib().gcmc_set_profiling(self.h, int(bool(on))), "gcmc_set_profiling")

    def get_profile(self):
        a, b, n = C.c_double(), C.c_double(), C.c_int64()
        self._check(lib().gcmc_get_profile(self.h, C.byref(a), C.byref(b), C.byref(n)), "gcmc_get_profile")
        return a.value, b.value, n.value

    def gather_bench(self, n_records, record_bytes=4, n_gathers=1 << 30):
        r = C.c_double()
        self._check(lib().gcmc_gather_bench(self.h, int(n_records), int(record_bytes), int(n_gathers), C.byref(r)),
                    "gcmc_gather_bench")
        return r.value

    def selftest_philox(self, ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32)
        key = np.ascontiguousarray(key, np.uint32)
        n = len(ctr)
        a = np.zeros((n, 4), np.uint32)
        b = np.zeros((n, 4), np.uint32)
        self._check(lib().gcmc_selftest_philox(self.h, _ptr(ctr), _ptr(key), n, _ptr(a), _ptr(b)), "gcmc_selftest_philox")
        return a, b


def emission_pdf_noalloc(lum, ncell, beta, cdf, wcell, totals, stream=None):
    """Allocation-free emission pdf stage: every argument array is caller-owned device memory (torch
    CUDA tensors of float64).  Returns the gcmc status code; the work is queued on `stream`."""
    handle = getattr(stream, "cuda_stream", stream)
    return int(lib().gcmc_emission_pdf_noalloc(_ptr(lum), int(ncell), float(beta), _ptr(cdf), _ptr(wcell),
                                               _ptr(totals), C.c_void_p(int(handle) if handle else 0)))


def kernel_launches():
    return int(lib().gcmc_kernel_launches())


def stats_dict(st):
    return dict(packets=st.packets, steps=st.steps, ledger=list(st.ledger), l_tot=st.l_tot, cdf_total=st.cdf_total,
                n_emit_cells=st.n_emit_cells)


def workload_arrays(wl, where):
    """The grid and opacity input arrays of a workload as torch tensors on `where` ('cuda' or
    'pinned' host memory), keyed like the descriptor fields."""
    import torch

    def put(a, dt):
        if a is None:
            return None
        t = torch.as_tensor(np.ascontiguousarray(a, dt))
        return t.cuda() if where == "cuda" else t.pin_memory()

    g = wl.grid
    ga = dict(r_edges=put(g.r_edges, np.float64), lat_edges=put(g.lat_edges, np.float64),
              lon_edges=put(g.lon_edges, np.float64), T=put(g.T, np.float32), p=put(g.p, np.float32),
              rho=put(g.rho, np.float32), wind=put(None if g.wind is None else g.wind.reshape(-1), np.float32))
    o = wl.opac
    if o.kind == OPAC_ALBEDO:
        oa = dict(kabs=put(o.kabs, np.float64), kray=put(o.kray, np.float64), qcld=put(o.qcld, np.float64),
                  wcld=put(o.wcld, np.float64), gcld=put(o.gcld, np.float64), acld=put(o.acld, np.float32))
    elif o.kind == OPAC_KTABLE:
        oa = dict(lam=put(o.lam, np.float64), Tg=put(o.Tg, np.float64), pg=put(o.pg, np.float64),
                  k=put(o.k, np.float32), gw=put(o.wg, np.float64))
    else:
        oa = dict(xlam=put(o.lam, np.float64), Tg=put(o.Tg, np.float64), pg=put(o.pg, np.float64),
                  sigma=put(o.sigma, np.float32))
    return ga, oa


def array_bytes(d):
    return int(sum(t.numel() * t.element_size() for t in d.values() if t is not None))


def load_workload(ctx, wl, precision=FP32, device_inputs=False):
    """Upload a synth.Workload (grid, opacity, source) and return (grid_id, opac_id, source_id, jobs).
    device_inputs=True stages the arrays in torch CUDA tensors first and uploads from device memory."""
    if device_inputs:
        import torch

        g = wl.grid

        def dev(a, dt):
            return None if a is None else torch.as_tensor(np.ascontiguousarray(a, dt)).cuda()

        ga = dict(r_edges=dev(g.r_edges, np.float64), lat_edges=dev(g.lat_edges, np.float64),
                  lon_edges=dev(g.lon_edges, np.float64), T=dev(g.T, np.float32), p=dev(g.p, np.float32),
                  rho=dev(g.rho, np.float32), wind=dev(None if g.wind is None else g.wind.reshape(-1), np.float32))
        torch.cuda.synchronize()
        gid = ctx.upload_grid(g, device_arrays=ga)
        o = wl.opac
        if o.kind == OPAC_ALBEDO:
            oa = dict(kabs=dev(o.kabs, np.float64), kray=dev(o.kray, np.float64), qcld=dev(o.qcld, np.float64),
                      wcld=dev(o.wcld, np.float64), gcld=dev(o.gcld, np.float64), acld=dev(o.acld, np.float32))
        elif o.kind == OPAC_KTABLE:
            oa = dict(lam=dev(o.lam, np.float64), Tg=dev(o.Tg, np.float64), pg=dev(o.pg, np.float64),
                      k=dev(o.k, np.float32), gw=dev(o.wg, np.float64))
        else:
            oa = dict(xlam=dev(o.lam, np.float64), Tg=dev(o.Tg, np.float64), pg=dev(o.pg, np.float64),
                      sigma=dev(o.sigma, np.float32))
        torch.cuda.synchronize()
        oid = ctx.upload_opacity(gid, o, device_arrays=oa)
    else:
        gid = ctx.upload_grid(wl.grid)
        oid = ctx.upload_opacity(gid, wl.opac)
    sids = ctx.set_sources(gid, wl.source, precision)
    jobs = workload_jobs(wl, gid, oid, sids)
    return gid, oid, sids[0], jobs


def workload_jobs(wl, gid, oid, sids):
    """gcmc_job structs of a workload's jobs; a job that tallies one observer o (obs_idx >= 0) uses
    source o // MAX_OBS, entry o % MAX_OBS (sources from Context.set_sources)."""
    jobs = []
    for j in wl.jobs:
        o = getattr(j, "obs_idx", -1)
        if o < 0 and len(sids) > 1:
            raise ValueError("a job that tallies every observer needs at most MAX_OBS observers")
        sid = sids[o // MAX_OBS] if o >= 0 else sids[0]
        jobs.append(Context.job(gid, oid, sid, wl.mode, j.lam_idx, j.g_idx, j.n_packets, wl.seed, j.key,
                                o % MAX_OBS if o >= 0 else -1))
    return jobs


def load_serving(ctx, sw, precision=FP32):
    """Upload every scene of a synth.ServingWorkload (grid, three opacities, three sources) and return
    the requests as gcmc_job structs, in request order."""
    from . import synth as S
    ids = []
    for sc in sw.scenes:
        gid = ctx.upload_grid(sc.grid)
        oa = ctx.upload_opacity(gid, sc.albedo)
        ok = ctx.upload_opacity(gid, sc.ktable)
        ox = ctx.upload_opacity(gid, sc.xsec)
        sa = ctx.set_source(gid, sc.src_albedo, precision)
        se = ctx.set_source(gid, sc.src_emission, precision)
        st = ctx.set_source(gid, sc.src_transmission, precision)
        ids.append({S.MODE_ALBEDO: (gid, oa, sa), S.MODE_EMISSION: (gid, ok, se), S.MODE_TRANSMISSION: (gid, ox, st)})
    jobs = []
    for r in sw.requests:
        gid, oid, sid = ids[r.scene][r.mode]
        jobs.append(Context.job(gid, oid, sid, r.mode, r.lam_idx, r.g_idx, r.n_packets, sw.seed, r.key, r.obs_idx))
    return jobs


class Server:
    """The continuous-batching request loop of one context (gcmc_server_*): submit jobs as they arrive,
    call progress() often, and take results of the tickets progress() reports complete."""

    def __init__(self, ctx: Context, block=128, blocks_per_sm=0, chunk=256, interval=4, refill_min=8,
                 max_jobs=1024, hbm_budget=8 << 30, idle_us=2000):
        self.ctx = ctx
        self.h = C.c_void_p()
        cfg = gcmc_server_cfg(block, blocks_per_sm, chunk, interval, refill_min, max_jobs, int(hbm_budget),
                              idle_us, 0)
        ctx._check(lib().gcmc_server_create(ctx.h, C.byref(cfg), C.byref(self.h)), "gcmc_server_create")
        self._done = (C.c_uint64 * 4096)()

    def submit(self, job: gcmc_job) -> int:
        t = C.c_uint64()
        self.ctx._check(lib().gcmc_server_submit(self.h, C.byref(job), C.byref(t)), "gcmc_server_submit")
        return int(t.value)

    def progress(self):
        """One pass of the loop; returns the tickets that completed in it."""
        n = C.c_int()
        self.ctx._check(lib().gcmc_server_progress(self.h, self._done, len(self._done), C.byref(n)),
                        "gcmc_server_progress")
        if n.value > len(self._done):
            raise GcmcError(ERR_RANGE, "more completions in one pass than the ticket buffer holds")
        return [int(self._done[i]) for i in range(n.value)]

    def times(self, ticket: int):
        """(submitted, admitted, published, completed) host times in s of a completed, untaken ticket."""
        t = (C.c_double * 4)()
        self.ctx._check(lib().gcmc_server_times(self.h, C.c_uint64(ticket), t), "gcmc_server_times")
        return tuple(t)

    def result(self, ticket: int):
        """(tallies [MAX_OBS], gcmc_stats) of a completed ticket."""
        out = np.zeros(MAX_OBS, np.float64)
        st = gcmc_stats()
        self.ctx._check(lib().gcmc_server_result(self.h, C.c_uint64(ticket), _ptr(out), C.byref(st)),
                        "gcmc_server_result")
        return out, st

    def query(self) -> gcmc_server_stats:
        st = gcmc_server_stats()
        self.ctx._check(lib().gcmc_server_query(self.h, C.byref(st)), "gcmc_server_query")
        return st

    def close(self, timeout_s=60.0):
        if self.h:
            self.ctx._check(lib().gcmc_server_destroy(self.h, float(timeout_s)), "gcmc_server_destroy")
            self.h = C.c_void_p()

    def run_all(self, jobs, timeout_s=120.0):
        """Submit every job at once and loop until all have completed; returns [(tallies, stats)]."""
        import time
        tickets = [self.submit(j) for j in jobs]
        want, got = set(tickets), {}
        t0 = time.perf_counter()
        while len(got) < len(want):
            for t in self.progress():
                got[t] = self.result(t)
            if time.perf_counter() - t0 > timeout_s:
                raise GcmcError(ERR_TIMEOUT, f"{len(want) - len(got)} served jobs still open after {timeout_s} s")
        return [got[t] for t in tickets]


class Graph:
    """A batch captured into a CUDA graph (gcmc_graph_*)."""

    def __init__(self, ctx: Context, jobs, cfg=None):
        self.ctx = ctx
        self.n = len(jobs)
        arr = (gcmc_job * len(jobs))(*jobs)
        self.h = C.c_void_p()
        ctx._check(lib().gcmc_graph_create(ctx.h, arr, len(jobs), C.byref(cfg) if cfg is not None else None,
                                           C.byref(self.h)), "gcmc_graph_create")

    def launch(self, tallies=None):
        """Replay asynchronously; tallies: optional torch CUDA tensor [n_jobs][MAX_OBS] float64."""
        self.ctx._check(lib().gcmc_graph_launch(self.h, _ptr(tallies)), "gcmc_graph_launch")

    def read(self):
        """(tallies [n_jobs][MAX_OBS], stats [n_jobs]) of the last replay (synchronises)."""
        out = np.zeros((self.n, MAX_OBS))
        sts = (gcmc_stats * self.n)()
        self.ctx._check(lib().gcmc_graph_read(self.h, _ptr(out), sts), "gcmc_graph_read")
        return out, sts

    def close(self):
        if self.h:
            lib().gcmc_graph_destroy(self.h)
            self.h = C.c_void_p()
