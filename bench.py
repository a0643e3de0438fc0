#!/usr/bin/env python
"""Benchmark of the photon-transport hot path on GB300.

Workload (default): thermal emission spectrum of a hot-Jupiter-shaped grid, 128 lon x 64 lat x 50
levels (1e-6..100 bar), correlated-k with 30 bands x 8 g-ordinates, 1e6 packets per (band, g) job,
FP32 march with FP64 emission CDF and fixed-point tallies.  One step = the whole path for all 240
jobs: cell tables (S1) and one persistent transport launch (S2-S8) with device tallies.

Prints ONE JSON line (rank 0): packet-steps/s of the batched form (value), the plain one-launch-
per-job form beside it, spectra/s, the end-to-end number through the C ABI from pinned host
buffers, the transport kernel against the measured random-gather rate of this GPU (the gather
roofline, `roofline`) and against its ALU issue ceiling (`alu_roofline`), the oracle's CPU baseline,
the clocks seen, the other configuration workloads at full size (`workloads`: albedo 32x16x20 FP64,
the 960-job phase curve, the 9532-wavelength transmission spectrum, transit with multiple
scattering; batched and plain form, gather fraction and clocks of each), and the serving stream of
10,000 Poisson-arriving mixed requests (p50/p99 latency and packet-steps/s of the server and of the
plain form).  `--impl reference` times the FP64 CPU oracle on the same workload instead.

Other workloads (--workload): albedo (32x16x20, FP64), phasecurve (40 wavelengths x 24 phases),
transmission (9532 wavelengths, Doppler cross sections), transit-scatter (40 optical wavelengths in
transit with multiple scattering and limb darkening), band (the emission workload as 30 band jobs
whose packets draw their g-ordinate), emission-hires (952 of the 9532 high-resolution wavelengths in
emission with Doppler-shifted cross-sections), serving (the full request stream).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OPS_PER_STEP = 64          # FP32-pipe operations of one cell step (counted from the formulas)
# DRAM bytes (read + write) of the persistent transport kernel per emission job of the 128x64x50 grid,
# from ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the 8-job band-0 launch of the current
# kernel, or None when the kernel has changed since the counters were taken: the traffic grows with the
# number of job tables the launch touches
TRAFFIC_PER_EMISSION_JOB = (48.625408e6 + 1.36704e6) / 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gcmc", choices=["gcmc", "reference"])
    ap.add_argument("--packets", type=int, default=1_000_000, help="packets per (band, g) job")
    ap.add_argument("--bands", type=int, default=30)
    ap.add_argument("--gpoints", type=int, default=8)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--interval", type=int, default=0)
    ap.add_argument("--refill", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="skip the launch autotuner")
    ap.add_argument("--workload", default="emission", choices=["emission", "albedo", "phasecurve", "transmission", "transit-scatter", "band",
                             "emission-hires", "serving"])
    ap.add_argument("--forced-first", action="store_true", help="scattering workloads: forced first scattering")
    ap.add_argument("--cont-abs", action="store_true", help="scattering workloads: continuous absorption")
    ap.add_argument("--requests", type=int, default=10_000, help="serving: requests in the stream")
    ap.add_argument("--hbm-budget-gb", type=float, default=16.0, help="serving: admitted workspace")
    ap.add_argument("--serving-requests", type=int, default=10_000,
                    help="emission bench: requests of the serving stream in its JSON line (0: none)")
    ap.add_argument("--jobs", type=int, default=0,
                    help="run only N jobs spread evenly over the workload's job list (profiling a small case)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="emission bench: skip the other configuration workloads in its JSON line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, rank):
    """The synthetic workload of --workload (seeded; distinct packets per rank for weak scaling)."""
    from paper_2110_15640_gb300 import shard, synth
    if args.workload == "albedo":
        wl = synth.config1_albedo()
    elif args.workload == "phasecurve":
        wl = synth.config3_phase_curve()
    elif args.workload == "transmission":
        wl = synth.config4_transmission()
    elif args.workload == "transit-scatter":
        wl = synth.config6_transit_scatter()
    elif args.workload == "emission-hires":
        wl = synth.config7_emission_hires(lam_subset=range(0, 9532, 10))
    elif args.workload == "band":
        wl = synth.config2_emission(n_packets=args.packets * args.gpoints, nb=30, ng=8, bands=range(args.bands),
                                    per_packet_g=True, g_bias=2)
    else:
        wl = synth.config2_emission(n_packets=args.packets, nb=30, ng=8, bands=range(args.bands),
                                    gpoints=range(args.gpoints))
    if args.forced_first or args.cont_abs:
        wl.source.opts.forced_first = int(args.forced_first)
        wl.source.opts.cont_abs = int(args.cont_abs)
        wl.name += ("_forced" if args.forced_first else "") + ("_contabs" if args.cont_abs else "")
    if getattr(args, "jobs", 0) and args.jobs < len(wl.jobs):
        n = len(wl.jobs)
        wl.jobs = [wl.jobs[(q * n) // args.jobs] for q in range(args.jobs)]
    wl.seed = shard.rank_seed(wl.seed, rank)
    return wl


# oracle sample per workload for the CPU baseline: (jobs, packets per job or None for all)
CPU_SAMPLE = {"emission": (48, 1_000_000), "albedo": (1, None), "phasecurve": (24, None), "transmission": (480, None),
              "transit-scatter": (8, 400_000), "band": (12, 1_000_000), "emission-hires": (40, None)}
REF_SAMPLE = {"emission": (2, 1_000_000), "albedo": (1, None), "phasecurve": (2, None), "transmission": (96, None),
              "transit-scatter": (2, None), "band": (2, 1_000_000), "emission-hires": (4, None)}


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = [l.split(",") for l in (self.out or "").strip().splitlines() if l.count(",") >= 6]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if "Active" in r[3 + q] and "Not" not in r[3 + q]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(dev):
    try:
        import torch
        u = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
        return f"GPU-{u}" if u is not None else None
    except Exception:  # noqa: BLE001
        return None


def cpu_oracle_rate(wl, n_jobs, n_packets, nthreads):
    """Oracle (FP64 CPU) packet-steps/s on a sample of the workload's jobs (spread over the job list),
    S1 included; n_packets None runs each job's full packet count."""
    from oracle import oracle as O
    steps = 0
    t0 = time.perf_counter()
    for job in wl.jobs[::max(1, len(wl.jobs) // n_jobs)][:n_jobs]:
        cells = O.prep_cells(wl, job)
        npk = job.n_packets if n_packets is None else min(n_packets, job.n_packets)
        r = O.run(wl, job, cells=cells, packet0=0, n_run=npk, nthreads=nthreads)
        steps += r["steps"]
    dt = time.perf_counter() - t0
    return steps / dt, dt, steps


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    wl = workload(args, 0)
    cores = os.cpu_count() or 1
    nj, npk = REF_SAMPLE[args.workload]
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, 1, 20_000, cores)
    rates, total_steps, total_t = [], 0, 0.0
    for _ in range(args.steps):
        r, dt, st = cpu_oracle_rate(wl, nj, npk, cores)
        rates.append(r)
        total_steps += st
        total_t += dt
    value = total_steps / total_t
    g = wl.grid
    sample = (f"{nj} of {len(wl.jobs)} jobs x {npk or 'all their'} packets per step (S1 + transport), "
              f"full {g.nlon}x{g.nlat}x{g.nr} grid")
    line = {"metric": "packet-steps/s", "value": value, "unit": "packet-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "jobs": len(wl.jobs), "packets": wl.total_packets},
            "cpu_baseline": {"value": value, "unit": "packet-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "packet-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serve_stream(sv, jobs, arrivals, timeout_s=600.0):
    """Submit jobs[i] at arrivals[i] seconds after the start and run the server's loop until all have
    completed; returns (per-request latency in s, total packet-steps, wall seconds)."""
    n = len(jobs)
    lat = [0.0] * n
    who = {}
    steps, done, i = 0, 0, 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            who[sv.submit(jobs[i])] = i
            i += 1
        for tk in sv.progress():
            q = who.pop(tk)
            _, st = sv.result(tk)
            lat[q] = time.perf_counter() - t0 - arrivals[q]
            steps += st.steps
            done += 1
        if now > timeout_s:
            raise RuntimeError(f"serving stream: {n - done} requests open after {timeout_s} s")
        if i < n and not who:
            time.sleep(max(0.0, min(arrivals[i] - now, 1e-3)))
    return lat, steps, time.perf_counter() - t0


def plain_stream(ctx, jobs, arrivals):
    """The same stream on the plain form: one request at a time, in arrival order, one cell-table
    preparation and one transport launch each (gcmc_run_packets)."""
    n = len(jobs)
    lat = [0.0] * n
    steps, busy = 0, 0.0
    t0 = time.perf_counter()
    for q in range(n):
        now = time.perf_counter() - t0
        if arrivals[q] > now:
            time.sleep(arrivals[q] - now)
        ts = time.perf_counter()
        _, st = ctx.run_packets(jobs[q])
        te = time.perf_counter()
        busy += te - ts
        steps += st.steps
        lat[q] = te - t0 - arrivals[q]
    return lat, steps, time.perf_counter() - t0, busy


def pct(xs, p):
    import numpy as np
    return float(np.percentile(np.asarray(xs) * 1e3, p))


def serving_run(n_requests, hbm_budget_gb, loads=(0.7, 0.9)):
    """Serving workload: a Poisson stream of mixed requests on four resident grids through the
    continuous-batching server, at the given fractions of the server's saturated request rate, and the
    same stream (at the first load) on the plain one-launch-per-request form.  Returns a dict."""
    import numpy as np
    from paper_2110_15640_gb300 import gcmc, synth
    sw = synth.config5_serving(n_requests=n_requests)
    ctx = gcmc.Context(0)
    jobs = gcmc.load_serving(ctx, sw)
    sv = gcmc.Server(ctx, hbm_budget=int(hbm_budget_gb * (1 << 30)))
    sv.run_all(jobs[:32])                                   # warm-up (first launches, pools)
    # saturated: every request queued at t = 0
    lat_s, steps_s, wall_s = serve_stream(sv, jobs, [0.0] * len(jobs))
    rate_sat = len(jobs) / wall_s
    rng = np.random.default_rng(55)
    runs = {}
    for load in loads:
        arr = np.cumsum(rng.exponential(1.0 / (load * rate_sat), len(jobs))).tolist()
        lat, steps, wall = serve_stream(sv, jobs, arr)
        runs[load] = {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "packet_steps_per_s": steps / wall,
                      "requests_per_s": len(jobs) / wall, "wall_s": wall}
    stq = sv.query()
    sv.close()
    arr = np.cumsum(rng.exponential(1.0 / (loads[0] * rate_sat), len(jobs))).tolist()
    lat_p, steps_p, wall_p, busy_p = plain_stream(ctx, jobs, arr)
    ctx.close()
    out = {"workload": sw.name, "requests": len(jobs),
           "grids": ["x".join(map(str, g)) for g in synth.SERVING_GRIDS],
           "packets": "log-uniform 1e4..1e7", "modes": "albedo / emission / transmission, 1/3 each",
           "hbm_budget_gb": hbm_budget_gb,
           "saturated": {"packet_steps_per_s": steps_s / wall_s, "requests_per_s": rate_sat, "wall_s": wall_s,
                         "p50_ms": pct(lat_s, 50), "p99_ms": pct(lat_s, 99)},
           f"plain_form_at_{loads[0]}": {"p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99),
                                         "packet_steps_per_s": steps_p / wall_p,
                                         "packet_steps_per_s_busy": steps_p / busy_p, "wall_s": wall_p},
           "server": {"kernel_launches": stq.kernel_launches, "grid_blocks": stq.grid_blocks}}
    for load in loads:
        out[f"poisson_{load}"] = runs[load]
    return out


def serving_bench(args):
    import torch
    from paper_2110_15640_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    sv = serving_run(args.requests, args.hbm_budget_gb)
    line = {
        "metric": "packet-steps/s", "value": sv["saturated"]["packet_steps_per_s"], "unit": "packet-steps/s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * sv["saturated"]["wall_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": sv["workload"], "requests": sv["requests"], "grids": sv["grids"],
                   "packets": sv["packets"], "modes": sv["modes"], "hbm_budget_gb": sv["hbm_budget_gb"]},
        "serving": sv,
    }
    print(json.dumps(line), flush=True)
    return 0


def device_sm_count(dev):
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def tune_cfg(args, ctx, jobs, stream):
    """The launch configuration: the flags' fixed one, or the autotuner's (untimed; tallies do not depend on
    the launch parameters)."""
    from paper_2110_15640_gb300 import autotune, gcmc
    if args.no_tune or args.block or args.chunk or args.interval or args.refill or args.blocks_per_sm:
        cfg = gcmc.gcmc_launch_cfg(args.block, args.blocks_per_sm, args.chunk, args.interval, args.refill, 0)
        tuned = {"block": args.block or 128, "blocks_per_sm": args.blocks_per_sm, "chunk": args.chunk or 1024,
                 "interval": args.interval or 1, "refill_min": args.refill or 16}
        return cfg, tuned
    cfg, tuned, _ = autotune.tune(ctx, autotune.sample_jobs(jobs), stream, reps=2, full_jobs=jobs)
    return cfg, tuned


def measure(ctx, stream, jobs, cfg, steps, warmup, plain_steps, world=1, graph=False):
    """Device-timed batched steps (max over ranks), then the plain one-launch-per-job form on the same jobs.
    Returns a dict of the measurements; `clocks` is the nvidia-smi record of the batched timed region."""
    import torch
    from paper_2110_15640_gb300 import gcmc

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        tall = torch.zeros((len(jobs), gcmc.MAX_OBS), dtype=torch.float64, device="cuda")
        _, sts = ctx.run_batch(jobs, cfg=cfg)                       # untimed: exact packet-step count
    steps_per_step = int(sum(s.steps for s in sts))
    out = {"packet_steps_per_step": steps_per_step, "packets_per_step": int(sum(s.packets for s in sts)),
           "capped_weight": float(sum(s.ledger[6] for s in sts))}
    for _ in range(warmup):
        ctx.run_batch(jobs, cfg=cfg, tallies=tall, stats=False)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    l0 = gcmc.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_uuid(torch.cuda.current_device())) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            ctx.run_batch(jobs, cfg=cfg, tallies=tall, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    out["gpu_launches"] = gcmc.kernel_launches() - l0
    prep_ms, tr_ms, ntr = ctx.get_profile()
    ctx.set_profiling(False)
    t = e0.elapsed_time(e1) / 1e3
    if world > 1:
        tt = torch.tensor([t], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t = float(tt.item())
    out.update(value=steps_per_step * steps * world / t, ms_per_step=1e3 * t / steps, seconds=t,
               kernel_ms=tr_ms / max(ntr, 1), prep_ms=prep_ms / max(ntr, 1), clocks=clk.summary())
    out["spectra_per_s"] = world * steps / t          # one step computes the workload's whole spectrum
    if graph:
        gr = ctx.graph(jobs, cfg)
        for _ in range(2):
            gr.launch(tall)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(steps):
            gr.launch(tall)
        g1.record(stream)
        torch.cuda.synchronize()
        tg = g0.elapsed_time(g1) / 1e3
        gr.close()
        out["graph_form"] = {"value": steps_per_step * steps / tg, "unit": "packet-steps/s",
                             "ms_per_step": 1e3 * tg / steps}
    if plain_steps:
        outp = torch.zeros(gcmc.MAX_OBS, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for j in jobs[:8]:
                ctx.run_packets(j, tallies=outp)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(plain_steps):
            for j in jobs:
                ctx.run_packets(j, tallies=outp)
        p1.record(stream)
        torch.cuda.synchronize()
        tp = p0.elapsed_time(p1) / 1e3
        out["plain_form"] = {"value": steps_per_step * plain_steps / tp, "unit": "packet-steps/s",
                             "ms_per_step": 1e3 * tp / plain_steps, "launches_per_step": len(jobs)}
        out["batched_over_plain"] = out["value"] / out["plain_form"]["value"]
    return out


def rooflines(ctx, wl, m, prec, dev, traffic):
    """The transport kernel against its bound, the measured random-gather rate of this GPU for a table of the
    job's size and record width (the gather roofline), with the ALU issue ceiling beside it.  The gather
    roofline is stated in GB/s of algorithmic record bytes, so achieved / peak is packet-steps/s over
    gathers/s."""
    from paper_2110_15640_gb300 import gcmc
    f64 = prec == gcmc.FP64
    rec_bytes = 16 if wl.opac.kind == gcmc.OPAC_ALBEDO else 4
    if f64:
        rec_bytes *= 2
    gather = ctx.gather_bench(wl.grid.ncell, 16 if wl.opac.kind == gcmc.OPAC_ALBEDO else 4, 1 << 30)
    k_s = m["kernel_ms"] / 1e3
    steps_s = m["packet_steps_per_step"] / k_s
    nsm = device_sm_count(dev)
    mhz = m["clocks"].get("sm_mhz") or m["clocks"].get("sm_max_mhz") or 2070.0
    lanes = 2 if f64 else 128                      # FP64 / FP32 lanes per SM and clock
    peak_ops = nsm * lanes * mhz * 1e6
    roof = {"bound": "gather", "achieved": steps_s * rec_bytes / 1e9, "peak": gather * rec_bytes / 1e9, "unit": "GB/s",
            "frac": steps_s / gather, "traffic": traffic,
            "kernel": f"k_transport_persistent<{'double' if f64 else 'float'}>", "kernel_ms": m["kernel_ms"],
            "prep_ms": m["prep_ms"], "packet_steps_per_s": steps_s, "gathers_per_s": gather,
            "record_bytes": rec_bytes, "table_records": wl.grid.ncell,
            "peak_source": "measured: gcmc_gather_bench on this GPU, random records of a table of the job's size"}
    alu = {"bound": "fp64" if f64 else "alu", "achieved": OPS_PER_STEP * steps_s / 1e12, "peak": peak_ops / 1e12,
           "unit": "TFLOP/s", "frac": OPS_PER_STEP * steps_s / peak_ops, "ops_per_step": OPS_PER_STEP, "sm_count": nsm,
           "sm_mhz": mhz, "peak_source": "SMs x lanes x median SM clock sampled during the timed steps"}
    if traffic:
        roof["dram_GBps"] = traffic / k_s / 1e9
        peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(peaks):
            with open(peaks) as f:
                hbm = json.load(f).get("hbm_gbs")
            if hbm:
                roof["dram_frac_of_measured_hbm"] = roof["dram_GBps"] / hbm
    return roof, alu


def workload_line(args, name, ctx, stream, dev):
    """One workload of the configuration list at its full size: batched (autotuned) and plain form, gather
    fraction and clocks; grids are released afterwards."""
    import copy
    from paper_2110_15640_gb300 import gcmc
    a2 = copy.copy(args)
    a2.workload = name
    wl = workload(a2, 0)
    prec = gcmc.FP64 if name == "albedo" else gcmc.FP32
    with __import__("torch").cuda.stream(stream):
        gid, oid, sid, jobs = gcmc.load_workload(ctx, wl, prec, device_inputs=True)
    cfg, tuned = tune_cfg(a2, ctx, jobs, stream)
    steps, plain = WORKLOAD_STEPS[name]
    m = measure(ctx, stream, jobs, cfg, steps, 1, plain)
    roof, alu = rooflines(ctx, wl, m, prec, dev, None)
    g = wl.grid
    ctx.release_grid(gid)
    return {"workload": wl.name, "grid": f"{g.nlon}x{g.nlat}x{g.nr}", "jobs": len(jobs),
            "dtype": "f64" if prec == gcmc.FP64 else "f32", "launch": tuned, "steps": steps,
            "value": m["value"], "unit": "packet-steps/s", "ms_per_step": m["ms_per_step"],
            "spectra_per_s": m["spectra_per_s"], "packet_steps_per_step": m["packet_steps_per_step"],
            "plain_form": m.get("plain_form"), "batched_over_plain": m.get("batched_over_plain"),
            "gather_roofline": {"frac": roof["frac"], "kernel_ms": roof["kernel_ms"],
                                "gathers_per_s": roof["gathers_per_s"], "record_bytes": roof["record_bytes"]},
            "alu_frac": alu["frac"], "clocks": m["clocks"]}


# configuration workloads timed in the default line beside the emission batch: (timed steps, plain steps)
WORKLOAD_STEPS = {"albedo": (5, 3), "phasecurve": (1, 1), "transmission": (3, 1), "transit-scatter": (2, 1)}


def main():
    args = parse()
    if args.workload == "serving":
        return serving_bench(args)
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2110_15640_gb300 import build, gcmc
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()

    wl = workload(args, rank)
    prec = gcmc.FP64 if args.workload == "albedo" else gcmc.FP32     # the 32x16x20 albedo case runs FP64
    stream = torch.cuda.Stream()
    ctx = gcmc.Context(local, stream=stream)
    with torch.cuda.stream(stream):
        gid, oid, sid, jobs = gcmc.load_workload(ctx, wl, prec, device_inputs=True)
    cfg, tuned = tune_cfg(args, ctx, jobs, stream)
    m = measure(ctx, stream, jobs, cfg, args.steps, args.warmup, args.plain_steps, world=world, graph=world == 1)

    # ---------------- end to end through the C ABI from pinned host buffers
    ga, oa = gcmc.workload_arrays(wl, "pinned")
    h2d = gcmc.array_bytes(ga) + gcmc.array_bytes(oa)
    d2h = len(jobs) * (32 * 8 + 4 * 8)
    torch.cuda.synchronize()
    te = time.perf_counter()
    F_band = None
    for _ in range(args.e2e_steps):
        g2 = ctx.upload_grid(wl.grid, device_arrays=ga, memory=gcmc.MEM_HOST)
        o2 = ctx.upload_opacity(g2, wl.opac, device_arrays=oa, memory=gcmc.MEM_HOST)
        jb = gcmc.workload_jobs(wl, g2, o2, ctx.set_sources(g2, wl.source, prec))
        tl, st2 = ctx.run_batch(jb, cfg=cfg)
        obs = [ctx.postscale(g2, wl.mode, tl[q][0], j.n_packets, st2[q].l_tot) for q, j in enumerate(wl.jobs)]
        if wl.mode == gcmc.EMISSION and (wl.jobs[0].g_idx < 0 or wl.opac.kind == gcmc.OPAC_XSEC):
            # band jobs (L_p sums over g) and high-resolution wavelengths: the mean over jobs
            F_band = {"spectrum_F_p_band_mean": float(np.mean([o["F_p"] for o in obs]))}
        elif wl.mode == gcmc.EMISSION:
            F = np.zeros((args.bands, args.gpoints))
            for q, j in enumerate(wl.jobs):
                F[j.lam_idx, j.g_idx] = obs[q]["F_p"]
            F_band = {"spectrum_F_p_band_mean": float(np.mean(F @ wl.opac.wg[:args.gpoints]))}
        elif wl.mode == gcmc.ALBEDO:
            F_band = {"A_g_mean": float(np.mean([o["A_g"] for o in obs]))}
        else:
            F_band = {"area_mean": float(np.mean([o["area"] for o in obs]))}
        ctx.release_grid(g2)
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - te) / max(args.e2e_steps, 1)
    e2e_value = m["packet_steps_per_step"] / t_e2e if args.e2e_steps else None

    g = wl.grid
    traffic = (TRAFFIC_PER_EMISSION_JOB * len(jobs)
               if TRAFFIC_PER_EMISSION_JOB and args.workload == "emission" and g.nlon * g.nlat * g.nr == 409600 else None)
    roof, alu = rooflines(ctx, wl, m, prec, local, traffic)

    workloads = None
    if rank == 0 and world == 1 and args.workload == "emission" and not args.no_workloads:
        ctx.release_grid(gid)
        workloads = {name: workload_line(args, name, ctx, stream, local) for name in WORKLOAD_STEPS}

    serving = None
    if rank == 0 and world == 1 and args.workload == "emission" and args.serving_requests > 0:
        # the serving stream: Poisson arrivals of mixed requests through the continuous-batching server
        serving = serving_run(args.serving_requests, args.hbm_budget_gb)
        del serving["grids"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        nj, npk = CPU_SAMPLE[args.workload]
        rate, dt, _ = cpu_oracle_rate(wl, nj, npk, cores)
        cpu = {"value": rate, "unit": "packet-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{min(nj, len(jobs))} of {len(jobs)} jobs x {npk or 'all their'} packets, S1 + transport, "
                         f"{dt:.1f} s"}
    if rank == 0:
        rec_bytes = 16 if wl.opac.kind == gcmc.OPAC_ALBEDO else 4
        tables = len(jobs) * (len(wl.opac.wg) if wl.mode == gcmc.EMISSION and wl.jobs[0].g_idx < 0 else 1)
        per_step_bytes = tables * g.ncell * (rec_bytes + (12 if wl.mode == gcmc.EMISSION else 0))
        f64 = prec == gcmc.FP64
        line = {
            "metric": "packet-steps/s", "value": m["value"], "unit": "packet-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if f64 else "f32",
            "data": "synthetic",
            "spectra_per_s": m["spectra_per_s"],
            "config": {"workload": wl.name, "jobs": len(jobs), "packets_per_step": m["packets_per_step"],
                       "grid": f"{g.nlon}x{g.nlat}x{g.nr}", "packet_steps_per_step": m["packet_steps_per_step"],
                       "capped_weight": m["capped_weight"],
                       "l2": (f"inputs larger than L2 (per-step cell tables {per_step_bytes / 1e9:.2f} GB)"
                              if per_step_bytes > 129e6 else
                              f"per-step cell tables {per_step_bytes / 1e6:.1f} MB fit in L2 (the workload's own size)"),
                       "precision": ("FP64 march, tables and tallies" if f64 else
                                     "FP32 march and opacities, FP64 luminosities, 64-bit fixed-point pdf and tallies"),
                       "launch": tuned},
            "plain_form": m.get("plain_form"),
            "batched_over_plain": m.get("batched_over_plain"),
            "graph_form": m.get("graph_form"),
            "e2e": {"value": e2e_value, "unit": "packet-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * t_e2e},
            "roofline": roof,
            "alu_roofline": alu,
            "cpu_baseline": cpu,
            "gpu_launches": m["gpu_launches"],
            "clocks": m["clocks"],
            "observables": F_band,
            "workloads": workloads,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
