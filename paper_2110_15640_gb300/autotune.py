"""Launch-parameter autotuner for the persistent transport kernel.

Searches the launch shape (block size and blocks per SM), packets per work item (chunk), refill
threshold and refill interval of gcmc_run_batch on a sample of the caller's jobs, timing each
candidate with CUDA events on the context's stream, and returns the fastest gcmc_launch_cfg.  Results do not depend on the launch
parameters (tallies are order-independent fixed point), so tuning never changes a spectrum.
"""
from __future__ import annotations

import itertools
import json
import os

from . import gcmc

# The block size and the blocks per SM form one axis (launch shapes): a kernel holds as many blocks per
# SM as its registers allow, so with one axis per parameter a coordinate search could stop at a block
# size whose best blocks-per-SM value lies on another block size's row.  blocks_per_sm 0: as many as fit.
SHAPES = [(128, 8), (128, 6), (128, 5), (128, 0), (64, 0), (256, 0)]
DEFAULT_SPACE = {
    "shape": SHAPES,
    "chunk": [32, 64, 128, 256, 512, 1024, 2048],
    "refill_min": [4, 8, 16, 32],
    "interval": [2, 4, 8, 16, 24, 32],
}
# where the coordinate search starts: 128-thread blocks, 8 per SM where the kernel fits them (the
# scattering kernels hold 5), 512-packet work items, refill at 16 idle lanes every 16 steps (the region
# of the fastest launches measured for the emission and phase-curve batches on a GB300)
DEFAULT_START = {"shape": (128, 8), "chunk": 512, "refill_min": 16, "interval": 16}


def as_cfg_dict(c):
    """a search point as the launch configuration's fields"""
    return {"block": c["shape"][0], "blocks_per_sm": c["shape"][1], "chunk": c["chunk"], "refill_min": c["refill_min"],
            "interval": c["interval"]}


def sample_jobs(jobs, min_jobs=16, min_packets=64_000_000):
    """Jobs spread evenly over the list, at least min_jobs of them and at least min_packets packets in
    all (or every job): enough work items that every resident warp takes a dozen even at the largest
    chunk size the search tries (a smaller sample ends in a tail of half-empty waves that favours
    small items), so workloads of many small jobs are tuned on the load they present."""
    n = len(jobs)
    mean = max(1.0, sum(j.n_packets for j in jobs) / max(n, 1))
    want = min(n, max(min_jobs, int(-(-min_packets // mean))))
    return [jobs[(q * n) // want] for q in range(want)]


def _time_cfg(ctx, jobs, cfg, reps, stream):
    import torch

    out = torch.zeros((len(jobs), gcmc.MAX_OBS), dtype=torch.float64, device="cuda")
    ctx.run_batch(jobs, cfg=cfg, tallies=out, stats=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        ctx.run_batch(jobs, cfg=cfg, tallies=out, stats=False)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune(ctx, jobs, stream, space=None, reps=2, coordinate=True, log=None, full_jobs=None, finalists=4):
    """Return (best gcmc_launch_cfg, table of (cfg dict, ms)).  coordinate=True searches one axis at a
    time from the defaults, twice over (about thirty runs), instead of the full product.  With full_jobs
    (the whole batch the sample was drawn from), the `finalists` fastest configurations on the sample are
    timed once more on the whole batch and the fastest there is returned: a sample can favour work-item
    sizes and refill settings that do not carry over to the batch."""
    space = space or DEFAULT_SPACE
    best = dict(DEFAULT_START)
    table = []

    def run(c):
        d = as_cfg_dict(c)
        cfg = gcmc.gcmc_launch_cfg(d["block"], d["blocks_per_sm"], d["chunk"], d["interval"], d["refill_min"], 0)
        ms = _time_cfg(ctx, jobs, cfg, reps, stream)
        table.append((d, ms))
        if log:
            log(f"autotune {d} {ms:.2f} ms")
        return ms

    if coordinate:
        best_ms = run(best)
        for _ in range(2):
            for axis, values in space.items():
                for v in values:
                    if v == best[axis]:
                        continue
                    c = dict(best, **{axis: v})
                    ms = run(c)
                    if ms < best_ms:
                        best, best_ms = c, ms
    else:
        keys = list(space)
        best_ms = float("inf")
        for vals in itertools.product(*(space[k] for k in keys)):
            c = dict(zip(keys, vals))
            ms = run(c)
            if ms < best_ms:
                best, best_ms = c, ms
    best = as_cfg_dict(best)
    if full_jobs is not None and len(full_jobs) > len(jobs):
        seen, cands = set(), []
        for c, _ in sorted(table, key=lambda t: t[1]):
            key = tuple(sorted(c.items()))
            if key not in seen:
                seen.add(key)
                cands.append(c)
            if len(cands) == finalists:
                break
        best_full = float("inf")
        for c in cands:
            cfg = gcmc.gcmc_launch_cfg(c["block"], c["blocks_per_sm"], c["chunk"], c["interval"], c["refill_min"], 0)
            ms = _time_cfg(ctx, full_jobs, cfg, 2, stream)
            if log:
                log(f"autotune (whole batch) {c} {ms:.2f} ms")
            if ms < best_full:
                best, best_full = c, ms
    cfg = gcmc.gcmc_launch_cfg(best["block"], best["blocks_per_sm"], best["chunk"], best["interval"], best["refill_min"], 0)
    return cfg, best, table


def save(path, best, table):
    with open(path, "w") as f:
        json.dump({"best": best, "table": [{"cfg": c, "ms": ms} for c, ms in table]}, f, indent=1)


def load(path):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        b = json.load(f)["best"]
    return gcmc.gcmc_launch_cfg(b["block"], b.get("blocks_per_sm", 0), b["chunk"], b["interval"], b["refill_min"], 0), b
