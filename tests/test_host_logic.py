"""Host-side logic that needs no GPU: the autotuner's job sample and its search, and the saved
launch configuration."""
import pytest

from paper_2110_15640_gb300 import autotune
from paper_2110_15640_gb300 import synth as S


def _jobs(n, packets):
    return [S.Job(lam_idx=q, g_idx=0, n_packets=packets, key=q) for q in range(n)]


@pytest.mark.parametrize("n,packets", [(9532, 10_000), (240, 1_000_000), (960, 500_000), (40, 1_000_000), (5, 100), (1, 10)])
def test_sample_jobs_fills_the_gpu_or_takes_everything(n, packets):
    jobs = _jobs(n, packets)
    s = autotune.sample_jobs(jobs)
    assert len(s) == len({id(j) for j in s})
    assert all(j in jobs for j in s)
    total = sum(j.n_packets for j in s)
    if n * packets >= 64_000_000 and n >= 16:
        assert total >= 64_000_000 * (1 - 1.0 / len(s)) and len(s) >= 16
    else:
        assert s == jobs
    # spread evenly over the list, not its head
    if len(s) < n:
        keys = [j.key for j in s]
        assert keys[0] == 0 and keys[-1] >= n - n / len(s) - 1
        gaps = [b - a for a, b in zip(keys, keys[1:])]
        assert max(gaps) - min(gaps) <= 1


def test_coordinate_search_finds_a_separable_minimum(monkeypatch):
    """With a cost that is a sum over the axes, the coordinate search reaches the global minimum."""
    target = {"shape": (64, 0), "chunk": 128, "refill_min": 16, "interval": 8}
    space = autotune.DEFAULT_SPACE

    def cost(cfg):
        c = {"shape": (cfg.block, cfg.blocks_per_sm), "chunk": cfg.chunk, "refill_min": cfg.refill_min,
             "interval": cfg.interval}
        return 10.0 + sum(abs(space[k].index(c[k]) - space[k].index(target[k])) for k in target)

    monkeypatch.setattr(autotune, "_time_cfg", lambda ctx, jobs, cfg, reps, stream: cost(cfg))
    cfg, best, table = autotune.tune(None, [], None)
    assert best == autotune.as_cfg_dict(target)
    assert (cfg.block, cfg.blocks_per_sm, cfg.chunk, cfg.refill_min, cfg.interval) == (64, 0, 128, 16, 8)
    assert min(ms for _, ms in table) == 10.0
    # two passes over the axes; a value is re-run at most once per axis after the best one moved
    assert len(table) <= 1 + 2 * sum(len(v) for v in space.values())


def test_launch_shape_is_one_axis(monkeypatch):
    """A cost whose best blocks-per-SM value depends on the block size (as occupancy does): searching the
    block size and the blocks per SM as one axis of shapes still finds the minimum from the start point."""
    def cost(cfg):
        shape = {(128, 6): 1.0, (256, 0): 2.0, (128, 8): 5.0}.get((cfg.block, cfg.blocks_per_sm), 9.0)
        return shape + abs(cfg.chunk - 256) / 1e4

    monkeypatch.setattr(autotune, "_time_cfg", lambda ctx, jobs, cfg, reps, stream: cost(cfg))
    cfg, best, table = autotune.tune(None, [], None)
    assert (best["block"], best["blocks_per_sm"], best["chunk"]) == (128, 6, 256)


def test_saved_configuration_round_trips(tmp_path):
    best = {"block": 64, "blocks_per_sm": 6, "chunk": 256, "refill_min": 4, "interval": 16}
    p = tmp_path / "tune.json"
    autotune.save(str(p), best, [(best, 1.5)])
    cfg, b = autotune.load(str(p))
    assert b == best
    assert (cfg.block, cfg.blocks_per_sm, cfg.chunk, cfg.interval, cfg.refill_min) == (64, 6, 256, 16, 4)
    assert autotune.load(str(tmp_path / "missing.json")) is None
