"""World-size-2 gloo tests (CPU) of the multi-GPU host logic: packet and job sharding with an exact
fixed-point all-reduce of the tallies, distinct per-rank seeds, and max-over-ranks timing.  The
ranks compute with the FP64 oracle, which gives each packet the same contribution on any rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2110_15640_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2110_15640_gb300 import synth as S

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # packet sharding of one job
        wl = S.config1_albedo(n_packets=3000, nlon=8, nlat=6, nr=10)
        job = wl.jobs[0]
        p0, nrun = shard.split_packets(job.n_packets, rank, world)
        r = O.run(wl, job, packet0=p0, n_run=nrun, per_packet=True)
        total = shard.reduce_fixed(shard.to_fixed(r["pk_f"][:, 0]).sum())
        # job sharding of a small batch (emission, 4 jobs)
        we = S.config2_emission(n_packets=500, nlon=12, nlat=6, nr=8, nb=2, ng=2)
        loc = np.zeros(len(we.jobs), np.int64)
        for q in shard.split_jobs(len(we.jobs), rank, world):
            rr = O.run(we, we.jobs[q], per_packet=True)
            loc[q] = shard.to_fixed(rr["pk_f"][:, 0]).sum()
        jt = shard.reduce_fixed(loc)
        tmax = shard.max_over_ranks(1.0 + rank)
        out[rank] = (int(total.item()), jt.numpy().tolist(), tmax, shard.rank_seed(2, rank))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_is_exact():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    from oracle import oracle as O
    from paper_2110_15640_gb300 import synth as S
    wl = S.config1_albedo(n_packets=3000, nlon=8, nlat=6, nr=10)
    ref = O.run(wl, wl.jobs[0], per_packet=True)
    want = int(shard.to_fixed(ref["pk_f"][:, 0]).sum())
    we = S.config2_emission(n_packets=500, nlon=12, nlat=6, nr=8, nb=2, ng=2)
    want_jobs = [int(shard.to_fixed(O.run(we, j, per_packet=True)["pk_f"][:, 0]).sum()) for j in we.jobs]
    for rank in range(world):
        total, jt, tmax, seed = out[rank]
        assert total == want
        assert jt == want_jobs
        assert tmax == 2.0
    assert out[0][3] != out[1][3]


@pytest.mark.parametrize("n,world", [(10, 3), (7, 2), (2, 4), (0, 2)])
def test_packet_split_covers_range(n, world):
    seen = []
    for r in range(world):
        p0, k = shard.split_packets(n, r, world)
        seen += list(range(p0, p0 + k))
    assert seen == list(range(n))
