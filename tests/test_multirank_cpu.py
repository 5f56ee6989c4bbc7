"""The multi-GPU path of the benchmark is replicas only: every rank advances its own run with
its own seed, no collective touches the data path, the slowest rank's time is taken (max over
ranks) and the whole-job rate sums the ranks' particles.  Checked here with two gloo ranks on
the host (the same collectives NCCL performs on the GPUs)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import bench
    import plasma
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench._rank_env()
    # each replica's timed region: a different duration per rank; the job takes the slowest
    ms = 10.0 + 5.0 * rank
    bench._barrier(True)
    ms_max = bench._max_over_ranks(ms, True)
    # the replica workloads differ (seed + rank) but have the same shape
    wl = plasma.fill(workloads.config_large(scheme=1, seed=workloads.BASE_SEED + rank, scale=64),
                     count=8)
    x0 = torch.from_numpy(wl.species[0].x[:, :8].copy())
    gathered = [torch.zeros_like(x0) for _ in range(world)]
    dist.all_gather(gathered, x0)
    n = wl.n_particles
    out[rank] = (r, w, loc, ms_max, bench.replica_rate(n, w, 10, ms_max), n,
                 bool(torch.equal(gathered[0], gathered[1])))
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r, w, loc, ms_max, rate, n, same = res[rank]
        assert (r, w, loc) == (rank, world, rank)
        assert ms_max == 15.0                      # the slowest rank
        assert rate == n * world * 10 / 15e-3      # both replicas' particles over that time
        assert not same                            # independent seeds per replica
    assert res[0][5] == res[1][5]                  # same workload shape on every rank
