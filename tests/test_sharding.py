"""Multi-process host logic of the sharded batch (gloo, world size 2, CPU):
the ranks' zone slices tile the global batch exactly, and the reported time
is the max over ranks while the work is the sum."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from kn_inputs import net150, profile_zones
    from paper_1409_5826_gb300 import shard
    z = profile_zones(net150(), 6, base_seed=shard.zone_seed_base(rank, world, 6))
    ms, steps, ok = shard.aggregate(100.0 + 50.0 * rank, 1000 * (rank + 1), 6)
    out[rank] = (z.T0.tolist(), z.rho0.tolist(), ms, steps, ok)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_and_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from kn_inputs import net150, profile_zones
    whole = profile_zones(net150(), 12, base_seed=1000)
    T0 = np.concatenate([out[0][0], out[1][0]])
    rho0 = np.concatenate([out[0][1], out[1][1]])
    assert np.array_equal(T0, whole.T0) and np.array_equal(rho0, whole.rho0)
    for r in range(2):
        assert out[r][2] == 150.0          # max of 100, 150 ms
        assert out[r][3] == 3000           # 1000 + 2000 steps
        assert out[r][4] == 12             # zones summed


def test_zone_slice_bounds():
    from paper_1409_5826_gb300 import shard
    assert shard.zone_slice(3, 4, 10) == (30, 40)
    with pytest.raises(ValueError):
        shard.zone_slice(4, 4, 10)


def _strong_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from kn_inputs import net150, profile_zones
    from paper_1409_5826_gb300 import shard
    whole = profile_zones(net150(), 37)
    parts = shard.balanced_partition(shard.cost_key(net150(), whole), world)
    out[rank] = parts[rank].tolist()
    dist.barrier()
    dist.destroy_process_group()


def test_strong_partition_two_ranks_cover_the_batch():
    """Each rank computes the cost-balanced split on its own; together the
    ranks hold every zone of the batch exactly once, sizes within one."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_strong_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    allz = sorted(out[0] + out[1])
    assert allz == list(range(37))
    assert abs(len(out[0]) - len(out[1])) <= 1


def test_strong_partition_balances_oracle_steps(oracle_mod):
    """The serpentine deal by predicted cost balances the measured work (the
    oracle's accepted steps) far better than contiguous slices of the batch
    sorted by that cost would, and about as well as a random split."""
    from kn_inputs import net150, profile_zones
    from paper_1409_5826_gb300 import shard
    net = net150()
    z = profile_zones(net, 48, t_end=2e-11)
    steps = oracle_mod.Oracle(net).integrate_batch(z, threads=8)["steps"].astype(float)
    key = shard.cost_key(net, z)
    assert np.corrcoef(key, steps)[0, 1] > 0.5  # the key predicts the cost
    for world in (2, 4):
        parts = shard.balanced_partition(key, world)
        loads = np.array([steps[p].sum() for p in parts])
        order = np.argsort(-key)
        contiguous = np.array([steps[c].sum() for c in np.array_split(order, world)])
        assert loads.max() / loads.mean() < 1.15, loads
        assert loads.max() / loads.mean() < contiguous.max() / contiguous.mean()
