"""The multi-rank path on CPU: active-range sharding of one system over
world_size-2 gloo ranks (each rank holding its own replica of the tree) must
give exactly the single-process result, and the step-time reduction must
return the slowest rank's time.  The per-rank force evaluation here is the
FP64 oracle walk; on GPUs it is each rank's ``System.compute_forces``."""
import os
import socket

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def shard():
    import __graft_entry__ as g

    g.build()
    from paper_1909_04667_gb300 import shard as m

    return m


def test_active_range_partitions(shard):
    for n in (0, 1, 2, 7, 8, 1000, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.active_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.active_range(10, 2, 2)


def test_weighted_ranges_balance_work(shard):
    """Ranges weighted by per-particle cost (interaction counts) cover the set
    in order and hold equal work to within one item's weight."""
    rng = np.random.default_rng(1)
    for n, world in ((1000, 2), (1001, 3), (5000, 8), (3, 4), (1, 2)):
        w = rng.lognormal(0.0, 1.5, n) * 700  # a halo's centre costs far more than its outskirts
        w[: n // 10] *= 5
        ranges = [shard.active_range(n, r, world, w) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        for (a, b), (c, d) in zip(ranges, ranges[1:]):
            assert b == c and a <= b
        loads = [w[a:b].sum() for a, b in ranges]
        assert max(loads) <= w.sum() / world + w.max() + 1e-9 * w.sum()
    # zero weights fall back to equal counts
    assert [shard.active_range(10, r, 2, np.zeros(10)) for r in range(2)] == [(0, 5), (5, 10)]
    with pytest.raises(ValueError):
        shard.active_range(4, 0, 2, [1.0, 2.0])
    with pytest.raises(ValueError):
        shard.active_range(2, 0, 2, [1.0, -1.0])


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, n, n_active, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1909_04667_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pos, mass = W.plummer(n, 77)
        tree = oracle.Tree(pos, mass, bucket=4, shift=tuple(W.root_shift(77)))  # this rank's replica
        ids = np.random.default_rng(3).choice(n, n_active, replace=False).astype(np.uint32)

        def compute(part):
            acc, pot, nint = tree.walk(part, 1.0, 0.01, theta=0.6, nthreads=1)
            return torch.from_numpy(acc), torch.from_numpy(pot), torch.from_numpy(nint.astype(np.int64))

        # ranges balanced by each particle's interaction count from a previous
        # evaluation (the same on every rank)
        weights = tree.walk(ids, 1.0, 0.01, theta=0.6, nthreads=1)[2].astype(np.float64) if n_active > 1 else None
        acc, pot, nint = shard.sharded_compute_forces(compute, ids, rank, world, weights=weights)
        slowest = shard.max_over_ranks(1.5 + rank)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), acc=acc.numpy(), pot=pot.numpy(), nint=nint.numpy(),
                 slowest=slowest)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_active", [1, 2001])
def test_two_gloo_ranks_match_one_process(shard, oracle_mod, tmp_path, n_active):
    import torch.multiprocessing as mp

    n, world = 3000, 2
    mp.start_processes(rank_main, args=(world, free_port(), n, n_active, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    pos, mass = W.plummer(n, 77)
    tree = oracle_mod.Tree(pos, mass, bucket=4, shift=tuple(W.root_shift(77)))
    ids = np.random.default_rng(3).choice(n, n_active, replace=False).astype(np.uint32)
    acc, pot, nint = tree.walk(ids, 1.0, 0.01, theta=0.6, nthreads=1)
    for r in range(world):
        got = np.load(tmp_path / ("rank%d.npz" % r))
        # every rank ends with the whole result, bit for bit the single-process walk
        np.testing.assert_array_equal(got["acc"], acc)
        np.testing.assert_array_equal(got["pot"], pot)
        np.testing.assert_array_equal(got["nint"], nint.astype(np.int64))
        assert float(got["slowest"]) == 1.5 + (world - 1)
