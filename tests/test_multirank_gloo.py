"""The multi-rank path on CPU: two gloo ranks split one batch with the
longest-first partition, each runs the CPU oracle on its share (the data path
has no collective), the results are gathered on rank 0 and must equal a
single-process run; the step-time reduction returns the largest rank time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2401_10089_gb300 import shard, workloads  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _mats():
    mats = [workloads.identity_plus(1, n, seed=300 + n, lo=0.1, hi=2.0)[0] for n in (3, 5, 8, 12, 16, 20, 24, 9)]
    mats += list(workloads.spd(4, 10, seed=310, lo=0.1, hi=10.0))
    return mats


def _worker(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    mats = _mats()
    parts = shard.partition(shard.batch_costs(mats), world)
    mine = parts[rank]
    Ls, ds = oracle.logm_batch([mats[i] for i in mine], nthreads=1)
    got = shard.gather_to_root({i: L for i, L in zip(mine, Ls)})
    t = shard.max_over_ranks(float(rank + 1) * 0.5)
    if rank == 0:
        merged = {}
        for g in got:
            merged.update(g)
        np.savez(os.path.join(outdir, "merged.npz"), **{str(k): v for k, v in merged.items()})
        with open(os.path.join(outdir, "tmax.txt"), "w") as f:
            f.write(repr(t))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_covers_and_balances():
    costs = np.array([100.0, 1.0, 50.0, 49.0, 3.0, 2.0])
    parts = shard.partition(costs, 2)
    assert sorted(parts[0] + parts[1]) == list(range(6))
    loads = [costs[p].sum() for p in parts]
    assert max(loads) - min(loads) <= 5.0
    assert shard.partition([], 3) == [[], [], []]


def test_two_gloo_ranks_match_single_process(tmp_path):
    import oracle
    oracle.build()
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    merged = np.load(tmp_path / "merged.npz")
    mats = _mats()
    ref, _ = oracle.logm_batch(mats, nthreads=1)
    assert sorted(int(k) for k in merged.files) == list(range(len(mats)))
    for i, L in enumerate(ref):
        assert np.array_equal(merged[str(i)], L)
    assert float((tmp_path / "tmax.txt").read_text()) == 1.0
