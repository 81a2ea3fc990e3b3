"""Data-parallel host logic on CPU: shard ranges, and the shard / all-reduce /
finish sequence run as two gloo ranks with the oracle as the per-shard engine.
The combined result must equal the oracle over all units, which pins the
additivity of the Accum sums over a partition of the units (Sec. 2.3.2)."""
import socket

import pytest
import torch.multiprocessing as mp

import dp_worker
from paper_2104_05372_b300.data_parallel import shard_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n", [0, 1, 127, 128, 129, 1000, 4096, 100003])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("align", [1, 128])
def test_shard_range_partitions(n, world, align):
    got = [shard_range(n, r, world, align) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == n
    for (b0, e0), (b1, e1) in zip(got, got[1:]):
        assert e0 == b1  # contiguous, disjoint, in rank order
    sizes = [e - b for b, e in got]
    assert sum(sizes) == n
    assert all(b % align == 0 for b, e in got if e > b)
    assert max(sizes) - min(sizes) <= align


def test_shard_range_rejects_bad_arguments():
    for args in [(-1, 0, 1), (10, 1, 1), (10, -1, 2), (10, 0, 0)]:
        with pytest.raises(ValueError):
            shard_range(*args)


@pytest.mark.parametrize("n,d,k", [(1000, 5, 3), (300, 3, 4)])
def test_gmm_gradient_two_gloo_ranks(n, d, k):
    mp.spawn(dp_worker.gmm_worker, args=(2, _free_port(), n, d, k, 11), nprocs=2, join=True)


def test_gmm_gradient_rank_with_empty_shard():
    # 100 points in 128-point blocks: rank 0 of 2 holds nothing
    mp.spawn(dp_worker.gmm_worker, args=(2, _free_port(), 100, 4, 2, 12), nprocs=2, join=True)


def test_reprojection_vjp_two_gloo_ranks():
    mp.spawn(dp_worker.reproj_worker, args=(2, _free_port(), 7, 50, 999, 13), nprocs=2, join=True)
