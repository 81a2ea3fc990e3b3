"""The data-parallel paths as two real ranks (processes of a gloo group) on
one GPU: each rank runs the library on its shard, the ranks all-reduce their
Accum vectors (the mixture's exchange vector; the reprojection's camera and
point cotangents) and every rank must hold the oracle's result over all units
(Accum sums over a partition of the units combine by addition, Sec. 2.3.2).
The ranks' kernels do not wait on one another; the collective runs between
launches on the host side of gloo."""
import socket

import pytest
import torch.multiprocessing as mp

import dp_gpu_worker

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,d,k,prec,from_host", [(20000, 64, 20, 0, False), (9000, 10, 5, 0, True),
                                                   (12000, 48, 9, 1, False), (7000, 128, 6, 1, True)])
def test_gmm_two_ranks_on_one_gpu(n, d, k, prec, from_host):
    mp.spawn(dp_gpu_worker.gmm_ranks, args=(2, _free_port(), n, d, k, 21, prec, from_host), nprocs=2, join=True)


@pytest.mark.parametrize("strat", ["atomic", "sort"])
def test_reprojection_two_ranks_on_one_gpu(strat):
    mp.spawn(dp_gpu_worker.reproj_ranks, args=(2, _free_port(), 300, 2000, 50001, 22, strat), nprocs=2,
             join=True)
