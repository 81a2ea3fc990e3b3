"""Rank bodies for the data-parallel tests (run as gloo ranks on CPU; no GPU).

Every rank builds the same seeded inputs, keeps its shard of the units
(shard_range), accumulates over the shard with the oracle, sums with the
library's all-reduce helper and finishes; the result must equal the oracle
over all units. Failures raise, which fails the spawning test."""
import dataclasses
import os

import numpy as np
import torch
import torch.distributed as dist


def _init(rank, world, port):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def gmm_worker(rank, world, port, n, d, k, seed):
    import oracle
    import synth
    from paper_2104_05372_b300 import data_parallel as dp
    _init(rank, world, port)
    try:
        g = synth.gmm_inputs(n, d, k, seed=seed)
        b, e = dp.shard_range(n, rank, world)
        shard = dataclasses.replace(g, x=np.ascontiguousarray(g.x[b:e]))
        sums = torch.from_numpy(oracle.gmm_accum(shard, seed=0.5) if e > b else
                                np.zeros(k + k * d + k * d * d + 1))
        n_total = dp.total_units(e - b, "cpu")
        assert n_total == n, (n_total, n)
        dp.combine(sums)
        got = oracle.gmm_finish(g, n_total, sums.numpy(), seed=0.5)
        ref = oracle.gmm_grad(g, seed=0.5)
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0]), (got[0], ref[0])
        for a, r in zip(got[1:], ref[1:]):
            assert _rel(a, r) <= 1e-12, _rel(a, r)
    finally:
        dist.destroy_process_group()


def reproj_worker(rank, world, port, n_cams, n_pts, n_obs, seed):
    import oracle
    import synth
    from paper_2104_05372_b300 import data_parallel as dp
    _init(rank, world, port)
    try:
        r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=seed)
        b, e = dp.shard_range(n_obs, rank, world, align=1)
        shard = dataclasses.replace(r, obs=np.ascontiguousarray(r.obs[b:e]), tgt=np.ascontiguousarray(r.tgt[b:e]),
                                    w=np.ascontiguousarray(r.w[b:e]))
        dc, dpt, _ = oracle.reproj_vjp(shard)
        dc, dpt = torch.from_numpy(np.ascontiguousarray(dc)), torch.from_numpy(np.ascontiguousarray(dpt))
        dp.combine(dc)
        dp.combine(dpt)
        rc, rp, _ = oracle.reproj_vjp(r)
        assert _rel(dc.numpy(), rc) <= 1e-12 and _rel(dpt.numpy(), rp) <= 1e-12
    finally:
        dist.destroy_process_group()
