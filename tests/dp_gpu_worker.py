"""Rank bodies for the multi-process test of the data-parallel paths on one
GPU: each process is one rank of a gloo group, runs the library on its shard
of the units on cuda:0 (the CUDA path itself, not the oracle), and the ranks
sum their Accum vectors with the library's all-reduce helper. Every rank
checks the combined result against the FP64 oracle over all units. The ranks'
kernels never wait on one another: the only exchange is the gloo all-reduce
between launches."""
import numpy as np
import torch
import torch.distributed as dist

TOL_OBJ_FP32, TOL_GRAD_FP32, TOL_BF16 = 1e-5, 1e-4, 3e-3


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gmm_ranks(rank, world, port, n, d, k, seed, prec, from_host):
    import oracle
    import synth
    from paper_2104_05372_b300 import _lib
    from paper_2104_05372_b300 import data_parallel as dp
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        g = synth.gmm_inputs(n, d, k, seed=seed)
        b, e = dp.shard_range(n, rank, world)
        a, mu, q, l = (torch.from_numpy(t).to(dev) for t in (g.alpha, g.mu, g.q, g.l))
        out = torch.zeros(1, dtype=torch.float64, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        if from_host:
            xh = torch.from_numpy(np.ascontiguousarray(g.x[b:e])).pin_memory()
            grads = dp.gmm_vjp_from_host(xh, a, mu, q, l, g.gamma, g.m, prec, seed=0.5, chunk_points=2048,
                                         out=out)
        else:
            xs = torch.from_numpy(np.ascontiguousarray(g.x[b:e])).to(dev)
            grads = dp.gmm_vjp(xs, a, mu, q, l, g.gamma, g.m, prec, seed=0.5, out=out, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        f_ref, *gref = oracle.gmm_grad(g, seed=0.5)
        f = float(out.item())
        tol_f, tol_g = (TOL_OBJ_FP32, TOL_GRAD_FP32) if prec == _lib.PREC_FP32 else (TOL_BF16, TOL_BF16)
        assert abs(f - f_ref) <= tol_f * abs(f_ref), (rank, f, f_ref)
        for name, got, ref in zip(("alpha", "mu", "q", "l"), grads, gref):
            err = _rel(got.cpu().numpy(), ref)
            assert err <= tol_g, (rank, name, err)
    finally:
        dist.destroy_process_group()


def reproj_ranks(rank, world, port, n_cams, n_pts, n_obs, seed, strat):
    import oracle
    import synth
    from paper_2104_05372_b300 import _lib
    from paper_2104_05372_b300 import data_parallel as dp
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=seed)
        b, e = dp.shard_range(n_obs, rank, world, align=1)
        cams, pts = torch.from_numpy(r.cams).to(dev), torch.from_numpy(r.pts).to(dev)
        obs = torch.from_numpy(np.ascontiguousarray(r.obs[b:e])).to(dev)
        w = torch.from_numpy(np.ascontiguousarray(r.w[b:e])).to(dev)
        plan = _lib.gpa_obs_plan_build(obs, n_cams, n_pts) if strat == "sort" else None
        dc = torch.zeros(n_cams, 11, device=dev)
        dpt = torch.zeros(n_pts, 3, device=dev)
        dp.reproj_vjp(cams, pts, obs, w, dc, dpt, strat=strat, plan=plan)
        torch.cuda.synchronize()
        rc, rp, _ = oracle.reproj_vjp(r)
        assert _rel(dc.cpu().numpy(), rc) <= TOL_GRAD_FP32, (rank, _rel(dc.cpu().numpy(), rc))
        assert _rel(dpt.cpu().numpy(), rp) <= TOL_GRAD_FP32, (rank, _rel(dpt.cpu().numpy(), rp))
    finally:
        dist.destroy_process_group()
