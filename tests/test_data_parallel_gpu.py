"""Data-parallel GMM gradient on one GPU: the points split into shards,
gmm_vjp_partial per shard, the exchange vectors summed on the device (the
all-reduce's arithmetic), gmm_vjp_finalize; compared with gmm_vjp over all
points and with the FP64 oracle. Also the one-rank path of the helpers."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_BF16, TOL_GRAD_FP32, TOL_OBJ_FP32, gmm_dev, host, rel_norm, status

pytestmark = pytest.mark.gpu


def _shards_then_finalize(g, world, prec, seed=1.0):
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300.data_parallel import shard_range
    x, a, mu, q, l = gmm_dev(g)
    st = status()
    total = torch.zeros(gpa.gpa_gmm_exchange_len(g.d, g.k), dtype=torch.float64, device="cuda")
    for r in range(world):
        b, e = shard_range(g.n, r, world)
        if e > b:
            total += gpa.gmm_vjp_partial(x[b:e].contiguous(), a, mu, q, l, g.gamma, g.m, prec, seed=seed, status=st)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    grads = gpa.gmm_vjp_finalize(a, mu, q, l, g.n, total, g.gamma, g.m, prec, seed=seed, out=out, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return float(out.item()), [host(t) for t in grads]


@pytest.mark.parametrize("n,d,k,world", [(1000, 10, 5, 2), (5000, 64, 33, 3), ((1 << 14) + 5, 17, 8, 4),
                                         (300, 2, 3, 8)])
def test_fp32_shards_match_single_call_and_oracle(n, d, k, world):
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(n, d, k, seed=n + k)
    f, grads = _shards_then_finalize(g, world, gpa.PREC_FP32, seed=0.75)
    x, a, mu, q, l = gmm_dev(g)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    one = [host(t) for t in gpa.gmm_vjp(x, a, mu, q, l, g.gamma, g.m, seed=0.75, out=out)]
    f_ref, *gref = oracle.gmm_grad(g, seed=0.75)
    assert abs(f - f_ref) <= TOL_OBJ_FP32 * abs(f_ref)
    assert abs(f - float(out.item())) <= 1e-6 * abs(f_ref)
    for s, o, r in zip(grads, one, gref):
        assert rel_norm(s, r) <= TOL_GRAD_FP32
        assert rel_norm(s, o) <= 1e-5


@pytest.mark.parametrize("n,d,k,world", [(3000, 48, 9, 2), (4000, 128, 5, 3)])
def test_tensor_core_shards_match_oracle(n, d, k, world):
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(n, d, k, seed=n + k)
    f, grads = _shards_then_finalize(g, world, gpa.PREC_BF16_TC)
    f_ref, *gref = oracle.gmm_grad(g)
    assert abs(f - f_ref) <= TOL_BF16 * abs(f_ref)
    for s, r in zip(grads, gref):
        assert rel_norm(s, r) <= TOL_BF16


def test_exchange_vector_is_additive_over_shards():
    """partial(all points) == partial(first half) + partial(second half), up to
    FP32 rounding of the per-chunk sums; successive calls accumulate (+=)."""
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(4096, 24, 6, seed=5)
    x, a, mu, q, l = gmm_dev(g)
    full = gpa.gmm_vjp_partial(x, a, mu, q, l, g.gamma, g.m)
    h = gpa.gmm_vjp_partial(x[:2048].contiguous(), a, mu, q, l, g.gamma, g.m)
    gpa.gmm_vjp_partial(x[2048:].contiguous(), a, mu, q, l, g.gamma, g.m, exch=h)
    assert rel_norm(host(h), host(full)) <= 1e-5


def test_helpers_without_a_process_group():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300 import data_parallel as dp
    g = synth.gmm_inputs(2000, 12, 4, seed=6)
    x, a, mu, q, l = gmm_dev(g)
    one = [host(t) for t in gpa.gmm_vjp(x, a, mu, q, l, g.gamma, g.m)]
    dpg = [host(t) for t in dp.gmm_vjp(x, a, mu, q, l, g.gamma, g.m)]
    for u, v in zip(dpg, one):
        assert rel_norm(u, v) <= 1e-5
    r = synth.reproj_inputs(16, 200, 3000, seed=7)
    cams, pts = torch.from_numpy(r.cams).cuda(), torch.from_numpy(r.pts).cuda()
    obs, w = torch.from_numpy(r.obs).cuda(), torch.from_numpy(r.w).cuda()
    dc, dpt = torch.zeros(16, 11, device="cuda"), torch.zeros(200, 3, device="cuda")
    dp.reproj_vjp(cams, pts, obs, w, dc, dpt)
    rc, rp, _ = oracle.reproj_vjp(r)
    assert rel_norm(host(dc), rc) <= TOL_GRAD_FP32 and rel_norm(host(dpt), rp) <= TOL_GRAD_FP32


def test_finalize_rejects_bad_arguments():
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(100, 8, 3, seed=1)
    x, a, mu, q, l = gmm_dev(g)
    exch = gpa.gmm_vjp_partial(x, a, mu, q, l)
    with pytest.raises(gpa.GpaError):
        gpa.gmm_vjp_finalize(a, mu, q, l, 0, exch)
    with pytest.raises(gpa.GpaError) as e:
        gpa.gmm_vjp_finalize(a, mu, q, l, 100, exch, prec=gpa.PREC_BF16_TC)
    assert e.value.code == 6


@pytest.mark.parametrize("n,chunk", [(5000, 1024), (300, 1 << 18), (1 << 15, 4096)])
def test_streamed_from_host_matches_device_call(n, chunk):
    """Points in pinned host memory, copied chunk by chunk on a side stream while
    the previous chunk accumulates: the same gradient and objective as one call
    on device-resident points (float32 partial sums in another grouping)."""
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300 import data_parallel as dp
    g = synth.gmm_inputs(n, 24, 7, seed=n)
    x, a, mu, q, l = gmm_dev(g)
    out1 = torch.empty(1, dtype=torch.float64, device="cuda")
    one = [host(t) for t in gpa.gmm_vjp(x, a, mu, q, l, g.gamma, g.m, out=out1)]
    xh = torch.from_numpy(g.x).pin_memory()
    out2 = torch.empty(1, dtype=torch.float64, device="cuda")
    st = status()
    grads = dp.gmm_vjp_from_host(xh, a, mu, q, l, g.gamma, g.m, chunk_points=chunk, out=out2)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert abs(float(out2.item()) - float(out1.item())) <= 1e-9 * abs(float(out1.item()))
    for u, v in zip([host(t) for t in grads], one):
        assert rel_norm(u, v) <= 1e-5
