"""gmm_vjp_host: the mixture objective and gradient from host memory (points
streamed in chunks, copies overlapping the reverse pass), against gmm_vjp on
device copies of the same inputs and against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_BF16, TOL_GRAD_FP32, TOL_OBJ_FP32, rel_norm

pytestmark = pytest.mark.gpu


def _host(g, pinned=True):
    ts = [torch.from_numpy(np.ascontiguousarray(a)) for a in (g.x, g.alpha, g.mu, g.q, g.l)]
    return [t.pin_memory() if pinned else t for t in ts]


@pytest.mark.parametrize("n,d,k,prec,chunk,pinned", [
    (5000, 10, 7, 0, 1024, True),      # several chunks, ragged last one
    (1, 1, 1, 0, 0, True),             # one point, no strict-lower entries
    (70000, 64, 20, 0, 0, True),       # default chunk (2^19 > n): one quarter-size chunk, then the rest
    (3000, 64, 33, 1, 512, True),      # tensor-core precision form
    (2000, 16, 5, 0, 384, False),      # pageable host memory
])
def test_host_entry_matches_device_call_and_oracle(n, d, k, prec, chunk, pinned):
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(n, d, k, seed=n + d + k)
    x, a, mu, q, l = _host(g, pinned)
    da, dm, dq, dl, out = gpa.gmm_vjp_host(x, a, mu, q, l, g.gamma, g.m, prec, seed=0.75, chunk_points=chunk)
    torch.cuda.synchronize()
    dev = [t.cuda() for t in (x, a, mu, q, l)]
    o1 = torch.empty(1, dtype=torch.float64, device="cuda")
    ref = gpa.gmm_vjp(*dev, g.gamma, g.m, prec, seed=0.75, out=o1)
    f_ref, *gref = oracle.gmm_grad(g, seed=0.75)
    f0 = oracle.gmm_objective(g)
    tol = TOL_BF16 if prec else TOL_GRAD_FP32
    assert abs(float(out[0]) - float(o1.item())) <= 1e-9 * abs(float(o1.item())) + 1e-9
    assert abs(float(out[0]) - f0) <= (TOL_BF16 if prec else TOL_OBJ_FP32) * abs(f0)
    for h, r_dev, r_or in zip((da, dm, dq, dl), ref, gref):
        if r_or.size:
            assert rel_norm(h.numpy(), r_dev.cpu().numpy()) <= (1e-4 if prec else 1e-5)
            assert rel_norm(h.numpy(), r_or) <= tol


def test_host_entry_rejects_bad_arguments():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300 import _lib
    g = synth.gmm_inputs(100, 16, 3, seed=2)
    x, a, mu, q, l = _host(g)
    with pytest.raises(gpa.GpaError) as e:
        gpa.gmm_vjp_host(x, a, mu, q, l, prec=1)  # D = 16 has no tensor-core form
    assert e.value.code == 6
    assert gpa.gpa_gmm_vjp_host_workspace_bytes(0, 16, 3) == 0
    assert gpa.gpa_gmm_vjp_host_workspace_bytes(10, 129, 3) == 0
    small = _lib.workspace(1024, "cuda")
    with pytest.raises(gpa.GpaError) as e:
        gpa.gmm_vjp_host(x, a, mu, q, l, ws=small)
    assert e.value.code == _lib.ERR_WORKSPACE
