"""The device-side failure path: a bounded wait that runs out reports
GPA_ERR_TIMEOUT through the status word and the kernel returns, leaving the
context usable. The wait is on a shared-memory mbarrier that nothing arrives
at (no copies, no tensor memory), so the failure is made without a fault."""
import time

import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL_GRAD_FP32, gmm_dev, host, rel_norm, status

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_ns", [1_000, 2_000_000, 50_000_000])
def test_wait_on_a_barrier_nobody_arrives_at_times_out(limit_ns):
    from paper_2104_05372_b300 import _lib
    st = status()
    gave_up = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lib.gpa_check_bounded_wait(limit_ns, st, gave_up)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(st.item()) == _lib.ERR_TIMEOUT
    assert int(gave_up.item()) == 64  # every thread of both wait forms gave up
    assert dt >= limit_ns * 1e-9 * 0.5
    assert dt < limit_ns * 1e-9 + 2.0


def test_library_works_after_a_timed_out_wait():
    import oracle
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300 import _lib
    st = status()
    gave_up = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.gpa_check_bounded_wait(1_000_000, st, gave_up)
    g = synth.gmm_inputs(1000, 10, 5, seed=0)
    st2 = status()
    grads = gpa.gmm_vjp(*gmm_dev(g), g.gamma, g.m, status=st2)
    torch.cuda.synchronize()
    assert int(st.item()) == _lib.ERR_TIMEOUT and int(st2.item()) == 0
    _, *ref = oracle.gmm_grad(g)
    for got, r in zip(grads, ref):
        assert rel_norm(host(got), r) <= TOL_GRAD_FP32
    assert np.isfinite(host(grads[0])).all()
