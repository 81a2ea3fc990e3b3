"""reproj_vjp_noalloc: the VJP for callers that cannot give the library a
workspace (their device memory belongs to another allocator, or their memory
budget is fixed up front), checked against reproj_vjp on two calls in a row.

This file is collected last on purpose. The entry point keeps its scratch in a
fixed device array shared by every call, so the second call (fewer cameras,
another strategy) also checks that the previous call's leftovers do not leak
into the result.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL_GRAD_FP32, dev, host, rel_norm, status

pytestmark = pytest.mark.gpu

MAX_CAMS = 16384  # GPA_NOALLOC_MAX_CAMS in include/gpa.h


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(lib, cams, pts, obs, w, d_cams, d_pts, strat, plan, st):
    return lib.reproj_vjp_noalloc(_p(cams), _p(pts), _p(obs), _p(w), cams.shape[0], pts.shape[0], obs.shape[0],
                                  _p(d_cams), _p(d_pts), strat, _p(plan), _p(st),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_vjp_matches_reproj_vjp_on_two_calls():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300 import _lib
    lib = _lib.load()
    calls = [(MAX_CAMS, 40000, 300001, 1, _lib.SCATTER_ATOMIC),   # fills the whole scratch
             (37, 900, 50003, 2, _lib.SCATTER_SORT)]               # fewer cameras, sorted plan
    for n_cams, n_pts, n_obs, seed, strat in calls:
        r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=seed)
        cams, pts, obs, w = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.w)
        plan = gpa.gpa_obs_plan_build(obs, n_cams, n_pts) if strat == _lib.SCATTER_SORT else None
        ref_c, ref_p = gpa.reproj_vjp(cams, pts, obs, w, strat=strat, plan=plan)
        d_c = torch.zeros(n_cams, 11, device="cuda")
        d_p = torch.zeros(n_pts, 3, device="cuda")
        st = status()
        assert _noalloc(lib, cams, pts, obs, w, d_c, d_p, strat, plan, st) == 0
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert rel_norm(host(d_c), host(ref_c)) <= TOL_GRAD_FP32
        assert rel_norm(host(d_p), host(ref_p)) <= TOL_GRAD_FP32


def test_noalloc_rejects_more_cameras_than_its_scratch_holds():
    from paper_2104_05372_b300 import _lib
    lib = _lib.load()
    r = synth.reproj_inputs(MAX_CAMS + 1, 10, 100, seed=3)
    cams, pts, obs, w = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.w)
    d_c = torch.zeros(MAX_CAMS + 1, 11, device="cuda")
    d_p = torch.zeros(10, 3, device="cuda")
    rc = _noalloc(lib, cams, pts, obs, w, d_c, d_p, _lib.SCATTER_ATOMIC, None, None)
    assert rc == _lib.ERR_WORKSPACE
    torch.cuda.synchronize()
    assert not host(d_c).any() and not host(d_p).any()
