"""reproj_vjp_noalloc: the VJP for callers that cannot give the library a
workspace (their device memory belongs to another allocator, or their memory
budget is fixed up front), checked against reproj_vjp on two calls in a row.

This file is collected last on purpose, so that a run that stops at the first
failure has run every other test before it. The entry point keeps its scratch
in a fixed device array shared by every call; the second test fills that array
with NaN records (a call on NaN cameras) before a call with fewer cameras, so a
record that is read without having been rewritten by the same call shows up as
a NaN in the result.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL_GRAD_FP32, dev, host, rel_norm, status

pytestmark = pytest.mark.gpu



def _header_max_cams():
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gpa.h")
    m = re.search(r"#define\s+GPA_NOALLOC_MAX_CAMS\s+(\d+)", open(hdr).read())
    assert m, "GPA_NOALLOC_MAX_CAMS not declared in gpa.h"
    return int(m.group(1))


MAX_CAMS = _header_max_cams()


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


def test_noalloc_rewrites_every_record_it_reads():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300 import _lib
    lib = _lib.load()
    # poison the whole scratch: NaN cameras expand to NaN records
    r = synth.reproj_inputs(MAX_CAMS, 100, 1000, seed=4)
    cams = dev(np.full_like(r.cams, np.nan))
    pts, obs, w = dev(r.pts), dev(r.obs), dev(r.w)
    d_c = torch.zeros(MAX_CAMS, 11, device="cuda")
    d_p = torch.zeros(100, 3, device="cuda")
    assert _noalloc(lib, cams, pts, obs, w, d_c, d_p, _lib.SCATTER_ATOMIC, None, None) == 0
    torch.cuda.synchronize()
    assert np.isnan(host(d_c)).any()
    for strat in (_lib.SCATTER_WARPAGG, _lib.SCATTER_SORT):
        r = synth.reproj_inputs(1000, 3000, 40007, seed=5)
        cams, pts, obs, w = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.w)
        plan = gpa.gpa_obs_plan_build(obs, 1000, 3000) if strat == _lib.SCATTER_SORT else None
        ref_c, ref_p = gpa.reproj_vjp(cams, pts, obs, w, strat=strat, plan=plan)
        d_c = torch.zeros(1000, 11, device="cuda")
        d_p = torch.zeros(3000, 3, device="cuda")
        st = status()
        assert _noalloc(lib, cams, pts, obs, w, d_c, d_p, strat, plan, st) == 0
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        hc, hp = host(d_c), host(d_p)
        assert np.isfinite(hc).all() and np.isfinite(hp).all()
        assert rel_norm(hc, host(ref_c)) <= TOL_GRAD_FP32
        assert rel_norm(hp, host(ref_p)) <= TOL_GRAD_FP32


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
