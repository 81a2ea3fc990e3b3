"""GPU parity of the reprojection residual and its VJP against the FP64 oracle.

Residual: normwise relative error <= 1e-5 (and elementwise). VJP: normwise
relative error per output (cameras, points) <= 1e-4 for every Accum strategy.
Integer plan contents (stable sort by camera) are bit-exact.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_GRAD_FP32, dev, host, rel_norm, status

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "reproj_worked_example.json")
STRATS = ["atomic", "warpagg", "sort"]


def _dev_inputs(r):
    return dev(r.cams), dev(r.pts), dev(r.obs), dev(r.tgt), dev(r.w)


def _near_plane(r, n_bad=6):
    """Move a few points close to (in front of and behind) their camera's image
    plane: depth Y_z of order 1e-3 .. 1e-4, the worst-conditioned observations."""
    from scipy.spatial.transform import Rotation
    for j in range(n_bad):
        ci, pi = r.obs[j]
        c = r.cams[ci, 3:6].astype(np.float64)
        y = np.array([0.7, -0.4, (-1) ** j * 10.0 ** (-3 - j % 2)])
        u = Rotation.from_rotvec(r.cams[ci, 0:3].astype(np.float64)).inv().apply(y)
        r.pts[pi] = (c + u).astype(np.float32)
    return r


def test_worked_example():
    import paper_2104_05372_b300 as gpa
    gd = json.load(open(GOLD))
    cams = dev(np.asarray(gd["cams"], np.float32))
    pts = dev(np.asarray(gd["pts"], np.float32))
    obs = dev(np.asarray(gd["obs"], np.int32))
    tgt = dev(np.asarray(gd["tgt"], np.float32))
    res = host(gpa.reproj_residual(cams, pts, obs, tgt))
    assert np.allclose(res, np.asarray(gd["res"]), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("n_cams,n_pts,n_obs", [(1, 1, 1), (3, 7, 33), (50, 300, 20000), (200, 5000, 100003)])
def test_residual_matches_oracle(n_cams, n_pts, n_obs):
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=n_obs)
    if n_obs > 1000:
        _near_plane(r)
    ref, bad = oracle.reproj_residual(r)
    assert bad == 0
    cams, pts, obs, tgt, _ = _dev_inputs(r)
    st = status()
    res = host(gpa.reproj_residual(cams, pts, obs, tgt, status=st))
    assert int(st.item()) == 0
    assert rel_norm(res, ref) <= 1e-5
    assert np.allclose(res, ref, rtol=2e-5, atol=1e-3)


@pytest.mark.parametrize("n_cams,n_pts,n_obs", [(1, 1, 1), (3, 7, 33), (50, 300, 20000), (200, 5000, 100003)])
def test_sorted_residual_is_bit_identical(n_cams, n_pts, n_obs):
    """The camera-sorted residual visits observations in plan order and writes
    them back in input order with the same per-observation arithmetic."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=n_obs + 3)
    if n_obs > 1000:
        _near_plane(r)
    ref, _ = oracle.reproj_residual(r)
    cams, pts, obs, tgt, _ = _dev_inputs(r)
    plan = gpa.gpa_obs_plan_build(obs, n_cams, n_pts)
    st = status()
    res_s = host(gpa.reproj_residual(cams, pts, obs, tgt, plan=plan, status=st))
    res_n = host(gpa.reproj_residual(cams, pts, obs, tgt))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(res_s, res_n)
    assert rel_norm(res_s, ref) <= 1e-5


def test_sorted_residual_invalid_indices():
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(10, 20, 500, seed=16)
    r.obs[3, 0] = 10
    r.obs[9, 1] = -1
    cams, pts, obs, tgt, _ = _dev_inputs(r)
    st = status()
    plan = gpa.gpa_obs_plan_build(obs, 10, 20)
    st.zero_()
    res = host(gpa.reproj_residual(cams, pts, obs, tgt, plan=plan, status=st))
    torch.cuda.synchronize()
    assert int(st.item()) == 2
    assert np.isnan(res[[3, 9]]).all() and np.isfinite(np.delete(res, [3, 9], axis=0)).all()
    ref, _ = oracle.reproj_residual(r)
    ok = np.delete(np.arange(500), [3, 9])
    assert rel_norm(res[ok], ref[ok]) <= 1e-5


@pytest.mark.parametrize("strat", STRATS)
@pytest.mark.parametrize("n_cams,n_pts,n_obs", [(1, 1, 1), (3, 7, 33), (50, 300, 20000), (200, 5000, 100003)])
def test_vjp_matches_oracle(strat, n_cams, n_pts, n_obs):
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=n_obs + 1)
    if n_obs > 1000:
        _near_plane(r)
    dcm_ref, dpt_ref, _ = oracle.reproj_vjp(r)
    cams, pts, obs, _, w = _dev_inputs(r)
    plan = gpa.gpa_obs_plan_build(obs, n_cams, n_pts) if strat == "sort" else None
    st = status()
    dcm, dpt = gpa.reproj_vjp(cams, pts, obs, w, strat=strat, plan=plan, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert rel_norm(host(dcm), dcm_ref) <= TOL_GRAD_FP32
    assert rel_norm(host(dpt), dpt_ref) <= TOL_GRAD_FP32


def _rotation_sweep():
    """Cameras whose rotation angles span 0 .. 6.2 rad (both sides of theta = 4,
    where the camera expansion switches from the power series of the Rodrigues
    coefficients to sin / cos of theta), each observing its own points placed
    3 .. 8 units in front of it."""
    from scipy.spatial.transform import Rotation
    angles = np.array([0.0, 1e-12, 1e-7, 1e-4, 0.03, 0.5, 1.0, 2.0, 3.0, 3.1416, 3.5, 3.99, 3.9999,
                       4.0, 4.0001, 4.01, 4.5, 5.0, 5.9, 6.2])
    nc, per = angles.size, 40
    r = synth.reproj_inputs(nc, nc * per, nc * per, seed=77)
    rng = np.random.default_rng(77)
    axes = rng.standard_normal((nc, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    r.cams[:, 0:3] = (axes * angles[:, None]).astype(np.float32)
    for ci in range(nc):
        rot = Rotation.from_rotvec(r.cams[ci, 0:3].astype(np.float64))
        y = np.column_stack([rng.uniform(-1, 1, per), rng.uniform(-1, 1, per), rng.uniform(3, 8, per)])
        js = np.arange(ci * per, (ci + 1) * per)
        r.pts[js] = (r.cams[ci, 3:6].astype(np.float64) + rot.inv().apply(y)).astype(np.float32)
        r.obs[js, 0] = ci
        r.obs[js, 1] = js
    return r


def test_rotation_angles_across_expansion_branches():
    import paper_2104_05372_b300 as gpa
    r = _rotation_sweep()
    cams, pts, obs, tgt, w = _dev_inputs(r)
    res_ref, bad = oracle.reproj_residual(r)
    assert bad == 0
    res = host(gpa.reproj_residual(cams, pts, obs, tgt))
    assert rel_norm(res, res_ref) <= 1e-5
    dcm_ref, dpt_ref, _ = oracle.reproj_vjp(r)
    for strat in STRATS:
        plan = gpa.gpa_obs_plan_build(obs, r.n_cams, r.n_pts) if strat == "sort" else None
        dcm, dpt = gpa.reproj_vjp(cams, pts, obs, w, strat=strat, plan=plan)
        assert rel_norm(host(dcm), dcm_ref) <= TOL_GRAD_FP32, strat
        assert rel_norm(host(dpt), dpt_ref) <= TOL_GRAD_FP32, strat
    vc, vp = synth.reproj_tangents(r.n_cams, r.n_pts, seed=5)
    vc32, vp32 = vc.astype(np.float32), vp.astype(np.float32)
    jv_ref, _ = oracle.reproj_jvp(r, vc32.astype(np.float64), vp32.astype(np.float64))
    jv = host(gpa.reproj_jvp(cams, pts, obs, dev(vc32), dev(vp32)))
    assert rel_norm(jv, jv_ref) <= 1e-5


def test_dot_product_adjoint_against_oracle_jvp():
    """<J v, w> (oracle, forward mode) = <v, J^T w> (GPU, Accum scatter)."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(64, 2000, 50000, seed=3)
    cams, pts, obs, _, w = _dev_inputs(r)
    dcm, dpt = gpa.reproj_vjp(cams, pts, obs, w)
    dcm, dpt = host(dcm).astype(np.float64), host(dpt).astype(np.float64)
    for s in range(8):
        vc, vp = synth.reproj_tangents(r.n_cams, r.n_pts, seed=100 + s)
        jv, _ = oracle.reproj_jvp(r, vc, vp)
        lhs = np.sum(jv * r.w.astype(np.float64))
        rhs = np.sum(dcm * vc) + np.sum(dpt * vp)
        scale = np.sqrt(np.sum(jv ** 2) * np.sum(r.w.astype(np.float64) ** 2))
        assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs)


def test_plan_is_bit_exact_stable_sort():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import plan_arrays
    r = synth.reproj_inputs(8192, 1000, 300001, seed=4)
    r.obs[5, 0] = 8192     # invalid camera
    r.obs[77, 1] = -3      # invalid point
    st = status()
    plan = gpa.gpa_obs_plan_build(dev(r.obs), 8192, 1000, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 2  # GPA_ERR_INDEX
    hdr, perm, keys, aux, seg = (host(t) for t in plan_arrays(plan, r.n_obs, 8192))
    keys_in = r.obs[:, 0].copy()
    keys_in[[5, 77]] = 8192
    perm_ref, seg_ref, bad = oracle.stable_sort_by_key(keys_in, 8192)
    n_valid = r.n_obs - 2
    assert bad == 2 and hdr[2] == n_valid
    assert np.array_equal(perm[:n_valid], perm_ref)
    assert np.array_equal(seg, seg_ref.astype(np.int32))
    assert np.array_equal(np.sort(perm[n_valid:]), [5, 77])
    assert np.array_equal(keys[:n_valid], keys_in[perm_ref])
    assert np.array_equal(aux[:n_valid], r.obs[perm_ref, 1])


def test_invalid_indices_reported_and_skipped():
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(10, 20, 500, seed=6)
    r.obs[3, 0] = 10
    r.obs[9, 1] = -1
    cams, pts, obs, tgt, w = _dev_inputs(r)
    st = status()
    res = host(gpa.reproj_residual(cams, pts, obs, tgt, status=st))
    torch.cuda.synchronize()
    assert int(st.item()) == 2
    assert np.isnan(res[[3, 9]]).all() and np.isfinite(np.delete(res, [3, 9], axis=0)).all()
    ref_c, ref_p, bad = oracle.reproj_vjp(r)
    assert bad == 2
    for strat in STRATS:
        plan = gpa.gpa_obs_plan_build(obs, 10, 20) if strat == "sort" else None
        st.zero_()
        dcm, dpt = gpa.reproj_vjp(cams, pts, obs, w, strat=strat, plan=plan, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 2
        assert rel_norm(host(dcm), ref_c) <= TOL_GRAD_FP32
        assert rel_norm(host(dpt), ref_p) <= TOL_GRAD_FP32


@pytest.mark.parametrize("strat", STRATS)
def test_fused_residual_vjp(strat):
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(40, 400, 30000, seed=8)
    res_ref, _ = oracle.reproj_residual(r)
    dcm_ref, dpt_ref, _ = oracle.reproj_vjp(r, w=res_ref.astype(np.float32))
    cams, pts, obs, tgt, _ = _dev_inputs(r)
    plan = gpa.gpa_obs_plan_build(obs, 40, 400) if strat == "sort" else None
    res, dcm, dpt = gpa.reproj_residual_vjp(cams, pts, obs, tgt, 1.0, strat=strat, plan=plan)
    assert rel_norm(host(res), res_ref) <= 1e-5
    # the GPU uses its own float32 residual as the cotangent
    assert rel_norm(host(dcm), dcm_ref) <= TOL_GRAD_FP32
    assert rel_norm(host(dpt), dpt_ref) <= TOL_GRAD_FP32


@pytest.mark.slow
@pytest.mark.parametrize("strat", STRATS)
def test_full_size_workload_matches_oracle(strat):
    """8192 cameras, 500 000 points, 4 000 000 observations, full oracle."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(8192, 500000, 4000000, seed=0)
    res_ref, _ = oracle.reproj_residual(r)
    dcm_ref, dpt_ref, _ = oracle.reproj_vjp(r)
    cams, pts, obs, tgt, w = _dev_inputs(r)
    res = host(gpa.reproj_residual(cams, pts, obs, tgt))
    assert rel_norm(res, res_ref) <= 1e-5
    plan = gpa.gpa_obs_plan_build(obs, 8192, 500000) if strat == "sort" else None
    dcm, dpt = gpa.reproj_vjp(cams, pts, obs, w, strat=strat, plan=plan)
    assert rel_norm(host(dcm), dcm_ref) <= TOL_GRAD_FP32
    assert rel_norm(host(dpt), dpt_ref) <= TOL_GRAD_FP32


def test_autograd_reprojection():
    from paper_2104_05372_b300.autograd import reproj_residual
    r = synth.reproj_inputs(30, 200, 5000, seed=12)
    cams, pts, obs, tgt, w = _dev_inputs(r)
    cams.requires_grad_(True)
    pts.requires_grad_(True)
    res = reproj_residual(cams, pts, obs, tgt)
    res.backward(w)
    dcm_ref, dpt_ref, _ = oracle.reproj_vjp(r)
    assert rel_norm(host(cams.grad), dcm_ref) <= TOL_GRAD_FP32
    assert rel_norm(host(pts.grad), dpt_ref) <= TOL_GRAD_FP32
    # with a plan: camera-sorted forward (bit-identical residual) and SORT backward
    import paper_2104_05372_b300 as gpa
    plan = gpa.gpa_obs_plan_build(obs, r.n_cams, r.n_pts)
    cams.grad = pts.grad = None
    res_p = reproj_residual(cams, pts, obs, tgt, plan=plan)
    assert torch.equal(res_p.detach(), res.detach())
    res_p.backward(w)
    assert rel_norm(host(cams.grad), dcm_ref) <= TOL_GRAD_FP32
    assert rel_norm(host(pts.grad), dpt_ref) <= TOL_GRAD_FP32


@pytest.mark.parametrize("n_cams,n_pts,n_obs", [(1, 1, 1), (50, 300, 20000), (200, 5000, 100003)])
def test_jvp_matches_oracle(n_cams, n_pts, n_obs):
    """Forward mode (linearize) on the GPU against the oracle's dual numbers."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=n_obs + 7)
    if n_obs > 1000:
        _near_plane(r)
    vc, vp = synth.reproj_tangents(n_cams, n_pts, seed=4)
    ref, _ = oracle.reproj_jvp(r, vc, vp)
    cams, pts, obs, _, _ = _dev_inputs(r)
    st = status()
    jv = host(gpa.reproj_jvp(cams, pts, obs, dev(vc.astype(np.float32)), dev(vp.astype(np.float32)), status=st))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    # the oracle used float64 tangents; the GPU their float32 rounding
    ref32, _ = oracle.reproj_jvp(r, vc.astype(np.float32).astype(np.float64), vp.astype(np.float32).astype(np.float64))
    assert rel_norm(jv, ref32) <= 1e-5


def test_dot_product_adjoint_entirely_on_gpu():
    """<J v, w> with the GPU JVP equals <v, J^T w> with the GPU VJP."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(64, 2000, 50000, seed=13)
    cams, pts, obs, _, w = _dev_inputs(r)
    dcm, dpt = gpa.reproj_vjp(cams, pts, obs, w)
    for s in range(4):
        vc, vp = synth.reproj_tangents(r.n_cams, r.n_pts, seed=200 + s)
        vc32, vp32 = vc.astype(np.float32), vp.astype(np.float32)
        jv = host(gpa.reproj_jvp(cams, pts, obs, dev(vc32), dev(vp32))).astype(np.float64)
        lhs = np.sum(jv * r.w.astype(np.float64))
        rhs = np.sum(host(dcm).astype(np.float64) * vc32) + np.sum(host(dpt).astype(np.float64) * vp32)
        scale = np.sqrt(np.sum(jv ** 2) * np.sum(r.w.astype(np.float64) ** 2))
        assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs)


def _offset4(a):
    """A device copy of float32 array a whose data pointer is 4 mod 8 bytes:
    4-byte aligned as the header allows, but not 8-byte aligned."""
    buf = torch.zeros(a.size + 1, dtype=torch.float32, device="cuda")
    t = buf[1:].view(*a.shape)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a, np.float32)))
    assert t.data_ptr() % 8 == 4
    return t


@pytest.mark.parametrize("strat", STRATS)
def test_point_arrays_aligned_to_four_bytes_only(strat):
    """pts and d_pts at 4 mod 8 bytes: every entry point takes its 4-byte paths."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(40, 1001, 20000, seed=77)
    dcm_ref, dpt_ref, _ = oracle.reproj_vjp(r)
    res_ref, _ = oracle.reproj_residual(r)
    cams, _, obs, tgt, w = _dev_inputs(r)
    pts = _offset4(r.pts)
    plan = gpa.gpa_obs_plan_build(obs, r.n_cams, r.n_pts) if strat == "sort" else None
    st = status()
    res = host(gpa.reproj_residual(cams, pts, obs, tgt, status=st))
    d_pts = _offset4(np.zeros((r.n_pts, 3), np.float32))
    dcm, dpt = gpa.reproj_vjp(cams, pts, obs, w, d_pts=d_pts, strat=strat, plan=plan, status=st)
    d_pts2 = _offset4(np.zeros((r.n_pts, 3), np.float32))
    dcm2, dpt2 = gpa._lib.reproj_vjp_noalloc(cams, pts, obs, w, d_pts=d_pts2, strat=strat, plan=plan, status=st)
    vc, vp = synth.reproj_tangents(r.n_cams, r.n_pts, seed=5)
    jv = host(gpa.reproj_jvp(cams, pts, obs, dev(vc.astype(np.float32)), _offset4(vp), status=st))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert rel_norm(res, res_ref) <= 1e-5
    for a, b in ((dcm, dcm_ref), (dpt, dpt_ref), (dcm2, dcm_ref), (dpt2, dpt_ref)):
        assert rel_norm(host(a), b) <= TOL_GRAD_FP32
    ref32, _ = oracle.reproj_jvp(r, vc.astype(np.float32).astype(np.float64), vp.astype(np.float32).astype(np.float64))
    assert rel_norm(jv, ref32) <= 1e-5


def test_plan_ordered_arrays_match_input_order():
    """obs_order 'plan': the cotangents, targets and residuals indexed by plan
    position (row i = observation perm[i]) give the same cotangent sums as the
    input order, and the residuals are the input-order residuals permuted."""
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import plan_arrays
    r = synth.reproj_inputs(300, 4000, 60013, seed=31)
    obs = r.obs.copy()
    obs[[5, 77]] = [[300, 1], [2, 4000]]  # two observations outside their index sets
    cams, pts, o, tgt, w = dev(r.cams), dev(r.pts), dev(obs), dev(r.tgt), dev(r.w)
    plan = gpa.gpa_obs_plan_build(o, 300, 4000)
    perm = plan_arrays(plan, r.n_obs, 300)[1].long()
    ref_c, ref_p = gpa.reproj_vjp(cams, pts, o, w, strat="sort", plan=plan)
    st = status()
    got_c, got_p = gpa.reproj_vjp(cams, pts, o, w[perm].contiguous(), strat="sort", plan=plan, obs_order="plan",
                                  status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 2  # GPA_ERR_INDEX for the two bad observations
    assert rel_norm(host(got_c), host(ref_c)) <= 1e-6 and rel_norm(host(got_p), host(ref_p)) <= 1e-6
    res = gpa.reproj_residual(cams, pts, o, tgt)
    res_p = gpa.reproj_residual(cams, pts, o, tgt[perm].contiguous(), plan=plan, obs_order="plan")
    assert np.array_equal(host(res_p), host(res)[host(perm)], equal_nan=True)
    rf, fc, fp = gpa.reproj_residual_vjp(cams, pts, o, tgt, 0.5, strat="sort", plan=plan)
    rfp, fcp, fpp = gpa.reproj_residual_vjp(cams, pts, o, tgt[perm].contiguous(), 0.5, strat="sort", plan=plan,
                                            obs_order="plan")
    assert np.array_equal(host(rfp), host(rf)[host(perm)], equal_nan=True)
    assert rel_norm(host(fcp), host(fc)) <= 1e-6 and rel_norm(host(fpp), host(fp)) <= 1e-6
    with pytest.raises(gpa.GpaError):
        gpa.reproj_vjp(cams, pts, o, w, strat="atomic", obs_order="plan")
