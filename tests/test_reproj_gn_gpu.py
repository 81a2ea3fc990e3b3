"""Gauss-Newton normal equations of the reprojection on the GPU
(reproj_normal_eqs) against the FP64 oracle, and the identity
(J^T J) v = J^T (J v) with every side on the GPU at the full workload size."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_GRAD_FP32, dev, host, rel_norm, status

pytestmark = pytest.mark.gpu


def _near_plane(r, n_bad=4):
    """A few points at depth 0.05 .. 0.1 in front of and behind their camera. The
    normal equations square the Jacobian, whose entries grow like the inverse
    depth to high powers through the distortion: much closer to the image plane
    J^T J leaves the float32 range (depth 1e-3 gives entries near 1e42)."""
    from scipy.spatial.transform import Rotation
    for j in range(n_bad):
        ci, pi = r.obs[j]
        c = r.cams[ci, 3:6].astype(np.float64)
        y = np.array([0.7, -0.4, (-1) ** j * (0.05 if j % 2 else 0.1)])
        u = Rotation.from_rotvec(r.cams[ci, 0:3].astype(np.float64)).inv().apply(y)
        r.pts[pi] = (c + u).astype(np.float32)


FP32_SAFE = 1e30  # rows whose FP64 entries stay below this fit float32 with room for the sums


def _compare_rows(got, ref, max_out=0.01):
    """Normwise parity over the rows (cameras, points or observations) whose FP64
    blocks fit float32; the rest come from observations within ~1e-3 of the
    image plane, whose squared Jacobian leaves the float32 range: there the GPU
    must overflow too, and they must be few."""
    ok = np.all(np.abs(ref) < FP32_SAFE, axis=1)
    assert np.mean(~ok) <= max_out
    assert rel_norm(got[ok], ref[ok]) <= TOL_GRAD_FP32, rel_norm(got[ok], ref[ok])
    if np.any(~ok):
        big = ~np.isfinite(got[~ok]) | (np.abs(got[~ok]) >= 1e29)
        assert np.all(np.any(big, axis=1))


def _gpu(r, strat, want_w=True):
    import paper_2104_05372_b300 as gpa
    cams, pts, obs, tgt = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.tgt)
    st = status()
    plan = gpa.gpa_obs_plan_build(obs, r.n_cams, r.n_pts, status=st) if strat == "sort" else None
    out = gpa.reproj_normal_eqs(cams, pts, obs, tgt, want_w=want_w, want_res=True, strat=strat, plan=plan,
                                status=st)
    torch.cuda.synchronize()
    return [None if t is None else host(t) for t in out], int(st.item())


@pytest.mark.parametrize("strat", ["sort", "atomic"])
@pytest.mark.parametrize("n_cams,n_pts,n_obs", [(1, 1, 1), (3, 7, 33), (50, 300, 20000), (200, 5000, 100003)])
def test_normal_equations_match_oracle(strat, n_cams, n_pts, n_obs):
    r = synth.reproj_inputs(n_cams, n_pts, n_obs, seed=n_obs + 3)
    if n_obs > 1000:
        _near_plane(r)
    U, V, W, gc, gp, res, bad = oracle.reproj_normal_eqs(r)
    (Ug, Vg, Wg, gcg, gpg, resg), st = _gpu(r, strat)
    assert bad == 0 and st == 0
    assert Wg.shape == (n_obs, 40) and np.all(Wg[:, 33:] == 0)  # padded rows: whole 32-byte sectors
    for got, ref in ((Ug, U), (Vg, V), (Wg[:, :33], W), (gcg, gc), (gpg, gp)):
        _compare_rows(got, ref)
    assert rel_norm(resg, res) <= 1e-5


@pytest.mark.parametrize("w_ld", [33, 48, 64])
def test_w_leading_dimension(w_ld):
    """W [M][w_ld]: the same blocks in columns 0..32 for any 33 <= w_ld <= 64,
    zeros after; other leading dimensions are rejected before any work."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(40, 500, 7001, seed=8)
    cams, pts, obs, tgt = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.tgt)
    plan = gpa.gpa_obs_plan_build(obs, r.n_cams, r.n_pts)
    W = torch.full((r.n_obs, w_ld), 7.0, device="cuda")
    gpa.reproj_normal_eqs(cams, pts, obs, tgt, W=W, strat="sort", plan=plan)
    W40 = gpa.reproj_normal_eqs(cams, pts, obs, tgt, want_w=True, strat="sort", plan=plan)[2]
    torch.cuda.synchronize()
    Wh, W40h = host(W), host(W40)
    assert np.array_equal(Wh[:, :33], W40h[:, :33])  # same arithmetic, same order
    assert np.all(Wh[:, 33:] == 0)
    for bad_ld in (32, 65):
        with pytest.raises(ValueError):
            gpa.reproj_normal_eqs(cams, pts, obs, tgt, W=torch.empty(r.n_obs, bad_ld, device="cuda"),
                                  strat="sort", plan=plan)


def test_w_in_plan_order():
    """w_order "plan": row i of W is the block of the observation at position i
    of the camera-sorted plan, bit for bit the input-order row perm[i]; an
    invalid observation (sorted last) gets a NaN row; plan order without a plan
    is rejected."""
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import plan_arrays
    r = synth.reproj_inputs(40, 500, 7001, seed=9)
    r.obs[11] = (40, 3)  # camera out of range
    cams, pts, obs, tgt = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.tgt)
    plan = gpa.gpa_obs_plan_build(obs, r.n_cams, r.n_pts)
    Wi = gpa.reproj_normal_eqs(cams, pts, obs, tgt, want_w=True, strat="sort", plan=plan)[2]
    Wp = gpa.reproj_normal_eqs(cams, pts, obs, tgt, want_w=True, strat="sort", plan=plan, w_order="plan")[2]
    torch.cuda.synchronize()
    _, perm, _, _, _ = (host(t) for t in plan_arrays(plan, r.n_obs, r.n_cams))
    Wi, Wp = host(Wi), host(Wp)
    n_valid = r.n_obs - 1
    assert np.array_equal(Wp[:n_valid], Wi[perm[:n_valid]])
    assert np.all(np.isnan(Wp[n_valid:, :33])) and np.all(np.isnan(Wi[11, :33]))
    with pytest.raises(RuntimeError):
        gpa.reproj_normal_eqs(cams, pts, obs, tgt, want_w=True, strat="atomic", w_order="plan")


def test_blocks_accumulate_and_invalid_observations_are_marked():
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(20, 100, 3000, seed=5)
    r.obs[7] = (20, 3)   # camera out of range
    r.obs[11] = (2, -1)  # point out of range
    cams, pts, obs, tgt = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.tgt)
    st = status()
    U, V, W, gc, gp, res = gpa.reproj_normal_eqs(cams, pts, obs, tgt, want_w=True, want_res=True, strat="atomic",
                                                 status=st)
    U1 = U.clone()
    gpa.reproj_normal_eqs(cams, pts, obs, tgt, U=U, V=V, g_cams=gc, g_pts=gp, strat="atomic", status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 2  # GPA_ERR_INDEX
    assert rel_norm(host(U), 2 * host(U1)) <= 1e-6
    Wh, rh = host(W), host(res)
    assert np.all(np.isnan(Wh[[7, 11], :33])) and np.all(np.isnan(rh[[7, 11]]))
    keep = np.ones(r.n_obs, bool)
    keep[[7, 11]] = False
    assert np.all(np.isfinite(Wh[keep])) and np.all(np.isfinite(rh[keep]))


@pytest.mark.slow
def test_full_size_normal_action_equals_vjp_of_jvp():
    """8192 cameras, 500 000 points, 4 000 000 observations: the blocks applied
    to a direction v equal reproj_vjp(reproj_jvp(v)), all on the GPU."""
    import paper_2104_05372_b300 as gpa
    r = synth.reproj_inputs(8192, 500000, 4000000, seed=0)
    cams, pts, obs, tgt = dev(r.cams), dev(r.pts), dev(r.obs), dev(r.tgt)
    plan = gpa.gpa_obs_plan_build(obs, r.n_cams, r.n_pts)
    U, V, W, _, _, _ = gpa.reproj_normal_eqs(cams, pts, obs, tgt, want_w=True, plan=plan)
    vc, vp = synth.reproj_tangents(r.n_cams, r.n_pts, seed=9)
    vc, vp = dev(vc.astype(np.float32)), dev(vp.astype(np.float32))
    jv = gpa.reproj_jvp(cams, pts, obs, vc, vp)
    dc, dp = gpa.reproj_vjp(cams, pts, obs, jv, plan=plan)
    iu = torch.triu_indices(11, 11, device="cuda")
    Uf = torch.zeros(r.n_cams, 11, 11, device="cuda", dtype=torch.float64)
    Uf[:, iu[0], iu[1]] = U.double()
    Uf[:, iu[1], iu[0]] = U.double()
    iv = torch.triu_indices(3, 3, device="cuda")
    Vf = torch.zeros(r.n_pts, 3, 3, device="cuda", dtype=torch.float64)
    Vf[:, iv[0], iv[1]] = V.double()
    Vf[:, iv[1], iv[0]] = V.double()
    Wm = W[:, :33].double().reshape(-1, 11, 3)
    ci, pi = obs[:, 0].long(), obs[:, 1].long()
    ac = torch.einsum("cab,cb->ca", Uf, vc.double())
    ac.index_add_(0, ci, torch.einsum("jab,jb->ja", Wm, vp.double()[pi]))
    ap = torch.einsum("pab,pb->pa", Vf, vp.double())
    ap.index_add_(0, pi, torch.einsum("jab,ja->jb", Wm, vc.double()[ci]))
    ac, ap, dc, dp = host(ac), host(ap), host(dc), host(dp)
    okc = np.all(np.abs(ac) < FP32_SAFE, axis=1) & np.all(np.isfinite(ac), axis=1)
    okp = np.all(np.abs(ap) < FP32_SAFE, axis=1) & np.all(np.isfinite(ap), axis=1)
    ec, ep = rel_norm(dc[okc], ac[okc]), rel_norm(dp[okp], ap[okp])
    print(f"\nfull size: (J^T J) v against J^T (J v): cameras {ec:.2e} ({np.sum(~okc)} of {len(okc)} overflow), "
          f"points {ep:.2e} ({np.sum(~okp)} of {len(okp)} overflow)")
    assert np.mean(~okc) <= 0.01 and np.mean(~okp) <= 0.001
    assert ec <= TOL_GRAD_FP32 and ep <= TOL_GRAD_FP32
