"""Pins for the FP64 reprojection oracle (CPU only).

Checked against: a hand-worked example (tests/golden), scipy's rotation-vector
rotation (an independent Rodrigues implementation), the identity camera's
closed form, central differences of every Jacobian column, continuity of the
small-angle branch, and the dot-product identity <J v, w> = <v, J^T w> that
defines the transpose (Sec. 5.2).
"""
import json
import os

import numpy as np
from scipy.spatial.transform import Rotation

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "reproj_worked_example.json")


def _inputs(cams, pts, obs, tgt, w=None):
    cams = np.asarray(cams, np.float32)
    pts = np.asarray(pts, np.float32)
    obs = np.asarray(obs, np.int32)
    tgt = np.asarray(tgt, np.float32)
    w = np.zeros_like(tgt) if w is None else np.asarray(w, np.float32)
    return synth.ReprojInputs(cams, pts, obs, tgt, w)


def test_worked_example():
    gd = json.load(open(GOLD))
    r = _inputs(gd["cams"], gd["pts"], gd["obs"], gd["tgt"])
    res, bad = oracle.reproj_residual(r)
    assert bad == 0
    assert np.allclose(res, np.asarray(gd["res"]), rtol=0, atol=1e-12)


def test_rotation_matches_scipy_rotvec():
    r = synth.reproj_inputs(50, 80, 400, seed=3)
    r.cams[:, 0:3] *= 10.0  # angles up to a few radians
    r.cams[:, 9:11] = 0.0   # no distortion: proj = f Y_xy / Y_z + pp
    res, _ = oracle.reproj_residual(r)
    cams = r.cams.astype(np.float64)
    ci, pi = r.obs[:, 0], r.obs[:, 1]
    u = r.pts[pi].astype(np.float64) - cams[ci, 3:6]
    Y = Rotation.from_rotvec(cams[ci, 0:3]).apply(u)
    proj = cams[ci, 6:7] * Y[:, 0:2] / Y[:, 2:3] + cams[ci, 7:9]
    ref = proj - r.tgt
    assert np.allclose(res, ref, rtol=1e-10, atol=1e-9)


def test_identity_camera():
    r = synth.reproj_inputs(4, 30, 60, seed=1)
    r.cams[:] = 0.0
    r.cams[:, 6] = 1.0
    res, _ = oracle.reproj_residual(r)
    X = r.pts[r.obs[:, 1]].astype(np.float64)
    assert np.allclose(res, X[:, 0:2] / X[:, 2:3] - r.tgt, rtol=1e-13, atol=1e-13)


def _scipy_residual(r):
    cams = r.cams.astype(np.float64)
    ci, pi = r.obs[:, 0], r.obs[:, 1]
    Y = Rotation.from_rotvec(cams[ci, 0:3]).apply(r.pts[pi].astype(np.float64) - cams[ci, 3:6])
    p = Y[:, 0:2] / Y[:, 2:3]
    rho = np.sum(p * p, axis=1, keepdims=True)
    L = 1.0 + cams[ci, 9:10] * rho + cams[ci, 10:11] * rho * rho
    return cams[ci, 6:7] * L * p + cams[ci, 7:9] - r.tgt


def test_small_angle_branch_continuity():
    """Just above and below the Rodrigues threshold (|w| = 1e-8) both branches
    agree with scipy's rotation, and the Jacobians of the two branches agree."""
    base = synth.reproj_inputs(1, 5, 5, seed=4)
    base.obs[:, 1] = np.arange(5)
    jacs = []
    for th in (2e-8, 5e-9):
        r = synth.ReprojInputs(base.cams.copy(), base.pts, base.obs, base.tgt, base.w)
        r.cams[0, 0:3] = np.array([0.6, -0.48, 0.64], np.float32) * np.float32(th)
        res, _ = oracle.reproj_residual(r)
        assert np.allclose(res, _scipy_residual(r), rtol=1e-12, atol=1e-10)
        jacs.append(oracle.reproj_jacobian(r))
    # the first-order branch drops an O(|w| |u|) term of the derivative
    assert np.allclose(jacs[0], jacs[1], rtol=1e-6, atol=1e-7 * np.abs(jacs[0]).max())


def test_jacobian_matches_central_differences():
    r = synth.reproj_inputs(3, 6, 12, seed=5)
    jac = oracle.reproj_jacobian(r)
    for j in range(r.n_obs):
        ci, pi = r.obs[j]
        for a in range(14):
            arr, row, col = (r.cams, ci, a) if a < 11 else (r.pts, pi, a - 11)
            v0 = float(arr[row, col])
            h = 2.0 ** -12 * max(1.0, abs(v0))
            vals = []
            for s in (+1, -1, +0.5, -0.5):
                arr[row, col] = np.float32(v0 + s * h)
                step = float(arr[row, col]) - v0
                res, _ = oracle.reproj_residual(r)
                vals.append((res[j], step))
            arr[row, col] = np.float32(v0)
            (fp, sp), (fm, sm), (fp2, sp2), (fm2, sm2) = vals
            d1 = (fp - fm) / (sp - sm)
            d2 = (fp2 - fm2) / (sp2 - sm2)
            fd = (4 * d2 - d1) / 3
            scale = max(1.0, np.abs(jac[j]).max())
            assert np.allclose(jac[j, :, a], fd, rtol=1e-5, atol=1e-6 * scale), (j, a, jac[j, :, a], fd)


def test_dot_product_vjp_jvp():
    r = synth.reproj_inputs(20, 50, 700, seed=6)
    vc, vp = synth.reproj_tangents(r.n_cams, r.n_pts, seed=2)
    jv, _ = oracle.reproj_jvp(r, vc, vp)
    dcm, dpt, _ = oracle.reproj_vjp(r)
    lhs = np.sum(jv * r.w.astype(np.float64))
    rhs = np.sum(dcm * vc) + np.sum(dpt * vp)
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_vjp_equals_scattered_per_observation_jacobians():
    r = synth.reproj_inputs(7, 9, 200, seed=8)
    jac = oracle.reproj_jacobian(r)
    g = np.einsum("jo,joa->ja", r.w.astype(np.float64), jac)
    dcm_ref = np.zeros((r.n_cams, 11))
    dpt_ref = np.zeros((r.n_pts, 3))
    np.add.at(dcm_ref, r.obs[:, 0], g[:, :11])
    np.add.at(dpt_ref, r.obs[:, 1], g[:, 11:])
    dcm, dpt, bad = oracle.reproj_vjp(r)
    assert bad == 0
    assert np.allclose(dcm, dcm_ref, rtol=1e-12, atol=1e-9)
    assert np.allclose(dpt, dpt_ref, rtol=1e-12, atol=1e-9)


def test_out_of_range_observations_are_skipped():
    r = synth.reproj_inputs(5, 6, 40, seed=9)
    r.obs[3, 0] = 5
    r.obs[7, 1] = -1
    res, bad = oracle.reproj_residual(r)
    assert bad == 2 and np.isnan(res[3]).all() and np.isnan(res[7]).all()
    dcm, dpt, bad = oracle.reproj_vjp(r)
    assert bad == 2
    keep = np.ones(r.n_obs, bool)
    keep[[3, 7]] = False
    r2 = synth.ReprojInputs(r.cams, r.pts, r.obs[keep].copy(), r.tgt[keep].copy(), r.w[keep].copy())
    dcm2, dpt2, _ = oracle.reproj_vjp(r2)
    assert np.allclose(dcm, dcm2) and np.allclose(dpt, dpt2)


def _unpack_upper(packed, n):
    """Symmetric n x n blocks from upper triangles packed by rows (last axis)."""
    iu = np.triu_indices(n)
    out = np.zeros(packed.shape[:-1] + (n, n))
    out[..., iu[0], iu[1]] = packed
    out[..., iu[1], iu[0]] = packed
    return out


def _normal_action(r, U, V, W, vc, vp):
    """(J^T J) v from the blocks: camera rows U v_c + sum_j W_j v_p, point rows
    V v_p + sum_j W_j^T v_c."""
    Uf, Vf = _unpack_upper(U, 11), _unpack_upper(V, 3)
    ac = np.einsum("cab,cb->ca", Uf, vc)
    ap = np.einsum("pab,pb->pa", Vf, vp)
    Wm = W.reshape(-1, 11, 3)
    ci, pi = r.obs[:, 0], r.obs[:, 1]
    np.add.at(ac, ci, np.einsum("jab,jb->ja", Wm, vp[pi]))
    np.add.at(ap, pi, np.einsum("jab,ja->jb", Wm, vc[ci]))
    return ac, ap


def test_normal_equations_act_as_jt_j():
    """(J^T J) v = J^T (J v) with J v from the forward mode and J^T w from the
    reverse mode (both pinned by central differences of the residual)."""
    r = synth.reproj_inputs(12, 90, 700, seed=21)
    U, V, W, gc, gp, res, bad = oracle.reproj_normal_eqs(r)
    assert bad == 0
    for s in range(3):
        vc, vp = synth.reproj_tangents(r.n_cams, r.n_pts, seed=50 + s)
        jv, _ = oracle.reproj_jvp(r, vc, vp)
        # the VJP takes float32 cotangents: J v rounded once, about 6e-8 relative
        rc, rp, _ = oracle.reproj_vjp(r, w=jv.astype(np.float32))
        ac, ap = _normal_action(r, U, V, W, vc, vp)
        assert np.max(np.abs(ac - rc)) <= 1e-6 * np.max(np.abs(ac))
        assert np.max(np.abs(ap - rp)) <= 1e-6 * np.max(np.abs(ap))


def test_normal_equations_match_dense_jt_j_on_tiny_inputs():
    """Every block against the dense (2M x (11C + 3P)) Jacobian's J^T J and J^T r."""
    r = synth.reproj_inputs(3, 5, 17, seed=8)
    U, V, W, gc, gp, res, _ = oracle.reproj_normal_eqs(r)
    jac = oracle.reproj_jacobian(r)  # (M, 2, 14)
    nc, npt = r.n_cams, r.n_pts
    J = np.zeros((2 * r.n_obs, 11 * nc + 3 * npt))
    for j, (c, p) in enumerate(r.obs):
        J[2 * j:2 * j + 2, 11 * c:11 * c + 11] = jac[j, :, :11]
        J[2 * j:2 * j + 2, 11 * nc + 3 * p:11 * nc + 3 * p + 3] = jac[j, :, 11:]
    H = J.T @ J
    g = J.T @ res.reshape(-1)
    Uf, Vf = _unpack_upper(U, 11), _unpack_upper(V, 3)
    for c in range(nc):
        assert np.allclose(Uf[c], H[11 * c:11 * c + 11, 11 * c:11 * c + 11], rtol=1e-12, atol=1e-9)
        assert np.allclose(gc[c], g[11 * c:11 * c + 11], rtol=1e-12, atol=1e-9)
    for p in range(npt):
        o = 11 * nc + 3 * p
        assert np.allclose(Vf[p], H[o:o + 3, o:o + 3], rtol=1e-12, atol=1e-9)
        assert np.allclose(gp[p], g[o:o + 3], rtol=1e-12, atol=1e-9)
    # off-diagonal blocks: sums of W over observations of the same (camera, point) pair
    for c in range(nc):
        for p in range(npt):
            o = 11 * nc + 3 * p
            Wsum = sum(W[j].reshape(11, 3) for j in range(r.n_obs) if tuple(r.obs[j]) == (c, p))
            assert np.allclose(Wsum if np.ndim(Wsum) else np.zeros((11, 3)), H[11 * c:11 * c + 11, o:o + 3],
                               rtol=1e-12, atol=1e-9)
    # the residual agrees with the residual function
    ref, _ = oracle.reproj_residual(r)
    assert np.allclose(res, ref, rtol=0, atol=0)
