"""Pins for the FP64 GMM oracle (CPU only).

Each test checks the oracle against something other than its own formula:
scipy's Gaussian and Wishart log-densities (an independent parameterisation
through the covariance matrix), per-dimension normal densities for the diagonal
case, and central finite differences of the objective for the reverse- and
forward-mode derivatives.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

import oracle
import synth


def _Q(g, kk):
    d = g.d
    Q = np.zeros((d, d))
    Q[np.diag_indices(d)] = np.exp(g.q[kk].astype(np.float64))
    rows, cols = np.tril_indices(d, -1)  # row-major order over (r, c), r > c
    Q[rows, cols] = g.l[kk].astype(np.float64)
    return Q


def _scipy_objective(g):
    """Mixture log-likelihood + Wishart log-prior through scipy densities."""
    x = g.x.astype(np.float64)
    logw = g.alpha.astype(np.float64) - logsumexp(g.alpha.astype(np.float64))
    comp = np.empty((g.n, g.k))
    lp = 0.0
    for kk in range(g.k):
        Q = _Q(g, kk)
        prec = Q.T @ Q
        cov = np.linalg.inv(prec)
        comp[:, kk] = logw[kk] + stats.multivariate_normal.logpdf(x, mean=g.mu[kk].astype(np.float64), cov=cov)
        lp += stats.wishart.logpdf(prec, df=g.d + g.m + 1, scale=np.eye(g.d) / g.gamma ** 2)
    return logsumexp(comp, axis=1).sum() + lp


@pytest.mark.parametrize("n,d,k,gamma,m", [(50, 3, 1, 1.0, 0), (40, 5, 1, 1.7, 2), (64, 4, 3, 0.6, 1),
                                           (100, 6, 5, 1.0, 0)])
def test_objective_matches_scipy_densities(n, d, k, gamma, m):
    g = synth.gmm_inputs(n, d, k, seed=n + d + k, gamma=gamma, m=m)
    f = oracle.gmm_objective(g)
    ref = _scipy_objective(g)
    assert abs(f - ref) <= 1e-10 * abs(ref), (f, ref)


def test_objective_diagonal_closed_form():
    """l = 0: each component is a product of 1-D normals with sd exp(-q)."""
    g = synth.gmm_inputs(80, 4, 3, seed=7)
    g.l[:] = 0.0
    x = g.x.astype(np.float64)
    comp = np.empty((g.n, g.k))
    logw = g.alpha - logsumexp(g.alpha.astype(np.float64))
    for kk in range(g.k):
        sd = np.exp(-g.q[kk].astype(np.float64))
        comp[:, kk] = logw[kk] + stats.norm.logpdf(x, g.mu[kk].astype(np.float64), sd).sum(axis=1)
    lp = sum(stats.wishart.logpdf(np.diag(np.exp(2.0 * g.q[kk].astype(np.float64))), df=g.d + 1,
                                  scale=np.eye(g.d)) for kk in range(g.k))
    ref = logsumexp(comp, axis=1).sum() + lp
    f = oracle.gmm_objective(g)
    assert abs(f - ref) <= 1e-10 * abs(ref)


def test_lse_per_point_matches_scipy():
    g = synth.gmm_inputs(30, 3, 4, seed=3)
    f, lse = oracle.gmm_objective(g, want_lse=True)
    comp = np.empty((g.n, g.k))
    for kk in range(g.k):
        Q = _Q(g, kk)
        ld = np.sum(g.q[kk].astype(np.float64))
        xc = g.x.astype(np.float64) - g.mu[kk]
        comp[:, kk] = g.alpha[kk] + ld - 0.5 * np.sum((xc @ Q.T) ** 2, axis=1)
    # lse_i is logsumexp of the unnormalised log-joint; adding the constants
    # gives scipy's per-point mixture density (checked above), here only the
    # sampled-point entry points are compared with the full run.
    s, lse2 = oracle.gmm_logjoint_at(g, np.arange(g.n))
    assert np.allclose(lse, lse2, rtol=0, atol=1e-12)
    assert np.allclose(s, comp, rtol=1e-13, atol=1e-12)
    idx = np.array([5, 0, 29, 5])
    s3, lse3 = oracle.gmm_logjoint_at(g, idx)
    assert np.array_equal(lse3, lse[idx])


def _set(g, block, j, val):
    getattr(g, block).reshape(-1)[j] = np.float32(val)


def _fd(g, block, j, h):
    """Central difference of f along one coordinate (exact realised step)."""
    arr = getattr(g, block).reshape(-1)
    v0 = float(arr[j])
    vp, vm = np.float32(v0 + h), np.float32(v0 - h)
    _set(g, block, j, vp)
    fp = oracle.gmm_objective(g)
    _set(g, block, j, vm)
    fm = oracle.gmm_objective(g)
    _set(g, block, j, v0)
    return (fp - fm) / (float(vp) - float(vm))


def test_gradient_matches_central_differences_all_coordinates():
    """Config-0 shape (N=1000, D=10, K=5): every parameter coordinate."""
    g = synth.gmm_inputs(1000, 10, 5, seed=0)
    g.gamma, g.m = 1.3, 2  # exercise the prior's gamma and m terms
    f, da, dm, dq, dl = oracle.gmm_grad(g)
    assert abs(f - oracle.gmm_objective(g)) < 1e-9 * abs(f)
    h = 2.0 ** -11
    for block, grad in (("alpha", da), ("mu", dm), ("q", dq), ("l", dl)):
        fd = np.array([_fd(g, block, j, h) for j in range(grad.size)])
        err = np.linalg.norm(fd - grad.reshape(-1)) / np.linalg.norm(fd)
        assert err < 2e-6, (block, err)


def test_gradient_seed_scales_linearly():
    g = synth.gmm_inputs(200, 5, 3, seed=2)
    _, *g1 = oracle.gmm_grad(g, 1.0)
    _, *g2 = oracle.gmm_grad(g, -2.5)
    for a, b in zip(g1, g2):
        assert np.allclose(b, -2.5 * a, rtol=1e-13, atol=1e-12)


def _exact_direction(vals, v, h):
    """Integer direction v, zeroed where theta +- h v is not exact in float32."""
    v = v.astype(np.float64)
    base = vals.astype(np.float64)
    p = (base + h * v).astype(np.float32).astype(np.float64)
    m = (base - h * v).astype(np.float32).astype(np.float64)
    ok = (p - base == h * v) & (base - m == h * v)
    return np.where(ok, v, 0.0)


def test_jvp_matches_central_difference_along_direction():
    """Steps theta +- h v exact in float32 (symmetric differences); Richardson
    extrapolation of two step sizes removes the O(h^2) truncation term."""
    g = synth.gmm_inputs(300, 6, 4, seed=11)
    g.gamma, g.m = 0.8, 1
    r = np.random.default_rng(123)
    blocks = ["alpha", "mu", "q", "l"]
    h = 2.0 ** -13
    vs = [_exact_direction(getattr(g, b), r.integers(-2, 3, getattr(g, b).shape), h / 2) for b in blocks]
    vs = [_exact_direction(getattr(g, b), v, h) for b, v in zip(blocks, vs)]
    saved = {b: getattr(g, b).copy() for b in blocks}

    def central(step):
        for b, v in zip(blocks, vs):
            setattr(g, b, (saved[b] + step * v).astype(np.float32))
        fp = oracle.gmm_objective(g)
        for b, v in zip(blocks, vs):
            setattr(g, b, (saved[b] - step * v).astype(np.float32))
        fm = oracle.gmm_objective(g)
        for b in blocks:
            setattr(g, b, saved[b])
        return (fp - fm) / (2 * step)

    fd = (4.0 * central(h / 2) - central(h)) / 3.0
    df, f, lse_dot = oracle.gmm_jvp(g, *vs, want_lse_dot=True)
    assert abs(f - oracle.gmm_objective(g)) < 1e-9 * abs(f)
    assert abs(df - fd) <= 1e-8 * abs(fd), (df, fd)

    # per point: the tangent of logsumexp_k s_ik against the same differences
    def central_lse(step):
        for b, v in zip(blocks, vs):
            setattr(g, b, (saved[b] + step * v).astype(np.float32))
        lp = oracle.gmm_objective(g, want_lse=True)[1]
        for b, v in zip(blocks, vs):
            setattr(g, b, (saved[b] - step * v).astype(np.float32))
        lm = oracle.gmm_objective(g, want_lse=True)[1]
        for b in blocks:
            setattr(g, b, saved[b])
        return (lp - lm) / (2 * step)

    fd_lse = (4.0 * central_lse(h / 2) - central_lse(h)) / 3.0
    assert np.max(np.abs(lse_dot - fd_lse)) <= 1e-7 * np.max(np.abs(fd_lse))


def test_dot_product_reverse_equals_forward():
    """<grad f, v> = df[v]: transpose of the linearisation (Sec. 5.2)."""
    g = synth.gmm_inputs(500, 8, 6, seed=5)
    _, da, dm, dq, dl = oracle.gmm_grad(g)
    for s in range(3):
        va, vm, vq, vl = synth.gmm_tangents(g.d, g.k, seed=10 + s)
        df, _ = oracle.gmm_jvp(g, va, vm, vq, vl)
        dot = np.sum(da * va) + np.sum(dm * vm) + np.sum(dq * vq) + np.sum(dl * vl)
        assert abs(dot - df) <= 1e-10 * max(1.0, abs(df))


def test_single_component_alpha_gradient_is_zero():
    """K=1: f does not depend on alpha (softmax of one weight is 1)."""
    g = synth.gmm_inputs(100, 3, 1, seed=9)
    _, da, *_ = oracle.gmm_grad(g)
    assert abs(da[0]) < 1e-9
