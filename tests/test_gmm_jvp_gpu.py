"""GPU forward-mode GMM derivative (gmm_jvp) against the FP64 oracle, and the
dot-product test <grad f, v> = df[v] (Sec. 5.2) with both sides on the GPU:
the reverse pass reduces over points first (Accum sums), the forward pass
carries tangents point by point, so they share no intermediate."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_GRAD_FP32, TOL_OBJ_FP32, gmm_dev, host, rel_norm, status

pytestmark = pytest.mark.gpu


def _dirs(g, seed, scale=1.0):
    """Tangent directions rounded to float32 (the GPU's inputs), as float64 for the oracle."""
    vs = [np.asarray(v * scale, np.float32) for v in synth.gmm_tangents(g.d, g.k, seed=seed)]
    return vs, [v.astype(np.float64) for v in vs]


def _jvp(g, vs32, lse_dot=True):
    import paper_2104_05372_b300 as gpa
    x, a, mu, q, l = gmm_dev(g)
    v = [torch.from_numpy(t).cuda() for t in vs32]
    f = torch.empty(1, dtype=torch.float64, device="cuda")
    ld = torch.empty(g.n, device="cuda") if lse_dot else None
    st = status()
    df = gpa.gmm_jvp(x, a, mu, q, l, *v, gamma=g.gamma, m=g.m, f_out=f, lse_dot_out=ld, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return float(df.item()), float(f.item()), (host(ld) if lse_dot else None)


@pytest.mark.parametrize("n,d,k", [(1000, 10, 5), (3000, 64, 17), ((1 << 13) + 37, 128, 9), (777, 1, 3),
                                   (500, 33, 2), (129, 16, 40)])
def test_jvp_matches_oracle(n, d, k):
    g = synth.gmm_inputs(n, d, k, seed=n + d)
    g.gamma, g.m = 0.9, 2
    vs32, vs64 = _dirs(g, seed=7)
    df, f, ld = _jvp(g, vs32)
    df_ref, f_ref, ld_ref = oracle.gmm_jvp(g, *vs64, want_lse_dot=True)
    print(f"\njvp N={n} D={d} K={k}: df rel {abs(df - df_ref) / abs(df_ref):.2e}, "
          f"lse_dot rel {rel_norm(ld, ld_ref):.2e}, f rel {abs(f - f_ref) / abs(f_ref):.2e}")
    assert abs(f - f_ref) <= TOL_OBJ_FP32 * abs(f_ref)
    assert abs(df - df_ref) <= TOL_GRAD_FP32 * abs(df_ref)
    assert rel_norm(ld, ld_ref) <= TOL_GRAD_FP32


@pytest.mark.parametrize("n,d,k", [(4000, 20, 7), (2048, 64, 30)])
def test_dot_product_both_sides_on_gpu(n, d, k):
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(n, d, k, seed=3 * n + k)
    x, a, mu, q, l = gmm_dev(g)
    grads = [host(t).astype(np.float64) for t in gpa.gmm_vjp(x, a, mu, q, l, g.gamma, g.m)]
    for s in range(3):
        vs32, vs64 = _dirs(g, seed=20 + s)
        df, _, _ = _jvp(g, vs32, lse_dot=False)
        dot = sum(float(np.sum(gr * v)) for gr, v in zip(grads, vs64))
        assert abs(dot - df) <= TOL_GRAD_FP32 * max(abs(df), 1.0), (dot, df)


def test_jvp_is_linear_in_the_direction():
    g = synth.gmm_inputs(2000, 24, 6, seed=8)
    v1, _ = _dirs(g, seed=1)
    v2, _ = _dirs(g, seed=2)
    d1, _, l1 = _jvp(g, v1)
    d2, _, l2 = _jvp(g, v2)
    # 0.5 and 0.25 keep the combination exact in float32
    v12 = [np.asarray(0.5 * a + 0.25 * b, np.float32) for a, b in zip(v1, v2)]
    d12, _, l12 = _jvp(g, v12)
    assert abs(d12 - (0.5 * d1 + 0.25 * d2)) <= 1e-5 * (abs(0.5 * d1) + abs(0.25 * d2))
    assert rel_norm(l12, 0.5 * l1 + 0.25 * l2) <= 1e-5


def test_zero_direction_gives_zero():
    g = synth.gmm_inputs(500, 9, 4, seed=9)
    zeros = [np.zeros(s, np.float32) for s in [(g.k,), (g.k, g.d), (g.k, g.d), (g.k, g.d * (g.d - 1) // 2)]]
    df, f, ld = _jvp(g, zeros)
    assert df == 0.0 and np.all(ld == 0.0)
    assert abs(f - oracle.gmm_objective(g)) <= TOL_OBJ_FP32 * abs(f)


def test_jvp_rejects_bad_arguments():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300 import _lib
    g = synth.gmm_inputs(100, 4, 2, seed=1)
    x, a, mu, q, l = gmm_dev(g)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = _lib.workspace(1024, "cuda")
    rc = _lib.load().gmm_jvp(_lib._ptr(x), _lib._ptr(a), _lib._ptr(mu), _lib._ptr(q), _lib._ptr(l), 100, 4, 2, 1.0,
                             0, None, None, None, None, _lib._ptr(out), None, None, _lib._ptr(ws), ws.numel(), None,
                             None)
    assert rc == 1  # GPA_ERR_ARG: no direction
    assert _lib.load().gpa_gmm_jvp_workspace_bytes(100, 129, 2) == 0


@pytest.mark.slow
def test_full_size_dot_product():
    """N=2^20, D=64, K=200: <grad f, v> = df[v] with both sides on the GPU."""
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(1 << 20, 64, 200, seed=0)
    x, a, mu, q, l = gmm_dev(g)
    grads = [host(t).astype(np.float64) for t in gpa.gmm_vjp(x, a, mu, q, l, g.gamma, g.m)]
    vs32, vs64 = _dirs(g, seed=99)
    df, _, _ = _jvp(g, vs32, lse_dot=False)
    dot = sum(float(np.sum(gr * v)) for gr, v in zip(grads, vs64))
    print(f"\nfull size dot test: <grad, v> = {dot:.9e}, df[v] = {df:.9e}, rel {abs(dot - df) / abs(df):.2e}")
    assert abs(dot - df) <= TOL_GRAD_FP32 * abs(df)
