"""GPU parity of the tensor-core GMM path (GPA_PREC_BF16_TC: BF16 operands,
FP32 accumulation in tensor memory) against the FP64 oracle.

Stated bound for BF16-contraction results: relative 3e-3 (objective; per-point
statistics; gradients normwise per parameter block). The measured errors are
printed per output (pytest -s shows them).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_BF16, gmm_dev, host, rel_norm, status

pytestmark = pytest.mark.gpu
PREC = 1  # GPA_PREC_BF16_TC


def _run(g, stored=True, logjoint_points=0):
    import paper_2104_05372_b300 as gpa
    x, a, mu, q, l = gmm_dev(g)
    lse = torch.empty(g.n, device="cuda")
    lj = torch.empty(g.k, g.n, device="cuda")
    st = status()
    f = gpa.gmm_objective(x, a, mu, q, l, g.gamma, g.m, PREC, lse_out=lse, logjoint_out=lj, status=st)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    grads = gpa.gmm_vjp(x, a, mu, q, l, g.gamma, g.m, PREC, logjoint_in=lj if stored else None,
                        lse_in=lse if stored else None, out=out, logjoint_points=logjoint_points, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return float(f.item()), float(out.item()), host(lse), host(lj), [host(t) for t in grads]


def lse_error(lse, lse_ref):
    """Worst per-point error of lse_i = log sum_k exp(s_ik), in nats, relative
    to max(|lse_i|, 1). lse is a log density: an absolute error of e nats is a
    relative error of about e in the density. A plain relative error is
    ill-conditioned where lse_i crosses zero (the s_ik terms, each of size
    ~D/2, cancel there), so the floor of one nat."""
    return float(np.max(np.abs(lse - lse_ref) / np.maximum(np.abs(lse_ref), 1.0)))


def _errors(g, f, f2, lse, grads, f_ref, lse_ref, gref):
    e = {"objective": abs(f - f_ref) / abs(f_ref), "objective_vjp": abs(f2 - f_ref) / abs(f_ref),
         "lse_max": lse_error(lse, lse_ref)}
    for name, gb, rb in zip(("alpha", "mu", "q", "l"), grads, gref):
        e["grad_" + name] = rel_norm(gb, rb)
    print(f"\nBF16 tensor-core path N={g.n} D={g.d} K={g.k}: " +
          ", ".join(f"{k}={v:.2e}" for k, v in e.items()))
    return e


@pytest.mark.parametrize("n,d,k", [(300, 33, 3), (1000, 40, 7), (5000, 64, 33), (2000, 64, 1),
                                   (300, 65, 3), (1000, 100, 7), (5000, 128, 33),
                                   ((1 << 13) + 37, 128, 256), ((1 << 13) + 37, 64, 255)])
def test_tc_path_matches_oracle(n, d, k):
    g = synth.gmm_inputs(n, d, k, seed=n + d + k)
    f_ref, lse_ref = oracle.gmm_objective(g, want_lse=True)
    _, *gref = oracle.gmm_grad(g)
    f, f2, lse, lj, grads = _run(g)
    e = _errors(g, f, f2, lse, grads, f_ref, lse_ref, gref)
    for name, v in e.items():
        assert v <= TOL_BF16, (name, v)


@pytest.mark.parametrize("n,d,k", [(8192, 64, 255), (8229, 64, 254), (4096, 128, 64), (3000, 33, 120),
                                   (6000, 100, 200)])
def test_tc_forward_is_deterministic_run_to_run(n, d, k):
    """The forward's stages are refilled by bulk copies while the epilogue
    warps still use the previous contents; a missing ordering shows up as
    values that change from run to run (it did, twice: a component constant
    read after its tail slot was released). Three runs must give bit-identical
    log-joint and lse, also with a partial last round of components."""
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(n, d, k, seed=n + d + k)
    x, a, mu, q, l = gmm_dev(g)
    outs = []
    for _ in range(3):
        lse = torch.empty(g.n, device="cuda")
        lj = torch.empty(g.k, g.n, device="cuda")
        gpa.gmm_objective(x, a, mu, q, l, g.gamma, g.m, PREC, lse_out=lse, logjoint_out=lj)
        torch.cuda.synchronize()
        outs.append((host(lse), host(lj)))
    for lse_i, lj_i in outs[1:]:
        assert np.array_equal(lse_i, outs[0][0])
        assert np.array_equal(lj_i, outs[0][1])


@pytest.mark.parametrize("d", [48, 128])
def test_tc_recompute_mode_matches_stored_mode(d):
    g = synth.gmm_inputs(3000, d, 21, seed=3)
    _, *gref = oracle.gmm_grad(g)
    _, _, _, _, g_st = _run(g, stored=True)
    _, f2, _, _, g_rc = _run(g, stored=False, logjoint_points=256)
    for a, b, r in zip(g_st, g_rc, gref):
        assert rel_norm(b, r) <= TOL_BF16
        assert rel_norm(a, b) <= 1e-5


def test_tc_rejects_small_dimensions():
    import paper_2104_05372_b300 as gpa
    g = synth.gmm_inputs(100, 32, 3, seed=1)
    x, a, mu, q, l = gmm_dev(g)
    with pytest.raises(gpa.GpaError) as e:
        gpa.gmm_objective(x, a, mu, q, l, prec=PREC)
    assert e.value.code == 6  # GPA_ERR_UNSUPPORTED


@pytest.mark.slow
def test_tc_full_size_errors_per_output():
    """N=2^20, D=128, K=256 in the benchmark's launch configuration (the
    log-joint recomputed inside gmm_vjp): every output against the FP64 oracle
    at full size -- the objective (from gmm_objective and as gmm_vjp's
    by-product), every point's lse, and 64 gradient coordinates (16 per block)
    against central differences of the oracle objective (fd_util) -- each
    within the BF16 bound; the gradient is also invariant under a permutation
    of the points (Accum is associative, Sec. 2.3.2)."""
    import paper_2104_05372_b300 as gpa
    from fd_util import fd_coordinates, per_block_errors
    g = synth.gmm_inputs(1 << 20, 128, 256, seed=0)
    x, a, mu, q, l = gmm_dev(g)
    lse = torch.empty(g.n, device="cuda")
    st = status()
    f = float(gpa.gmm_objective(x, a, mu, q, l, g.gamma, g.m, PREC, lse_out=lse, status=st).item())
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    grads = [host(t).astype(np.float64) for t in gpa.gmm_vjp(x, a, mu, q, l, g.gamma, g.m, PREC, out=out,
                                                              status=st)]
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    f_ref, lse_ref = oracle.gmm_objective(g, want_lse=True)
    lse_h = host(lse).astype(np.float64)
    e = {"objective": abs(f - f_ref) / abs(f_ref),
         "objective_vjp": abs(float(out.item()) - f_ref) / abs(f_ref),
         "lse_max": lse_error(lse_h, lse_ref),
         "lse_max_plain_relative": float(np.max(np.abs(lse_h - lse_ref) / np.abs(lse_ref)))}
    rows = fd_coordinates(g, lse_ref, grads, per_block=16, seed=128)
    for block, v in per_block_errors(rows).items():
        e[f"grad_{block}_max"] = v["max"]
        e[f"grad_{block}_normwise"] = v["normwise"]
    print(f"\nBF16 full size N={g.n} D={g.d} K={g.k} vs FP64 oracle: " +
          ", ".join(f"{k}={v:.2e}" for k, v in e.items()))
    for name, v in e.items():
        assert v <= TOL_BF16, (name, v)
    perm = torch.from_numpy(np.random.default_rng(1).permutation(g.n)).cuda()
    pm = [host(t) for t in gpa.gmm_vjp(x[perm].contiguous(), a, mu, q, l, g.gamma, g.m, PREC)]
    for u, v in zip(grads, pm):
        assert rel_norm(v, u) <= 1e-4
