"""GPU parity of the batched GMM path (persistent work-queue kernels) against
the FP64 oracle, per instance, plus its CUDA-graph replay and the autotuner."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_BF16, TOL_GRAD_FP32, TOL_OBJ_FP32, host, rel_norm, status

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (130, 3, 4), (1000, 8, 9), (3000, 16, 40), (777, 20, 5), (2500, 32, 17), (64, 64, 2),
          (4100, 64, 33), (900, 100, 3), (129, 128, 7), (50, 5, 120), (2049, 12, 1)]


def _instances(shapes, seed=0):
    gs = [synth.gmm_inputs(n, d, k, seed=seed + 17 * i, gamma=1.0 + 0.1 * (i % 3), m=i % 2)
          for i, (n, d, k) in enumerate(shapes)]
    inst = [dict(x=torch.from_numpy(g.x).cuda(), alpha=torch.from_numpy(g.alpha).cuda(),
                 mu=torch.from_numpy(g.mu).cuda(), q=torch.from_numpy(g.q).cuda(),
                 l=torch.from_numpy(g.l).cuda(), gamma=g.gamma, m=g.m, seed=1.0 if i % 4 else -0.5)
            for i, g in enumerate(gs)]
    return gs, inst


def _check(gs, inst, batch, which=None):
    res = batch.results()
    for i in (range(len(gs)) if which is None else which):
        g = gs[i]
        f_ref, *gref = oracle.gmm_grad(g, seed=inst[i]["seed"])
        f_ref0 = oracle.gmm_objective(g)
        out, grads = res[i]
        tc = inst[i].get("prec", 0) == 1
        tol_f, tol_g = (TOL_BF16, TOL_BF16) if tc else (TOL_OBJ_FP32, TOL_GRAD_FP32)
        assert abs(float(out.item()) - f_ref0) <= tol_f * abs(f_ref0), (i, float(out.item()), f_ref0)
        for name, gb, rb in zip(("alpha", "mu", "q", "l"), grads, gref):
            if rb.size:
                assert rel_norm(host(gb), rb) <= tol_g, (i, name)


@pytest.mark.parametrize("chunk", [64, 1024])
def test_batched_matches_oracle_per_instance(chunk):
    from paper_2104_05372_b300._lib import GmmBatch
    gs, inst = _instances(SHAPES)
    b = GmmBatch(inst, chunk_points=chunk)
    b.prepare()
    st = status()
    b.run(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    _check(gs, inst, b)


def test_batched_equals_per_instance_calls():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import GmmBatch
    gs, inst = _instances(SHAPES[:8], seed=5)
    b = GmmBatch(inst, chunk_points=2048)
    b.prepare()
    b.run(ctas_per_sm=1)
    for (out, grads), i in zip(b.results(), inst):
        single = gpa.gmm_vjp(i["x"], i["alpha"], i["mu"], i["q"], i["l"], i["gamma"], i["m"], seed=i["seed"])
        for u, v in zip(grads, single):
            if u.numel():
                assert rel_norm(host(u), host(v)) <= 1e-5


def test_graph_capture_and_replay():
    from paper_2104_05372_b300._lib import GmmBatch
    gs, inst = _instances(SHAPES[:6], seed=9)
    b = GmmBatch(inst, chunk_points=1024)
    b.prepare()
    b.run()  # warm-up outside the capture
    torch.cuda.synchronize()
    ref = [(float(o.item()), [host(t).copy() for t in g]) for o, g in b.results()]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    for _ in range(2):
        b.zero_grads()
        graph.replay()
    torch.cuda.synchronize()
    for (o, g), (fo, fg) in zip(b.results(), ref):
        assert float(o.item()) == fo
        for u, v in zip(g, fg):
            assert np.array_equal(host(u), v)


def test_autotuner_picks_per_class_and_caches(tmp_path):
    """SHAPES[:5] holds classes D <= 8 (three instances), D <= 16 and D <= 32:
    each is tuned on its own instances, the two with small component groups
    over both group sizes."""
    from paper_2104_05372_b300 import autotune
    _, inst = _instances(SHAPES[:5], seed=3)
    path = str(tmp_path / "tune.json")
    r1 = autotune.tune_batched(inst, chunks=(256, 4096), ctas=(0,), reps=1, cache_path=path)
    assert sorted(r1["opts"]) == [0, 1, 2]
    assert [len(r1["classes"][c]["table"]) for c in (0, 1, 2)] == [2, 4, 4]
    for c, o in r1["opts"].items():
        assert o["chunk_points"] in (256, 4096) and o["ctas_per_sm"] == 0
        assert o["small_groups"] in ((0, 1) if c in (1, 2) else (0,))
    r2 = autotune.tune_batched(inst, chunks=(256, 4096), ctas=(0,), reps=1, cache_path=path)
    assert r2 == r1


@pytest.mark.parametrize("small", [0, 1])
def test_batched_per_class_options_match_oracle(small):
    """Per-class settings (chunk sizes, CTAs per SM, the small component
    groups of D <= 16 and D <= 32): every instance against the oracle, and
    against the uniform-settings run within float32 rounding."""
    from paper_2104_05372_b300._lib import GmmBatch
    shapes = SHAPES + [(600, 14, 3), (2000, 30, 7), (333, 16, 11), (1500, 24, 31)]
    gs, inst = _instances(shapes, seed=13)
    opts = {0: {"chunk_points": 256}, 1: {"chunk_points": 1024, "ctas_per_sm": 1, "small_groups": small},
            2: {"chunk_points": 128, "small_groups": small}, 3: {"chunk_points": 4096}, 4: {"chunk_points": 64}}
    b = GmmBatch(inst, opts=opts)
    b.prepare()
    st = status()
    b.run(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    _check(gs, inst, b)
    u = GmmBatch(inst, chunk_points=2048)
    u.prepare()
    u.run()
    for (_, g1), (_, g2) in zip(b.results(), u.results()):
        for a, c in zip(g1, g2):
            if a.numel():
                assert rel_norm(host(a), host(c)) <= 1e-5


@pytest.mark.slow
def test_full_batched_workload_sampled_instances():
    """512 instances with the batched workload's shape law (D = 64 instances on the
    tensor cores); 12 sampled instances compared with the oracle."""
    from paper_2104_05372_b300._lib import GmmBatch
    shapes = synth.batched_shapes(512, seed=0)
    gs = synth.batched_inputs(shapes, seed=0)
    inst = [dict(x=torch.from_numpy(g.x).cuda(), alpha=torch.from_numpy(g.alpha).cuda(),
                 mu=torch.from_numpy(g.mu).cuda(), q=torch.from_numpy(g.q).cuda(),
                 l=torch.from_numpy(g.l).cuda(), gamma=g.gamma, m=g.m, seed=1.0) for g in gs]
    inst = _tensor_cores_where_supported(inst)  # the D = 64 instances: BF16 contraction
    b = GmmBatch(inst, chunk_points=4096)
    b.prepare()
    b.run()
    torch.cuda.synchronize()
    which = sorted(set(np.random.default_rng(0).choice(512, 12, replace=False).tolist()))
    _check(gs, inst, b, which=which)


def _tensor_cores_where_supported(inst):
    for i in inst:
        if 32 < i["x"].shape[1] <= 128:
            i["prec"] = 1  # GPA_PREC_BF16_TC
    return inst


def test_mixed_precision_batch_matches_oracle():
    """Instances with 32 < D <= 128 on the tensor-core path (BF16 bound), the
    rest on the FP32 persistent kernels, in one batch."""
    from paper_2104_05372_b300._lib import GmmBatch
    gs, inst = _instances(SHAPES, seed=21)
    inst = _tensor_cores_where_supported(inst)
    assert sum(i.get("prec", 0) for i in inst) == 4
    b = GmmBatch(inst, chunk_points=1024)
    b.prepare()
    st = status()
    b.run(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    _check(gs, inst, b)


def test_mixed_precision_graph_replay():
    from paper_2104_05372_b300._lib import GmmBatch
    gs, inst = _instances(SHAPES[4:10], seed=23)
    inst = _tensor_cores_where_supported(inst)
    b = GmmBatch(inst, chunk_points=1024)
    b.prepare()
    b.run()
    torch.cuda.synchronize()
    ref = [(float(o.item()), [host(t).copy() for t in g]) for o, g in b.results()]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    b.zero_grads()
    graph.replay()
    torch.cuda.synchronize()
    for (o, g), (fo, fg) in zip(b.results(), ref):
        assert abs(float(o.item()) - fo) <= 1e-9 * abs(fo)
        for u, v in zip(g, fg):
            assert rel_norm(host(u), v) <= 1e-6


def test_tensor_core_instance_outside_its_range_is_rejected():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import GmmBatch
    _, inst = _instances([(100, 32, 3)], seed=1)
    inst[0]["prec"] = 1
    with pytest.raises(gpa.GpaError):
        GmmBatch(inst).prepare()


@pytest.mark.parametrize("shapes", [[(257, 8, 17), (300, 2, 16), (129, 7, 15), (5000, 8, 33)],
                                    [(128, 8, 1), (1, 4, 3), (4096, 6, 64)]])
def test_batched_d8_class_matches_oracle(shapes):
    """D <= 8 instances run in kernels of their own (one thread per point in
    the forward; component groups of up to 16 split over point slices in the
    backward): group sizes around 16, a single point, ragged tiles."""
    from paper_2104_05372_b300._lib import GmmBatch
    gs, inst = _instances(shapes, seed=21)
    for chunk in (128, 4096):
        b = GmmBatch(inst, chunk_points=chunk)
        b.prepare()
        st = status()
        b.run(status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        _check(gs, inst, b)


def test_concatenated_tensor_core_class_equals_per_call_path():
    """The batched form runs its tensor-core instances of one padded dimension
    as one concatenated class (shared operand buffers, one launch per stage):
    every instance's objective and gradient equal the per-call tensor-core
    path's within float32 summation order (the backward's chunking differs)."""
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import GmmBatch
    shapes = [(5000, 64, 33), (64, 40, 2), (1, 48, 9), (3000, 33, 120), (900, 100, 3), (129, 128, 7),
              (2500, 65, 40), (300, 128, 260)]
    gs, inst = _instances(shapes, seed=31)
    inst = _tensor_cores_where_supported(inst)
    b = GmmBatch(inst, chunk_points=512)
    b.prepare()
    st = status()
    b.run(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    _check(gs, inst, b)
    for (out, grads), i in zip(b.results(), inst):
        o1 = torch.empty(1, dtype=torch.float64, device="cuda")
        single = gpa.gmm_vjp(i["x"], i["alpha"], i["mu"], i["q"], i["l"], i["gamma"], i["m"], 1, seed=i["seed"],
                             out=o1)
        assert abs(float(out.item()) - float(o1.item())) <= 1e-6 * abs(float(o1.item()))
        for u, v in zip(grads, single):
            if u.numel():
                assert rel_norm(host(u), host(v)) <= 1e-4
