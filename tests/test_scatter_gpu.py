"""GPU parity of accum_scatter_add (every strategy) and of index plans.

int32 values: bit-exact against the oracle (exact int64 sums). float32 values:
per bucket within the summation bound (n_b - 1) u sum_j |v_j| (u = 2^-24) plus
the final rounding, checked against the oracle's float64 sums.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev, host, status

pytestmark = pytest.mark.gpu
STRATS = ["atomic", "warpagg", "sort", "smem", "runs"]


def _run(idx, vals, nb, strat):
    import paper_2104_05372_b300 as gpa
    idx_d = dev(idx)
    vals_d = dev(vals)
    acc = torch.zeros((nb,) + vals.shape[1:], dtype=vals_d.dtype, device="cuda")
    st = status()
    # with SORT, invalid indices are reported where the plan is built
    plan = gpa.gpa_index_plan_build(idx_d, nb, status=st) if strat == "sort" else None
    gpa.accum_scatter_add(idx_d, vals_d, acc, strat=strat, plan=plan, status=st)
    torch.cuda.synchronize()
    return host(acc), int(st.item())


@pytest.mark.parametrize("strat", STRATS)
@pytest.mark.parametrize("m,w,nb,skew", [(1, 1, 1, 0.0), (5, 1, 4, 0.0), (100000, 1, 1000, 0.0),
                                         (100000, 3, 50, 1.5), (33333, 11, 7, 0.0), (4096, 64, 1, 0.0),
                                         (1000003, 1, 1, 0.0), (300000, 2, 12288, 0.5)])
def test_int32_histogram_bit_exact(strat, m, w, nb, skew):
    idx, vals = synth.scatter_inputs(m, w, nb, "i32", seed=m + w, skew=skew)
    ref, bad = oracle.scatter_add(idx, vals, nb)
    got, st = _run(idx, vals, nb, strat)
    assert bad == 0 and st == 0
    assert np.array_equal(got.reshape(nb, w).astype(np.int64), ref)


@pytest.mark.parametrize("strat", STRATS)
@pytest.mark.parametrize("m,w,nb,skew", [(100000, 1, 1000, 0.0), (200000, 4, 300, 1.2), (50000, 14, 3, 0.0)])
def test_float_scatter_within_summation_bound(strat, m, w, nb, skew):
    idx, vals = synth.scatter_inputs(m, w, nb, "f32", seed=7 + w, skew=skew)
    ref, _ = oracle.scatter_add(idx, vals, nb)
    got, st = _run(idx, vals, nb, strat)
    assert st == 0
    nbk = np.bincount(idx, minlength=nb).astype(np.float64)[:, None]
    absum, _ = oracle.scatter_add(idx, np.abs(vals), nb)
    bound = (np.maximum(nbk - 1, 0) * 2.0 ** -24) * absum + 2.0 ** -24 * np.abs(ref) + 1e-30
    assert np.all(np.abs(got.reshape(nb, w) - ref) <= bound)


def test_paper_histogram_example():
    # hist!(x.i) += 1 over x = [2, 0, 2, 3, 2], 4 bins -> [1, 0, 3, 1]
    for strat in STRATS:
        got, _ = _run(np.array([2, 0, 2, 3, 2], np.int32), np.ones(5, np.int32), 4, strat)
        assert got.tolist() == [1, 0, 3, 1]


def test_invalid_indices_skipped_and_reported():
    idx = np.array([0, 7, -1, 2, 2, 3], np.int32)
    vals = np.arange(1, 7, dtype=np.int32)
    for strat in STRATS:
        got, st = _run(idx, vals, 4, strat)
        assert st == 2
        assert got.tolist() == [1, 0, 4 + 5, 6]


def test_index_plan_bit_exact():
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import plan_arrays
    for m, nk in [(1, 1), (1000, 7), (123457, 70000), (300000, 3)]:
        idx, _ = synth.scatter_inputs(m, 1, nk, "i32", seed=m, skew=0.8 if nk > 10 else 0.0)
        plan = gpa.gpa_index_plan_build(dev(idx), nk)
        hdr, perm, keys, _, seg = (host(t) for t in plan_arrays(plan, m, nk))
        perm_ref, seg_ref, _ = oracle.stable_sort_by_key(idx, nk)
        assert hdr[2] == m
        assert np.array_equal(perm, perm_ref)
        assert np.array_equal(keys, idx[perm_ref])
        assert np.array_equal(seg, seg_ref.astype(np.int32))


def test_index_plan_segments_empty_and_invalid_keys():
    """Segment offsets of the sorted plan: keys with no updates (leading,
    interior and trailing) get empty segments, invalid indices sort after
    every valid key and are counted, not placed in a segment."""
    import paper_2104_05372_b300 as gpa
    from paper_2104_05372_b300._lib import plan_arrays
    rng = np.random.default_rng(21)
    nk = 50000
    cases = []
    # 3.5 sort tiles of keys drawn from [1000, 20000): keys 0..999 and
    # 20000..nk-1 are empty; every 97th index is out of range.
    idx = rng.integers(1000, 20000, 14336).astype(np.int32)
    idx[::97] = nk + 5
    idx[1::211] = -7
    cases.append((idx, nk))
    cases.append((np.full(5000, -1, np.int32), nk))      # every index invalid
    cases.append((np.full(9000, nk - 1, np.int32), nk))  # one key, the last
    # 2^16 keys: the invalid key 2^16 needs a third 8-bit radix pass.
    idx = rng.integers(0, 1 << 16, 20000).astype(np.int32)
    idx[::13] = 1 << 16
    cases.append((idx, 1 << 16))
    for idx, nk in cases:
        m = idx.shape[0]
        st = status()
        plan = gpa.gpa_index_plan_build(dev(idx), nk, status=st)
        hdr, perm, keys, _, seg = (host(t) for t in plan_arrays(plan, m, nk))
        keys_in = np.where((idx >= 0) & (idx < nk), idx, nk).astype(np.int32)
        perm_ref, seg_ref, bad = oracle.stable_sort_by_key(keys_in, nk)
        n_valid = m - int(np.sum(keys_in == nk))
        assert bad == m - n_valid and hdr[2] == n_valid
        assert int(st.item()) == (2 if n_valid < m else 0)
        assert np.array_equal(seg, seg_ref.astype(np.int32))
        assert seg[0] == 0 and seg[-1] == n_valid
        assert np.array_equal(perm[:n_valid], perm_ref)
        assert np.array_equal(keys[:n_valid], keys_in[perm_ref])
        assert np.array_equal(np.sort(perm[n_valid:]), np.flatnonzero(keys_in == nk))


def test_partition_invariance_bit_exact_int32():
    """Accum: splitting the updates into shards and adding the shard sums
    gives the same histogram (Sec. 2.3.2)."""
    import paper_2104_05372_b300 as gpa
    idx, vals = synth.scatter_inputs(200000, 2, 500, "i32", seed=11, skew=1.0)
    whole, _ = _run(idx, vals, 500, "atomic")
    acc = torch.zeros(500, 2, dtype=torch.int32, device="cuda")
    cuts = [0, 12345, 100000, 177777, 200000]
    for a, b in zip(cuts[:-1], cuts[1:]):
        gpa.accum_scatter_add(dev(idx[a:b]), dev(vals[a:b]), acc, strat="warpagg")
    assert np.array_equal(host(acc), whole)


@pytest.mark.parametrize("dtype", ["i32", "f32"])
@pytest.mark.parametrize("seg", [1, 7, 256, 5000])
def test_runs_regular_segmented(dtype, seg):
    """idx = j // seg: the regular segmented pattern (Sec. 6.1.3) through RUNS,
    against the oracle (int bit-exact, float within the summation bound)."""
    m, w = 200003, 3
    nb = (m + seg - 1) // seg
    idx = (np.arange(m) // seg).astype(np.int32)
    _, vals = synth.scatter_inputs(m, w, nb, dtype, seed=seg)
    ref, _ = oracle.scatter_add(idx, vals, nb)
    for strat in ("runs", "auto"):
        got, st = _run(idx, vals, nb, strat)
        assert st == 0
        if dtype == "i32":
            assert np.array_equal(got.reshape(nb, w).astype(np.int64), ref)
        else:
            absum, _ = oracle.scatter_add(idx, np.abs(vals), nb)
            bound = (seg - 1) * 2.0 ** -24 * absum + 2.0 ** -24 * np.abs(ref) + 1e-30
            assert np.all(np.abs(got.reshape(nb, w) - ref) <= bound)


@pytest.mark.parametrize("w", [1, 11, 31, 33])
def test_runs_unaligned_values_bit_exact(w):
    """RUNS with the value rows at a 4-byte offset and a ragged last block
    gives the oracle's integer sums."""
    import paper_2104_05372_b300 as gpa
    m, seg = 70001, 37
    nb = (m + seg - 1) // seg
    idx = (np.arange(m) // seg).astype(np.int32)
    _, vals = synth.scatter_inputs(m, w, nb, "i32", seed=w)
    ref, _ = oracle.scatter_add(idx, vals, nb)
    buf = torch.empty(m * w + 1, dtype=torch.int32, device="cuda")
    off = buf[1:].view(m, w)
    off.copy_(dev(vals))
    assert off.data_ptr() % 16 == 4
    acc = torch.zeros(nb, w, dtype=torch.int32, device="cuda")
    st = status()
    gpa.accum_scatter_add(dev(idx), off, acc, strat="runs", status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(host(acc).astype(np.int64), ref)


def test_complete_reduction_float_within_bound():
    """One bucket, width 1: the complete pattern (tree sums, one atomic per CTA)."""
    m = 3000017
    idx = np.zeros(m, np.int32)
    _, vals = synth.scatter_inputs(m, 1, 1, "f32", seed=3)
    ref, _ = oracle.scatter_add(idx, vals, 1)
    got, st = _run(idx, vals, 1, "smem")
    assert st == 0
    bound = (m - 1) * 2.0 ** -24 * float(np.sum(np.abs(vals.astype(np.float64)))) + 1e-30
    assert abs(float(got.reshape(-1)[0]) - float(ref.reshape(-1)[0])) <= bound


def test_smem_rejects_too_many_buckets_and_auto_falls_back():
    import paper_2104_05372_b300 as gpa
    idx, vals = synth.scatter_inputs(1000, 2, 20000, "i32", seed=1)
    acc = torch.zeros(20000, 2, dtype=torch.int32, device="cuda")
    with pytest.raises(gpa.GpaError) as e:
        gpa.accum_scatter_add(dev(idx), dev(vals), acc, strat="smem")
    assert e.value.code == 6
    got, st = _run(idx, vals, 20000, "auto")  # 40000 entries: ATOMIC
    ref, _ = oracle.scatter_add(idx, vals, 20000)
    assert st == 0 and np.array_equal(got.reshape(20000, 2).astype(np.int64), ref)
