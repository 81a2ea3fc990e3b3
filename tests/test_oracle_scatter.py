"""Pins for the oracle's Accum scatter and stable sort (CPU only).

Against numpy's own primitives (bincount, add.at, stable argsort) and the
paper's tiny worked programs: the sum, histogram and segmented reduction of
Sec. 2.3.2 / 6.1.2 / 6.1.3 written out by hand.
"""
import numpy as np
import pytest

import oracle
import synth


def test_histogram_worked_example():
    # hist!(x.i) += 1 over x = [2, 0, 2, 3, 2] with 4 bins -> [1, 0, 3, 1]
    x = np.array([2, 0, 2, 3, 2], np.int32)
    acc, bad = oracle.scatter_add(x, np.ones((5, 1), np.int32), 4)
    assert bad == 0 and acc[:, 0].tolist() == [1, 0, 3, 1]


def test_complete_and_segmented_reduction_worked_examples():
    # complete reduction: acc += values.i (one bucket)
    v = np.array([[1.5], [2.25], [-0.75]], np.float32)
    acc, _ = oracle.scatter_add(np.zeros(3, np.int32), v, 1)
    assert acc[0, 0] == 3.0
    # regular segmented reduction: acc!i += values.i.j over a 2 x 3 table
    vals = np.array([1, 2, 3, 10, 20, 30], np.float32)[:, None]
    acc, _ = oracle.scatter_add(np.array([0, 0, 0, 1, 1, 1], np.int32), vals, 2)
    assert acc[:, 0].tolist() == [6.0, 60.0]


@pytest.mark.parametrize("w,skew", [(1, 0.0), (3, 0.0), (11, 1.2)])
def test_float_scatter_matches_numpy_add_at(w, skew):
    idx, vals = synth.scatter_inputs(5000, w, 97, "f32", seed=w, skew=skew)
    acc, bad = oracle.scatter_add(idx, vals, 97)
    ref = np.zeros((97, w))
    np.add.at(ref, idx, vals.astype(np.float64))
    assert bad == 0
    assert np.allclose(acc, ref, rtol=1e-13, atol=1e-11)


def test_int_scatter_matches_bincount_exactly():
    idx, vals = synth.scatter_inputs(20000, 2, 300, "i32", seed=4, skew=1.0)
    acc, bad = oracle.scatter_add(idx, vals, 300)
    for c in range(2):
        ref = np.bincount(idx, weights=vals[:, c].astype(np.float64), minlength=300)
        assert np.array_equal(acc[:, c], ref.astype(np.int64))


def test_out_of_range_indices_are_skipped():
    idx = np.array([0, 5, -1, 2, 2], np.int32)
    acc, bad = oracle.scatter_add(idx, np.ones((5, 1), np.int32), 3)
    assert bad == 2 and acc[:, 0].tolist() == [1, 0, 2]


def test_stable_sort_matches_numpy_stable_argsort():
    keys = np.random.default_rng(0).integers(0, 50, 3000).astype(np.int32)
    perm, seg, bad = oracle.stable_sort_by_key(keys, 50)
    assert bad == 0
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))
    assert np.array_equal(seg, np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=50))]))


def test_stable_sort_drops_invalid_keys():
    keys = np.array([3, 1, 9, 1, -2, 0], np.int32)
    perm, seg, bad = oracle.stable_sort_by_key(keys, 4)
    assert bad == 2
    assert perm.tolist() == [5, 1, 3, 0]
    assert seg.tolist() == [0, 1, 3, 3, 4]
