"""The benchmark's accuracy methodology on the CPU: the exact distinct counts
bench.py measures its MRE against equal Definition 1 computed by the
oracle's exact module (and by plain Python sets on a small sample)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import exact  # noqa: E402
from synth import traffic  # noqa: E402


def test_exact_truth_matches_definition_1():
    gen = traffic.ZipfTraffic(3000, 1.05, 20_000, 30, seed=41, repeat_frac=0.1)
    slices = [gen.next_slice(200_000) for _ in range(4)]
    sample, truth = bench._exact_truth(gen, slices, n_sample=1500, seed=5)
    assert sample.size >= 1000  # the top hosts plus a uniform draw
    want = exact.window_cardinalities(slices, 3, 4, sample)
    np.testing.assert_array_equal(truth.astype(np.int64), np.asarray(want, dtype=np.int64))
    small = sample[:50]
    sets = exact.window_cardinalities_sets(slices, 3, 4, small)
    np.testing.assert_array_equal(truth[:50].astype(np.int64), np.asarray(sets, dtype=np.int64))


def test_exact_mre_of_the_truth_is_zero():
    gen = traffic.ZipfTraffic(500, 1.1, 5_000, 10, seed=42)
    slices = [gen.next_slice(50_000) for _ in range(2)]
    sample, truth = bench._exact_truth(gen, slices, n_sample=400, seed=6)
    out = bench._exact_mre(sample, truth, lambda s: truth.copy())
    assert out["mre"] == 0.0 and out["hosts"] == int((truth > 0).sum())
