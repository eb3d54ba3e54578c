"""Host arithmetic of the benchmark's accuracy census (bench.kappa_stats)
on small hand-made arrays: the error of each particle is the largest
component of |got - ref|, divided by the particle's condition number or by
|ref|_2."""
import numpy as np
import pytest


def test_kappa_stats_counts_and_maxima():
    bench = pytest.importorskip("bench")
    ref = np.array([[3.0, 4.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 5.0]])
    got = ref.copy()
    got[0, 1] += 4e-6        # kappa 10: ratio 4e-7, plain 8e-7
    got[1, 0] -= 9e-6        # kappa 10: ratio 9e-7, plain 9e-6
    got[2, 2] += 3e-5        # kappa 20: ratio 1.5e-6, plain 1.5e-5
    kappa = np.array([10.0, 10.0, 20.0, 5.0])
    st = bench.kappa_stats(got, ref, kappa, 1e-6)
    assert st["kappa_norm_max"] == pytest.approx(1.5e-6)
    assert st["above"] == {"5e-07": 2, "8e-07": 2, "1e-06": 1}
    assert st["plain_above_1e-06"] == pytest.approx(0.5)
    assert 9e-7 <= st["p999"] <= 1.5e-6


def test_kappa_stats_of_exact_results_are_zero():
    bench = pytest.importorskip("bench")
    ref = np.arange(12, dtype=float).reshape(4, 3) + 1.0
    st = bench.kappa_stats(ref, ref, np.ones(4), 1e-12)
    assert st["kappa_norm_max"] == 0.0 and st["p999"] == 0.0
    assert st["above"] == {"5e-13": 0, "8e-13": 0, "1e-12": 0}
    assert st["plain_above_1e-12"] == 0.0
