"""Host logic of the ensemble autotuner with a stand-in ensemble (no GPU):
every candidate runs on a fresh copy, rejected shapes are skipped, and the
highest interaction rate wins."""
import time

import pytest


class FakeEnsemble:
    made = 0

    def __init__(self):
        FakeEnsemble.made += 1
        self.precision = 3
        self.shape = None
        self.inter = 0.0

    def set_shape(self, g, thr, jt):
        if thr == 96:
            raise ValueError("shape does not fit")
        self.shape = (g, thr, jt)

    def stats(self):
        return None, self.inter, 0

    def run(self, t_end):
        g, thr, jt = self.shape
        time.sleep(0.002)
        self.inter += 1e6 * g * (2.0 if jt == 512 else 1.0)

    def close(self):
        pass


def test_tune_ensemble_picks_the_highest_rate_and_skips_rejected_shapes():
    autotune = pytest.importorskip("paper_1901_08532_gb300.autotune")
    FakeEnsemble.made = 0
    seen = []
    shapes = [(2, 128, 256), (8, 128, 512), (4, 96, 512), (8, 64, 256)]
    best, rate = autotune.tune_ensemble(FakeEnsemble, 0.125, shapes, seen.append)
    assert best == (8, 128, 512)
    assert rate > 0
    assert [r["shape"] for r in seen] == [(2, 128, 256), (8, 128, 512), (8, 64, 256)]
    assert FakeEnsemble.made == 4       # one fresh copy per candidate


def test_ensemble_candidates_start_with_the_default():
    autotune = pytest.importorskip("paper_1901_08532_gb300.autotune")
    assert next(iter(autotune.ensemble_candidates(1))) == (4, 128, 1024)
    ex = list(autotune.ensemble_candidates(3))
    assert ex[0] == (8, 128, 256) and len(ex) == len(set(ex)) == 36


def test_evaluation_candidates_cover_lanes_for_the_mixed_kernel():
    """The mixed kernel's search includes the lanes per i-particle (0: the
    library's own choice, which takes two lanes below 4096 active), and
    every candidate keeps to the kernel's limits (KI 2 and 3 at most 128
    threads, KI 3 with four j per iteration)."""
    autotune = pytest.importorskip("paper_1901_08532_gb300.autotune")
    cands = list(autotune.candidates(1))
    assert {c["lanes"] for c in cands} == {0, 1, 2, 4}
    assert all(c["threads"] <= 128 for c in cands if c["ki"] >= 2)
    assert all(c["junroll"] == 4 for c in cands if c["ki"] == 3)
    assert {"ki": 2, "junroll": 4, "threads": 128, "jtile": 512, "lanes": 2} in cands
