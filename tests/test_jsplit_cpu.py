"""Host logic of the multi-device j-split (the paper's section 3 item 3: each
device evaluates the active particles against its share of the j-particles
and the results are reduced across devices), run as two gloo ranks on the
CPU.  Each rank drives the library's own step (jsplit_step: schedule,
predict, partial sums over its j-range, all-reduce, load, correct) through
a stand-in context built from the FP64 oracle's primitives, whose
evaluation sees only the rank's j-range (zero masses elsewhere: a
zero-mass particle adds exactly 0 to every sum).  The reduced sums must
equal the oracle's unsplit evaluation to 1e-12, and a run of block steps
must take the unsplit oracle's decisions and end on its state."""
import json
import os
import socket
import sys

import numpy as np
import pytest

import nb_inputs as ni
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS = 1e-4


class OracleShard:
    """The context protocol of jsplit_step on the CPU oracle: the oracle's
    block step (predict all, evaluate the active set, correct, interpolate,
    new steps) written with its primitives, the evaluation restricted to
    j in [lo, hi)."""

    def __init__(self, m, x, v, eps, dt_max=2.0 ** -3):
        self.m, self.eps, self.dt_max = np.asarray(m, float), eps, dt_max
        self.st = O.System(m, x, v, eps, dt_max=dt_max).state()  # the oracle's start-up

    def schedule(self):
        tt = self.st["t"] + self.st["dt"]
        tn = tt.min()
        self.act = np.nonzero(tt == tn)[0].astype(np.int32)
        return float(tn), int(self.act.size)

    def active(self):
        return self.act

    def predict(self, t):
        s = self.st
        self.pred = O.predict(t, s["t"], s["x"], s["v"], s["a"], s["j"], s["s"], s["c"])
        self.tp = t

    def evaluate_partial(self, act, lo, hi, out="host"):
        import torch
        mm = np.zeros_like(self.m)
        mm[lo:hi] = self.m[lo:hi]
        a1, j1, s1 = O.evaluate(mm, *self.pred, self.eps, act)
        return torch.from_numpy(np.concatenate([a1.T, j1.T, s1.T]).copy())

    def set_forces(self, act, f):
        self.f = np.asarray(f).reshape(3, 3, len(act))   # [a|j|s][component][k]

    def correct(self, t):
        s = self.st
        for k, i in enumerate(self.act):
            a1, j1, s1 = (self.f[q][:, k] for q in range(3))
            h = t - s["t"][i]
            x1, v1 = O.correct(h, s["x"][i], s["v"][i], s["a"][i], s["j"][i], s["s"][i], a1, j1, s1)
            c1, d1, e1 = O.interpolate(h, s["a"][i], s["j"][i], s["s"][i], a1, j1, s1)
            crit = O.dt_crit(0.4, a1, j1, s1, c1, d1, e1)
            s["dt"][i], _ = O.dt_quantise(crit, s["dt"][i], t, dt_max=self.dt_max)
            s["x"][i], s["v"][i], s["a"][i], s["j"][i], s["s"][i], s["c"][i] = x1, v1, a1, j1, s1, c1
            s["t"][i] = t


def _system(n=96, seed=6):
    return ni.plummer(n, seed)


def _rank_main(rank, world, port, out_dir, steps):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1901_08532_gb300.jsplit import jsplit_step, reduce_partials, shard_bounds
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, x, v = _system()
    ctx = OracleShard(m, x, v, EPS)
    lo, hi = shard_bounds(m.size, world, rank, align=4)
    # one evaluation of every particle, reduced across the ranks
    ctx.predict(0.0)
    act = np.arange(m.size, dtype=np.int32)
    full = reduce_partials(ctx.evaluate_partial(act, lo, hi)).numpy()
    log = [jsplit_step(ctx, lo, hi, out="host") for _ in range(steps)]
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"lo": lo, "hi": hi, "full": full.tolist(), "log": log,
                   "state": {k: np.asarray(q).tolist() for k, q in ctx.st.items()}}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_unsplit_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    steps = 40
    torch.multiprocessing.spawn(_rank_main, args=(2, port, str(tmp_path), steps), nprocs=2, join=True)
    res = [json.loads((tmp_path / f"r{r}.json").read_text()) for r in range(2)]
    m, x, v = _system()
    n = m.size
    # the two j-ranges tile [0, n) at multiples of 4
    assert res[0]["lo"] == 0 and res[0]["hi"] == res[1]["lo"] and res[1]["hi"] == n
    assert res[0]["hi"] % 4 == 0
    # reduced sums: identical on both ranks, equal to the oracle's unsplit sums
    ref = O.System(m, x, v, EPS)
    st0 = ref.state()
    sums = O.evaluate(m, st0["x"], st0["v"], st0["a"], EPS)
    for r in res:
        f = np.asarray(r["full"]).reshape(3, 3, n)
        for q in range(3):
            got = f[q].T
            err = np.abs(got - sums[q]).max(axis=1) / np.linalg.norm(sums[q], axis=1)
            assert err.max() < 1e-12, (q, err.max())
    assert res[0]["full"] == res[1]["full"]
    # block steps: the unsplit oracle's decisions and state
    ref_log = [ref.step()[:2] for _ in range(steps)]
    st_ref = ref.state()
    for r in res:
        assert [tuple(e) for e in r["log"]] == ref_log
        for k in ("x", "v", "a", "j", "s"):
            got = np.asarray(r["state"][k])
            err = np.abs(got - st_ref[k]).max(axis=1) / np.linalg.norm(st_ref[k], axis=1)
            assert err.max() < 1e-11, (k, err.max())
        np.testing.assert_array_equal(np.asarray(r["state"]["t"]), st_ref["t"])
        np.testing.assert_array_equal(np.asarray(r["state"]["dt"]), st_ref["dt"])
    assert res[0]["state"] == res[1]["state"]   # the replicas never drift apart


@pytest.mark.parametrize("n, world, align", [(0, 1, 1), (1, 1, 4), (5, 2, 4), (1000, 3, 4), (1001, 8, 1),
                                             (1 << 20, 8, 4), (3, 8, 4)])
def test_shard_bounds_tile_the_range(n, world, align):
    sys.path.insert(0, ROOT)
    from paper_1901_08532_gb300.jsplit import shard_bounds
    b = [shard_bounds(n, world, r, align) for r in range(world)]
    assert b[0][0] == 0 and b[-1][1] == n
    for (lo0, hi0), (lo1, hi1) in zip(b, b[1:]):
        assert hi0 == lo1
    for lo, hi in b:
        assert lo <= hi and lo % align == 0 and (hi % align == 0 or hi == n)
    lens = [hi - lo for lo, hi in b]
    assert max(lens) - min(lens) <= align


def test_shard_bounds_rejects_bad_arguments():
    sys.path.insert(0, ROOT)
    from paper_1901_08532_gb300.jsplit import shard_bounds
    for args in ((10, 0, 0), (10, 2, 2), (10, 2, -1), (-1, 1, 0)):
        with pytest.raises(ValueError):
            shard_bounds(*args)
