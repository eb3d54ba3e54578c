"""The multi-device j-split on one GPU (section 3 item 3: the evaluation split
over devices, partial results reduced): the partial sums of nb_evaluate_partial
over j-ranges that tile [0, n) add up to the oracle's sums, and a j-split
integration on a single rank reproduces nb_step bit for bit.  The collective
itself (an all-reduce between ranks) is covered on the CPU by
test_jsplit_cpu.py; every run here has one GPU."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import check_parity, nb_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_partial_sums_over_tiled_ranges_match_oracle(prec):
    nb = nb_gpu()
    from paper_1901_08532_gb300.jsplit import shard_bounds
    n, eps = 1001, 1e-4
    m, x, v = ni.plummer(n, 13, imf="salpeter")
    a = ni.random_state(n, 14, scale=2.0)
    g = nb.NBody(m, x, v, eps, precision=prec, start_forces=False)
    g.set_state({"a": a})
    g.predict(0.0)
    act = ni.active_subset(n, 300, 15)
    align = 1 if prec == 0 else 4
    total = np.zeros((9, act.size))
    for r in range(3):
        lo, hi = shard_bounds(n, 3, r, align)
        _, before = g.counters()
        part = g.evaluate_partial(act, lo, hi, out="host" if r == 1 else "device")
        _, after = g.counters()
        # a rank's share counts its own interactions (the bench sums them over the ranks)
        assert after - before == act.size * (hi - lo)
        total += part if r == 1 else part.cpu().numpy()
    empty = g.evaluate_partial(act, 8, 8, out="host")      # an empty range adds nothing
    assert not empty.any()
    g.close()
    ref = O.evaluate(m, x, v, a, eps, act)
    kap = O.evaluate_kappa(m, x, v, a, eps, act)
    for q in range(3):
        got = total[3 * q:3 * q + 3].T
        if prec == 0:
            assert check_parity(0, got, ref[q]) <= 1.0, q
        else:
            tol = 1e-6 if prec == 1 else 1e-12
            assert check_parity(1, got, ref[q], kap[q], tol_mixed=tol) <= 1.0, q


@pytest.mark.parametrize("prec", [0, 1])
def test_single_rank_jsplit_reproduces_nb_step(prec):
    """One rank holds the whole j-range: schedule, predict, partial sums,
    load, correct must be nb_step bit for bit (same kernels, same launch)."""
    nb = nb_gpu()
    from paper_1901_08532_gb300.jsplit import JSplit
    m, x, v = ni.plummer(700, 16)
    ref = nb.NBody(m, x, v, 1e-4, precision=prec)
    log_ref = [ref.step() for _ in range(25)]
    st_ref = ref.state()
    ref.close()
    js = JSplit(m, x, v, 1e-4, precision=prec)
    assert (js.lo, js.hi) == (0, 700)
    log = [js.step() for _ in range(25)]
    st = js.state()
    js.close()
    assert log == log_ref
    for k in ("x", "v", "a", "j", "s", "c", "t", "dt"):
        np.testing.assert_array_equal(st[k], st_ref[k], err_msg=k)


def test_partial_and_set_forces_argument_errors():
    nb = nb_gpu()
    m, x, v = ni.plummer(64, 2)
    g = nb.NBody(m, x, v, 1e-3, precision=nb.NB_MIXED)
    act = np.arange(10, dtype=np.int32)
    with pytest.raises(nb.NBError) as e:
        g.evaluate_partial(act, 0, 64, out="host")
    assert e.value.status == nb.NB_ESTATE
    g.predict(0.0)
    for lo, hi in ((2, 64), (0, 62), (8, 4), (-4, 8), (0, 65)):
        with pytest.raises(nb.NBError) as e:
            g.evaluate_partial(act, lo, hi, out="host")
        assert e.value.status == nb.NB_EINVAL, (lo, hi)
    with pytest.raises(nb.NBError) as e:
        g.set_forces(act, np.full((9, 10), np.nan))
    assert e.value.status == nb.NB_ENONFINITE
    g.close()
