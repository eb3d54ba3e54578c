"""Failure detection without faulting the GPU: a device-side wait that runs
out (a tile copy whose expected byte count is never reached) is reported as
NB_ETIMEOUT through the normal status path, and the context stays usable."""
import numpy as np
import pytest

import nb_inputs as ni
from nbhelp import nb_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_timed_out_wait_reports_etimeout_and_context_recovers(prec):
    nb = nb_gpu()
    n = 2048
    m, x, v = ni.plummer(n, 51)
    g = nb.NBody(m, x, v, 1e-4, precision=prec, start_forces=False)
    g.set_state({"a": ni.random_state(n, 52)})
    g.predict(0.0)
    act = ni.active_subset(n, 64, 53)      # small set: split-j with arrival counters
    assert g.resolve_tiles(64)["split"] > 1
    ref = g.evaluate(act)
    g.inject_fault(1)
    with pytest.raises(nb.NBError) as e:
        g.evaluate(act)
    assert e.value.status == nb.NB_ETIMEOUT
    again = g.evaluate(act)
    for a_, r_ in zip(again, ref):
        assert rel_err(a_, r_).max() == 0.0
    g.close()


def test_host_side_faults_are_rejected_before_any_launch():
    nb = nb_gpu()
    m, x, v = ni.plummer(16, 54)
    g = nb.NBody(m, x, v, 1e-3)
    with pytest.raises(nb.NBError) as e:
        g.inject_fault(7)
    assert e.value.status == nb.NB_EINVAL
    with pytest.raises(nb.NBError) as e:
        g.set_tiles(lanes=3)
    assert e.value.status == nb.NB_EINVAL
    with pytest.raises(nb.NBError) as e:
        g.run_until(0.1)          # not a multiple of dt_max
    assert e.value.status == nb.NB_EINVAL
    st = g.state()
    bad = dict(st)
    bad["dt"] = st["dt"] * 3.0    # not a power of two
    with pytest.raises(nb.NBError) as e:
        g.set_state(bad)
    assert e.value.status == nb.NB_EINVAL
    g.close()
