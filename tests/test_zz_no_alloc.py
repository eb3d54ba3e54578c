"""Allocation-free evaluation entry point (nb_evaluate_fp64_static).

Some callers cannot allocate device memory (a host framework that owns all
GPU memory through its own pool, a latency-critical loop that must not let
cudaMalloc synchronise the device, a deployment whose memory is reserved up
front).  This entry point keeps its split-j scratch in a fixed array inside
the library; here its output is checked, through the C-ABI, against the
regular context path (nb_evaluate on an FP64 context) on the same predicted
particles, to the FP64 parity tolerance, on two calls in a row.

The file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import nb_inputs as ni
from nbhelp import nb_gpu, rel_err

pytestmark = pytest.mark.gpu


def _records(xp, vp, ap, m):
    """The documented input layout: 5 arrays of n (double, double) records."""
    n = m.size
    rec = np.empty((5, n, 2))
    rec[0, :, 0], rec[0, :, 1] = xp[:, 0], xp[:, 1]
    rec[1, :, 0], rec[1, :, 1] = xp[:, 2], m
    rec[2, :, 0], rec[2, :, 1] = vp[:, 0], vp[:, 1]
    rec[3, :, 0], rec[3, :, 1] = vp[:, 2], ap[:, 0]
    rec[4, :, 0], rec[4, :, 1] = ap[:, 1], ap[:, 2]
    return rec


@pytest.mark.parametrize("n,n_act,split", [(3000, 5, 0), (3000, 700, 0), (4099, 64, 9),
                                           (1 << 17, 1 << 17, 0)])
def test_static_scratch_entry_matches_context_path_twice(n, n_act, split):
    nb = nb_gpu()
    import torch
    eps = 1e-4
    m, x, v = ni.plummer(n, 17, imf="salpeter")
    a = ni.random_state(n, 18, scale=2.0)
    ctx = nb.NBody(m, x, v, eps, start_forces=False)
    ctx.set_state({"a": a})
    ctx.predict(0.0)
    act = ni.active_subset(n, n_act, 19)
    ref = ctx.evaluate(act)
    xp, vp, ap = ctx.predicted()
    ctx.close()

    rec = torch.from_numpy(_records(xp, vp, ap, m)).cuda()
    act_d = torch.from_numpy(act).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    lib = nb.lib()
    # two calls queued back to back on one stream (no synchronisation between
    # them): work on one stream runs in order, so the second call's clearing
    # of the shared scratch cannot overtake the first call's use of it
    outs = [torch.full((9, n_act), float("nan"), dtype=torch.float64, device="cuda")
            for _ in range(2)]
    for out in outs:
        st = lib.nb_evaluate_fp64_static(C.c_void_p(rec.data_ptr()), n, C.c_void_p(act_d.data_ptr()),
                                         n_act, eps, split, C.c_void_p(out.data_ptr()),
                                         C.c_void_p(stream))
        assert st == nb.NB_OK, lib.nb_last_error(None)
    torch.cuda.synchronize()
    for call, out in enumerate(outs):
        got = out.cpu().numpy()
        for q in range(3):
            g = got[3 * q:3 * q + 3].T
            assert rel_err(g, ref[q]).max() < 1e-12, (call, q)


def test_static_scratch_entry_rejects_oversized_split():
    nb = nb_gpu()
    import torch
    lib = nb.lib()
    n, n_act = 1 << 16, 1 << 14
    rec = torch.zeros((5, n, 2), dtype=torch.float64, device="cuda")
    act = torch.arange(n_act, dtype=torch.int32, device="cuda")
    out = torch.empty((9, n_act), dtype=torch.float64, device="cuda")
    st = lib.nb_evaluate_fp64_static(C.c_void_p(rec.data_ptr()), n, C.c_void_p(act.data_ptr()),
                                     n_act, 1e-3, 64, C.c_void_p(out.data_ptr()), None)
    assert st == nb.NB_EINVAL
    assert b"static scratch" in lib.nb_last_error(None)
