"""Launch-shape autotuner for the evaluation kernels.

For a given system size and active-set size it times candidate launch
shapes (i-particles per thread, threads per block, j-tile length, j per
inner iteration, and for the mixed kernel the lanes per i-particle, 0 being
the library's own choice; split-j is resolved by the library for each
shape) through the C-ABI (nb_set_tiles + nb_evaluate, CUDA events on the
context's stream) and keeps the fastest.  Results are cached per
(precision, n, n_act bucket) in memory and, optionally, in a JSON file.

Ensembles: tune_ensemble() times candidate cluster shapes (blocks per
system, threads, j-tile) on fresh copies of an ensemble and keeps the one
with the highest interaction rate.

Command line (prints one JSON line per timed shape, then the best):
    python -m paper_1901_08532_gb300.autotune --n 1048576 --n-act 1024 --prec mixed
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os

MIXED_SPACE = {"ki": (1, 2, 3), "junroll": (2, 4), "threads": (64, 128, 256), "jtile": (256, 512),
               "lanes": (0, 1, 2, 4)}
FP64_SPACE = {"ki": (1, 2), "threads": (64, 128, 256), "jtile": (128, 256)}
EX_SPACE = {"ki": (1,), "junroll": (1, 2), "threads": (64, 128), "jtile": (256, 512, 1024)}

_cache: dict = {}


def _bucket(n_act: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(1, n_act))))


def candidates(precision: int):
    space = MIXED_SPACE if precision in (1, 2) else EX_SPACE if precision == 3 else FP64_SPACE
    keys = sorted(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        shape = dict(zip(keys, vals))
        if precision in (1, 2) and shape["ki"] >= 2 and shape["threads"] > 128:
            continue
        if precision in (1, 2) and shape["ki"] == 3 and shape["junroll"] != 4:
            continue
        if shape["ki"] == 2 and shape["threads"] > 256:
            continue
        yield shape


def time_shape(ctx, shape, active, reps=3):
    """Mean seconds of one evaluation of `active` (a CUDA int32 tensor) with
    the given launch shape; None if the library rejects the shape."""
    import torch
    import paper_1901_08532_gb300 as nb
    try:
        ctx.set_tiles(**shape)
        ctx.evaluate(active, out=False)
    except nb.NBError:
        return None
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        ctx.evaluate(active, out=False)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def tune(ctx, active, reps=3, log=None, cache_file=None):
    """Pick the fastest shape for evaluating `active` on `ctx` and leave it
    set on the context.  Returns (shape, seconds)."""
    key = (ctx.precision, ctx.n, _bucket(int(active.numel())))
    if key not in _cache and cache_file and os.path.exists(cache_file):
        with open(cache_file) as f:
            for k, v in json.load(f).items():
                _cache[tuple(json.loads(k))] = (v["shape"], v["seconds"])
    if key in _cache:
        shape, sec = _cache[key]
        ctx.set_tiles(**shape)
        return shape, sec
    best = (None, float("inf"))
    for shape in candidates(ctx.precision):
        sec = time_shape(ctx, shape, active, reps)
        if log is not None:
            log({"shape": shape, "resolved": ctx.resolve_tiles(int(active.numel())) if sec else None,
                 "seconds": sec})
        if sec is not None and sec < best[1]:
            best = (shape, sec)
    if best[0] is None:
        ctx.set_tiles()
        return None, None
    _cache[key] = best
    ctx.set_tiles(**best[0])
    if cache_file:
        data = {}
        if os.path.exists(cache_file):
            with open(cache_file) as f:
                data = json.load(f)
        data[json.dumps(list(key))] = {"shape": best[0], "seconds": best[1]}
        with open(cache_file, "w") as f:
            json.dump(data, f, indent=1)
    return best


ENSEMBLE_SPACE = {"ctas_per_system": (2, 4, 8, 16), "threads": (64, 128, 256), "jtile": (256, 512, 1024)}


def ensemble_candidates(precision: int):
    """Ensemble launch shapes worth timing (blocks per system, threads per
    block, j-tile): a portable starting shape for the precision first (mixed
    4 x 128, j-tile 1024; otherwise 8 x 128, j-tile 256), then the space."""
    default = (4, 128, 1024) if precision == 1 else (8, 128, 256)
    yield default
    for g in ENSEMBLE_SPACE["ctas_per_system"]:
        for thr in ENSEMBLE_SPACE["threads"]:
            for jt in ENSEMBLE_SPACE["jtile"]:
                if (g, thr, jt) != default:
                    yield (g, thr, jt)


def tune_ensemble(make, t_probe, shapes=None, log=None):
    """Pick the fastest ensemble launch shape.

    make() must return a fresh Ensemble of the workload (each candidate runs
    on its own copy, because a run advances the state); every candidate is
    run to t_probe and timed on the host around Ensemble.run, which
    synchronises.  The score is interactions per second, so that shapes whose
    rounding leads to different (equally valid) trajectories compare fairly.
    Returns (shape, interactions_per_s)."""
    import time
    best = (None, 0.0)
    for shape in (shapes or ensemble_candidates(make().precision)):
        ens = make()
        try:
            ens.set_shape(*shape)
        except Exception:  # the library rejects shapes that do not fit
            ens.close()
            continue
        _, it0, _ = ens.stats()
        t0 = time.perf_counter()
        try:
            ens.run(t_probe)
        except Exception:
            ens.close()
            continue
        el = time.perf_counter() - t0
        _, it1, _ = ens.stats()
        ens.close()
        rate = (it1 - it0) / el if el > 0 else 0.0
        if log is not None:
            log({"shape": shape, "seconds": el, "interactions_per_s": rate})
        if rate > best[1]:
            best = (shape, rate)
    return best


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=1 << 20)
    p.add_argument("--n-act", type=int, nargs="+", default=[1024])
    p.add_argument("--prec", choices=["mixed", "fp64", "ex", "sp"], default="mixed")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--seed", type=int, default=3)
    args = p.parse_args()
    import torch

    import nb_inputs as ni
    import paper_1901_08532_gb300 as nb
    torch.cuda.set_device(0)
    m, x, v = ni.plummer(args.n, args.seed, imf="salpeter")
    prec = {"mixed": nb.NB_MIXED, "fp64": nb.NB_FP64, "ex": nb.NB_EX, "sp": nb.NB_SP}[args.prec]
    ctx = nb.NBody(m, x, v, 1e-4, precision=prec, start_forces=False)
    ctx.set_state({"a": ni.random_state(args.n, 5, scale=2.0)})
    ctx.predict(0.0)
    for n_act in args.n_act:
        act = torch.from_numpy(ni.active_subset(args.n, n_act, 7)).cuda()

        def log(rec, n_act=n_act):
            sec = rec["seconds"]
            rec.update(n=args.n, n_act=n_act, prec=args.prec,
                       interactions_per_s=(float(args.n) * n_act / sec) if sec else None)
            print(json.dumps(rec), flush=True)

        shape, sec = tune(ctx, act, args.reps, log=log)
        print(json.dumps({"best": shape, "n": args.n, "n_act": n_act, "prec": args.prec,
                          "seconds": sec,
                          "interactions_per_s": float(args.n) * n_act / sec if sec else None}),
              flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
