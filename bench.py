#!/usr/bin/env python3
"""Benchmark of the direct N-body hot path on GB300.

Metric: acc+jerk+snap interactions per second at N = 2^20 (one interaction
= one (i, j) pair evaluated, the i = j term included, so n_act * N per
evaluation), mixed precision against FP64, mixed error stated.

Workload (seeded, synthetic): Plummer sphere, N = 2^20, Salpeter masses
(slope 2.35 on [0.1, 100], total mass 1), Henon units, eps = 1e-4, seed 3.
One step = one shared block step of the whole path with every particle
active (the paper's shared-step scheme): predict all N, evaluate all N
against all N in the mixed kernel, correct + new step.  Inputs resident in
HBM; the L2 is flushed (256 MB write) before every step, inside the timed
region.  Secondary numbers: the FP64 kernel at active fraction 2^-5, the
mixed kernel at active fractions 2^-10 and 2^-5 (split-j), and the mixed
error against the FP64 GPU path.

The CPU leg runs the FP64 CPU oracle on the host cores: one core on 48
sampled i-particles, then one instance per core on disjoint rows of a seeded
4096-particle subset (all against the 2^20 j); the oracle's sums for that
subset check both GPU paths (err_vs_oracle).  --impl reference times the
oracle (the reference arm) on the host cores for the same workload: one
instance per core, 16 sampled i-particles each per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BODY = 1 << 20
EPS = 1e-4
SEED = 3
FLOPS_PER_INTERACTION = 78        # FMA = 2, rsqrt = 1 (counted against the pair formula)
# SM count and maximum SM clock: GB300's, replaced by the device's own
# (set_device_peaks) before any number is reported
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# plain-ALU peaks from unit counts (128 FP32 and 2 FP64 FMA lanes per SM) and
# the maximum SM clock
PEAK_FP32_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 80.5
PEAK_FP64_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12     # 1.26
# The extended-precision (double-word) kernel issues 496 FP32-pipe operations
# (add, sub, mul, fma; sign flips not counted) per interaction, counted from
# the operation sequence of its pair term; the FP32 pipe retires 128 of them
# per clock per SM.
EX_OPS_PER_INTERACTION = 496
PEAK_FP32_OPS = SM_COUNT * 128 * SM_MAX_MHZ * 1e6                 # 40.3e12 / s


def set_device_peaks(torch, dev):
    """Unit-count peaks of the current device: its SM count and maximum SM
    clock (nvidia-smi clocks.max.sm)."""
    global SM_COUNT, SM_MAX_MHZ, PEAK_FP32_TFLOPS, PEAK_FP64_TFLOPS, PEAK_FP32_OPS
    SM_COUNT = torch.cuda.get_device_properties(dev).multi_processor_count
    SM_MAX_MHZ = _max_sm_mhz(dev)
    PEAK_FP32_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    PEAK_FP64_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    PEAK_FP32_OPS = SM_COUNT * 128 * SM_MAX_MHZ * 1e6
# DRAM traffic of one mixed evaluation launch (the bench's own launch, one
# ncu pass); valid only for the kernel source it was measured on (the sha256
# prefix of csrc/k_eval.cu and csrc/nb_device.cuh).
TRAFFIC = {"kernel_sha": "3b4746f198356227", "bytes_per_launch": 147.528960e6 + 70.369280e6,
           "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass on this launch"}
WORKLOAD = "plummer_salpeter_N1048576_eps1e-4_shared_step_all_active"
METRIC = "acc+jerk+snap interactions/s at N=2^20, mixed vs FP64 at rel err <= 1e-6"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--shard", default="j", choices=["j", "replicas"],
                   help="with N > 1 ranks: 'j' splits the j-particles of the one system over the "
                        "ranks (the paper's multi-device evaluation: one all-reduce of the partial "
                        "sums per step, strong scaling); 'replicas' runs an independent copy per "
                        "rank (weak scaling)")
    p.add_argument("--n", type=int, default=N_BODY, help="particles (default 2^20)")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    p.add_argument("--no-extra", action="store_true", help="skip the secondary measurements")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other configurations' legs (ensemble, adjoint, N=65536 integration)")
    p.add_argument("--profile-eval", action="store_true",
                   help="only launch the evaluation kernel --reps times on --n particles with "
                        "--n-act active (a small case for ncu captures)")
    p.add_argument("--n-act", type=int, default=4096)
    p.add_argument("--prec", default="mixed", choices=["mixed", "fp64", "both", "ex", "sp", "mixed32"])
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--ensemble", action="store_true",
                   help="ensemble workload: 256 Plummer systems, N log-uniform in [256, 16384] "
                        "(seed 4), each to --ens-t-end; one persistent launch vs one at a time")
    p.add_argument("--ens-t-end", type=float, default=0.25)
    p.add_argument("--ens-systems", type=int, default=256)
    p.add_argument("--ens-shapes", default="",
                   help="comma-separated ctas_per_system x threads [x jtile] shapes to time "
                        "(default 0x128x0: the library's default blocks and j-tile)")
    p.add_argument("--ens-sample", type=int, default=8,
                   help="systems in the one-at-a-time comparison (0: skip)")
    p.add_argument("--ens-cmp-t-end", type=float, default=0.125)
    p.add_argument("--ens-tune", action="store_true",
                   help="pick the launch shape with the autotuner (candidate shapes timed on a "
                        "32-system sample to t = 1/8) instead of --ens-shapes")
    p.add_argument("--integrate", action="store_true",
                   help="Plummer N=65536 (equal masses, eps 1e-4, seed 2), FP64: one full-N "
                        "evaluation, then block steps to t = 1/16; interactions/s and the "
                        "active-set size histogram")
    p.add_argument("--adjoint", action="store_true",
                   help="differentiable fixed-step trajectory: Plummer N=--n (default 8192 in this "
                        "mode), eps 1e-3, dt 2^-10, 64 steps, checkpoints every 8; forward and "
                        "backward times")
    p.add_argument("--precision-study", action="store_true",
                   help="energy and angular-momentum errors against time (Eq. 1) for FP64, mixed, "
                        "extended (double-word FP32) and single-precision positions: Plummer N=--n (default 4096 in this mode), "
                        "equal masses, eps 1e-4, block steps, a device sample every --ps-dt")
    p.add_argument("--ps-t-end", type=float, default=1.0)
    p.add_argument("--ps-dt", type=float, default=2.0 ** -3)
    p.add_argument("--ps-precs", default="fp64,mixed,ex,sp",
                   help="comma-separated precisions; name@eps runs it with nb_config.step_noise = eps")
    p.add_argument("--step-noise", type=float, default=0.0,
                   help="nb_config.step_noise for --integrate and --ensemble (the rounding floor the "
                        "step criterion discounts; 0: the criterion as is)")
    p.add_argument("--census", action="store_true",
                   help="mixed and EX errors over every particle of the default model (--n) in units "
                        "of the sums' condition numbers, against the FP64 GPU path (about four minutes "
                        "at 2^20)")
    p.add_argument("--peaks", action="store_true",
                   help="throughput probes of the CUDA-core pipes (FP32 FMA scalar and f32x2, FP64 "
                        "FMA, special-function estimates, and packed FMAs mixed with estimates)")
    return p.parse_args()


# ----------------------------------------------------------------- CPU leg

def oracle_accel(ni, n):
    """The acceleration inputs of the oracle comparison: a seeded synthetic
    field (components uniform in [-2, 2]), so that the snap's a_j - a_i term
    is exercised; the positions and velocities are the model's own."""
    return ni.random_state(n, 5, scale=2.0)


def _oracle_worker(args):
    """Oracle evaluation of i-rows [lo, hi) of the sample; returns seconds
    (and, when asked, the sums and their condition numbers, untimed)."""
    lo, hi, n = args[:3]
    keep = len(args) > 3 and args[3]
    sample = args[4] if len(args) > 4 else 4096
    import numpy as np

    import nb_inputs as ni
    import oracle as O
    m, x, v = ni.plummer(n, SEED, imf="salpeter")
    a = oracle_accel(ni, n)
    act = ni.active_subset(n, sample, 31)[lo:hi]
    t0 = time.perf_counter()
    sums = O.evaluate(m, x, v, a, EPS, act)
    sec = time.perf_counter() - t0
    if not keep:
        return sec
    return sec, act, sums, O.evaluate_kappa(m, x, v, a, EPS, act)


def cpu_baseline(n, per_core_rows=48, sample=4096):
    """Single-threaded FP64 oracle timed on (a) one core, per_core_rows
    i-particles, and (b) one independent instance per usable core on
    disjoint i-rows covering the whole seeded `sample`-particle subset, each i
    against all n j.  The oracle's sums and condition numbers for the whole
    subset are kept (untimed) for the accuracy check of the GPU paths."""
    import multiprocessing as mp

    import numpy as np
    cores = len(os.sched_getaffinity(0))
    t1 = _oracle_worker((0, per_core_rows, n, False, sample))
    one = per_core_rows * n / t1
    ctx = mp.get_context("spawn")
    k = max(1, min(cores, sample))
    edges = [sample * r // k for r in range(k + 1)]
    jobs = [(edges[r], edges[r + 1], n, True, sample) for r in range(k)]
    with ctx.Pool(k) as pool:
        res = pool.map(_oracle_worker, jobs)
    secs = [r[0] for r in res]
    allc = sample * n / max(secs)   # instances run concurrently
    act = np.concatenate([r[1] for r in res])
    sums = tuple(np.concatenate([r[2][q] for r in res]) for q in range(3))
    kap = tuple(np.concatenate([r[3][q] for r in res]) for q in range(3))
    return {"value": allc, "unit": "interactions/s", "cores": k, "kind": "oracle",
            "one_core": one, "_ref": (act, sums, kap),
            "sample": f"{k} oracle instances on disjoint i-rows of a seeded {sample}-i subset "
                      f"x all {n} j (FP64, single-threaded C); one-core run: "
                      f"{per_core_rows} i x {n} j in {t1:.1f} s",
            "host_cpu": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands (single-threaded C),
    one independent instance per usable host core on disjoint i-rows of the
    seeded 4096-particle subset, each against all n j.  A step is one round of
    `rows` i-particles per instance; its time is the slowest instance's (they
    run concurrently)."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import multiprocessing as mp
    n, rows, sample = args.n, 16, 4096
    k = max(1, min(len(os.sched_getaffinity(0)), sample // rows))

    def jobs(s):
        return [(((s * k + r) * rows) % sample, ((s * k + r) * rows) % sample + rows, n)
                for r in range(k)]

    with mp.get_context("spawn").Pool(k) as pool:
        for w in range(args.warmup):
            pool.map(_oracle_worker, jobs(w))
        times = [max(pool.map(_oracle_worker, jobs(args.warmup + s))) for s in range(args.steps)]
    value = k * rows * n * len(times) / sum(times)
    sample_txt = (f"{k} oracle instances x {rows} i-particles of a seeded {sample}-i subset "
                  f"x all {n} j per step")
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "eps": EPS, "seed": SEED, "imf": "salpeter",
                       "arm": "FP64 CPU oracle (single-threaded C, one instance per host core), "
                              "the reference arm of a paper without code",
                       "step": f"oracle evaluation of {k * rows} sampled i x all {n} j"},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": k, "kind": "oracle",
                             "sample": sample_txt, "host_cpu": _cpu_model()},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- GPU leg

class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = str(dev)
        try:
            import torch
            self.dev = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            pass
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"nb_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [q.strip() for q in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    mhz.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for name, val in zip(names, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mhz.sort()
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


def _kernel_sha():
    h = hashlib.sha256()
    for name in ("k_eval.cu", "nb_device.cuh"):
        with open(os.path.join(ROOT, "paper_1901_08532_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def aggregate_ranks(elapsed, interactions, device="cpu"):
    """Whole-job figures over the ranks of an initialised process group: the
    slowest rank's elapsed time and the sum of the interactions every rank
    evaluated (each rank runs an independent replica).  Without a group (or
    with one rank) the local figures are returned."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(elapsed), float(interactions)
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    k = torch.tensor([float(interactions)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(k, op=dist.ReduceOp.SUM)
    return float(t.item()), float(k.item())


def run_ours(args):
    import numpy as np
    import torch

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    n = args.n

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(n)          # before any GPU work (spawned pool)

    torch.cuda.set_device(local)
    set_device_peaks(torch, local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import nb_inputs as ni
    import paper_1901_08532_gb300 as nb

    stream = torch.cuda.current_stream()
    m, x, v = ni.plummer(n, SEED, imf="salpeter")
    mixed = nb.NBody(m, x, v, EPS, precision=nb.NB_MIXED, dt_shared=2.0 ** -10, stream=stream)
    st = mixed.state()                      # starting a, jerk, snap from the mixed path
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    split = world > 1 and args.shard == "j"
    lo, hi = 0, n
    if split:
        from paper_1901_08532_gb300.jsplit import reduce_partials, shard_bounds
        lo, hi = shard_bounds(n, world, rank, 4)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def one_step(ctx, ev=None):
        """Shared block step: predict all, evaluate all (with N > 1 ranks in
        j-split mode: this rank's j-range, then the all-reduce of the
        partial sums), correct all."""
        flush.zero_()
        t = ctx_t[0] + 2.0 ** -10
        ctx.predict(t)
        if ev is not None:
            ev[0].record(stream)
        if split:
            part = ctx.evaluate_partial(None, lo, hi)
            if ev is not None:
                ev[1].record(stream)
            reduce_partials(part)
            ctx.set_forces(None, part)
        else:
            ctx.evaluate(None, out=False)
            if ev is not None:
                ev[1].record(stream)
        ctx.correct(t)
        ctx_t[0] = t

    ctx_t = [0.0]
    for _ in range(args.warmup):
        one_step(mixed)
    launches0, inter0 = mixed.counters()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        e_start.record(stream)
        for k in range(args.steps):
            one_step(mixed, evs[k])
        e_end.record(stream)
        barrier()
    elapsed = e_start.elapsed_time(e_end) / 1e3          # device time of the K steps
    launches1, inter1 = mixed.counters()
    eval_ms = [a.elapsed_time(b) for a, b in evs]
    elapsed, interactions = aggregate_ranks(elapsed, inter1 - inter0, "cuda")
    value = interactions / elapsed
    eval_s = sum(eval_ms) / len(eval_ms) / 1e3
    achieved = FLOPS_PER_INTERACTION * float(n) * (hi - lo) / eval_s / 1e12
    # the DRAM figure is of the whole-range launch; a rank's j-range launch is another workload
    traffic = (TRAFFIC["bytes_per_launch"] if TRAFFIC["kernel_sha"] == _kernel_sha() and not split
               else None)
    clocks = clk.summary()
    peaks = measure_peaks(nb, torch)
    peak_meas = peaks["fp32_tflops_at_max_clock"]

    extra = {}
    if not args.no_extra:
        extra = secondary(nb, np, torch, m, x, v, st, stream, n)

    e2e = end_to_end(nb, np, torch, mixed, n, stream, max(1, min(args.steps, 3)),
                     (lo, hi, reduce_partials) if split else None)
    mixed.close()
    if not args.no_configs and rank == 0 and world == 1:
        extra["configs"] = config_legs(nb, np, torch, local)
    err_oracle = None
    if cpu is not None:
        err_oracle = error_vs_oracle(nb, np, torch, m, x, v, stream, *cpu.pop("_ref"))

    line = {
        "metric": METRIC,
        "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "strong" if split else "weak", "vs_baseline": None,
        "dtype": "f32", "precision": "mixed: FP32 pair arithmetic; FP64 positions (hi+lo FP32 "
                                     "pairs), FP64 prediction/correction, compensated accumulation",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "eps": EPS, "seed": SEED, "imf": "salpeter",
                   "step": "shared block step, all N active: predict + mixed evaluation + correct",
                   "l2": "flushed before every step (256 MB write inside the timed region)",
                   "parallelism": (f"j-split x{world} (all-reduce of [9][N] FP64 partial sums per step)"
                                   if split else f"replicas x{world}" if world > 1 else "single GPU"),
                   "flops_per_interaction": FLOPS_PER_INTERACTION},
        "roofline": {"bound": "alu", "kernel": "eval_mixed_kernel",
                     "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / PEAK_FP32_TFLOPS, "traffic": traffic,
                     "peak_source": f"{SM_COUNT} SMs x 128 FP32 lanes x 2 flops x {SM_MAX_MHZ:g} MHz "
                                    "(unit counts and max clock)",
                     "peak_measured": peak_meas, "frac_measured": achieved / peak_meas,
                     "peak_measured_source": "nb_peak_probe: f32x2 FMA throughput "
                                             f"{peaks['fp32_fma_per_clk_per_sm']:.1f}/clk/SM x 2 flops x "
                                             f"{SM_COUNT} SMs x {SM_MAX_MHZ:g} MHz",
                     "eval_ms_mean": 1e3 * eval_s},
        "peaks": {k: peaks[k] for k in ("fp32_fma_per_clk_per_sm", "fp64_fma_per_clk_per_sm",
                                        "fp32_tflops_at_max_clock", "fp64_tflops_at_max_clock")} | {
            "per_clk_per_sm": {k: round(v["ops_per_clk_per_sm"], 2) for k, v in peaks["kinds"].items()},
            "est_per_clk_per_sm": {k: round(v["est_per_clk_per_sm"], 2) for k, v in peaks["kinds"].items()
                                   if v["est_per_clk_per_sm"] > 0}},
        "e2e": e2e,
        "gpu_launches": int(launches1 - launches0),
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if err_oracle is not None:
        line["err_vs_oracle"] = err_oracle
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _time_eval(ctx, torch, stream, act, reps, warm=True):
    if warm:
        ctx.evaluate(act, out=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        ctx.evaluate(act, out=False)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def secondary(nb, np, torch, m, x, v, st, stream, n):
    """FP64 and EX kernel throughput, split-j fractions, mixed and EX error vs FP64."""
    import nb_inputs as ni
    out = {}
    state = {k: st[k] for k in ("x", "v", "a", "j", "s", "c", "t", "dt")}
    fp64 = nb.NBody(m, x, v, EPS, precision=nb.NB_FP64, dt_shared=2.0 ** -10, stream=stream,
                    start_forces=False)
    fp64.set_state(state)
    mixed = nb.NBody(m, x, v, EPS, precision=nb.NB_MIXED, dt_shared=2.0 ** -10, stream=stream,
                     start_forces=False)
    mixed.set_state(state)
    ex = nb.NBody(m, x, v, EPS, precision=nb.NB_EX, dt_shared=2.0 ** -10, stream=stream,
                  start_forces=False)
    ex.set_state(state)
    t = 2.0 ** -10
    fp64.predict(t)
    mixed.predict(t)
    ex.predict(t)
    fr = {}
    act_32k = ni.active_subset(n, n // 32, 32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    a64, j64, s64_ = fp64.evaluate(act_32k)     # one FP64 launch, timed, results kept
    e1.record(stream)
    torch.cuda.synchronize()
    s64 = e0.elapsed_time(e1) / 1e3
    fr["fp64_2^-5"] = {"n_act": int(act_32k.size), "interactions_per_s": act_32k.size * n / s64,
                       "tflops": FLOPS_PER_INTERACTION * act_32k.size * n / s64 / 1e12,
                       "frac_of_fp64_peak": FLOPS_PER_INTERACTION * act_32k.size * n / s64 / 1e12
                       / PEAK_FP64_TFLOPS, "tiles": fp64.resolve_tiles(act_32k.size)}
    for frac, k in (("2^-10", 1024), ("2^-5", 32)):
        act = ni.active_subset(n, n // k, k)
        at = torch.from_numpy(act).cuda()
        sm = _time_eval(mixed, torch, stream, at, 5)
        fr[f"mixed_{frac}"] = {"n_act": int(act.size), "interactions_per_s": act.size * n / sm,
                               "frac_of_fp32_peak": FLOPS_PER_INTERACTION * act.size * n / sm / 1e12
                               / PEAK_FP32_TFLOPS, "tiles": mixed.resolve_tiles(act.size)}
    # the realistic, core-concentrated active set: the n particles with the
    # smallest starting steps (ties by index), in ascending index order
    core = np.sort(np.argsort(st["dt"], kind="stable")[: n // 32]).astype(np.int32)
    sm = _time_eval(mixed, torch, stream, torch.from_numpy(core).cuda(), 5)
    fr["mixed_core_2^-5"] = {"n_act": int(core.size), "interactions_per_s": core.size * n / sm,
                             "frac_of_fp32_peak": FLOPS_PER_INTERACTION * core.size * n / sm / 1e12
                             / PEAK_FP32_TFLOPS, "active_set": "smallest starting dt",
                             "tiles": mixed.resolve_tiles(core.size)}
    at32 = torch.from_numpy(act_32k).cuda()
    sx = _time_eval(ex, torch, stream, at32, 2)
    rate_ex = act_32k.size * n / sx
    fr["ex_2^-5"] = {"n_act": int(act_32k.size), "interactions_per_s": rate_ex,
                     "fp32_ops_per_interaction": EX_OPS_PER_INTERACTION,
                     "frac_of_fp32_pipe": EX_OPS_PER_INTERACTION * rate_ex / PEAK_FP32_OPS,
                     "fp64_equiv_tflops": FLOPS_PER_INTERACTION * rate_ex / 1e12,
                     "tiles": ex.resolve_tiles(act_32k.size)}
    out["fractions"] = fr

    def err_stats(got, ref, thr):
        errs = {}
        for name, g, r in zip(("acc", "jerk", "snap"), got, ref):
            e = np.abs(g - r).max(axis=1) / np.linalg.norm(r, axis=1)
            errs[name] = {"max": float(e.max()), "p99": float(np.percentile(e, 99)),
                          "median": float(np.median(e)), f"frac_above_{thr:g}": float((e > thr).mean())}
        return errs

    # mixed and EX vs FP64 on the same predicted inputs (the 2^-5 active set)
    ref = (a64, j64, s64_)
    out["mixed_vs_fp64_err"] = {"n_act": int(act_32k.size), "metric": "|d|_inf/|ref|_2 per particle",
                                **err_stats(mixed.evaluate(act_32k), ref, 1e-6)}
    out["ex_vs_fp64_err"] = {"n_act": int(act_32k.size), "metric": "|d|_inf/|ref|_2 per particle",
                             **err_stats(ex.evaluate(act_32k), ref, 1e-12)}
    mixed_rate = fr["mixed_2^-5"]["interactions_per_s"]
    out["speedup_mixed_over_fp64"] = mixed_rate / fr["fp64_2^-5"]["interactions_per_s"]
    out["speedup_ex_over_fp64"] = rate_ex / fr["fp64_2^-5"]["interactions_per_s"]
    fp64.close()
    mixed.close()
    ex.close()
    return out


def error_vs_oracle(nb, np, torch, m, x, v, stream, act, sums, kap):
    """Both GPU precisions on the oracle's sample (same inputs: the start
    positions and velocities, the seeded acceleration field of
    oracle_accel, t = 0; the mixed path in the headline's all-active launch,
    the FP64 path on the sample alone): per particle |d|_inf / |ref|_2 (max
    and the fraction above 1e-6), and |d|_inf / sum_j |T_ij| (the error
    relative to the sum's condition number)."""
    import nb_inputs as ni
    out = {"sample": int(len(act)),
           "inputs": "start positions and velocities, seeded acceleration field (uniform [-2, 2])"}
    a = oracle_accel(ni, m.size)
    for name, prec in (("mixed", nb.NB_MIXED), ("fp64", nb.NB_FP64)):
        ctx = nb.NBody(m, x, v, EPS, precision=prec, stream=stream, start_forces=False)
        ctx.set_state({"a": a})
        ctx.predict(0.0)
        if prec == nb.NB_MIXED:
            # the headline's own launch (every particle active), read at the sample
            got = [q[act] for q in ctx.evaluate(None)]
        else:
            got = ctx.evaluate(act)
        ctx.close()
        rec = {}
        for q, g, r, k in zip(("acc", "jerk", "snap"), got, sums, kap):
            d = np.abs(g - r).max(axis=1)
            plain = d / np.linalg.norm(r, axis=1)
            rec[q] = {"max": float(plain.max()), "frac_above_1e-06": float((plain > 1e-6).mean()),
                      "kappa_norm_max": float((d / k).max())}
        out[name] = rec
    out["mixed_within_1e-6_of_condition_number"] = all(
        out["mixed"][q]["kappa_norm_max"] <= 1e-6 for q in ("acc", "jerk", "snap"))
    return out


def end_to_end(nb, np, torch, ctx, n, stream, steps, split=None):
    """Same metric through the public API with pinned host buffers: upload
    the full state, one shared block step, read back x and v.  split =
    (lo, hi, reduce): the step evaluates j in [lo, hi) and all-reduces."""
    def pinned(shape):
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    st = ctx.state()
    host = {k: pinned(st[k].shape) for k in ("x", "v", "a", "j", "s", "c", "t", "dt")}
    for k in host:
        host[k][...] = st[k]
    outx, outv = pinned((n, 3)), pinned((n, 3))
    ptr = lambda a: a.ctypes.data_as(nb._d)  # noqa: E731
    lib = nb.lib()
    h2d = sum(a.nbytes for a in host.values())
    d2h = outx.nbytes + outv.nbytes

    def step():
        ctx._check(lib.nb_set_state(ctx._ctx, *[ptr(host[k]) for k in ("x", "v", "a", "j", "s", "c",
                                                                        "t", "dt")]))
        if split is None:
            ctx.step()
        else:
            from paper_1901_08532_gb300.jsplit import jsplit_step
            jsplit_step(ctx, split[0], split[1])
        ctx._check(lib.nb_get_state(ctx._ctx, ptr(outx), ptr(outv), None, None, None, None, None,
                                    None))
    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    if split is not None:
        el, _ = aggregate_ranks(el, 0.0, "cuda")     # the slowest rank's time
    return {"value": float(n) * n * steps / el, "unit": "interactions/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "api": ("nb_set_state (pinned host) -> nb_step -> nb_get_state (pinned host)" if split is None
                    else "nb_set_state (pinned host) -> nb_schedule, nb_predict, nb_evaluate_partial, "
                         "all-reduce, nb_set_forces, nb_correct -> nb_get_state (pinned host)"),
            "steps": steps}


def profile_eval(args):
    """Evaluation launches only: Plummer/Salpeter N = --n, --n-act seeded
    active particles, --reps launches (for ncu; prints per-launch times)."""
    import numpy as np
    import torch

    import nb_inputs as ni
    import paper_1901_08532_gb300 as nb
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    m, x, v = ni.plummer(args.n, SEED, imf="salpeter")
    a = ni.random_state(args.n, 5, scale=2.0)
    prec = {"mixed": nb.NB_MIXED, "fp64": nb.NB_FP64, "ex": nb.NB_EX, "sp": nb.NB_SP}[args.prec]
    ctx = nb.NBody(m, x, v, EPS, precision=prec, stream=stream, start_forces=False)
    ctx.set_state({"a": a})
    ctx.predict(0.0)
    act = torch.from_numpy(ni.active_subset(args.n, args.n_act, 7)).cuda()
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.evaluate(act, out=False)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    inter = float(args.n) * args.n_act
    print(json.dumps({"profile_eval": args.prec, "n": args.n, "n_act": args.n_act,
                      "tiles": ctx.resolve_tiles(args.n_act), "ms": times,
                      "interactions_per_s": inter / (min(times) / 1e3)}))
    ctx.close()
    return 0


def ensemble_bench(args):
    """Batched ensemble (256 Plummer systems, N log-uniform in [256, 16384],
    seed 4, eps = 1e-4, own block steps): (1) all systems in one persistent,
    graph-captured launch to --ens-t-end; (2) the batching gain on a sample
    of --ens-sample systems spread over the size range, each advanced one at
    a time through nb_run_until, against the same sample as one ensemble, to
    --ens-cmp-t-end.  Interactions per second of each."""
    import numpy as np
    import torch

    import nb_inputs as ni
    import paper_1901_08532_gb300 as nb
    torch.cuda.set_device(0)
    sizes = ni.ensemble_sizes(args.ens_systems, 4)
    parts = [ni.plummer(int(n), 1000 + k) for k, n in enumerate(sizes)]

    def cat(idx):
        return (np.concatenate([parts[k][0] for k in idx]), np.concatenate([parts[k][1] for k in idx]),
                np.concatenate([parts[k][2] for k in idx]))

    def run_ens(idx, prec, shape, t_end):
        g, thr, jt = shape
        ens = nb.Ensemble(sizes[idx], *cat(idx), EPS, precision=prec, step_noise=args.step_noise)
        ens.set_shape(g or None, thr, jt or None)
        used = ens.shape()
        _, it0, _ = ens.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.run(t_end)
        el = time.perf_counter() - t0
        steps, it1, launches = ens.stats()
        ens.close()
        return {"shape_used": list(used), "seconds": el, "interactions": it1 - it0,
                "interactions_per_s": (it1 - it0) / el,
                "block_steps": int(steps.sum()), "max_steps": int(steps.max())}

    out = {"workload": f"ensemble_{args.ens_systems}_plummer_N256-16384_eps1e-4",
           "systems": int(sizes.size), "particles": int(sizes.sum())}
    precs = ("mixed", "fp64") if args.prec == "both" else (args.prec,)
    prec_of = {"mixed": nb.NB_MIXED, "fp64": nb.NB_FP64, "ex": nb.NB_EX, "mixed32": nb.NB_MIXED32}
    def shapes_for(prec_name):
        spec = args.ens_shapes or "0x128x0"      # 0: the library's default for the precision
        out = [tuple(int(q) for q in sh.split("x")) for sh in spec.split(",")]
        return [sh if len(sh) == 3 else (sh[0], sh[1], 0) for sh in out]
    everyone = list(range(sizes.size))
    for prec_name in precs:
        prec = prec_of[prec_name]
        res = {"t_end": args.ens_t_end, "shapes": {}}
        shapes = shapes_for(prec_name)
        if args.ens_tune:
            from paper_1901_08532_gb300.autotune import tune_ensemble
            order = np.argsort(sizes)
            pick = [int(order[q]) for q in np.linspace(0, sizes.size - 1, 32).astype(int)]
            jts = (512, 1024) if prec_name in ("mixed", "mixed32") else (256, 512)
            cands = [(g, thr, jt) for g in (2, 4, 8, 16) for thr in (64, 128) for jt in jts]

            def make(pick=pick, prec=prec):
                return nb.Ensemble(sizes[pick], *cat(pick), EPS, precision=prec)

            def log(rec, prec_name=prec_name):
                print(json.dumps({"tune": prec_name, **rec}), flush=True)

            best, _ = tune_ensemble(make, 0.125, cands, log)
            shapes = [best]
            res["tuned_on"] = {"systems": len(pick), "t_end": 0.125, "candidates": len(cands)}
        for sh in shapes:
            r = run_ens(everyone, prec, sh, args.ens_t_end)
            res["shapes"]["%dx%dx%d" % sh] = r
            print(json.dumps({"progress": prec_name, "shape": sh, **r}), flush=True)
        best_shape = max(res["shapes"], key=lambda k: res["shapes"][k]["interactions_per_s"])
        res["best_shape"] = best_shape
        res["interactions_per_s"] = res["shapes"][best_shape]["interactions_per_s"]
        if args.ens_sample > 0:
            order = np.argsort(sizes)
            idx = [int(order[q]) for q in np.linspace(0, sizes.size - 1, args.ens_sample).astype(int)]
            sh = tuple(int(q) for q in best_shape.split("x"))
            batched = run_ens(idx, prec, sh, args.ens_cmp_t_end)
            tot_el, tot_it = 0.0, 0.0
            for k in idx:
                ctx = nb.NBody(*parts[k], EPS, precision=prec)
                _, i0 = ctx.counters()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx.run_until(args.ens_cmp_t_end)
                tot_el += time.perf_counter() - t0
                _, i1 = ctx.counters()
                tot_it += i1 - i0
                ctx.close()
            res["sample"] = {"systems": idx, "sizes": [int(sizes[k]) for k in idx],
                             "t_end": args.ens_cmp_t_end, "ensemble": batched,
                             "one_at_a_time": {"seconds": tot_el, "interactions": tot_it,
                                               "interactions_per_s": tot_it / tot_el},
                             "speedup": batched["interactions_per_s"] / (tot_it / tot_el)}
            print(json.dumps({"progress": prec_name, "sample": res["sample"]}), flush=True)
        out[prec_name] = res
    print(json.dumps(out))
    return 0


def adjoint_run(torch, n=8192, steps=64, checkpoint_every=8):
    """Differentiable fixed-step trajectory: Plummer N = n (seed 5), eps =
    1e-3, shared step 2^-10, `steps` steps, loss = sum m |x(T)|^2, gradients
    with respect to x0, v0, m through the hand-written adjoints with
    checkpoints every `checkpoint_every` steps.  Forward and forward+backward
    timed with device synchronisation on both sides."""
    import nb_inputs as ni
    from paper_1901_08532_gb300 import adjoint as A
    eps, h = 1e-3, 2.0 ** -10
    m, x, v = ni.plummer(n, 5)
    mt, xt, vt = (torch.tensor(q, dtype=torch.float64, device="cuda") for q in (m, x, v))
    with torch.no_grad():
        A.trajectory(mt, xt, vt, eps, h, 2, 0)          # warm-up
    A.loss_and_grads(mt, xt, vt, eps, h, 2, checkpoint_every=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.no_grad():
        A.trajectory(mt, xt, vt, eps, h, steps, 0)
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    L, gx, gv, gm = A.loss_and_grads(mt, xt, vt, eps, h, steps, checkpoint_every=checkpoint_every)
    torch.cuda.synchronize()
    both = time.perf_counter() - t0
    inter_fwd = float(n) * n * (steps + 2)
    return {"workload": f"adjoint_plummer_N{n}_eps1e-3_dt2^-10_{steps}steps_ckpt{checkpoint_every}",
            "forward_s": fwd, "forward_interactions_per_s": inter_fwd / fwd,
            "forward_plus_backward_s": both, "backward_s": both - fwd,
            "backward_over_forward": (both - fwd) / fwd,
            "loss": float(L), "grad_norms": [float(g.norm()) for g in (gx, gv, gm)]}


def adjoint_bench(args):
    """Config: Plummer N = 8192, eps = 1e-3, shared step 2^-10, 64 steps,
    loss = sum m |x(T)|^2, gradients with respect to x0, v0, m through the
    hand-written adjoint kernels with checkpoints every 8 steps."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(adjoint_run(torch, args.n if args.n != N_BODY else 8192)))
    return 0


def integrate_run(nb, np, torch, n, prec_name, t_end=1.0 / 16, step_noise=0.0):
    """Plummer N = n (equal masses, eps 1e-4, seed 2): one full-N evaluation
    (n^2 interactions), then block-step integration to t_end through
    nb_run_until (active sets from 1 to N particles), dt_max = 2^-4 so that
    every particle synchronises at t_end."""
    import nb_inputs as ni
    prec = {"mixed": nb.NB_MIXED, "fp64": nb.NB_FP64, "ex": nb.NB_EX, "sp": nb.NB_SP}[prec_name]
    m, x, v = ni.plummer(n, 2)
    stream = torch.cuda.current_stream()
    ctx = nb.NBody(m, x, v, EPS, precision=prec, stream=stream, dt_max=2.0 ** -4, step_noise=step_noise)
    ctx.predict(0.0)
    ctx.evaluate(None, out=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.evaluate(None, out=False)
    e1.record(stream)
    torch.cuda.synchronize()
    full_s = e0.elapsed_time(e1) / 1e3
    E0 = sum(ctx.energy())
    _, i0 = ctx.counters()
    t0 = time.perf_counter()
    steps, (lt, ln) = ctx.run_until(t_end, log_cap=10 ** 7)
    el = time.perf_counter() - t0
    _, i1 = ctx.counters()
    E1 = sum(ctx.energy())
    ctx.close()
    hist = np.bincount(np.floor(np.log2(np.maximum(ln, 1))).astype(int))
    flops = FLOPS_PER_INTERACTION * float(n) * n / full_s / 1e12
    peak = PEAK_FP64_TFLOPS if prec == nb.NB_FP64 else PEAK_FP32_TFLOPS
    n_fp32_ops = {nb.NB_EX: EX_OPS_PER_INTERACTION}.get(prec)
    return {"workload": f"plummer_N{n}_eps1e-4_{prec_name}" + (f"_noise{step_noise:g}" if step_noise else ""),
            "full_eval_s": full_s,
            "full_eval_interactions_per_s": float(n) * n / full_s,
            "full_eval_frac_of_peak": (flops / peak if n_fp32_ops is None else
                                       n_fp32_ops * float(n) * n / full_s / PEAK_FP32_OPS),
            "integration_t_end": t_end, "block_steps": steps,
            "integration_s": el, "us_per_block_step": 1e6 * el / max(steps, 1),
            "integration_interactions": i1 - i0,
            "integration_interactions_per_s": (i1 - i0) / el,
            "mean_active": float(ln.mean()), "max_active": int(ln.max()),
            "active_log2_histogram": hist.tolist(), "energy_rel_error": abs((E1 - E0) / E0)}


def integrate_bench(args):
    """Plummer N = 65536 (--prec fp64 in this mode's reference config; ex and
    mixed also run): one full-N evaluation (2^32 interactions), then
    block-step integration to t = 1/16."""
    import numpy as np
    import torch

    import paper_1901_08532_gb300 as nb
    torch.cuda.set_device(0)
    set_device_peaks(torch, 0)
    n = args.n if args.n != N_BODY else 65536
    print(json.dumps(integrate_run(nb, np, torch, n, args.prec, step_noise=args.step_noise)))
    return 0


def ensemble_leg(nb, np, torch, prec_name="ex", t_end=0.25, sample=256, step_noise=0.0):
    """Batched ensemble (256 Plummer systems, N log-uniform in [256, 16384],
    seed 4, eps 1e-4, own block steps) to t_end in one persistent
    graph-captured launch at the library's default shape, then `sample`
    systems spread over the size range (all 256 by default) advanced one at
    a time through nb_run_until against the same systems as one ensemble."""
    import nb_inputs as ni
    prec = {"mixed": nb.NB_MIXED, "mixed32": nb.NB_MIXED32, "fp64": nb.NB_FP64, "ex": nb.NB_EX}[prec_name]
    sizes = ni.ensemble_sizes(256, 4)
    parts = [ni.plummer(int(k), 1000 + q) for q, k in enumerate(sizes)]

    def run(idx):
        cat = [np.concatenate([parts[k][f] for k in idx]) for f in range(3)]
        ens = nb.Ensemble(sizes[idx], *cat, EPS, precision=prec, step_noise=step_noise)
        _, it0, _ = ens.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.run(t_end)
        el = time.perf_counter() - t0
        steps, it1, _ = ens.stats()
        shape = ens.shape()
        ens.close()
        return {"seconds": el, "interactions": it1 - it0, "interactions_per_s": (it1 - it0) / el,
                "block_steps": int(steps.sum()), "shape": list(shape)}

    out = {"workload": f"ensemble_256_plummer_N256-16384_eps1e-4_{prec_name}_t{t_end:g}"
                       + (f"_floor{step_noise:g}" if step_noise else ""),
           "systems": int(sizes.size), "particles": int(sizes.sum()), "all": run(list(range(sizes.size)))}
    if sample <= 0:
        return out
    order = np.argsort(sizes)
    idx = [int(order[q]) for q in np.linspace(0, sizes.size - 1, sample).astype(int)]
    batched = out["all"] if len(idx) == sizes.size else run(idx)
    tot_el, tot_it = 0.0, 0.0
    for k in idx:
        ctx = nb.NBody(*parts[k], EPS, precision=prec)
        _, i0 = ctx.counters()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.run_until(t_end)
        tot_el += time.perf_counter() - t0
        _, i1 = ctx.counters()
        tot_it += i1 - i0
        ctx.close()
    out["sample"] = {"systems": len(idx), "ensemble": batched,
                     "one_at_a_time": {"seconds": tot_el, "interactions": tot_it,
                                       "interactions_per_s": tot_it / tot_el},
                     "speedup": batched["interactions_per_s"] / (tot_it / tot_el)}
    return out


def config_legs(nb, np, torch, local):
    """The other configurations, compact, each under its own clock record:
    the 256-system ensemble to t = 1/4 in EX (with all 256 systems also run
    one at a time), in FP64, and in mixed with the step criterion's rounding
    floor at 4e-7 (nb_config.step_noise), the differentiable N = 8192 trajectory (64
    steps, checkpoints every 8), and the N = 65536 block-step integration
    to t = 1/16 in EX, FP64 and mixed (with the step criterion as is, and
    with its rounding floor at 4e-7, nb_config.step_noise)."""
    legs = {}
    for name, fn in (("ensemble_ex_256", lambda: ensemble_leg(nb, np, torch, "ex")),
                     ("ensemble_fp64_256", lambda: ensemble_leg(nb, np, torch, "fp64", sample=0)),
                     ("ensemble_mixed_256_floor4e-7",
                      lambda: ensemble_leg(nb, np, torch, "mixed", sample=0, step_noise=4e-7)),
                     ("adjoint_n8192", lambda: adjoint_run(torch)),
                     ("integrate_n65536_ex", lambda: integrate_run(nb, np, torch, 65536, "ex")),
                     ("integrate_n65536_fp64", lambda: integrate_run(nb, np, torch, 65536, "fp64")),
                     ("integrate_n65536_mixed", lambda: integrate_run(nb, np, torch, 65536, "mixed")),
                     ("integrate_n65536_mixed_floor4e-7",
                      lambda: integrate_run(nb, np, torch, 65536, "mixed", step_noise=4e-7))):
        with Clocks(local) as clk:
            rec = fn()
        rec["clocks"] = clk.summary()
        legs[name] = rec
    return legs


def precision_study(args):
    """The precision experiment of section 3 item 6: the same Plummer system
    integrated with block steps in each arithmetic, sampling the energy and
    the angular momentum on the device (nb_run_diag) and reporting
    dE/E = |E_start - E(t)| / |E_start| and dL/L = |L_start - L(t)| / |L_start|
    (Eq. 1; L the vector, also relative to sum m |x cross v| because the net
    L of an isotropic model is small)."""
    import numpy as np
    import torch

    import nb_inputs as ni
    import paper_1901_08532_gb300 as nb
    torch.cuda.set_device(0)
    n = args.n if args.n != N_BODY else 4096
    m, x, v = ni.plummer(n, 1)
    precs = {"fp64": nb.NB_FP64, "mixed": nb.NB_MIXED, "ex": nb.NB_EX, "sp": nb.NB_SP}
    res = {"workload": f"precision_study_plummer_N{n}_equal_eps1e-4_t{args.ps_t_end:g}",
           "sample_dt": args.ps_dt, "t_end": args.ps_t_end}
    for name in args.ps_precs.split(","):
        base, _, noise = name.partition("@")
        ctx = nb.NBody(m, x, v, EPS, precision=precs[base], dt_max=args.ps_dt,
                       step_noise=float(noise) if noise else 0.0)
        t0 = time.perf_counter()
        steps, d = ctx.run_diag(args.ps_t_end, args.ps_dt)
        el = time.perf_counter() - t0
        _, inter = ctx.counters()
        ctx.close()
        E = d["ekin"] + d["epot"]
        dE = np.abs(E[0] - E) / abs(E[0])
        dL = np.linalg.norm(d["L"] - d["L"][0], axis=1)
        res[name] = {"block_steps": steps, "seconds": el, "interactions": inter,
                     "t": d["t"].tolist(), "dE_over_E": dE.tolist(),
                     "dL_over_L": (dL / np.linalg.norm(d["L"][0])).tolist(),
                     "dL_over_sum_m_xv": (dL / d["labs"][0]).tolist(),
                     "max_dE_over_E": float(dE.max()), "final_dE_over_E": float(dE[-1])}
        print(json.dumps({"prec": name, "block_steps": steps, "seconds": el,
                          "max_dE_over_E": float(dE.max()), "final_dE_over_E": float(dE[-1]),
                          "final_dL_over_L": res[name]["dL_over_L"][-1]}), flush=True)
    print(json.dumps(res))
    return 0


def measure_peaks(nb, torch, iters=4096):
    """Measured CUDA-core peaks of this device (nb_peak_probe): operations
    per clock per SM and the derived whole-GPU peaks at the device's maximum
    SM clock.  FP32 and FP64 flop peaks count an FMA as 2 flops."""
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = _max_sm_mhz(dev)
    res = {"sms": sms, "sm_max_mhz": max_mhz, "kinds": {}}
    # (label, probe kind, blocks per SM, threads): 32 warps per SM, and the
    # three-operand case also at the 12 warps per SM the mixed kernel runs
    for label, kind, bps, thr, it in (("ffma", "ffma", 4, 256, iters), ("ffma2", "ffma2", 4, 256, iters),
                                      ("dfma", "dfma", 4, 256, max(1, iters // 16)),
                                      ("rsqrt", "rsqrt", 4, 256, iters), ("rcp", "rcp", 4, 256, iters),
                                      ("ffma2+rsqrt", "ffma2+rsqrt", 4, 256, iters),
                                      ("ffma2+rsqrt_noftz", "ffma2+rsqrt_noftz", 4, 256, iters),
                                      ("ffma2+rsqrt+rcp", "ffma2+rsqrt+rcp", 4, 256, iters),
                                      ("ffma2_3reg", "ffma2_3reg", 4, 256, iters),
                                      ("ffma2_3reg@12warps", "ffma2_3reg", 3, 128, iters)):
        res["kinds"][label] = nb.peak_probe(kind, bps, thr, it)
    k = res["kinds"]
    fp32 = max(k["ffma"]["ops_per_clk_per_sm"], k["ffma2"]["ops_per_clk_per_sm"])
    res["fp32_fma_per_clk_per_sm"] = fp32
    res["fp64_fma_per_clk_per_sm"] = k["dfma"]["ops_per_clk_per_sm"]
    res["fp32_tflops_at_max_clock"] = 2 * fp32 * sms * max_mhz * 1e6 / 1e12
    res["fp64_tflops_at_max_clock"] = 2 * k["dfma"]["ops_per_clk_per_sm"] * sms * max_mhz * 1e6 / 1e12
    return res


def _max_sm_mhz(dev):
    """The device's maximum SM clock (nvidia-smi clocks.max.sm), else 2070."""
    try:
        import torch
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        out = subprocess.run(["nvidia-smi", f"--id={uuid}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=30)
        return float(out.stdout.strip().splitlines()[0])
    except Exception:
        return 2070.0


def peaks_bench(args):
    import torch

    import paper_1901_08532_gb300 as nb
    torch.cuda.set_device(0)
    with Clocks(0) as clk:
        res = measure_peaks(nb, torch)
    res["clocks"] = clk.summary()
    print(json.dumps(res))
    return 0


def census_bench(args):
    """The mixed and EX paths' errors over every particle of the headline
    model (Plummer with Salpeter masses, eps 1e-4, seed 3, the seeded
    acceleration field of the oracle comparison, t = 0, every particle
    active, the mixed path in the headline launch): |d|_inf against the FP64
    GPU path (whose own error is about 1e-15) in units of each sum's
    condition number sum_j |T_ij| (nb_evaluate_kappa), and in the plain
    reading |d|_inf / |ref|_2; counts against 1e-6 (mixed) and 1e-12 (EX)."""
    import numpy as np
    import torch

    import nb_inputs as ni
    import paper_1901_08532_gb300 as nb
    n = args.n
    torch.cuda.set_device(0)
    m, x, v = ni.plummer(n, SEED, imf="salpeter")
    a = oracle_accel(ni, n)
    res = {}
    for name, prec in (("fp64", nb.NB_FP64), ("mixed", nb.NB_MIXED), ("ex", nb.NB_EX)):
        ctx = nb.NBody(m, x, v, EPS, precision=prec, start_forces=False)
        ctx.set_state({"a": a})
        ctx.predict(0.0)
        t0 = time.perf_counter()
        res[name] = ctx.evaluate(None)
        res[name + "_s"] = time.perf_counter() - t0
        if prec == nb.NB_MIXED:
            res["kappa"] = ctx.evaluate_kappa(None)
            res["tiles"] = ctx.resolve_tiles(n)
        ctx.close()
    # the FP64 path once more on the inputs rounded to double words (hi + lo
    # FP32, as the EX buffer holds them): what separates EX's arithmetic from
    # its 48-bit representation of the inputs
    def dw(q):
        h = q.astype(np.float32).astype(np.float64)
        return h + (q - h).astype(np.float32).astype(np.float64)
    ctx = nb.NBody(dw(m), dw(x), dw(v), EPS, precision=nb.NB_FP64, start_forces=False)
    ctx.set_state({"a": dw(a)})
    ctx.predict(0.0)
    res["fp64_dw"] = ctx.evaluate(None)
    ctx.close()
    out = {"census": f"plummer_salpeter_N{n}_eps1e-4_all_active", "particles": n,
           "reference": "FP64 GPU path (ex_arith: on the double-word-rounded inputs)",
           "mixed_tiles": res["tiles"],
           "seconds": {k: res[k + "_s"] for k in ("fp64", "mixed", "ex")}}
    for path, ref, bound in (("mixed", "fp64", 1e-6), ("ex", "fp64", 1e-12), ("ex_arith", "fp64_dw", 1e-12)):
        got = res["ex" if path == "ex_arith" else path]
        out[path] = {name: kappa_stats(got[q], res[ref][q], res["kappa"][q], bound)
                     for q, name in enumerate(("acc", "jerk", "snap"))}
    print(json.dumps(out), flush=True)
    return 0


def kappa_stats(got, ref, kappa, bound):
    """Per particle |got - ref|_inf in units of the sum's condition number
    kappa (and of |ref|_2, the plain reading) against `bound`: the largest
    ratio, how many particles exceed half, 0.8 of and the whole bound, the
    99.9th percentile, and the fraction above the bound in the plain
    reading.  got, ref: [n][3]; kappa: [n]."""
    import numpy as np
    d = np.abs(np.asarray(got) - np.asarray(ref)).max(axis=1)
    r = d / np.asarray(kappa)
    plain = d / np.linalg.norm(ref, axis=1)
    return {"kappa_norm_max": float(r.max()),
            "above": {f"{t:g}": int((r > t).sum()) for t in (0.5 * bound, 0.8 * bound, bound)},
            "p999": float(np.quantile(r, 0.999)),
            f"plain_above_{bound:g}": float((plain > bound).mean())}


def main():
    args = parse()
    if args.peaks:
        return peaks_bench(args)
    if args.census:
        return census_bench(args)
    if args.precision_study:
        return precision_study(args)
    if args.integrate:
        return integrate_bench(args)
    if args.adjoint:
        return adjoint_bench(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_eval:
        return profile_eval(args)
    if args.ensemble:
        return ensemble_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
