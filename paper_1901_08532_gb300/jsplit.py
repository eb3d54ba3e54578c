"""Multi-device j-split of one system: the paper's decomposition of the
evaluation over devices (section 3 item 3: with n devices each one deals
with N/n particles and evaluates N (N/n) accelerations and derivatives, and
the results are collected and reduced across the nodes).

One process per GPU.  Every rank holds the whole system (state, predictor,
corrector and scheduler are replicated, and stay identical because every
rank applies the same reduced forces), but evaluates the active set only
against its own contiguous share [lo, hi) of the j-particles.  One
all-reduce (sum) of the [9][n_act] FP64 partial sums per block step is the
only exchange; the collective (NCCL between GPUs, gloo on CPU) returns the
same bits on every rank, so the replicas never drift apart.  The self term
needs no care: eps > 0 makes it exactly zero on whichever rank holds j = i.

The step itself is jsplit_step(), written against a small context protocol
(schedule, active, predict, evaluate_partial, set_forces, correct) that
NBody implements through the C-ABI.
"""
from __future__ import annotations


def shard_bounds(n: int, world: int, rank: int, align: int = 1):
    """Contiguous j-range [lo, hi) of `rank` among `world` ranks covering
    [0, n): boundaries are multiples of `align` (the FP32-row buffers are
    copied in 16-byte rows, so 4 particles), the last range ends at n, and
    the ranges differ in length by at most `align`."""
    if world < 1 or not 0 <= rank < world or n < 0 or align < 1:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0, align >= 1")
    units = -(-n // align)                     # ceil(n / align)
    lo_u = units * rank // world
    hi_u = units * (rank + 1) // world
    return min(n, lo_u * align), min(n, hi_u * align)


def reduce_partials(part, group=None):
    """Sum the ranks' partial sums in place (all-reduce); a no-op without an
    initialised process group or with one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part


def jsplit_step(ctx, lo: int, hi: int, group=None, out="device", scheduled=None):
    """One block step with the evaluation split over the ranks: schedule
    (unless `scheduled` holds the (t_next, n_act) of a schedule() call just
    made), predict, this rank's partial sums over j in [lo, hi), all-reduce,
    load the totals, correct.  Returns (t_next, n_act)."""
    t, n_act = scheduled if scheduled is not None else ctx.schedule()
    act = ctx.active()
    ctx.predict(t)
    part = ctx.evaluate_partial(act, lo, hi, out=out)
    reduce_partials(part, group)
    ctx.set_forces(act, part)
    ctx.correct(t)
    return t, n_act


class JSplit:
    """One system integrated by all ranks of `group` (torch.distributed),
    each evaluating its share of the j-particles.  m, x, v, eps and the
    keyword arguments are those of NBody; every rank passes the same
    system."""

    def __init__(self, m, x, v, eps, group=None, **kw):
        import torch.distributed as dist

        from . import NB_EX, NB_MIXED, NB_SP, NBody
        self.group = group
        if dist.is_available() and dist.is_initialized():
            self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        else:
            self.rank, self.world = 0, 1
        self.ctx = NBody(m, x, v, eps, **kw)
        rows = self.ctx.precision in (NB_MIXED, NB_SP, NB_EX)
        self.lo, self.hi = shard_bounds(self.ctx.n, self.world, self.rank, 4 if rows else 1)

    def step(self):
        return jsplit_step(self.ctx, self.lo, self.hi, self.group)

    def run_until(self, t_end):
        """Block steps until every particle reaches t_end (a multiple of
        dt_max); returns the number of steps."""
        steps = 0
        while True:
            t, n_act = self.ctx.schedule()
            if t > t_end:
                return steps
            jsplit_step(self.ctx, self.lo, self.hi, self.group, scheduled=(t, n_act))
            steps += 1

    def state(self):
        return self.ctx.state()

    def close(self):
        self.ctx.close()
