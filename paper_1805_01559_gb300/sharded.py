"""Row-sharded Algorithm 1 (Sec. III-C, Eqs. (3)-(5)).

Each rank holds a contiguous block of rows of the cost C with its row marginals p; the
column marginals q are replicated.  The row update of an iteration needs only a shard's own
rows; the column update needs the column sums of every shard.  So one iteration is a sweep
over every shard (``ot_assoc_shard_sweep``), one sum over the shards of J + 1 doubles (the
column sums and the row residual), and the same column update on every rank
(``ot_assoc_shard_update``).  The arithmetic is the library's (the C ABI through
``binding.Context``); this module orders the calls and the collective.

The result is the one ``Context.solve_cost`` defines (same cell, same iteration count
semantics, stop at row residual <= tol (1 - 2^-5)): potentials f (each shard's rows) and g
(natural units), transport cost, loads rho_j and the FP64 marginal residuals of the returned
plan.  Iteration 1 starts from g = 0 (or a warm g) in the log domain with a fixed 2^64 column
scale; when a column's scaled sum underflows it is taken again exactly (column maxima, then
shifted sums: two more sweeps and collectives).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import torch

from . import binding as B

STOP_MARGIN = 1.0 - 2.0 ** -5  # stop at residual <= tol (1 - 2^-5), as the single-GPU solver
AHEAD = 8  # iterations enqueued between two reads of the loop state
LOG2E = 1.0 / math.log(2.0)


@dataclasses.dataclass
class ShardResult:
    f: List[torch.Tensor]       # natural-unit row potentials, one tensor per local shard
    g: torch.Tensor             # natural-unit column potentials (J)
    rrh_load: torch.Tensor      # rho_j = sum_i C_ij pi_ij over all shards (J)
    transport_cost: float
    marg_err_row: float         # residuals of the returned plan, unit mass
    marg_err_col: float
    err_loop: float             # the residual that stopped the loop
    iters: int
    converged: bool


class DeviceOps:
    """The steps on this GPU, through the C ABI."""

    def __init__(self, ctx: "B.Context", stream=None):
        self.ctx = ctx
        self.stream = stream

    def new_F(self, I: int, like: torch.Tensor) -> torch.Tensor:
        return torch.empty((I, 2), dtype=torch.float32, device=like.device)

    def prepare(self, C: torch.Tensor) -> torch.Tensor:
        """The sweep reads 16-byte row pieces: a C whose rows are not 16-byte aligned is
        copied once into a padded buffer (a layout copy, no arithmetic)."""
        if C.stride(1) == 1 and C.stride(0) % 4 == 0 and C.data_ptr() % 16 == 0:
            return C
        I, J = C.shape
        buf = torch.empty((I, (J + 3) // 4 * 4), dtype=C.dtype, device=C.device)[:, :J]
        buf.copy_(C)
        return buf

    def mass(self, p, q, out):
        self.ctx.shard_mass(p, q, out, stream=self.stream)

    def sweep(self, mode, C, p, inv_mass, eps, G, F_in, F_out, colmax, col_out, row_out=None, f_out=None,
              state=None):
        self.ctx.shard_sweep(mode, C, p, inv_mass, eps, G, F_in, F_out, colmax, col_out, row_out, f_out, state,
                             stream=self.stream)

    def update(self, mode, q, inv_qmass, col, colmax, G_in, G_out, flag, err=None, it=0, tol_stop=0.0,
               max_iter=0, state=None):
        self.ctx.shard_update(mode, q, inv_qmass, col, colmax, G_in, G_out, flag, err, it, tol_stop, max_iter,
                              state, stream=self.stream)

    def finish(self, col2, row_err, q, mass, inv_qmass, eps, G, g_out, rho_out, summary):
        self.ctx.shard_finish(col2, row_err, q, mass, inv_qmass, eps, G, g_out, rho_out, summary,
                              stream=self.stream)


class DistReduce:
    """Sums (and maxima) over the ranks of a torch.distributed group (NCCL on GPUs)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def sum(self, t: torch.Tensor) -> None:
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def max(self, t: torch.Tensor) -> None:
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)


class LocalReduce:
    """One process holds every shard: the local combination is the whole reduction."""

    def sum(self, t: torch.Tensor) -> None:
        pass

    def max(self, t: torch.Tensor) -> None:
        pass


def _combine(parts: Sequence[torch.Tensor], how: str) -> torch.Tensor:
    if len(parts) == 1:
        return parts[0]
    out = parts[0].clone()
    for t in parts[1:]:
        if how == "sum":
            out += t
        else:
            torch.maximum(out, t, out=out)
    return out


def solve_sharded(ops, shards: Sequence[Tuple[torch.Tensor, torch.Tensor]], q: torch.Tensor, eps: float,
                  tol: float = 1e-6, max_iter: int = 2000, reduce=None,
                  warm_g: Optional[torch.Tensor] = None) -> ShardResult:
    """Algorithm 1 over row shards.  shards: this process's (C, p) blocks (one per rank in a
    multi-GPU run; several emulate ranks in one process); q: the replicated column marginals;
    reduce: DistReduce across ranks (default LocalReduce).  Raises ValueError on invalid
    marginals and FloatingPointError when a column sum is not positive and finite."""
    if not shards:
        raise ValueError("no shards")
    if not (eps > 0.0) or not math.isfinite(eps):
        raise ValueError("eps must be positive and finite")
    if max_iter < 1 or tol < 0.0:
        raise ValueError("max_iter >= 1 and tol >= 0 are required")
    reduce = reduce or LocalReduce()
    if hasattr(ops, "prepare"):
        shards = [(ops.prepare(C), p) for C, p in shards]
    J = q.numel()
    dev = q.device
    f64 = dict(dtype=torch.float64, device=dev)

    # total mass over every shard; the marginals must agree (as the single-GPU solver checks)
    outs = []
    for C, p in shards:
        if C.shape[0] != p.numel() or C.shape[1] != J:
            raise ValueError("shard shapes do not match q")
        o = torch.empty(3, **f64)
        ops.mass(p, q, o)
        outs.append(o)
    tot = torch.stack([_combine([o[0:1] for o in outs], "sum")[0], _combine([o[2:3] for o in outs], "sum")[0]])
    reduce.sum(tot)
    mass, bad = (float(x) for x in tot.cpu())
    qmass = float(outs[0][1].cpu())
    if bad > 0.0 or not (mass > 0.0) or not (qmass > 0.0):
        raise ValueError("p and q entries must be positive and finite")
    if not abs(mass - qmass) <= 1e-5 * mass:
        raise ValueError(f"sum p = {mass} and sum q = {qmass} differ")
    inv_mass, inv_qmass = 1.0 / mass, 1.0 / qmass

    G = torch.zeros(J, **f64) if warm_g is None else warm_g.to(**f64) * (LOG2E / eps)
    F = [(ops.new_F(C.shape[0], C), ops.new_F(C.shape[0], C)) for C, _ in shards]
    flag = torch.zeros(1, dtype=torch.int32, device=dev)

    # ---- iteration 1: F'^1 (buffer 1), then G^1 ------------------------------------------
    cols = []
    for (C, p), Fk in zip(shards, F):
        c = torch.empty(J, **f64)
        ops.sweep(B.OT_SHARD_FIRST, C, p, inv_mass, eps, G, None, Fk[1], None, c)
        cols.append(c)
    col = _combine(cols, "sum")
    reduce.sum(col)
    G1 = torch.empty(J, **f64)
    ops.update(B.OT_SHARD_FIRST, q, inv_qmass, col, None, G, G1, flag)
    if int(flag.cpu()[0]) & 1:  # a scaled column sum underflowed: exact iteration 1
        flag.zero_()
        maxes = []
        for (C, p), Fk in zip(shards, F):
            m = torch.empty(J, **f64)
            ops.sweep(B.OT_SHARD_COLMAX, C, p, inv_mass, eps, G, Fk[1], None, None, m)
            maxes.append(m)
        colmax = _combine(maxes, "max")
        reduce.max(colmax)
        cols = []
        for (C, p), Fk in zip(shards, F):
            c = torch.empty(J, **f64)
            ops.sweep(B.OT_SHARD_COLSUM, C, p, inv_mass, eps, G, Fk[1], None, colmax, c)
            cols.append(c)
        col = _combine(cols, "sum")
        reduce.sum(col)
        ops.update(B.OT_SHARD_COLSUM, q, inv_qmass, col, colmax, G, G1, flag)
    if int(flag.cpu()[0]):
        raise FloatingPointError("a column sum of iteration 1 is not positive and finite")
    G = G1

    # ---- iterations 2, 3, ...: sweep, one sum of J + 1 doubles, column update ----------------
    # The loop test runs in the update (a loop state on the device), so iterations are
    # enqueued AHEAD at a time and the host reads the state once per batch; launches after
    # the stop do nothing.  The collective still runs every enqueued iteration on every rank.
    state = torch.zeros(4, **f64)
    vbuf = [torch.empty(J + 1, **f64) for _ in shards]
    s = 2
    while True:
        for _ in range(AHEAD):
            old, new = (s - 1) & 1, s & 1
            for (C, p), Fk, v in zip(shards, F, vbuf):
                ops.sweep(B.OT_SHARD_ITER, C, p, inv_mass, eps, G, Fk[old], Fk[new], None, v[:J], v[J:], None,
                          state)
            vec = _combine(vbuf, "sum")
            reduce.sum(vec)
            ops.update(B.OT_SHARD_ITER, q, inv_qmass, vec[:J], None, G, G, flag, vec[J:], s, tol * STOP_MARGIN,
                       max_iter, state)
            s += 1
        st = torch.cat([state, flag.to(torch.float64)]).cpu()
        if st[0] != 0.0 or st[4] != 0.0:
            break
    reason, iters, ans, err = int(st[0]), int(st[1]), int(st[2]), float(st[3])
    if reason == 3 or st[4] != 0.0:
        raise FloatingPointError("a column sum is not positive and finite")
    conv = reason == 1

    # ---- finalize on the returned plan (F'^iters, G^iters) -------------------------------------
    parts, fs = [], []
    for (C, p), Fk in zip(shards, F):
        v = torch.empty(2 * J + 1, **f64)
        f_nat = torch.empty(C.shape[0], **f64)
        ops.sweep(B.OT_SHARD_FINAL, C, p, inv_mass, eps, G, Fk[ans], None, None, v[:2 * J], v[2 * J:], f_nat)
        parts.append(v)
        fs.append(f_nat)
    vec = _combine(parts, "sum")
    reduce.sum(vec)
    g_out, rho, summary = torch.empty(J, **f64), torch.empty(J, **f64), torch.empty(3, **f64)
    ops.finish(vec[:2 * J], vec[2 * J:], q, mass, inv_qmass, eps, G, g_out, rho, summary)
    cost, er, ec = (float(x) for x in summary.cpu())
    return ShardResult(f=fs, g=g_out, rrh_load=rho, transport_cost=cost, marg_err_row=er, marg_err_col=ec,
                       err_loop=err, iters=iters, converged=bool(conv))
