"""The association policies of Sec. IV compared by average job completion time (Sec. II-B).

  (a) maxSINR: every device on its strongest RRH (Sec. II-C);
  (b) OT with the Euclidean cost ||x_i - x_j|| and equal RRH traffic q_j = sum(lambda) / J;
  (c) OT with the load cost 1/(mu R_ij) and equal RRH traffic;
  (d) OT with the load cost and q_j = Lambda_j, the RRH traffic of maxSINR (Lemma 1).

Each OT policy is the entropic plan of Eq. (5) (Algorithm 1), evaluated on the load cost:
rho_j = sum_i C_ij x_ij and T = (1/I) sum_ij pi_ij C_ij / (1 - rho_j).  Every step runs in the
library's kernels (rates, costs, maxSINR, solves, evaluation); this module only marshals
arguments and moves J-vectors between host and device.

Choices the paper leaves open (each a reading of Sec. IV's experiment):
  * the traffic level: total traffic scaled so that maxSINR's most loaded RRH is at
    `load_target` (maxSINR must be feasible for Lemma 1);
  * eps: `eps_best` times the mean cost of the devices' cheapest links, per cost (the
    regularisation must be small next to the costs a plan actually uses for the plan to
    approach the LP solution Lemma 1 speaks of; a multiple of median(C) is not: the median
    is set by distant links);
  * RRHs that no device picks under maxSINR get Lambda_j floored to 1e-6 of an equal share
    (the solver needs q_j > 0), and q is renormalised to sum(lambda).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import binding


def _padded(I: int, J: int, dev) -> torch.Tensor:
    ld = (J + 3) // 4 * 4
    return torch.empty((I, ld), dtype=torch.float32, device=dev)[:, :J]


@dataclasses.dataclass
class Prepared:
    C: torch.Tensor          # load cost
    Ce: torch.Tensor         # Euclidean cost
    lam: torch.Tensor        # scaled traffic
    assoc: torch.Tensor      # maxSINR association
    T_a: float
    scale: float             # traffic scale applied to the unit-total cell
    eps_load: float
    eps_euclid: float
    instances: list          # binding.Instance for (b), (c), (d)


@dataclasses.dataclass
class PolicyResult:
    T: dict                  # average completion time per policy (s)
    ratio: dict              # T / T_a for b, c, d
    max_load: dict           # largest rho_j per policy
    total_load: dict         # sum_j rho_j per policy
    iters: dict
    converged: dict
    scale: float
    eps_load: float
    eps_euclid: float


def prepare(ctx: "binding.Context", cell, load_target: float = 0.3, eps_best: float = 0.01, tol: float = 1e-6,
            max_iter: int = 2000, device: Optional[torch.device] = None) -> Prepared:
    dev = device or torch.device("cuda", ctx.device if hasattr(ctx, "device") else 0)
    N, J = cell.G.shape
    G = _padded(N, J, dev)
    G.copy_(torch.from_numpy(np.ascontiguousarray(cell.G, dtype=np.float32)))
    P = torch.from_numpy(cell.P.astype(np.float32)).to(dev)
    R = ctx.build_rates(G, P, cell.N0, cell.W_hz, R_out=_padded(N, J, dev))
    C, _ = ctx.build_cost(R, cell.mu, C_out=_padded(N, J, dev))
    lam1 = torch.from_numpy(cell.lam.astype(np.float32)).to(dev)
    assoc, Lam1, _ = ctx.maxsinr(R, lam1, cell.mu)
    _, rho1 = ctx.completion_time(C, lam1, assoc=assoc)
    scale = load_target / float(rho1.cpu().numpy().max())
    lam_h = (cell.lam * scale).astype(np.float32)
    lam = torch.from_numpy(lam_h).to(dev)
    T_a, _ = ctx.completion_time(C, lam, assoc=assoc, want_rho=False)
    total = float(lam_h.astype(np.float64).sum())
    q_eq = torch.full((J,), total / J, dtype=torch.float32, device=dev)
    Lam = Lam1.cpu().numpy() * scale
    Lam = np.maximum(Lam, 1e-6 * total / J)
    q_d = torch.from_numpy((Lam * (total / Lam.sum())).astype(np.float32)).to(dev)
    Ce = ctx.euclid_cost(torch.from_numpy(np.ascontiguousarray(cell.dev_xy, np.float32)).to(dev),
                         torch.from_numpy(np.ascontiguousarray(cell.rrh_xy, np.float32)).to(dev),
                         C_out=_padded(N, J, dev))
    eps_l = eps_best * ctx.mean_row_min(C)
    eps_e = eps_best * ctx.mean_row_min(Ce)
    mk = lambda Cp, q, e: binding.Instance(C=Cp, p=lam, q=q, eps=e, tol=tol, max_iter=max_iter)
    inst = [mk(Ce, q_eq, eps_e), mk(C, q_eq, eps_l), mk(C, q_d, eps_l)]
    return Prepared(C=C, Ce=Ce, lam=lam, assoc=assoc, T_a=T_a, scale=scale, eps_load=eps_l, eps_euclid=eps_e,
                    instances=inst)


def finish(ctx: "binding.Context", prep: Prepared, results) -> PolicyResult:
    T = {"a": prep.T_a}
    ml, tl, its, conv = {}, {}, {}, {}
    _, rho_a = ctx.completion_time(prep.C, prep.lam, assoc=prep.assoc)
    rho_a = rho_a.cpu().numpy()
    ml["a"] = float(rho_a.max())
    tl["a"] = float(rho_a.sum())
    for name, inst, r in zip("bcd", prep.instances, results):
        Cp = prep.Ce if name == "b" else None
        eps = prep.eps_euclid if name == "b" else prep.eps_load
        T[name], rho = ctx.completion_time(prep.C, prep.lam, f=inst.f, g=inst.g, eps=eps, C_plan=Cp)
        rho = rho.cpu().numpy()
        ml[name] = float(rho.max())
        tl[name] = float(rho.sum())
        its[name] = r.iters
        conv[name] = r.converged
    ratio = {k: T[k] / T["a"] for k in "bcd"}
    return PolicyResult(T=T, ratio=ratio, max_load=ml, total_load=tl, iters=its, converged=conv, scale=prep.scale,
                        eps_load=prep.eps_load, eps_euclid=prep.eps_euclid)


def evaluate(ctx: "binding.Context", cell, **kw) -> PolicyResult:
    """All four policies on one cell: the three OT solves in one batched launch."""
    prep = prepare(ctx, cell, **kw)
    res = ctx.solve_batched(prep.instances)
    return finish(ctx, prep, res)
