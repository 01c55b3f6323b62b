"""Row-sharded Algorithm 1: the host driver (`paper_1805_01559_gb300.sharded`) and its
collectives, on CPU.  The per-shard steps run in an FP64 numpy stand-in for the device calls
(written from their definitions in include/ot_assoc.h); the ranks are a world_size-2 `gloo`
group.  The result after k iterations must be the oracle's Algorithm 1 iterate on the whole
matrix, and a converged solve must stop where the oracle's does (within one iteration)."""
from __future__ import annotations

import math
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

from paper_1805_01559_gb300 import sharded as S  # noqa: E402

FIRST, ITER, COLMAX, COLSUM, FINAL = 0, 1, 2, 3, 4
LN2 = math.log(2.0)


class NumpyOps:
    """FP64 stand-in for ot_assoc_shard_* (CPU tensors in, CPU tensors out)."""

    def new_F(self, I, like):
        return torch.zeros(I, dtype=torch.float64)

    def mass(self, p, q, out):
        pn, qn = p.numpy().astype(np.float64), q.numpy().astype(np.float64)  # FP64 sums, as the device
        bad = not (np.isfinite(pn).all() and (pn > 0).all() and np.isfinite(qn).all() and (qn > 0).all())
        out[0], out[1], out[2] = float(pn.sum()), float(qn.sum()), 1.0 if bad else 0.0

    def sweep(self, mode, C, p, inv_mass, eps, G, F_in, F_out, colmax, col_out, row_out=None, f_out=None,
              state=None):
        if state is not None and state[0] != 0.0:
            return
        k = 1.0 / (eps * LN2)  # log2(e) / eps
        Cn, Gn, pn = C.numpy().astype(np.float64), G.numpy(), p.numpy().astype(np.float64)
        ph = pn * inv_mass
        J = Gn.size
        y = Gn[None, :] - k * Cn
        if mode == FIRST:
            m = y.max(1)
            F1 = -(m + np.log2(np.exp2(y - m[:, None]).sum(1)))
            F_out.numpy()[:] = F1
            col_out.numpy()[:] = 2.0 ** 64 * (ph[:, None] * np.exp2(F1[:, None] + y)).sum(0)
            return
        F = F_in.numpy()
        x = F[:, None] + y
        if mode == ITER:
            r = np.exp2(x).sum(1)
            Fn = F - np.log2(r)
            F_out.numpy()[:] = Fn
            row_out.numpy()[0] = (ph * np.abs(r - 1.0)).sum()
            col_out.numpy()[:] = (ph[:, None] * np.exp2(Fn[:, None] + y)).sum(0)
        elif mode == COLMAX:
            col_out.numpy()[:] = (x + np.log2(ph)[:, None]).max(0)
        elif mode == COLSUM:
            col_out.numpy()[:] = np.exp2(x + np.log2(ph)[:, None] - colmax.numpy()[None, :]).sum(0)
        elif mode == FINAL:
            t = np.exp2(x)
            col_out.numpy()[:J] = (ph[:, None] * t).sum(0)
            col_out.numpy()[J:] = (ph[:, None] * np.where(t > 0, Cn * t, 0.0)).sum(0)
            row_out.numpy()[0] = (ph * np.abs(t.sum(1) - 1.0)).sum()
            if f_out is not None:
                f_out.numpy()[:] = eps * LN2 * (F + np.log2(pn))

    def update(self, mode, q, inv_qmass, col, colmax, G_in, G_out, flag, err=None, it=0, tol_stop=0.0,
               max_iter=0, state=None):
        if state is not None:
            if state[0] != 0.0:
                return
            if mode == ITER:
                e = float(err[0])
                if not math.isfinite(e) or e <= tol_stop or it - 1 >= max_iter:
                    state[1], state[2], state[3] = it - 1, (it - 1) & 1, e
                    state[0] = 3.0 if not math.isfinite(e) else (1.0 if e <= tol_stop else 2.0)
                    return
        lq = np.log2(q.numpy().astype(np.float64) * inv_qmass)
        c, g = col.numpy(), G_in.numpy().copy()
        if mode == FIRST:
            if not (np.isfinite(c).all() and (c >= 2.0 ** -60).all()):
                flag[0] |= 1
                return
            G_out.numpy()[:] = g + lq - (np.log2(c) - 64.0)
            return
        M = colmax.numpy() if mode == COLSUM else 0.0
        if not (np.isfinite(c).all() and (c > 0).all()):
            flag[0] |= 2
            if state is not None:
                state[0] = 3.0
            return
        G_out.numpy()[:] = g + lq - (M + np.log2(c))

    def finish(self, col2, row_err, q, mass, inv_qmass, eps, G, g_out, rho_out, summary):
        J = q.numel()
        c2 = col2.numpy()
        rho_out.numpy()[:] = c2[J:] * mass
        g_out.numpy()[:] = eps * LN2 * G.numpy()
        summary.numpy()[:] = [c2[J:].sum() * mass, float(row_err.numpy()[0]),
                              np.abs(c2[:J] - q.numpy() * inv_qmass).sum()]


def _instance(seed, I, J, underflow=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    if underflow:
        C[:, 0] += 3.0  # at eps = 0.02 the first half-step's column 0 is far below 2^-124
    p = rng.lognormal(0.0, 1.0, I)
    q = rng.uniform(0.5, 1.5, J)
    p = (p / p.sum()).astype(np.float32)
    q = (q / q.sum()).astype(np.float32)
    return C, p, q


def _shards(C, p, cuts):
    b = [0, *cuts, C.shape[0]]
    return [(torch.from_numpy(C[b[i]:b[i + 1]]), torch.from_numpy(p[b[i]:b[i + 1]])) for i in range(len(b) - 1)]


def _plan_close(C, f, g, f_or, g_or, eps, rtol):
    C64 = C.astype(np.float64)
    a, b = oracle.plan(C64, f, g, eps), oracle.plan(C64, f_or, g_or, eps)
    np.testing.assert_allclose(a, b, rtol=rtol, atol=1e-15)


@pytest.mark.parametrize("iters", [1, 2, 7])
def test_three_local_shards_equal_the_oracle_iterate(iters):
    C, p, q = _instance(3, 301, 23)
    eps = 0.1
    res = S.solve_sharded(NumpyOps(), _shards(C, p, [97, 98]), torch.from_numpy(q), eps, tol=0.0,
                          max_iter=iters)
    f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, eps, 0.0, iters)
    assert res.iters == iters
    f = np.concatenate([t.numpy() for t in res.f])
    _plan_close(C, f, res.g.numpy(), f_or, g_or, eps, 1e-9)


def test_converged_stop_and_summary_match_the_oracle():
    C, p, q = _instance(5, 400, 31)
    eps, tol = 0.05, 1e-6
    res = S.solve_sharded(NumpyOps(), _shards(C, p, [150]), torch.from_numpy(q), eps, tol=tol, max_iter=5000)
    C64 = C.astype(np.float64)
    f_or, g_or, it_or, _ = oracle.sinkhorn(C64, p, q, eps, tol, 5000)
    assert res.converged and abs(res.iters - it_or) <= 1
    f = np.concatenate([t.numpy() for t in res.f])
    cost, rho, er, ec = oracle.finalize(C64, f, res.g.numpy(), p, q, eps)
    assert er <= tol and ec <= tol
    assert res.transport_cost == pytest.approx(cost, rel=1e-12)
    assert res.marg_err_row == pytest.approx(er, rel=1e-9, abs=1e-15)
    # the device measures columns against q / sum q, the oracle against q / sum p: with float32
    # marginals the two differ by at most |sum q / sum p - 1|
    sp, sq = p.astype(np.float64).sum(), q.astype(np.float64).sum()
    assert res.marg_err_col == pytest.approx(ec, rel=1e-9, abs=abs(sq / sp - 1.0) + 1e-15)
    np.testing.assert_allclose(res.rrh_load.numpy(), rho, rtol=1e-12)


def test_invalid_marginals_are_rejected():
    C, p, q = _instance(7, 50, 5)
    p[3] = 0.0
    with pytest.raises(ValueError):
        S.solve_sharded(NumpyOps(), _shards(C, p, [20]), torch.from_numpy(q), 0.1)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        C, p, q, eps, tol, iters, cut = case
        lo, hi = (0, cut) if rank == 0 else (cut, C.shape[0])
        res = S.solve_sharded(NumpyOps(), [(torch.from_numpy(C[lo:hi]), torch.from_numpy(p[lo:hi]))],
                              torch.from_numpy(q), eps, tol=tol, max_iter=iters, reduce=S.DistReduce())
        out.put((rank, res.f[0].numpy(), res.g.numpy(), res.iters, res.transport_cost, res.marg_err_row))
    finally:
        dist.destroy_process_group()


def _run_world2(case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, case, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = sorted((out.get(timeout=120) for _ in range(2)), key=lambda x: x[0])
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    return got


@pytest.mark.parametrize("underflow", [False, True])
def test_two_gloo_ranks_equal_the_oracle_iterate(underflow):
    # iteration 1 with an underflowing column goes through the exact passes and a MAX reduce
    C, p, q = _instance(11, 257, 19, underflow=underflow)
    eps, iters = (0.02 if underflow else 0.1), 5
    got = _run_world2((C, p, q, eps, 0.0, iters, 131))
    f = np.concatenate([got[0][1], got[1][1]])
    g0, g1 = got[0][2], got[1][2]
    assert np.array_equal(g0, g1)  # every rank applies the same column update
    assert got[0][3] == got[1][3] == iters
    assert got[0][4] == got[1][4] and got[0][5] == got[1][5]  # the same totals on both ranks
    f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, eps, 0.0, iters)
    _plan_close(C, f, g0, f_or, g_or, eps, 1e-9)


def test_two_gloo_ranks_converge_like_the_oracle():
    C, p, q = _instance(13, 360, 27)
    eps, tol = 0.05, 1e-6
    got = _run_world2((C, p, q, eps, tol, 5000, 200))
    f_or, g_or, it_or, _ = oracle.sinkhorn(C.astype(np.float64), p, q, eps, tol, 5000)
    assert abs(got[0][3] - it_or) <= 1
    f = np.concatenate([got[0][1], got[1][1]])
    cost, _, er, ec = oracle.finalize(C.astype(np.float64), f, got[0][2], p, q, eps)
    assert er <= tol and ec <= tol
    assert got[0][4] == pytest.approx(cost, rel=1e-12)


def test_a_column_without_links_fails_loudly():
    # column 0 has no finite cost: its sum is 0 in iteration 1, the exact passes cannot repair
    # it, and the driver raises instead of returning potentials
    C, p, q = _instance(17, 120, 9)
    C[:, 0] = np.inf
    with np.errstate(all="ignore"), pytest.raises(FloatingPointError):
        S.solve_sharded(NumpyOps(), _shards(C, p, [60]), torch.from_numpy(q), 0.1, tol=1e-6, max_iter=50)


def test_max_iter_one_returns_the_first_iterate():
    C, p, q = _instance(19, 150, 11)
    res = S.solve_sharded(NumpyOps(), _shards(C, p, [70]), torch.from_numpy(q), 0.2, tol=1e-9, max_iter=1)
    f_or, g_or, it_or, err_or = oracle.sinkhorn(C.astype(np.float64), p, q, 0.2, 0.0, 1)
    assert res.iters == 1 and not res.converged
    assert res.err_loop == pytest.approx(err_or, rel=1e-9)
    _plan_close(C, np.concatenate([t.numpy() for t in res.f]), res.g.numpy(), f_or, g_or, 0.2, 1e-9)
