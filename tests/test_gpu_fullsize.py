"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

50,000 x 800 (the default benchmark step): the oracle finishes the whole instance in seconds,
so the rates are compared everywhere, the median bit for bit, and the three solves of the
step (eps = 0.1, 0.03, 0.01 x median, enqueued back to back as the benchmark does) against
the oracle's converged solves on the same FP32 cost, with the converged-solve tolerances of
test_gpu_parity.py.

400,000 x 4,096 (the stored-kernel configuration), twice:
  * the GPU's own pipeline (gains -> rates and cost on the device), checked on sampled outputs
    the oracle computes one by one (rates and cost of sampled rows, the plan's row sums of
    sampled rows) and on properties that hold at any size;
  * the whole instance against the FP64 oracle: the oracle builds C (rates with the O(I J)
    total-minus-own interference), solves Algorithm 1 to tol 1e-7 and evaluates the GPU's
    FP32 log-domain, BF16-K~ and FP16-K~ answers on the same C exactly: cost and marginal L1
    within 1e-6 for FP32 and within 1e-3 for the stored 16-bit kernels.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_REL = (0.1, 0.03, 0.01)
TOL = 1e-6
MARG_SLACK = 0.0  # the device stops at FP32 residual <= tol (1 - 2^-5)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_01559_gb300 import binding
    c = binding.Context(0)
    yield c
    c.close()


def test_step_50000x800_against_the_oracle(ctx):
    from paper_1805_01559_gb300 import instances as ins
    inst = ins.config2(0)
    I, J = inst.I, inst.J
    dev = torch.device("cuda", 0)
    G = torch.from_numpy(np.ascontiguousarray(inst.G, dtype=np.float32)).to(dev)
    P = torch.from_numpy(inst.P.astype(np.float32)).to(dev)
    lam = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    q = torch.from_numpy(inst.q.astype(np.float32)).to(dev)
    R = torch.empty((I, J), dtype=torch.float32, device=dev)
    ctx.build_cost_from_gains(G, P, inst.N0, inst.W_hz, inst.mu, R_out=R)
    # rates on the oracle for the whole instance (it forms each interference sum directly);
    # the device's rates within the rate tolerance everywhere
    R_or = oracle.rates(inst.G.astype(np.float32).astype(np.float64), inst.P, inst.N0, inst.W_hz)
    np.testing.assert_allclose(R.cpu().numpy(), R_or, rtol=1e-6)
    # the solves run on the oracle's cost rounded to FP32, the same matrix on both sides
    C32 = oracle.cost(R_or, inst.mu).astype(np.float32)
    C64 = C32.astype(np.float64)
    C = torch.from_numpy(C32).to(dev)
    med = ctx.median_f32(C.view(-1))
    assert med == oracle.median(C64)  # exact
    lam64 = inst.lam.astype(np.float32).astype(np.float64)
    q64 = inst.q.astype(np.float32).astype(np.float64)
    pend = [ctx.solve_cost_async(C, lam, q, er * med, tol=TOL, max_iter=2000) for er in EPS_REL]
    results = [x.wait() for x in pend]
    for er, r in zip(EPS_REL, results):
        eps = er * med
        f_o, g_o, it_o, _ = oracle.sinkhorn(C64, lam64, q64, eps, TOL, 2000)
        cost_o = oracle.finalize(C64, f_o, g_o, lam64, q64, eps)[0]
        assert r.status == 0
        assert abs(r.iters - it_o) <= 2, (er, r.iters, it_o)
        assert r.transport_cost == pytest.approx(cost_o, rel=1e-6)
        _, rho, e_r, e_c = oracle.finalize(C64, r.f.cpu().numpy(), r.g.cpu().numpy(), lam64, q64, eps)
        assert e_r <= TOL + MARG_SLACK and e_c <= TOL + MARG_SLACK
        np.testing.assert_allclose(r.rrh_load.cpu().numpy(), rho, rtol=1e-5)


def _c4_block(args):
    from paper_1805_01559_gb300 import instances as ins
    seed, I, J, block, b = args
    return b, ins.config4_blocked(seed, I, J, block).gains_block(b)


def test_stored_kernel_400000x4096_sampled_and_properties(ctx):
    from paper_1805_01559_gb300 import binding, instances as ins
    I, J, block = 400_000, 4096, 8192
    inst = ins.config4_blocked(0, I, J, block)
    dev = torch.device("cuda", 0)
    P = torch.from_numpy(inst.P.astype(np.float32)).to(dev)
    C = torch.empty((I, J), dtype=torch.float32, device=dev)
    rng = np.random.Generator(np.random.PCG64(9))
    sample = np.sort(rng.choice(I, 8, replace=False))
    sampled_G = {}
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        for b, Gb in pool.imap_unordered(_c4_block, [(0, I, J, block, b) for b in range(inst.nblocks)]):
            r0 = b * block
            for i in sample[(sample >= r0) & (sample < r0 + Gb.shape[0])]:
                sampled_G[int(i)] = Gb[i - r0].copy()
            Gd = torch.from_numpy(Gb).to(dev)
            ctx.build_cost_from_gains(Gd, P, inst.N0, inst.W_hz, inst.mu, C_out=C[r0:r0 + Gb.shape[0]])
            del Gd
    # rates and cost of sampled rows, one by one on the oracle
    Gs = np.stack([sampled_G[int(i)] for i in sample]).astype(np.float64)
    C_or = oracle.cost(oracle.rates(Gs, inst.P, inst.N0, inst.W_hz), inst.mu)
    C_rows = C[torch.from_numpy(sample).to(dev)].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(C_rows, C_or, rtol=2e-6)
    med = ctx.median_f32(C.view(-1))
    eps = 0.05 * med
    p = torch.from_numpy(inst.lam.astype(np.float32)).to(dev)
    q = torch.from_numpy(inst.q.astype(np.float32)).to(dev)
    ref = ctx.solve_cost(C, p, q, eps, tol=TOL, max_iter=2000)
    assert ref.status == 0
    assert ref.marg_err_row <= TOL + MARG_SLACK and ref.marg_err_col <= TOL + MARG_SLACK
    assert float(ref.rrh_load.sum().item()) == pytest.approx(ref.transport_cost, rel=1e-9)
    # the plan's rows of sampled devices, from the returned potentials, in FP64 on the host
    p64 = inst.lam.astype(np.float32).astype(np.float64)
    f, g = ref.f.cpu().numpy(), ref.g.cpu().numpy()
    rows = np.exp((f[sample, None] + g[None, :] - C_or) / eps).sum(axis=1)
    np.testing.assert_allclose(rows, p64[sample], rtol=5e-4)  # per row; the total L1 is <= tol
    for fmt, tol_cost, tol_marg in ((binding.OT_KERNEL_BF16, 1e-4, 1e-3), (binding.OT_KERNEL_F16, 1e-4, 1e-3)):
        r = ctx.solve_lowp(C, p, q, eps, tol=TOL, max_iter=2000, fmt=fmt)
        assert r.status in (0, 1)
        assert r.transport_cost == pytest.approx(ref.transport_cost, rel=tol_cost)
        assert r.marg_err_row <= tol_marg and r.marg_err_col <= tol_marg


def test_c4_full_instance_against_the_oracle(ctx):
    from paper_1805_01559_gb300 import binding, instances as ins
    I, J, block = 400_000, 4096, 8192
    inst = ins.config4_blocked(0, I, J, block)
    C32 = np.empty((I, J), np.float32)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        for b, Gb in pool.imap_unordered(_c4_block, [(0, I, J, block, b) for b in range(inst.nblocks)]):
            r0 = b * block
            C32[r0:r0 + Gb.shape[0]] = oracle.cost(oracle.rates_total(Gb, inst.P, inst.N0, inst.W_hz),
                                                   inst.mu).astype(np.float32)
    C64 = C32.astype(np.float64)
    eps = 0.05 * oracle.median(C64)
    p, q = inst.lam.astype(np.float32), inst.q.astype(np.float32)
    dev = torch.device("cuda", 0)
    Cd = torch.from_numpy(C32).to(dev)
    pd, qd = torch.from_numpy(p).to(dev), torch.from_numpy(q).to(dev)
    runs = {"f32": ctx.solve_cost(Cd, pd, qd, eps, tol=TOL, max_iter=2000)}
    for name, fmt in (("bf16", binding.OT_KERNEL_BF16), ("f16", binding.OT_KERNEL_F16)):
        runs[name] = ctx.solve_lowp(Cd, pd, qd, eps, tol=TOL, max_iter=2000, fmt=fmt)
    got = {k: (r.status, r.transport_cost, r.f.cpu().numpy(), r.g.cpu().numpy()) for k, r in runs.items()}
    del Cd
    torch.cuda.empty_cache()
    f_or, g_or, _, _ = oracle.sinkhorn(C64, p, q, eps, 1e-7, 2000)
    cost_or = oracle.finalize(C64, f_or, g_or, p, q, eps)[0]
    for name, (st, dev_cost, f, g) in got.items():
        bound = 1e-6 if name == "f32" else 1e-3
        assert st in (0, 1) and (st == 0 or name != "f32"), (name, st)
        cost, _, er, ec = oracle.finalize(C64, f, g, p, q, eps)
        assert abs(cost - cost_or) <= bound * cost_or, (name, cost, cost_or)
        assert abs(dev_cost - cost_or) <= bound * cost_or, (name, dev_cost, cost_or)
        assert er <= bound and ec <= bound, (name, er, ec)
