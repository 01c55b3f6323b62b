"""GPU parity of eps-scaling (annealed warm starts of Algorithm 1).

The stages only choose where the last stage's iteration starts; the answer is the solution
of Eq. (5) at the requested eps, so it is compared with the oracle's converged solve at that
eps with the converged-solve tolerances of test_gpu_parity.py (transport cost within 1e-6
relative for a shared starting point; the stages start the last solve elsewhere, so there
the costs agree to the size of the tol-ball: 1e-5), exact FP64 marginals of the returned
potentials within tol + 5e-7.  With one stage
the kernel is the single-instance solver's arithmetic, bit for bit.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARG_SLACK = 0.0  # the device stops at FP32 residual <= tol (1 - 2^-5)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_01559_gb300 import binding
    c = binding.Context(0)
    yield c
    c.close()


def _padded(C32):
    I, J = C32.shape
    ld = (J + 3) // 4 * 4
    buf = torch.full((I, ld), float("inf"), dtype=torch.float32, device="cuda")
    buf[:, :J] = torch.from_numpy(np.ascontiguousarray(C32)).cuda()
    return buf[:, :J]


def _c1():
    from paper_1805_01559_gb300 import instances as ins
    inst = ins.config1()
    R = oracle.rates(inst.G.astype(np.float32).astype(np.float64), inst.P, inst.N0, inst.W_hz)
    C32 = oracle.cost(R, inst.mu).astype(np.float32)
    return C32, inst.lam.astype(np.float32), inst.q.astype(np.float32)


@pytest.mark.parametrize("eps_rel,factor,tol_stage", [(0.01, 0.3, 1e-3), (0.003, 0.5, 1e-2)])
def test_eps_scaling_reaches_the_solution_at_eps(ctx, eps_rel, factor, tol_stage):
    C32, p32, q32 = _c1()
    C64, p64, q64 = C32.astype(np.float64), p32.astype(np.float64), q32.astype(np.float64)
    med = float(np.median(C64))
    eps, eps0, tol = eps_rel * med, 0.1 * med, 1e-6
    f_o, g_o, it_o, _ = oracle.sinkhorn(C64, p64, q64, eps, tol, 20000)
    cost_o = oracle.finalize(C64, f_o, g_o, p64, q64, eps)[0]
    res, stages = ctx.solve_eps_scaling(_padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(),
                                        eps, eps0, factor=factor, tol_stage=tol_stage, tol=tol, max_iter=20000)
    assert res.status == 0
    n_expect = 1
    e = eps0
    while e > eps * (1 + 1e-12):
        n_expect += 1
        e *= factor
    assert len(stages) == n_expect
    assert sum(stages) == res.iters
    # both solves stop inside the tol-ball around the solution, from different starting points,
    # so they end at different points of it: their costs agree to the ball's size, not to the
    # FP32 rounding of one shared iterate sequence (1.6e-6 relative measured at 0.003 median).
    # Against the oracle driven far past tol, the device is as close as the oracle's own stop.
    f_t, g_t, _, _ = oracle.sinkhorn(C64, p64, q64, eps, 1e-12, 200000)
    cost_t = oracle.finalize(C64, f_t, g_t, p64, q64, eps)[0]
    assert res.transport_cost == pytest.approx(cost_o, rel=1e-5)
    assert abs(res.transport_cost - cost_t) <= 4 * abs(cost_o - cost_t) + 1e-6 * cost_t
    _, _, er, ec = oracle.finalize(C64, res.f.cpu().numpy(), res.g.cpu().numpy(), p64, q64, eps)
    assert er <= tol + MARG_SLACK and ec <= tol + MARG_SLACK
    # the last stage starts from the previous stage's potentials: it needs no more
    # iterations than a start from b = 1 (the oracle's count, within the loop test's slack)
    assert stages[-1] <= it_o + 1


def test_one_stage_is_the_plain_solver(ctx):
    C32, p32, q32 = _c1()
    med = float(np.median(C32.astype(np.float64)))
    eps = 0.05 * med
    C, p, q = _padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
    res, stages = ctx.solve_eps_scaling(C, p, q, eps, eps, factor=0.5, tol=1e-6)
    ref = ctx.solve_cost(C, p, q, eps, tol=1e-6)
    assert stages == [ref.iters]
    assert res.transport_cost == pytest.approx(ref.transport_cost, rel=1e-12)
    np.testing.assert_allclose(res.g.cpu().numpy(), ref.g.cpu().numpy(), rtol=1e-12, atol=1e-12 * eps)
    np.testing.assert_allclose(res.f.cpu().numpy(), ref.f.cpu().numpy(), rtol=1e-12, atol=1e-12 * eps)


def test_warm_start_and_plan_output(ctx):
    C32, p32, q32 = _c1()
    C64 = C32.astype(np.float64)
    med = float(np.median(C64))
    eps = 0.02 * med
    C, p, q = _padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
    first, _ = ctx.solve_eps_scaling(C, p, q, eps, 0.1 * med, factor=0.3, tol=1e-7)
    again, stages = ctx.solve_eps_scaling(C, p, q, eps, eps, factor=0.3, tol=1e-7, warm_g=first.g, want_pi=True)
    assert stages[0] <= 2  # started at the answer
    pi = again.pi.cpu().numpy().astype(np.float64)
    want = oracle.plan(C64, again.f.cpu().numpy(), again.g.cpu().numpy(), eps)
    np.testing.assert_allclose(pi, want, rtol=2e-5, atol=1e-30)


def test_eps_scaling_rejects_bad_arguments(ctx):
    from paper_1805_01559_gb300 import binding
    C32, p32, q32 = _c1()
    C, p, q = _padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
    with pytest.raises(binding.OTError):
        ctx.solve_eps_scaling(C, p, q, 1.0, 0.5)  # eps0 < eps
    with pytest.raises(binding.OTError):
        ctx.solve_eps_scaling(C, p, q, 1.0, 2.0, factor=1.0)
    with pytest.raises(binding.OTError):
        ctx.solve_eps_scaling(C, p, q, 1e-30, 1e30, factor=0.5)  # too many stages
    bad = p.clone()
    bad[0] = 0.0
    with pytest.raises(binding.OTError):
        ctx.solve_eps_scaling(C, bad, q, 1.0, 4.0, factor=0.5)
