"""GPU parity of the FP64 solver (ot_assoc_solve_f64) against the FP64 oracle.

Both sides run Algorithm 1 in the log domain in double precision with the same stopping
rule, so the iteration counts match exactly on the 1000 x 50 configuration and the plans
agree to a few ulp per iteration: potentials and plans are compared at 1e-10 relative,
costs at 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_1805_01559_gb300 import instances as ins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_01559_gb300 import binding
    c = binding.Context(0)
    yield c
    c.close()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


def test_config1_fp64_matches_oracle(ctx):
    inst = ins.config1()
    R = oracle.rates(inst.G, inst.P, inst.N0, inst.W_hz)
    C = oracle.cost(R, inst.mu)
    eps = inst.eps_rel[0] * oracle.median(C)
    p, q = inst.lam, inst.q
    res = ctx.solve_f64(_t(C), _t(p), _t(q), eps, tol=inst.tol, max_iter=inst.max_iter, want_pi=True)
    _, _, it_or, _ = oracle.sinkhorn(C, p, q, eps, inst.tol, inst.max_iter)
    assert res.status == 0
    # the same test on the same residual; the two evaluate it in different (exact) forms, so
    # a residual within rounding of tol may stop one iteration apart
    assert abs(res.iters - it_or) <= 1, (res.iters, it_or)
    f_or, g_or, _, _ = oracle.sinkhorn(C, p, q, eps, 0.0, res.iters)
    pi_or = oracle.plan(C, f_or, g_or, eps)
    np.testing.assert_allclose(oracle.plan(C, _np(res.f), _np(res.g), eps), pi_or, rtol=1e-10, atol=1e-300)
    cost_or, rho_or, er_or, ec_or = oracle.finalize(C, f_or, g_or, p, q, eps)
    assert res.transport_cost == pytest.approx(cost_or, rel=1e-12)
    assert res.marg_err_row == pytest.approx(er_or, rel=1e-6, abs=1e-15)
    assert res.marg_err_col == pytest.approx(ec_or, rel=1e-6, abs=1e-15)
    np.testing.assert_allclose(_np(res.rrh_load), rho_or, rtol=1e-12)
    # float plan output: FP32 rounding of the FP64 plan (entries below FP32's range are 0)
    np.testing.assert_allclose(_np(res.pi), pi_or.astype(np.float32), rtol=1e-6, atol=1e-37)


@pytest.mark.parametrize("shape,iters", [((1, 1), 3), ((37, 129), 5), ((300, 7), 20), ((2000, 300), 8)])
def test_fp64_fixed_iterations(ctx, shape, iters):
    I, J = shape
    rng = np.random.Generator(np.random.PCG64(I * 31 + J))
    C = rng.uniform(0.0, 1.0, (I, J))
    p = rng.lognormal(0.0, 1.0, I)
    q = rng.uniform(0.5, 1.5, J)
    q *= p.sum() / q.sum()
    res = ctx.solve_f64(_t(C), _t(p), _t(q), 0.05, tol=0.0, max_iter=iters)
    f_or, g_or, it_or, _ = oracle.sinkhorn(C, p, q, 0.05, 0.0, iters)
    assert res.iters == it_or
    np.testing.assert_allclose(oracle.plan(C, _np(res.f), _np(res.g), 0.05), oracle.plan(C, f_or, g_or, 0.05),
                               rtol=1e-10, atol=1e-300)


def test_fp64_and_fp32_agree_on_config1(ctx):
    # Iteration counts of the FP32 and FP64 solvers stay within a few of each other.
    inst = ins.config1()
    R = oracle.rates(inst.G.astype(np.float32).astype(np.float64), inst.P, inst.N0, inst.W_hz)
    C = oracle.cost(R.astype(np.float32).astype(np.float64), inst.mu)
    eps = inst.eps_rel[0] * oracle.median(C)
    r64 = ctx.solve_f64(_t(C), _t(inst.lam), _t(inst.q), eps, tol=inst.tol, max_iter=inst.max_iter)
    C32 = torch.from_numpy(C.astype(np.float32)).cuda()
    r32 = ctx.solve_cost(C32, torch.from_numpy(inst.lam.astype(np.float32)).cuda(),
                         torch.from_numpy(inst.q.astype(np.float32)).cuda(), eps, tol=inst.tol,
                         max_iter=inst.max_iter)
    assert abs(r64.iters - r32.iters) <= 2
    assert r32.transport_cost == pytest.approx(r64.transport_cost, rel=1e-6)


def test_fp64_rejects_unbalanced(ctx):
    from paper_1805_01559_gb300 import binding
    C = np.ones((10, 4))
    with pytest.raises(binding.OTError) as e:
        ctx.solve_f64(_t(C), _t(np.full(10, 0.1)), _t(np.full(4, 0.5)), 0.1)
    assert e.value.status == binding.OT_EINVAL
