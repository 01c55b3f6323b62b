"""Several solves on one cost matrix in one launch (an eps sweep sharing each read of C).

Each solve follows the single-solve algorithm and stopping rule; the launch picks a wider
row team than a single solve of the same J (three solves' accumulators must fit the
registers), so results agree with ot_assoc_solve_cost and with the oracle at the
converged-solve tolerances of test_gpu_parity.py (transport cost within 1e-6 relative of
the oracle's, exact FP64 marginals of the returned potentials within tol + 5e-7), and a
solve's result is bit-identical whichever solves share its launch.
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


def _inst(I, J, seed):
    from paper_1805_01559_gb300 import instances as ins
    inst = ins.make_instance("multi", I, J, 2000.0, seed, hotspot=True, traffic_sigma=1.5, marginal="capacity",
                             dtype=np.float32)
    R = oracle.rates(inst.G.astype(np.float64), inst.P, inst.N0, inst.W_hz)
    C32 = oracle.cost(R, inst.mu).astype(np.float32)
    return C32, inst.lam.astype(np.float32), inst.q.astype(np.float32)


def _padded(C32):
    I, J = C32.shape
    ld = (J + 3) // 4 * 4
    buf = torch.full((I, ld), float("inf"), dtype=torch.float32, device="cuda")
    buf[:, :J] = torch.from_numpy(np.ascontiguousarray(C32)).cuda()
    return buf[:, :J]


@pytest.mark.parametrize("I,J,seed", [(3000, 64, 1), (6000, 200, 2), (4000, 800, 3), (2500, 1037, 4)])
def test_multi_matches_oracle(ctx, I, J, seed):
    C32, p32, q32 = _inst(I, J, seed)
    C64, p64, q64 = C32.astype(np.float64), p32.astype(np.float64), q32.astype(np.float64)
    med = float(np.median(C64))
    eps = [0.1 * med, 0.03 * med, 0.01 * med]
    tol = 1e-6
    res = ctx.solve_cost_multi(_padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps,
                               tol=tol)
    assert len(res) == 3
    for e, r in zip(eps, res):
        f_o, g_o, it_o, _ = oracle.sinkhorn(C64, p64, q64, e, tol, 2000)
        cost_o = oracle.finalize(C64, f_o, g_o, p64, q64, e)[0]
        assert r.status == 0
        assert abs(r.iters - it_o) <= 2, (r.iters, it_o)
        assert r.transport_cost == pytest.approx(cost_o, rel=1e-6)
        _, rho, er, ec = oracle.finalize(C64, r.f.cpu().numpy(), r.g.cpu().numpy(), p64, q64, e)
        assert er <= tol + MARG_SLACK and ec <= tol + MARG_SLACK
        np.testing.assert_allclose(r.rrh_load.cpu().numpy(), rho, rtol=1e-5)


@pytest.mark.parametrize("J", [400, 800])
def test_multi_result_does_not_depend_on_companions(ctx, J):
    # the kernel is chosen by J and by how many solves share it (above 512 columns, one or two
    # solves keep one-warp teams, three take wider ones): within one choice a solve's result
    # is the same bit for bit whichever solves share the launch
    C32, p32, q32 = _inst(5000, J, 5)
    med = float(np.median(C32))
    C, p, q = _padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
    trio = ctx.solve_cost_multi(C, p, q, [0.1 * med, 0.03 * med, 0.01 * med], tol=1e-6)
    alone = ctx.solve_cost_multi(C, p, q, [0.03 * med], tol=1e-6)[0]
    pair = ctx.solve_cost_multi(C, p, q, [0.01 * med, 0.03 * med], tol=1e-6)
    assert alone.iters == pair[1].iters and alone.transport_cost == pair[1].transport_cost
    assert torch.equal(alone.f, pair[1].f) and torch.equal(alone.g, pair[1].g)
    if J <= 512:
        assert torch.equal(alone.g, trio[1].g) and torch.equal(pair[0].g, trio[2].g)
    else:
        assert abs(alone.iters - trio[1].iters) <= 1
        assert alone.transport_cost == pytest.approx(trio[1].transport_cost, rel=1e-6)


def test_multi_pair_on_wide_rows_matches_oracle(ctx):
    # two solves on 800 columns: one-warp teams, cell values formed twice per row
    C32, p32, q32 = _inst(4000, 800, 9)
    C64, p64, q64 = C32.astype(np.float64), p32.astype(np.float64), q32.astype(np.float64)
    med = float(np.median(C64))
    eps = [0.03 * med, 0.01 * med]
    res = ctx.solve_cost_multi(_padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps,
                               tol=1e-6)
    for e, r in zip(eps, res):
        f_o, g_o, it_o, _ = oracle.sinkhorn(C64, p64, q64, e, 1e-6, 2000)
        cost_o = oracle.finalize(C64, f_o, g_o, p64, q64, e)[0]
        assert abs(r.iters - it_o) <= 2
        assert r.transport_cost == pytest.approx(cost_o, rel=1e-6)
        _, _, er, ec = oracle.finalize(C64, r.f.cpu().numpy(), r.g.cpu().numpy(), p64, q64, e)
        assert er <= 1e-6 + MARG_SLACK and ec <= 1e-6 + MARG_SLACK


def test_multi_agrees_with_single_solves(ctx):
    C32, p32, q32 = _inst(8000, 300, 6)
    med = float(np.median(C32))
    C, p, q = _padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
    eps = [0.1 * med, 0.02 * med]
    multi = ctx.solve_cost_multi(C, p, q, eps, tol=1e-7, want_pi=True)
    for e, m in zip(eps, multi):
        s = ctx.solve_cost(C, p, q, e, tol=1e-7, want_pi=True)
        assert abs(m.iters - s.iters) <= 1
        assert m.transport_cost == pytest.approx(s.transport_cost, rel=1e-6)
        np.testing.assert_allclose(m.pi.cpu().numpy(), s.pi.cpu().numpy(), rtol=1e-4, atol=1e-12)


def test_multi_stops_each_solve_at_its_own_iteration(ctx):
    C32, p32, q32 = _inst(3000, 128, 7)
    med = float(np.median(C32))
    C, p, q = _padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
    res = ctx.solve_cost_multi(C, p, q, [0.05 * med, 0.05 * med, 0.05 * med], tol=[1e-3, 1e-5, 0.0], max_iter=40)
    assert res[0].iters < res[1].iters < res[2].iters == 40
    assert res[2].status == 1  # not converged: max_iter
    ref = ctx.solve_cost_multi(C, p, q, [0.05 * med], tol=1e-3)[0]
    assert ref.iters == res[0].iters and torch.equal(ref.g, res[0].g)


def test_multi_rejects_bad_arguments(ctx):
    from paper_1805_01559_gb300 import binding
    C32, p32, q32 = _inst(500, 40, 8)
    C, p, q = _padded(C32), torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
    with pytest.raises(binding.OTError):
        ctx.solve_cost_multi(C, p, q, [1.0, 1.0, 1.0, 1.0])  # at most three
    with pytest.raises(binding.OTError):
        ctx.solve_cost_multi(C, p, q, [1.0, -1.0])
    bad = p.clone()
    bad[0] = float("nan")
    with pytest.raises(binding.OTError):
        ctx.solve_cost_multi(C, bad, q, [1.0, 2.0])
    ok = ctx.solve_cost_multi(C, p, q, [float(np.median(C32)) * 0.1])
    assert ok[0].status == 0
