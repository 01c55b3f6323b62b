"""The Euclidean cost of Sec. IV (cost choice (i)) formed inside the sweeps.

The kernel evaluates C_ij = sqrt((x_i - x_j)^2 + (y_i - y_j)^2) in FP32 with every operation
correctly rounded and none fused; numpy's float32 arithmetic evaluates the same formula the
same way, so the test builds that matrix on the host and (i) the on-the-fly solve equals
ot_assoc_solve_cost on it bit for bit (same partitions, teams and reduction orders), and
(ii) both match the oracle run on that matrix with the converged-solve tolerances of
test_gpu_parity.py.  The FP32 formula itself is checked against the oracle's FP64 distances.
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


def _geom(I, J, seed, side=1000.0):
    from paper_1805_01559_gb300 import instances as ins
    rng = np.random.Generator(np.random.PCG64(seed))
    rrh = ins.rrh_jittered_grid(J, side, rng).astype(np.float32)
    dev = ins.devices_hotspot(I, side, rng).astype(np.float32)
    dev[0] = rrh[0]  # a device on an RRH: a zero cost
    lam = ins.traffic_lognormal(I, 1.0, rng).astype(np.float32)
    q = ins.capacity_marginal(J, float(lam.astype(np.float64).sum()), rng).astype(np.float32)
    return dev, rrh, lam, q


def _c32(dev, rrh):
    dx = dev[:, None, 0] - rrh[None, :, 0]
    dy = dev[:, None, 1] - rrh[None, :, 1]
    return np.sqrt(dx * dx + dy * dy)  # float32 throughout, no fused operations


def _padded(C32):
    I, J = C32.shape
    ld = (J + 3) // 4 * 4
    buf = torch.full((I, ld), float("inf"), dtype=torch.float32, device="cuda")
    buf[:, :J] = torch.from_numpy(np.ascontiguousarray(C32)).cuda()
    return buf[:, :J]


def test_fp32_formula_against_the_oracle():
    dev, rrh, _, _ = _geom(500, 30, 1)
    C32 = _c32(dev, rrh)
    assert C32.dtype == np.float32
    C64 = oracle.euclid_cost(dev, rrh)
    np.testing.assert_allclose(C32, C64, rtol=3e-7, atol=1e-4)


@pytest.mark.parametrize("I,J,seed", [(3000, 50, 2), (20000, 800, 3), (5000, 1500, 4), (7, 9, 5)])
def test_euclid_on_the_fly_equals_the_matrix_solve(ctx, I, J, seed):
    dev, rrh, lam, q = _geom(I, J, seed)
    C32 = _c32(dev, rrh)
    C64 = C32.astype(np.float64)
    eps = 0.05 * float(np.median(C64))
    d_dev, d_rrh = torch.from_numpy(dev).cuda(), torch.from_numpy(rrh).cuda()
    p_t, q_t = torch.from_numpy(lam).cuda(), torch.from_numpy(q).cuda()
    fly = ctx.solve_euclid(d_dev, d_rrh, p_t, q_t, eps, tol=1e-6)
    mat = ctx.solve_cost(_padded(C32), p_t, q_t, eps, tol=1e-6)
    assert fly.iters == mat.iters and fly.status == mat.status == 0
    assert fly.transport_cost == mat.transport_cost
    assert torch.equal(fly.f, mat.f) and torch.equal(fly.g, mat.g)
    assert torch.equal(fly.rrh_load, mat.rrh_load)
    lam64, q64 = lam.astype(np.float64), q.astype(np.float64)
    f_o, g_o, it_o, _ = oracle.sinkhorn(C64, lam64, q64, eps, 1e-6, 2000)
    cost_o = oracle.finalize(C64, f_o, g_o, lam64, q64, eps)[0]
    assert abs(fly.iters - it_o) <= 2
    assert fly.transport_cost == pytest.approx(cost_o, rel=1e-6)
    _, _, er, ec = oracle.finalize(C64, fly.f.cpu().numpy(), fly.g.cpu().numpy(), lam64, q64, eps)
    assert er <= 1e-6 + MARG_SLACK and ec <= 1e-6 + MARG_SLACK


def test_euclid_plan_and_warm_start(ctx):
    dev, rrh, lam, q = _geom(2000, 40, 6)
    C64 = _c32(dev, rrh).astype(np.float64)
    eps = 0.05 * float(np.median(C64))
    d_dev, d_rrh = torch.from_numpy(dev).cuda(), torch.from_numpy(rrh).cuda()
    p_t, q_t = torch.from_numpy(lam).cuda(), torch.from_numpy(q).cuda()
    a = ctx.solve_euclid(d_dev, d_rrh, p_t, q_t, eps, tol=1e-6, want_pi=True)
    want = oracle.plan(C64, a.f.cpu().numpy(), a.g.cpu().numpy(), eps)
    np.testing.assert_allclose(a.pi.cpu().numpy().astype(np.float64), want, rtol=2e-5, atol=1e-30)
    b = ctx.solve_euclid(d_dev, d_rrh, p_t, q_t, eps, tol=1e-6, warm_g=a.g)
    assert b.iters <= 2


def test_euclid_rejects_bad_arguments(ctx):
    from paper_1805_01559_gb300 import binding
    dev, rrh, lam, q = _geom(100, 8, 7)
    d_dev, d_rrh = torch.from_numpy(dev).cuda(), torch.from_numpy(rrh).cuda()
    p_t, q_t = torch.from_numpy(lam).cuda(), torch.from_numpy(q).cuda()
    with pytest.raises(binding.OTError):
        ctx.solve_euclid(d_dev, d_rrh, p_t, q_t, -1.0)
    bad = p_t.clone()
    bad[3] = 0.0
    with pytest.raises(binding.OTError):
        ctx.solve_euclid(d_dev, d_rrh, bad, q_t, 10.0)
