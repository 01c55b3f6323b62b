"""GPU parity of the adaptive Sinkhorn association (Algorithm 2, Sec. V) against the oracle.

Every outer step solves Algorithm 1 with the FP32 log-domain solver, so the per-step plans
carry the converged-solve tolerances of test_gpu_parity.py (loads within 1e-5 relative of
the oracle's).  The choice j* = argmax rho_j is an integer decided from those loads: it is
compared step by step where the oracle's two largest loads differ by more than 1e-4
relative (far above the solve tolerance), and the test asserts that the instances used
here keep every step above that margin.  Given equal choices the FP64 targets follow the
same updates, so q matches the oracle's to 1e-12 relative (the equal split's total is summed
in another order).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAP = 1e-4


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


def _cell(I, J, seed, side=1000.0, hotspot=True, scale=1.0):
    """A hot-spot cell (Sec. V's setting): FP32 load costs from the Sec. II-A rates."""
    from paper_1805_01559_gb300 import instances as ins
    inst = ins.make_instance(f"adaptive_{I}x{J}", I, J, side, seed, hotspot=hotspot, traffic_sigma=1.0,
                             marginal="uniform", dtype=np.float32)
    R = oracle.rates(inst.G.astype(np.float64), inst.P, inst.N0, inst.W_hz)
    C32 = oracle.cost(R, inst.mu).astype(np.float32)
    lam32 = (inst.lam * scale).astype(np.float32)
    return C32, lam32


def _top2_gap(rho):
    s = np.sort(rho)[::-1]
    return (s[0] - s[1]) / s[0]


@pytest.mark.parametrize("I,J,seed,outer", [(2000, 25, 3, 8), (1500, 4, 5, 6), (4000, 64, 9, 5)])
def test_adaptive_matches_oracle(ctx, I, J, seed, outer):
    C32, lam32 = _cell(I, J, seed)
    C64, lam64 = C32.astype(np.float64), lam32.astype(np.float64)
    eps = 0.05 * float(np.median(C64))
    delta = 0.1 * lam64.sum() / J
    tol = 1e-6
    f_o, g_o, q_o, ml_o, js_o, rho_o = oracle.adaptive_trace(C64, lam64, eps, tol, 2000, outer, delta)
    gaps = [_top2_gap(r) for r in rho_o]
    assert min(gaps) > GAP, f"instance has a near tie in the oracle's loads: {gaps}"
    res = ctx.adaptive(_padded(C32), torch.from_numpy(lam32).cuda(), eps, delta, outer, tol=tol, max_iter=2000)
    assert res.status == 0, res.steps
    js = [s["jstar"] for s in res.steps]
    assert js == list(js_o)
    ml = np.array([s["max_load"] for s in res.steps])
    np.testing.assert_allclose(ml, ml_o, rtol=1e-5)
    np.testing.assert_allclose(res.q.cpu().numpy(), q_o, rtol=1e-12)
    # the last plan: its loads and transport cost against the oracle's last solve
    np.testing.assert_allclose(res.rrh_load.cpu().numpy(), rho_o[-1], rtol=1e-5)
    cost_o = oracle.finalize(C64, f_o, g_o, lam64, q_o, eps)[0]
    assert res.steps[-1]["transport_cost"] == pytest.approx(cost_o, rel=1e-6)
    # the returned potentials are a plan of the q it reports, to the solve tolerance
    _, _, er, ec = oracle.finalize(C64, res.f.cpu().numpy(), res.g.cpu().numpy(), lam64, res.q.cpu().numpy(), eps)
    assert er <= tol + 5e-7 and ec <= tol + 5e-7
    for s, so in zip(res.steps, rho_o):
        assert s["converged"] == 1 and s["iters"] >= 1


def test_one_step_equals_a_plain_solve_with_the_equal_split(ctx):
    C32, lam32 = _cell(3000, 32, 11)
    eps = 0.05 * float(np.median(C32))
    C = _padded(C32)
    lam = torch.from_numpy(lam32).cuda()
    res = ctx.adaptive(C, lam, eps, 0.01, 1, tol=1e-6, max_iter=2000)
    q0 = float(lam32.astype(np.float64).sum()) / 32
    q = torch.full((32,), q0, dtype=torch.float32, device="cuda")
    ref = ctx.solve_cost(C, lam, q, eps, tol=1e-6, max_iter=2000)
    assert res.steps[0]["iters"] == ref.iters
    assert res.steps[0]["transport_cost"] == pytest.approx(ref.transport_cost, rel=1e-12)
    np.testing.assert_allclose(res.g.cpu().numpy(), ref.g.cpu().numpy(), rtol=1e-12, atol=1e-12 * eps)
    np.testing.assert_allclose(res.rrh_load.cpu().numpy(), ref.rrh_load.cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(res.q.cpu().numpy(), np.full(32, q0), rtol=1e-13)


def test_half_moves_and_mass_conservation(ctx):
    # delta above every target: each step halves the chosen target (the oracle does the same)
    C32, lam32 = _cell(1200, 6, 13)
    C64, lam64 = C32.astype(np.float64), lam32.astype(np.float64)
    eps = 0.05 * float(np.median(C64))
    delta = 10.0 * lam64.sum()
    _, _, q_o, ml_o, js_o, rho_o = oracle.adaptive_trace(C64, lam64, eps, 1e-6, 2000, 4, delta)
    assert min(_top2_gap(r) for r in rho_o) > GAP
    res = ctx.adaptive(_padded(C32), torch.from_numpy(lam32).cuda(), eps, delta, 4, tol=1e-6)
    assert [s["jstar"] for s in res.steps] == list(js_o)
    q = res.q.cpu().numpy()
    np.testing.assert_allclose(q, q_o, rtol=1e-12)
    assert q.sum() == pytest.approx(lam64.sum(), rel=1e-12)
    assert (q > 0).all()


def test_adaptive_balances_a_hot_spot(ctx):
    # Sec. V: moving target traffic off the most loaded RRH lowers the largest load
    C32, lam32 = _cell(4000, 16, 17, side=800.0)
    eps = 0.05 * float(np.median(C32))
    delta = 0.05 * float(lam32.sum()) / 16
    res = ctx.adaptive(_padded(C32), torch.from_numpy(lam32).cuda(), eps, delta, 12, tol=1e-6)
    ml = [s["max_load"] for s in res.steps]
    assert min(ml[1:]) < ml[0]


def test_adaptive_cold_start_agrees(ctx):
    C32, lam32 = _cell(2000, 20, 19)
    eps = 0.05 * float(np.median(C32))
    delta = 0.1 * float(lam32.sum()) / 20
    C, lam = _padded(C32), torch.from_numpy(lam32).cuda()
    warm = ctx.adaptive(C, lam, eps, delta, 5, tol=1e-7)
    cold = ctx.adaptive(C, lam, eps, delta, 5, tol=1e-7, cold_start=True)
    assert [s["jstar"] for s in warm.steps] == [s["jstar"] for s in cold.steps]
    # warm starts need fewer iterations after the first step
    assert sum(s["iters"] for s in warm.steps[1:]) < sum(s["iters"] for s in cold.steps[1:])
    np.testing.assert_allclose(warm.rrh_load.cpu().numpy(), cold.rrh_load.cpu().numpy(), rtol=1e-5)


def test_adaptive_writes_the_last_plan(ctx):
    C32, lam32 = _cell(1000, 12, 23)
    C64, lam64 = C32.astype(np.float64), lam32.astype(np.float64)
    eps = 0.05 * float(np.median(C64))
    res = ctx.adaptive(_padded(C32), torch.from_numpy(lam32).cuda(), eps, 0.002, 3, tol=1e-6, want_pi=True)
    pi = res.pi.cpu().numpy().astype(np.float64)
    want = oracle.plan(C64, res.f.cpu().numpy(), res.g.cpu().numpy(), eps)
    np.testing.assert_allclose(pi, want, rtol=2e-5, atol=1e-30)
    np.testing.assert_allclose((C64 * pi).sum(axis=0), res.rrh_load.cpu().numpy(), rtol=1e-5)


def test_adaptive_rejects_bad_arguments(ctx):
    from paper_1805_01559_gb300 import binding
    C32, lam32 = _cell(100, 8, 29)
    C, lam = _padded(C32), torch.from_numpy(lam32).cuda()
    with pytest.raises(binding.OTError):
        ctx.adaptive(C, lam, 0.1, 0.01, 0)  # no outer step
    with pytest.raises(binding.OTError):
        ctx.adaptive(C, lam, -1.0, 0.01, 2)  # eps
    with pytest.raises(binding.OTError):
        ctx.adaptive(C, lam, 0.1, -0.5, 2)  # delta
    with pytest.raises(binding.OTError):
        ctx.adaptive(C[:, :1], lam, 0.1, 0.01, 2)  # one RRH
    big = torch.ones((16, 1028), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.OTError):
        ctx.adaptive(big, torch.ones(16, device="cuda"), 0.1, 0.01, 2)  # J above 1024
    # a bad traffic entry fails the first step; the rest report the same failure
    bad = lam.clone()
    bad[3] = -1.0
    with pytest.raises(binding.OTError):
        ctx.adaptive(C, bad, 0.1, 0.01, 3)
    # the context still works afterwards
    ok = ctx.adaptive(C, lam, 0.05 * float(np.median(C32)), 0.001, 2)
    assert ok.status == 0
