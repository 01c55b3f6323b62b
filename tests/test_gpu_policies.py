"""GPU parity of the policy-evaluation kernels (Sec. II-B completion time, Sec. IV Euclidean
cost) against the oracle, and the four-policy comparison of Sec. IV on small cells.

Tolerances: the Euclidean cost is formed in FP64 with explicit roundings on both sides and
rounded once, so it is bit-exact.  Completion times of a hard association sum the same FP64
products (1e-12 relative).  For an entropic plan the kernel evaluates each entry with an FP32
exponential of an FP64 exponent (relative error about 1e-7 per entry), so loads and T agree
to 1e-5 relative.
"""
import math

import numpy as np
import pytest

import oracle

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


def _padded(A32):
    I, J = A32.shape
    ld = (J + 3) // 4 * 4
    buf = torch.full((I, ld), float("inf"), dtype=torch.float32, device="cuda")
    buf[:, :J] = torch.from_numpy(np.ascontiguousarray(A32)).cuda()
    return buf[:, :J]


def _cell(N, seed, J=25):
    from paper_1805_01559_gb300 import instances as ins
    cell = ins.policy_cell(N, seed, J=J)
    R = oracle.rates(cell.G.astype(np.float64), cell.P, cell.N0, cell.W_hz)
    C32 = oracle.cost(R, cell.mu).astype(np.float32)
    return cell, R, C32


@pytest.mark.parametrize("I,J", [(1, 1), (257, 25), (3000, 130)])
def test_euclid_cost_bit_exact(ctx, I, J):
    rng = np.random.Generator(np.random.PCG64(I * 7 + J))
    dev = rng.uniform(-500, 1500, (I, 2)).astype(np.float32)
    rrh = rng.uniform(0, 1000, (J, 2)).astype(np.float32)
    rrh[0] = dev[0]  # a zero distance
    C = ctx.euclid_cost(torch.from_numpy(dev).cuda(), torch.from_numpy(rrh).cuda())
    want = oracle.euclid_cost(dev, rrh).astype(np.float32)
    np.testing.assert_array_equal(C.cpu().numpy(), want)


def test_mean_row_min(ctx):
    _, _, C32 = _cell(777, 3)
    got = ctx.mean_row_min(_padded(C32))
    assert got == pytest.approx(C32.astype(np.float64).min(axis=1).mean(), rel=1e-13)


def test_completion_time_of_maxsinr(ctx):
    cell, R, C32 = _cell(1000, 5)
    C64 = C32.astype(np.float64)
    lam32 = (cell.lam * 30.0).astype(np.float32)
    lam64 = lam32.astype(np.float64)
    Rd = _padded(R.astype(np.float32))
    assoc, _, _ = ctx.maxsinr(Rd, torch.from_numpy(lam32).cuda(), cell.mu)
    a = assoc.cpu().numpy()
    T, rho = ctx.completion_time(_padded(C32), torch.from_numpy(lam32).cuda(), assoc=assoc)
    x = np.zeros_like(C64)
    x[np.arange(len(a)), a] = lam64
    T_o, rho_o = oracle.completion_time(C64, x, lam64)
    assert rho_o.max() < 1.0
    np.testing.assert_allclose(rho.cpu().numpy(), rho_o, rtol=1e-12)
    assert T == pytest.approx(T_o, rel=1e-12)


@pytest.mark.parametrize("plan_cost", ["load", "euclid"])
def test_completion_time_of_an_entropic_plan(ctx, plan_cost):
    cell, R, C32 = _cell(1500, 7, J=40)
    C64 = C32.astype(np.float64)
    lam32 = (cell.lam * 2.0).astype(np.float32)
    lam64 = lam32.astype(np.float64)
    if plan_cost == "load":
        Cp32 = C32
    else:
        Cp32 = oracle.euclid_cost(cell.dev_xy, cell.rrh_xy).astype(np.float32)
    Cp64 = Cp32.astype(np.float64)
    eps = 0.03 * Cp64.min(axis=1).mean()
    q = np.full(40, lam64.sum() / 40)
    f, g, _, _ = oracle.sinkhorn(Cp64, lam64, q, eps, 1e-9, 5000)
    x = oracle.plan(Cp64, f, g, eps)
    T_o, rho_o = oracle.completion_time(C64, x, lam64)
    T, rho = ctx.completion_time(_padded(C32), torch.from_numpy(lam32).cuda(),
                                 f=torch.from_numpy(f).cuda(), g=torch.from_numpy(g).cuda(), eps=eps,
                                 C_plan=None if plan_cost == "load" else _padded(Cp32))
    np.testing.assert_allclose(rho.cpu().numpy(), rho_o, rtol=1e-5)
    if math.isinf(T_o):
        assert math.isinf(T)
    else:
        assert T == pytest.approx(T_o, rel=1e-5)


def test_completion_time_overload_and_errors(ctx):
    from paper_1805_01559_gb300 import binding
    C = np.array([[1.0, 2.0], [0.5, 0.5]], np.float32)
    lam = np.array([0.2, 0.4], np.float32)
    # device 1 on RRH 1, device 0 on RRH 0: rho = (0.2, 0.2)
    T, rho = ctx.completion_time(_padded(C), torch.from_numpy(lam).cuda(),
                                 assoc=torch.tensor([0, 1], dtype=torch.int32, device="cuda"))
    l64 = lam.astype(np.float64)
    x = np.array([[l64[0], 0.0], [0.0, l64[1]]])
    T_o, _ = oracle.completion_time(C.astype(np.float64), x, l64)
    assert T == pytest.approx(T_o, rel=1e-14)
    # the same association with 10x the load: RRH 1 at rho = 2 carries traffic -> inf
    T, rho = ctx.completion_time(_padded(C * 10), torch.from_numpy(lam).cuda(),
                                 assoc=torch.tensor([0, 1], dtype=torch.int32, device="cuda"))
    assert math.isinf(T) and rho.cpu().numpy()[1] >= 1.0
    with pytest.raises(binding.OTError):
        ctx.completion_time(_padded(C), torch.tensor([0.2, -0.4], device="cuda"),
                            assoc=torch.tensor([0, 1], dtype=torch.int32, device="cuda"))
    with pytest.raises(binding.OTError):  # neither an association nor potentials
        ctx.completion_time(_padded(C), torch.from_numpy(lam).cuda())


@pytest.mark.parametrize("N", [200, 2000])
def test_four_policies_against_the_oracle(ctx, N):
    from paper_1805_01559_gb300 import policies
    cell, R, _ = _cell(N, 1)
    prep = policies.prepare(ctx, cell, load_target=0.3, eps_best=0.01, tol=1e-6, max_iter=2000)
    res = policies.finish(ctx, prep, ctx.solve_batched(prep.instances))
    # the oracle evaluates the same inputs: the device's FP32 load cost and association
    C64 = prep.C.cpu().numpy().astype(np.float64)
    Ce64 = prep.Ce.cpu().numpy().astype(np.float64)
    lam64 = prep.lam.cpu().numpy().astype(np.float64)
    a = prep.assoc.cpu().numpy()
    # the association is maxSINR: the oracle's argmax wherever its rates are not tied
    R64 = np.sort(R, axis=1)
    clear = (R64[:, -1] - R64[:, -2]) > 1e-5 * R64[:, -1]
    np.testing.assert_array_equal(a[clear], np.argmax(R, axis=1)[clear])
    x = np.zeros_like(C64)
    x[np.arange(N), a] = lam64
    T_a, rho_a = oracle.completion_time(C64, x, lam64)
    assert rho_a.max() == pytest.approx(0.3, rel=1e-6)
    assert res.T["a"] == pytest.approx(T_a, rel=1e-12)
    # each OT policy: the oracle's completion time of the device's potentials
    for k, inst in zip("bcd", prep.instances):
        Cp = Ce64 if k == "b" else C64
        xp = oracle.plan(Cp, inst.f.cpu().numpy(), inst.g.cpu().numpy(), inst.eps)
        T_o, _ = oracle.completion_time(C64, xp, lam64)
        if math.isinf(T_o):
            assert math.isinf(res.T[k])
        else:
            assert res.T[k] == pytest.approx(T_o, rel=1e-5)
    # Lemma 1: OT with load costs and q = Lambda reaches maxSINR's total load (the entropic
    # plan to within its regularisation) and its completion time
    assert res.total_load["d"] == pytest.approx(res.total_load["a"], rel=1e-3)
    assert res.ratio["d"] == pytest.approx(1.0, rel=2e-2)
    # (c) with an equal split is no better than maxSINR on a random drop
    assert res.ratio["c"] >= 0.999
