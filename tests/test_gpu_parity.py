"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same inputs.

Tolerances (FP32 per-cell arithmetic against an FP64 reference):
  * rates: relative 1e-6 -- the SINR keeps ~2^-23 relative accuracy (compensated row total,
    exact own term), log1pf and the product with W/ln2 add a few ulp;
  * cost: relative 2^-22 -- one correctly rounded FP32 division plus the rounding of 1/mu;
  * median, argmax, association: bit-exact (both sides decide on the same FP32 values);
  * Sinkhorn iterates at a fixed iteration count: every plan entry within
    RTOL_ITER = 2e-5 relative (plus 1e-12 of the total mass absolute).  The exponent of a
    cell is formed from values of magnitude |k C| + |F'| + |G| (a few tens at most on the
    support of these instances) rounded at 2^-24, plus ex2.approx (2 ulp) and FP32 row and
    column sums of up to 8192 terms; these give < 2e-6 per iteration and the Sinkhorn map
    does not amplify them;
  * converged solves (tol = 1e-6 on the unit-mass row residual): transport cost relative
    error <= 1e-6 against the oracle's converged cost, and the exact (FP64) marginal L1 of
    the GPU potentials <= tol (MARG_SLACK = 0).  The sweeps hold the column potentials as
    FP32 pairs, so the plan the device measures is the plan of the FP64 potentials it
    returns; its FP32 residual then sits within about 1e-8 of the exact one, and the device
    stops at FP32 residual <= tol (1 - 2^-5).
"""
import numpy as np
import pytest

import oracle
from paper_1805_01559_gb300 import instances as ins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_ITER = 2e-5
MARG_SLACK = 0.0  # the device stops at FP32 residual <= tol (1 - 2^-5)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_01559_gb300 import binding
    c = binding.Context(0)
    yield c
    c.close()


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _np(t):
    return t.detach().cpu().numpy()


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


def _marg(rng, I, J):
    p = rng.lognormal(0.0, 1.0, I)
    q = rng.uniform(0.5, 1.5, J)
    p /= p.sum()
    q = q / q.sum()
    return p.astype(np.float32), q.astype(np.float32)


# ------------------------------------------------------------------------------ rates / cost
@pytest.mark.parametrize("shape", [(1000, 50), (101, 37), (64, 1), (257, 1030)])
def test_rates_match_oracle(ctx, shape):
    I, J = shape
    inst = ins.make_instance("t", I, J, 1000.0, 11, hotspot=True, traffic_sigma=1.0, marginal="uniform")
    G32 = inst.G.astype(np.float32)
    R = _np(ctx.build_rates(_t(G32), _t(inst.P), inst.N0, inst.W_hz))
    R_or = oracle.rates(G32.astype(np.float64), inst.P.astype(np.float32), inst.N0, inst.W_hz)
    np.testing.assert_allclose(R, R_or, rtol=1e-6)


def test_cost_matches_oracle(ctx):
    inst = ins.config1()
    R_or = oracle.rates(inst.G.astype(np.float32), inst.P, inst.N0, inst.W_hz)
    R32 = R_or.astype(np.float32)
    C, eps = ctx.build_cost(_t(R32), inst.mu, eps_rel=0.05)
    C_or = oracle.cost(R32.astype(np.float64), inst.mu)
    np.testing.assert_allclose(_np(C), C_or, rtol=2.0 ** -22)
    # eps = 0.05 * median of the FP32 cost the GPU built (oracle median of the same floats)
    assert eps == 0.05 * oracle.median(_np(C).astype(np.float64))


def test_cost_rejects_bad_rates(ctx):
    from paper_1805_01559_gb300 import binding
    R = np.ones((8, 5), np.float32)
    R[3, 2] = -1.0
    with pytest.raises(binding.OTError) as e:
        ctx.build_cost(_t(R), 1.0, eps_rel=0.05)
    assert e.value.status == binding.OT_EINVAL


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 1001, 65536, 3_000_001])
def test_median_bit_exact(ctx, n):
    rng = _rng(n)
    x = rng.lognormal(0.0, 4.0, n).astype(np.float32)
    if n > 10:
        x[: n // 10] = x[n // 2]          # duplicates
        x[n // 10: n // 5] *= -1.0        # negatives
        x[-1] = np.inf
    assert ctx.median_f32(_t(x)) == oracle.median(x.astype(np.float64))


@pytest.mark.parametrize("kind", ["sample_misses", "heavy_ties", "even_large"])
def test_median_bracket_fallback(ctx, kind):
    """Above 2^20 entries the median brackets the middle ranks with a strided sample.  A
    sample that misses the middle (every 20th entry tiny) or a bracket holding far too many
    ties must fall back to the full select and stay exact."""
    n = 65536 * 20
    rng = _rng(n + len(kind))
    x = rng.lognormal(0.0, 2.0, n).astype(np.float32)
    if kind == "sample_misses":
        x[::20] = 0.0
    elif kind == "heavy_ties":
        x[: (3 * n) // 4] = np.float32(1.5)
    else:
        x = x[: n - 2]
    assert ctx.median_f32(_t(x)) == oracle.median(x.astype(np.float64))


def test_cost_median_strided_large(ctx):
    """Cost median over a padded (ld > J) matrix large enough for the sampled bracket."""
    rng = _rng(7)
    I, J = 2000, 801
    R32 = rng.lognormal(np.log(2e7), 1.5, (I, J)).astype(np.float32)
    C, eps = ctx.build_cost(_t(R32), 1e-6, eps_rel=1.0)
    assert eps == oracle.median(_np(C).astype(np.float64))


def test_maxsinr_matches_oracle(ctx):
    inst = ins.config1()
    R32 = oracle.rates(inst.G.astype(np.float32), inst.P, inst.N0, inst.W_hz).astype(np.float32)
    R32[5, [3, 17]] = R32[5].max() * 2   # a tie: lowest index
    lam32 = inst.lam.astype(np.float32)
    assoc, Lam, tot = ctx.maxsinr(_t(R32), _t(lam32), inst.mu)
    R64 = R32.astype(np.float64)
    a_or, L_or, t_or = oracle.maxsinr(R64, oracle.cost(R64, inst.mu), lam32)
    np.testing.assert_array_equal(_np(assoc), a_or)
    assert _np(assoc)[5] == 3
    np.testing.assert_allclose(_np(Lam), L_or, rtol=1e-12, atol=1e-300)
    assert tot == pytest.approx(t_or, rel=1e-12)


# --------------------------------------------------------------------------- Sinkhorn parity
def _plan_check(pi_gpu, C, f_or, g_or, eps, mass):
    pi_or = oracle.plan(C, f_or, g_or, eps)
    err = np.abs(pi_gpu.astype(np.float64) - pi_or)
    tol = RTOL_ITER * pi_or + 1e-12 * mass
    bad = err > tol
    assert not bad.any(), (int(bad.sum()), float((err / np.maximum(pi_or, 1e-300)).max()))


SHAPES = [(1, 1), (2, 3), (37, 129), (1000, 50), (2049, 1023), (513, 1025), (300, 2049), (100, 4099),
          (64, 8192)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("iters", [1, 3, 12])
def test_fixed_iterations_match_oracle(ctx, shape, iters):
    # The GPU iterate after k iterations of Algorithm 1 equals the oracle's, entry by entry.
    I, J = shape
    rng = _rng(I * 7919 + J)
    C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    p, q = _marg(rng, I, J)
    eps = 0.1
    res = ctx.solve_cost(_t(C), _t(p), _t(q), eps, tol=0.0, max_iter=iters, want_pi=True)
    f_or, g_or, it_or, _ = oracle.sinkhorn(C.astype(np.float64), p, q, eps, 0.0, iters)
    # tol = 0 runs to max_iter unless the residual is exactly zero (trivial shapes)
    assert res.iters == iters or (res.iters < iters and (I == 1 or J == 1)), (res.iters, iters)
    _plan_check(_np(res.pi), C.astype(np.float64), f_or, g_or, eps, 1.0)
    # the returned potentials reproduce the same plan (gauge-free comparison)
    pi_fg = oracle.plan(C.astype(np.float64), _np(res.f), _np(res.g), eps)
    np.testing.assert_allclose(pi_fg, oracle.plan(C.astype(np.float64), f_or, g_or, eps),
                               rtol=RTOL_ITER, atol=1e-12)


@pytest.mark.parametrize("iters", [1, 3])
def test_first_iteration_with_an_underflowing_column(ctx, iters):
    # Column 0 costs 3 more than any row's cheapest link at eps = 0.02: in the first half-step
    # its entries are about 2^-216 of each row's largest, below the range of the first
    # sweep's fixed 2^64 column scale, so the solver takes the first iteration again in the
    # exact (online max, sum) form; the iterates still equal the oracle's.
    I, J = 3000, 50
    rng = _rng(77)
    C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    C[:, 0] += 3.0
    p, q = _marg(rng, I, J)
    eps = 0.02
    res = ctx.solve_cost(_t(C), _t(p), _t(q), eps, tol=0.0, max_iter=iters, want_pi=True)
    f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, eps, 0.0, iters)
    assert res.iters == iters
    _plan_check(_np(res.pi), C.astype(np.float64), f_or, g_or, eps, 1.0)


@pytest.mark.parametrize("eps", [0.01, 0.02, 0.05, 0.1, 0.3, 1.0, 7.0])
def test_forbidden_links_and_eps_values(ctx, eps):
    # +inf costs (no link) carry no mass for every eps; J = 45 leaves a masked tail chunk.
    rng = _rng(31)
    I, J = 600, 45
    C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    C[rng.uniform(size=(I, J)) < 0.2] = np.inf
    C[:, 0] = rng.uniform(0.0, 1.0, I).astype(np.float32)      # every row keeps a link
    C[np.arange(J), np.arange(J)] = 0.5                          # every column keeps a link
    p, q = _marg(rng, I, J)
    res = ctx.solve_cost(_t(C), _t(p), _t(q), eps, tol=0.0, max_iter=6, want_pi=True)
    pi = _np(res.pi)
    assert np.isfinite(pi).all() and (pi[np.isinf(C)] == 0).all()
    f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, eps, 0.0, 6)
    _plan_check(pi, C.astype(np.float64), f_or, g_or, eps, 1.0)


def test_padded_leading_dimension(ctx):
    rng = _rng(3)
    I, J, ld = 300, 37, 48
    big = rng.uniform(0, 1, (I, ld)).astype(np.float32)
    p, q = _marg(rng, I, J)
    Ct = _t(big)[:, :J]
    assert Ct.stride(0) == ld
    res = ctx.solve_cost(Ct, _t(p), _t(q), 0.1, tol=0.0, max_iter=5, want_pi=True)
    f_or, g_or, _, _ = oracle.sinkhorn(big[:, :J].astype(np.float64), p, q, 0.1, 0.0, 5)
    _plan_check(_np(res.pi), big[:, :J].astype(np.float64), f_or, g_or, 0.1, 1.0)


def test_single_rrh_gives_pi_equal_p(ctx):
    rng = _rng(4)
    I = 333
    C = rng.uniform(0, 10, (I, 1)).astype(np.float32)
    p = rng.uniform(0.1, 1, I).astype(np.float32)
    q = np.array([p.astype(np.float64).sum()], np.float32)
    res = ctx.solve_cost(_t(C), _t(p), _t(q), 0.01, tol=1e-6, max_iter=50, want_pi=True)
    assert res.iters == 1
    np.testing.assert_allclose(_np(res.pi)[:, 0], p, rtol=2e-6)


def test_separable_cost_gives_product_plan(ctx):
    rng = _rng(5)
    I, J = 700, 33
    C = (rng.uniform(0, 3, I)[:, None] + rng.uniform(0, 3, J)[None, :]).astype(np.float32)
    p, q = _marg(rng, I, J)
    res = ctx.solve_cost(_t(C), _t(p), _t(q), 0.05, tol=0.0, max_iter=1, want_pi=True)
    want = np.outer(p.astype(np.float64), q.astype(np.float64) / q.astype(np.float64).sum())
    np.testing.assert_allclose(_np(res.pi), want, rtol=RTOL_ITER, atol=1e-14)


def _converged_check(res, C64, p, q, eps, tol, it_or, cost_or):
    assert res.status == 0
    assert abs(res.iters - it_or) <= 2, (res.iters, it_or)
    cost, rho, er, ec = oracle.finalize(C64, _np(res.f), _np(res.g), p, q, eps)
    assert er <= tol + MARG_SLACK and ec <= tol + MARG_SLACK, (er, ec)
    assert abs(res.transport_cost - cost_or) <= 1e-6 * cost_or, (res.transport_cost, cost_or)
    assert abs(cost - cost_or) <= 1e-6 * cost_or
    # the device's own FP64 summary agrees with the exact evaluation
    assert res.marg_err_row == pytest.approx(er, abs=3e-7)
    np.testing.assert_allclose(_np(res.rrh_load), rho, rtol=1e-5, atol=1e-9 * rho.max())


def test_config1_fp32_matches_oracle(ctx):
    inst = ins.config1()
    R32 = oracle.rates(inst.G.astype(np.float32), inst.P, inst.N0, inst.W_hz).astype(np.float32)
    C64 = oracle.cost(R32.astype(np.float64), inst.mu)
    eps = inst.eps_rel[0] * oracle.median(C64)
    p, q = inst.lam.astype(np.float32), inst.q.astype(np.float32)
    res = ctx.solve(_t(R32), _t(p), _t(q), inst.mu, eps, tol=inst.tol, max_iter=inst.max_iter)
    f_or, g_or, it_or, err_or = oracle.sinkhorn(C64, p, q, eps, inst.tol, inst.max_iter)
    cost_or = oracle.finalize(C64, f_or, g_or, p, q, eps)[0]
    _converged_check(res, C64, p, q, eps, inst.tol, it_or, cost_or)


@pytest.mark.parametrize("shape,eps", [((4000, 300), 0.02), ((2500, 1111), 0.05), ((1500, 5000), 0.1)])
def test_converged_random_costs(ctx, shape, eps):
    I, J = shape
    rng = _rng(I + J)
    C = rng.uniform(0, 1, (I, J)).astype(np.float32)
    p, q = _marg(rng, I, J)
    res = ctx.solve_cost(_t(C), _t(p), _t(q), eps, tol=1e-6, max_iter=5000)
    C64 = C.astype(np.float64)
    f_or, g_or, it_or, _ = oracle.sinkhorn(C64, p, q, eps, 1e-6, 5000)
    cost_or = oracle.finalize(C64, f_or, g_or, p, q, eps)[0]
    _converged_check(res, C64, p, q, eps, 1e-6, it_or, cost_or)


def test_warm_start_resumes(ctx):
    rng = _rng(6)
    I, J = 3000, 200
    C = rng.uniform(0, 1, (I, J)).astype(np.float32)
    p, q = _marg(rng, I, J)
    a = ctx.solve_cost(_t(C), _t(p), _t(q), 0.05, tol=1e-6, max_iter=5000)
    b = ctx.solve_cost(_t(C), _t(p), _t(q), 0.05, tol=1e-6, max_iter=5000, warm_g=a.g.clone())
    assert b.iters <= 2
    assert b.transport_cost == pytest.approx(a.transport_cost, rel=1e-6)


def test_deterministic(ctx):
    rng = _rng(7)
    C = rng.uniform(0, 1, (5000, 640)).astype(np.float32)
    p, q = _marg(rng, 5000, 640)
    a = ctx.solve_cost(_t(C), _t(p), _t(q), 0.05, tol=1e-6, max_iter=500)
    b = ctx.solve_cost(_t(C), _t(p), _t(q), 0.05, tol=1e-6, max_iter=500)
    assert torch.equal(a.f, b.f) and torch.equal(a.g, b.g)
    assert a.transport_cost == b.transport_cost


def test_invalid_inputs_are_rejected(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(8)
    C = rng.uniform(0, 1, (50, 10)).astype(np.float32)
    p, q = _marg(rng, 50, 10)
    cases = []
    p0 = p.copy(); p0[4] = 0.0; cases.append((C, p0, q, 0.1))
    q2 = q * 1.5; cases.append((C, p, q2, 0.1))
    cases.append((C, p, q, 0.0))
    pn = p.copy(); pn[1] = np.nan; cases.append((C, pn, q, 0.1))
    for Cc, pp, qq, eps in cases:
        with pytest.raises(binding.OTError) as e:
            ctx.solve_cost(_t(Cc), _t(pp), _t(qq), eps, tol=1e-6, max_iter=10)
        assert e.value.status == binding.OT_EINVAL
    R = np.ones((50, 10), np.float32); R[2, 2] = 0.0
    with pytest.raises(binding.OTError) as e:
        ctx.solve(_t(R), _t(p), _t(q), 1.0, 0.1, tol=1e-6, max_iter=10)
    assert e.value.status == binding.OT_EINVAL
    with pytest.raises(binding.OTError) as e:
        ctx.solve_cost(_t(np.ones((4, 8200), np.float32)), _t(np.full(4, .25, np.float32)),
                       _t(np.full(8200, 1 / 8200, np.float32)), 0.1)
    assert e.value.status == binding.OT_EUNSUPPORTED
    # the context is still usable
    ctx.solve_cost(_t(C), _t(p), _t(q), 0.1, tol=1e-6, max_iter=100)


def test_bounded_barrier_reports_timeout(ctx):
    # A grid barrier whose spin limit is one poll gives up and reports OT_ETIMEOUT through
    # the device status word instead of waiting; the context stays usable afterwards.
    from paper_1805_01559_gb300 import binding
    rng = _rng(9)
    I, J = 60000, 256
    C = rng.uniform(0, 1, (I, J)).astype(np.float32)
    p, q = _marg(rng, I, J)
    ctx.set_spin_limit(1)
    try:
        with pytest.raises(binding.OTError) as e:
            ctx.solve_cost(_t(C), _t(p), _t(q), 0.05, tol=0.0, max_iter=50)
        assert e.value.status == binding.OT_ETIMEOUT
    finally:
        ctx.set_spin_limit(0)
    res = ctx.solve_cost(_t(C), _t(p), _t(q), 0.05, tol=1e-6, max_iter=2000)
    assert res.status == binding.OT_OK



def test_cost_from_gains_equals_rates_then_cost(ctx):
    """Rates and cost in one pass give the same values as the two calls."""
    from paper_1805_01559_gb300 import instances
    inst = instances.config1()
    G = torch.from_numpy(inst.G.astype(np.float32)).cuda()
    P = torch.from_numpy(inst.P.astype(np.float32)).cuda()
    R = ctx.build_rates(G, P, inst.N0, inst.W_hz)
    C_ref, eps_ref = ctx.build_cost(R, inst.mu, eps_rel=0.05)
    R2 = torch.empty_like(R)
    C, eps = ctx.build_cost_from_gains(G, P, inst.N0, inst.W_hz, inst.mu, eps_rel=0.05, R_out=R2)
    assert torch.equal(R2, R) and torch.equal(C, C_ref) and eps == eps_ref
    C3, none = ctx.build_cost_from_gains(G, P, inst.N0, inst.W_hz, inst.mu)
    assert none is None and torch.equal(C3, C_ref)
    G0 = G.clone()
    G0[5, :] = 0.0  # a device that hears nothing: zero rates
    from paper_1805_01559_gb300 import binding
    with pytest.raises(binding.OTError):
        ctx.build_cost_from_gains(G0, P, inst.N0, inst.W_hz, inst.mu, eps_rel=0.05)
