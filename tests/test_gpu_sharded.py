"""GPU parity of the row-sharded Algorithm 1 (ot_assoc_shard_* through the C ABI, strung
together by paper_1805_01559_gb300.sharded) against the FP64 oracle on the whole matrix.

The ranks are emulated as several shards in one process on the one GPU: every shard's sweep
is its own launch and the sum over the shards is formed on the host side between launches,
so no kernel waits on another.  Tolerances are the single-GPU solver's (test_gpu_parity.py):
the plan after k iterations within RTOL_ITER = 2e-5 entry by entry; converged solves with
the exact FP64 marginal residuals of the returned potentials <= tol and the transport cost
within 1e-6 of the oracle's."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_ITER = 2e-5


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


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


def _marg(rng, I, J):
    p = rng.lognormal(0.0, 1.0, I)
    q = rng.uniform(0.5, 1.5, J)
    return (p / p.sum()).astype(np.float32), (q / q.sum()).astype(np.float32)


def _solve(ctx, C, p, q, eps, cuts, **kw):
    from paper_1805_01559_gb300 import sharded as S
    b = [0, *cuts, C.shape[0]]
    Ct, pt = _t(C), _t(p)
    shards = [(Ct[b[i]:b[i + 1]], pt[b[i]:b[i + 1]]) for i in range(len(b) - 1)]
    res = S.solve_sharded(S.DeviceOps(ctx), shards, _t(q), eps, **kw)
    f = np.concatenate([t.cpu().numpy() for t in res.f])
    return res, f, res.g.cpu().numpy()


def _plan_check(C, f, g, f_or, g_or, eps):
    C64 = C.astype(np.float64)
    pi, pi_or = oracle.plan(C64, f, g, eps), oracle.plan(C64, f_or, g_or, eps)
    bad = np.abs(pi - pi_or) > RTOL_ITER * pi_or + 1e-12
    assert not bad.any(), (int(bad.sum()), float((np.abs(pi - pi_or) / np.maximum(pi_or, 1e-300)).max()))


# one-, two-, four- and eight-warp teams; ragged shard cuts
SHAPES = [((1000, 50), [333]), ((2049, 1023), [1000, 1001]), ((513, 1025), [7]), ((300, 2049), [150]),
          ((100, 4099), [50]), ((64, 8192), [10, 40])]


@pytest.mark.parametrize("shape,cuts", SHAPES)
@pytest.mark.parametrize("iters", [1, 4])
def test_fixed_iterations_match_oracle(ctx, shape, cuts, iters):
    I, J = shape
    rng = _rng(I * 31 + J)
    C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    p, q = _marg(rng, I, J)
    eps = 0.1
    res, f, g = _solve(ctx, C, p, q, eps, cuts, tol=0.0, max_iter=iters)
    assert res.iters == iters
    f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, eps, 0.0, iters)
    _plan_check(C, f, g, f_or, g_or, eps)


def test_underflowing_column_takes_the_exact_first_iteration(ctx):
    # column 0 lies 3 above every row's cheapest link at eps = 0.02: its scaled first sums
    # underflow, so iteration 1 goes through the column maxima and the shifted sums
    I, J = 3000, 50
    rng = _rng(77)
    C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    C[:, 0] += 3.0
    p, q = _marg(rng, I, J)
    for iters in (1, 3):
        res, f, g = _solve(ctx, C, p, q, 0.02, [1234], tol=0.0, max_iter=iters)
        f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, 0.02, 0.0, iters)
        _plan_check(C, f, g, f_or, g_or, 0.02)


@pytest.mark.parametrize("shape,eps,cuts", [((4000, 300), 0.02, [1500, 3000]), ((2500, 1111), 0.05, [1249])])
def test_converged_matches_oracle_and_the_single_gpu_solver(ctx, shape, eps, cuts):
    I, J = shape
    rng = _rng(I + J)
    C = rng.uniform(0, 1, (I, J)).astype(np.float32)
    p, q = _marg(rng, I, J)
    tol = 1e-6
    res, f, g = _solve(ctx, C, p, q, eps, cuts, tol=tol, max_iter=5000)
    C64 = C.astype(np.float64)
    f_or, g_or, it_or, _ = oracle.sinkhorn(C64, p, q, eps, tol, 5000)
    cost_or = oracle.finalize(C64, f_or, g_or, p, q, eps)[0]
    assert res.converged and abs(res.iters - it_or) <= 2, (res.iters, it_or)
    cost, rho, er, ec = oracle.finalize(C64, f, g, p, q, eps)
    assert er <= tol and ec <= tol, (er, ec)
    assert abs(res.transport_cost - cost_or) <= 1e-6 * cost_or
    assert res.marg_err_row == pytest.approx(er, abs=3e-7)
    np.testing.assert_allclose(res.rrh_load.cpu().numpy(), rho, rtol=1e-5, atol=1e-9 * rho.max())
    one = ctx.solve_cost(_t(C), _t(p), _t(q), eps, tol=tol, max_iter=5000)
    assert abs(one.iters - res.iters) <= 1
    assert res.transport_cost == pytest.approx(one.transport_cost, rel=1e-6)


def test_unaligned_rows_and_determinism(ctx):
    rng = _rng(5)
    I, J = 700, 37  # rows of 37 floats: the driver pads them once
    C = rng.uniform(0, 1, (I, J)).astype(np.float32)
    p, q = _marg(rng, I, J)
    a, fa, ga = _solve(ctx, C, p, q, 0.1, [300], tol=0.0, max_iter=6)
    b, fb, gb = _solve(ctx, C, p, q, 0.1, [300], tol=0.0, max_iter=6)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.transport_cost == b.transport_cost
    f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, 0.1, 0.0, 6)
    _plan_check(C, fa, ga, f_or, g_or, 0.1)


def test_invalid_marginals_are_rejected(ctx):
    rng = _rng(9)
    C = rng.uniform(0, 1, (100, 8)).astype(np.float32)
    p, q = _marg(rng, 100, 8)
    p[5] = -1.0
    with pytest.raises(ValueError):
        _solve(ctx, C, p, q, 0.1, [50])
