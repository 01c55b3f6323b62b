"""GPU parity of the batched ragged solver (one persistent launch for many instances).

Each instance of a batch is solved by a group of CTAs with the same arithmetic as the
single-instance solver, so the tolerances of test_gpu_parity.py apply unchanged: fixed
iteration counts are compared plan entry by plan entry (RTOL_ITER), converged solves by
transport cost (1e-6 relative) and exact FP64 marginals of the returned potentials.
An instance's arithmetic depends only on its own data and its group size and stage
geometry, so results are bit-identical alone and inside any mix that plans it the same way.
"""
import numpy as np
import pytest

import oracle

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


def _padded(C):
    """Device copy of C with rows padded to a multiple of 4 floats (16-byte rows)."""
    I, J = C.shape
    ld = (J + 3) // 4 * 4
    buf = torch.full((I, ld), float("inf"), dtype=torch.float32, device="cuda")
    buf[:, :J] = _t(C)
    return buf[:, :J]


def _inst(rng, I, J, eps=0.1, tol=0.0, max_iter=5, kind="uniform"):
    from paper_1805_01559_gb300 import binding
    if kind == "uniform":
        C = rng.uniform(0.0, 1.0, (I, J)).astype(np.float32)
    else:
        C = rng.lognormal(0.0, 0.7, (I, J)).astype(np.float32)
    p = rng.lognormal(0.0, 1.0, I)
    q = rng.uniform(0.5, 1.5, J)
    p /= p.sum()
    q *= p.sum() / q.sum()
    p32, q32 = p.astype(np.float32), q.astype(np.float32)
    x = binding.Instance(C=_padded(C), p=_t(p32), q=_t(q32), eps=eps, tol=tol, max_iter=max_iter)
    return x, C, p32, q32


RAGGED = [(1, 1), (3, 2), (37, 129), (1000, 50), (2049, 1023), (513, 1024), (5000, 64), (12, 257),
          (700, 3), (20000, 100), (64, 700), (4099, 511)]


def test_batch_fixed_iterations_match_oracle(ctx):
    rng = _rng(11)
    batch = [_inst(rng, I, J, eps=0.1, tol=0.0, max_iter=4) for I, J in RAGGED]
    for x, *_ in batch:
        x.pi = torch.empty((x.C.shape[0], x.C.shape[1]), dtype=torch.float32, device="cuda")
    res = ctx.solve_batched([b[0] for b in batch])
    for (x, C, p, q), r in zip(batch, res):
        I, J = C.shape
        assert r.status in (0, 1), r
        assert r.iters == 4 or (r.iters < 4 and (I == 1 or J == 1)), (I, J, r.iters)
        f_or, g_or, _, _ = oracle.sinkhorn(C.astype(np.float64), p, q, 0.1, 0.0, r.iters)
        pi_or = oracle.plan(C.astype(np.float64), f_or, g_or, 0.1)
        err = np.abs(_np(x.pi).astype(np.float64) - pi_or)
        assert (err <= RTOL_ITER * pi_or + 1e-12).all(), (I, J, float(err.max()))
        pi_fg = oracle.plan(C.astype(np.float64), _np(x.f), _np(x.g), 0.1)
        np.testing.assert_allclose(pi_fg, pi_or, rtol=RTOL_ITER, atol=1e-12)


def test_batch_converged_match_oracle(ctx):
    rng = _rng(12)
    shapes = [(3000, 200, 0.05), (1500, 1000, 0.1), (800, 77, 0.02), (6000, 512, 0.05)]
    batch = [_inst(rng, I, J, eps=e, tol=1e-6, max_iter=5000, kind="lognormal") for I, J, e in shapes]
    res = ctx.solve_batched([b[0] for b in batch])
    for (x, C, p, q), r, (I, J, eps) in zip(batch, res, shapes):
        assert r.status == 0 and r.converged, r
        C64 = C.astype(np.float64)
        f_or, g_or, it_or, _ = oracle.sinkhorn(C64, p, q, eps, 1e-6, 5000)
        cost_or = oracle.finalize(C64, f_or, g_or, p, q, eps)[0]
        assert abs(r.iters - it_or) <= 2, (r.iters, it_or)
        cost, rho, er, ec = oracle.finalize(C64, _np(x.f), _np(x.g), p, q, eps)
        assert er <= 1e-6 + MARG_SLACK and ec <= 1e-6 + MARG_SLACK, (er, ec)
        assert abs(r.transport_cost - cost_or) <= 1e-6 * cost_or, (r.transport_cost, cost_or)
        assert r.marg_err_row == pytest.approx(er, abs=3e-7)
        assert r.marg_err_col == pytest.approx(ec, abs=3e-7)
        np.testing.assert_allclose(_np(x.rrh_load), rho, rtol=1e-5, atol=1e-9 * rho.max())


@pytest.mark.parametrize("shape", [(4000, 300), (60000, 1024), (777, 64), (5000, 3)])
def test_batch_matches_single_solver(ctx, shape):
    # Same instance through the single-instance entry point and inside a batch (untuned: the
    # same stage size).  Every reduction runs over the same row partitions in the same order,
    # so the potentials, loads and iteration count are bit-identical; the cost total is
    # summed over columns in a different order.
    I, J = shape
    rng = _rng(13 + I)
    x, C, p, q = _inst(rng, I, J, eps=0.05, tol=1e-6, max_iter=3000)
    single = ctx.solve_cost(x.C, x.p, x.q, 0.05, tol=1e-6, max_iter=3000)
    (r,) = ctx.solve_batched([x])
    assert r.iters == single.iters
    assert torch.equal(x.f, single.f) and torch.equal(x.g, single.g)
    assert torch.equal(x.rrh_load, single.rrh_load)
    assert r.transport_cost == pytest.approx(single.transport_cost, rel=1e-12)


def test_alone_and_in_the_mix_are_identical(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(14)
    mix = [_inst(rng, I, J, eps=0.05, tol=1e-6, max_iter=2000) for I, J in
           [(9000, 333), (700, 1000), (30000, 64), (2500, 900), (4000, 200), (128, 16)]]
    res_mix = ctx.solve_batched([m[0] for m in mix])
    f_mix = [m[0].f.clone() for m in mix]
    g_mix = [m[0].g.clone() for m in mix]
    for k, (x, C, p, q) in enumerate(mix):
        alone = binding.Instance(C=x.C, p=x.p, q=x.q, eps=x.eps, tol=x.tol, max_iter=x.max_iter)
        (r,) = ctx.solve_batched([alone])
        assert r.iters == res_mix[k].iters
        assert r.transport_cost == res_mix[k].transport_cost
        assert torch.equal(alone.f, f_mix[k]) and torch.equal(alone.g, g_mix[k])


def test_graph_replay_and_update(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(15)
    items = [_inst(rng, I, J, eps=0.05, tol=1e-6, max_iter=2000) for I, J in [(5000, 128), (3000, 700), (800, 40)]]
    b = ctx.batch([it[0] for it in items], graph=True)
    r1 = b.run()
    f1 = [it[0].f.clone() for it in items]
    r2 = b.run()
    for a, c in zip(r1, r2):
        assert a.iters == c.iters and a.transport_cost == c.transport_cost
    for it, f in zip(items, f1):
        assert torch.equal(it[0].f, f)
    # change eps of instance 1 without re-planning; the replay must use it
    x, C, p, q = items[1]
    y = binding.Instance(C=x.C, p=x.p, q=x.q, eps=0.1, tol=1e-6, max_iter=2000)
    b.set(1, y)
    r3 = b.run()
    single = ctx.solve_cost(_t(C), _t(p), _t(q), 0.1, tol=1e-6, max_iter=2000)
    assert r3[1].transport_cost == pytest.approx(single.transport_cost, rel=1e-6)
    assert r3[0].transport_cost == r1[0].transport_cost
    b.close()


def test_deterministic_batch(ctx):
    rng = _rng(16)
    mk = lambda: [_inst(_rng(16 + k), I, J, eps=0.05, tol=1e-6, max_iter=1000)
                  for k, (I, J) in enumerate([(7000, 640), (3000, 100), (900, 1024)])]
    a, b = mk(), mk()
    ra = ctx.solve_batched([x[0] for x in a])
    rb = ctx.solve_batched([x[0] for x in b])
    for xa, xb, u, v in zip(a, b, ra, rb):
        assert torch.equal(xa[0].f, xb[0].f) and torch.equal(xa[0].g, xb[0].g)
        assert u.transport_cost == v.transport_cost


def test_failed_instance_does_not_stop_the_others(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(17)
    good1, _, _, _ = _inst(rng, 2000, 100, eps=0.05, tol=1e-6, max_iter=2000)
    bad, C, p, q = _inst(rng, 1500, 50, eps=0.05, tol=1e-6, max_iter=2000)
    p0 = p.copy()
    p0[7] = 0.0
    bad.p = _t(p0)
    unbalanced, C2, p2, q2 = _inst(rng, 900, 30, eps=0.05, tol=1e-6, max_iter=2000)
    unbalanced.q = _t(q2 * 2.0)
    good2, _, _, _ = _inst(rng, 3000, 700, eps=0.05, tol=1e-6, max_iter=2000)
    res = ctx.solve_batched([good1, bad, unbalanced, good2])
    assert res[0].status == binding.OT_OK and res[3].status == binding.OT_OK
    assert res[1].status == binding.OT_EINVAL and res[2].status == binding.OT_EINVAL


def test_warm_start_in_batch(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(18)
    x, C, p, q = _inst(rng, 6000, 256, eps=0.05, tol=1e-6, max_iter=3000)
    (r0,) = ctx.solve_batched([x])
    y = binding.Instance(C=x.C, p=x.p, q=x.q, eps=x.eps, tol=1e-6, max_iter=3000, warm_start=True,
                         g=x.g.clone())
    (r1,) = ctx.solve_batched([y])
    assert r1.iters <= 2 < r0.iters
    assert r1.transport_cost == pytest.approx(r0.transport_cost, rel=1e-6)


def test_group_sizes_agree(ctx):
    # The same instance planned on different group sizes (tuning table) gives the same solve
    # up to summation order.
    from paper_1805_01559_gb300 import binding
    rng = _rng(19)
    x, C, p, q = _inst(rng, 20000, 400, eps=0.05, tol=1e-6, max_iter=3000)
    bk = binding.bucket(20000, 400)
    out = []
    try:
        for gs in (1, 4, 19, 152):
            ctx.set_tuning(bk, gs, 24576)
            y = binding.Instance(C=x.C, p=x.p, q=x.q, eps=x.eps, tol=1e-6, max_iter=3000)
            (r,) = ctx.solve_batched([y])
            out.append(r)
    finally:
        ctx.set_tuning(bk, 0, 0)
    for r in out[1:]:
        assert abs(r.iters - out[0].iters) <= 1
        assert r.transport_cost == pytest.approx(out[0].transport_cost, rel=1e-6)


def test_autotune_fills_the_table(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(20)
    items = [_inst(rng, I, J, eps=0.05, tol=1e-6, max_iter=2000)[0].prepare()
             for I, J in [(4000, 128), (30000, 700), (900, 64)]]
    f_before = [x.f.clone() for x in items]
    ctx.autotune(items, iters=4)
    tab = ctx.tuning()
    for x in items:
        e = tab[binding.bucket(*x.C.shape)]
        assert e["gsize"] > 0 and e["stage"] > 0 and e["rate"] > 0
    for x, f in zip(items, f_before):
        assert torch.equal(x.f, f)  # the callers' buffers are untouched by tuning
    res = ctx.solve_batched(items)
    assert all(r.status == binding.OT_OK for r in res)
    for b in range(15):
        ctx.set_tuning(b, 0, 0)


def test_batch_rejects_bad_arguments(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(21)
    x, *_ = _inst(rng, 100, 1030)
    with pytest.raises(binding.OTError) as e:
        ctx.solve_batched([x])
    assert e.value.status == binding.OT_EUNSUPPORTED
    C = _t(rng.uniform(0, 1, (100, 7)).astype(np.float32))  # ld 7: rows not 16-byte aligned
    y = binding.Instance(C=C, p=_t(np.full(100, 0.01, np.float32)), q=_t(np.full(7, 1 / 7, np.float32)), eps=0.1)
    with pytest.raises(binding.OTError) as e:
        ctx.solve_batched([y])
    assert e.value.status == binding.OT_EINVAL
    ok, *_ = _inst(rng, 100, 8)
    ok.eps = 0.0
    with pytest.raises(binding.OTError) as e:
        ctx.solve_batched([ok])
    assert e.value.status == binding.OT_EINVAL


def test_batch_timeout_is_reported(ctx):
    from paper_1805_01559_gb300 import binding
    rng = _rng(22)
    items = [_inst(rng, 60000, 256, eps=0.05, tol=0.0, max_iter=50)[0]]
    ctx.set_spin_limit(1)
    try:
        with pytest.raises(binding.OTError) as e:
            ctx.solve_batched(items)
        assert e.value.status == binding.OT_ETIMEOUT
    finally:
        ctx.set_spin_limit(0)
    res = ctx.solve_batched(items)
    assert res[0].status in (binding.OT_OK, binding.OT_NOT_CONVERGED)
