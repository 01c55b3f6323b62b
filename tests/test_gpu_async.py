"""Asynchronous solves (ot_assoc_solve_cost_async + ot_assoc_wait): the same arithmetic as the
synchronous call, so results are bit-identical; tickets, the in-flight limit and device-side
errors reported at the wait."""
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


def _inst(seed=0, I=3000, J=120):
    from paper_1805_01559_gb300 import instances as ins
    inst = ins.make_instance("async", I, J, 1000.0, seed, hotspot=True, traffic_sigma=1.0, marginal="capacity",
                             dtype=np.float32)
    R = oracle.rates(inst.G.astype(np.float64), inst.P, inst.N0, inst.W_hz)
    C = oracle.cost(R, inst.mu).astype(np.float32)
    return (torch.from_numpy(C).cuda(), torch.from_numpy(inst.lam.astype(np.float32)).cuda(),
            torch.from_numpy(inst.q.astype(np.float32)).cuda(), float(np.median(C)))


def test_async_equals_sync_bit_for_bit(ctx):
    C, p, q, med = _inst()
    eps = [0.1 * med, 0.03 * med, 0.01 * med]
    sync = [ctx.solve_cost(C, p, q, e, tol=1e-6) for e in eps]
    pend = [ctx.solve_cost_async(C, p, q, e, tol=1e-6) for e in eps]
    got = [x.wait() for x in pend]
    for a, b in zip(sync, got):
        assert a.iters == b.iters and a.status == b.status
        assert a.transport_cost == b.transport_cost
        assert torch.equal(a.f, b.f) and torch.equal(a.g, b.g) and torch.equal(a.rrh_load, b.rrh_load)


def test_async_waits_out_of_order_and_timings(ctx):
    C, p, q, med = _inst(1)
    ctx.enable_timing(True)
    try:
        pend = [ctx.solve_cost_async(C, p, q, e * med, tol=1e-6) for e in (0.1, 0.05)]
        second = pend[1].wait()
        t = ctx.last_timings()
        assert t["valid"] == 1 and t["loop_ms"] > 0 and t["sweeps"] == second.iters
        first = pend[0].wait()
        ref = ctx.solve_cost(C, p, q, 0.1 * med, tol=1e-6)
        assert first.transport_cost == ref.transport_cost
    finally:
        ctx.enable_timing(False)


def test_async_ticket_rules(ctx):
    from paper_1805_01559_gb300 import binding
    C, p, q, med = _inst(2, I=500, J=20)
    x = ctx.solve_cost_async(C, p, q, 0.1 * med)
    x.wait()
    with pytest.raises(binding.OTError):
        x.wait()  # a ticket is waited for once
    pend = [ctx.solve_cost_async(C, p, q, 0.1 * med, max_iter=3) for _ in range(16)]
    with pytest.raises(binding.OTError):
        ctx.solve_cost_async(C, p, q, 0.1 * med)  # 16 in flight
    for x in pend:
        x.wait()
    # an invalid marginal is found on the device and reported by the wait
    bad = p.clone()
    bad[7] = -1.0
    y = ctx.solve_cost_async(C, bad, q, 0.1 * med)
    with pytest.raises(binding.OTError):
        y.wait()
    ok = ctx.solve_cost_async(C, p, q, 0.1 * med).wait()
    assert ok.status == 0
