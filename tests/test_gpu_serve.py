"""GPU tests of the serving path (ot_assoc_server_*): resident cells, warm-started solves of
successive time instances, continuous batching on one persistent launch.

Parity: every served solve is a converged solve of that time instance's cost, so it is
checked against the FP64 oracle on the same gains (transport cost within 5e-6: the rates
are rebuilt from the gains in FP32 on the device), and the device's FP64 marginals of the
returned potentials are within tol + 5e-7 as for the FP32 solver.
Determinism: a cell's sequence of results is bit-identical served alone and in a mix.
"""
import numpy as np
import pytest

import oracle
from paper_1805_01559_gb300 import instances as ins

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


def _cell(I, J, seed):
    return ins.serving_cell(I, J, seed)


def _gains_dev(G):
    """Device copy of the gains with rows padded to 16 bytes."""
    I, J = G.shape
    ld = (J + 3) // 4 * 4
    buf = torch.zeros((I, ld), dtype=torch.float32, device="cuda")
    buf[:, :J] = torch.from_numpy(np.ascontiguousarray(G, np.float32)).cuda()
    return buf[:, :J]


def _eps_of(cell):
    G0 = cell.gains(np.float32).astype(np.float64)
    R = oracle.rates(G0, np.ones(cell.J), ins.noise_power_w(), ins.W_HZ)
    return 0.05 * oracle.median(oracle.cost(R.astype(np.float32).astype(np.float64), ins.MU_PER_BIT))


def _add(srv, cell, eps, drift=False):
    kw = {}
    if drift:
        kw = dict(dev_xy=cell.dev_xy, dev_v=cell.vel, rrh_xy=cell.rrh_xy, shadow_db=cell.shadow_db, side_m=cell.side)
    return srv.add_cell(cell.I, cell.J, eps, np.ones(cell.J), cell.lam, cell.q, ins.MU_PER_BIT, ins.noise_power_w(),
                        ins.W_HZ, tol=1e-6, max_iter=3000, **kw)


def _sequence(cell, steps, dt):
    """Gains of `steps` successive time instances of a moving cell (host generator)."""
    out = []
    for _ in range(steps):
        out.append(cell.gains(np.float32))
        cell.advance(dt)
    return out


def test_served_solves_match_oracle(ctx):
    srv = ctx.server(group_ctas=8)
    cells = [_cell(3000, 64, 1), _cell(1500, 200, 2)]
    seqs = [_sequence(_cell(3000, 64, 1), 3, 0.05), _sequence(_cell(1500, 200, 2), 3, 0.05)]
    ids = [_add(srv, c, _eps_of(c)) for c in cells]
    epss = [_eps_of(c) for c in cells]
    G_dev = {}
    for step in range(3):
        for k in range(2):
            G_dev[(k, step)] = _gains_dev(seqs[k][step])
            srv.submit(ids[k], G_dev[(k, step)])
    res = srv.drain()
    assert len(res) == 6 and all(r.status == 0 for r in res), [r.status for r in res]
    by_cell = {0: [], 1: []}
    for r in sorted(res, key=lambda r: r.ticket):
        by_cell[ids.index(r.cell)].append(r)
    for k in range(2):
        iters = [r.iters for r in by_cell[k]]
        assert iters[1] < iters[0] and iters[2] < iters[0], iters  # warm starts
        G = seqs[k][2].astype(np.float64)
        R = oracle.rates(G, np.ones(cells[k].J), ins.noise_power_w(), ins.W_HZ).astype(np.float32)
        C64 = oracle.cost(R.astype(np.float64), ins.MU_PER_BIT)
        p, q = cells[k].lam.astype(np.float32), cells[k].q.astype(np.float32)
        f_or, g_or, _, _ = oracle.sinkhorn(C64, p, q, epss[k], 1e-6, 5000)
        cost_or = oracle.finalize(C64, f_or, g_or, p, q, epss[k])[0]
        last = by_cell[k][-1]
        # the server builds the rates from the gains in FP32 (1e-6 relative to the FP64
        # formula, see the rates parity test), which moves the optimum by as much
        assert abs(last.transport_cost - cost_or) <= 5e-6 * cost_or, (last.transport_cost, cost_or)
        # the device's FP64 evaluation of the returned potentials on the cell's own cost
        assert last.marg_err_row <= 1e-6 + MARG_SLACK and last.marg_err_col <= 1e-6 + MARG_SLACK
    srv.close()


def _run(ctx, cells, order, dt=0.03):
    """Serve the drifting cells in the given request order; results per cell in order."""
    srv = ctx.server(group_ctas=8)
    ids = [_add(srv, c, eps, drift=True) for c, eps in cells]
    for k in order:
        srv.submit(ids[k], None, dt)
    res = srv.drain()
    out = {k: [] for k in range(len(cells))}
    for r in sorted(res, key=lambda r: r.ticket):
        out[ids.index(r.cell)].append(r)
    states = [srv.cell_state(ids[k], c.I, c.J) for k, (c, _) in enumerate(cells)]
    srv.close()
    return out, states


def test_alone_and_in_the_mix_are_identical(ctx):
    specs = [(4000, 128, 11), (2000, 512, 12), (6000, 64, 13), (1000, 1000, 14)]
    mk = lambda: [(_cell(I, J, s), None) for I, J, s in specs]
    cells = mk()
    cells = [(c, _eps_of(c)) for c, _ in cells]
    # cell 0 alone: 4 time instances
    alone, st_alone = _run(ctx, [(_cell(*specs[0]), cells[0][1])], [0, 0, 0, 0])
    # cell 0 among the others, requests interleaved
    mixed_cells = [(_cell(I, J, s), eps) for (I, J, s), (_, eps) in zip(specs, cells)]
    order = [0, 1, 2, 3, 0, 2, 1, 0, 3, 3, 0, 1]
    mix, st_mix = _run(ctx, mixed_cells, order)
    a, m = alone[0], mix[0]
    assert len(a) == len(m) == 4
    for x, y in zip(a, m):
        assert x.status == y.status == 0
        assert x.iters == y.iters
        assert x.transport_cost == y.transport_cost
        assert x.marg_err_row == y.marg_err_row
    for t_a, t_m in zip(st_alone[0], st_mix[0]):
        assert torch.equal(t_a, t_m)


def test_requests_overlap_and_drain(ctx):
    # Many requests at once: several groups work at the same time; every request finishes,
    # each cell's results come back in submission order.
    specs = [(3000 + 500 * k, 128 * (1 + k % 4), 20 + k) for k in range(12)]
    cells = [(_cell(I, J, s), None) for I, J, s in specs]
    cells = [(c, _eps_of(c)) for c, _ in cells]
    srv = ctx.server(group_ctas=8)
    ids = [_add(srv, c, eps, drift=True) for c, eps in cells]
    tickets = {cid: [] for cid in ids}
    for rep in range(5):
        for cid in ids:
            tickets[cid].append(srv.submit(cid, None, 0.02))
    res = srv.drain()
    assert len(res) == 60 and all(r.status == 0 for r in res)
    for cid in ids:
        got = [r for r in res if r.cell == cid]
        done_order = [r.ticket for r in sorted(got, key=lambda r: r.t_done_us)]
        assert done_order == tickets[cid]
    # the launch served requests side by side: some request started before another ended
    spans = sorted((r.t_start_us, r.t_done_us) for r in res)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    st = srv.stats()
    assert st["cells"] == 12 and st["inflight"] == 0
    srv.close()


def test_admission_by_hbm_budget(ctx):
    from paper_1805_01559_gb300 import binding
    c = _cell(20000, 512, 30)
    eps = _eps_of(c)
    srv = ctx.server(group_ctas=8, hbm_budget=100 << 20)  # 100 MiB
    _add(srv, c, eps, drift=True)                          # ~ 20000 x 512 x 8 B = 82 MB
    with pytest.raises(binding.OTError) as e:
        _add(srv, _cell(20000, 512, 31), eps, drift=True)
    assert e.value.status == binding.OT_EBUSY
    assert srv.stats()["cells"] == 1
    srv.close()


def test_server_rejects_bad_requests(ctx):
    from paper_1805_01559_gb300 import binding
    c = _cell(1000, 64, 40)
    srv = ctx.server(group_ctas=8)
    cid = _add(srv, c, _eps_of(c), drift=True)
    with pytest.raises(binding.OTError):
        srv.submit(cid + 5, None, 0.1)
    with pytest.raises(binding.OTError):
        srv.submit(cid, _gains_dev(c.gains()), 0.0)  # a drifting cell moves its own devices
    srv.close()


def test_mobile_cost_equals_the_servers_rebuild_and_the_host_model(ctx):
    """ot_assoc_build_cost_mobile moves the devices and rebuilds C with the server's own device
    code: after the same dt the cost is bit-identical to the served cell's, the positions follow
    the host mobility model (reflection at the walls), and the cost matches the oracle's rates
    (Sec. II-A) on the host model's gains to FP32/SFU accuracy."""
    from paper_1805_01559_gb300 import binding
    c0 = _cell(2000, 96, 41)
    dt = 3.7  # a few hundred metres for the fastest devices: some reflect
    srv = ctx.server(group_ctas=8)
    try:
        cid = srv.add_cell(c0.I, c0.J, 0.0, np.ones(c0.J), c0.lam, c0.q, ins.MU_PER_BIT, ins.noise_power_w(),
                           ins.W_HZ, tol=1e-6, max_iter=3000, dev_xy=c0.dev_xy, dev_v=c0.vel, rrh_xy=c0.rrh_xy,
                           shadow_db=c0.shadow_db, side_m=c0.side, eps_rel=0.05)
        srv.submit(cid, None, dt)
        res = srv.drain()
        assert len(res) == 1 and res[0].status == 0
        C_srv = srv.cell_state(cid, c0.I, c0.J)[0].clone()
        eps_srv = srv.cell_eps(cid)
    finally:
        srv.close()
    dev = torch.device("cuda", 0)
    xy = torch.from_numpy(np.ascontiguousarray(c0.dev_xy, np.float64)).to(dev)
    v = torch.from_numpy(np.ascontiguousarray(c0.vel, np.float64)).to(dev)
    rrh = torch.from_numpy(np.ascontiguousarray(c0.rrh_xy, np.float32)).to(dev)
    sh = torch.from_numpy(np.ascontiguousarray(c0.shadow_db, np.float32)).to(dev)
    P = torch.ones(c0.J, dtype=torch.float32, device=dev)
    args = (ins.noise_power_w(), ins.W_HZ, ins.MU_PER_BIT)
    _, eps = ctx.build_cost_mobile(xy, v, rrh, sh, P, 0.0, c0.side, *args, eps_rel=0.05)
    assert eps == eps_srv
    C, _ = ctx.build_cost_mobile(xy, v, rrh, sh, P, dt, c0.side, *args)
    assert torch.equal(C, C_srv)
    host = _cell(2000, 96, 41)
    host.advance(dt)
    np.testing.assert_allclose(xy.cpu().numpy(), host.dev_xy, atol=2e-3)
    np.testing.assert_array_equal(np.sign(v.cpu().numpy()), np.sign(host.vel))
    C_or = oracle.cost(oracle.rates(host.gains(np.float64), np.ones(c0.J), ins.noise_power_w(), ins.W_HZ),
                       ins.MU_PER_BIT)
    np.testing.assert_allclose(C.cpu().numpy().astype(np.float64), C_or, rtol=5e-5)
    with pytest.raises(binding.OTError):
        ctx.build_cost_mobile(xy, v, rrh, sh, P, -1.0, c0.side, *args)
