"""The seeded input generators (the one module both the CUDA path and the oracle use): they
draw what the input recipe states (positions in the area, the path-loss model, marginals
that balance), and a seed fixes every array."""
import math

import numpy as np
import pytest

from paper_1805_01559_gb300 import instances as ins


def test_same_seed_same_instance_other_seed_other_instance():
    a = ins.make_instance("t", 300, 20, 1000.0, 5, hotspot=True, traffic_sigma=1.5, marginal="capacity",
                          keep_geometry=True)
    b = ins.make_instance("t", 300, 20, 1000.0, 5, hotspot=True, traffic_sigma=1.5, marginal="capacity",
                          keep_geometry=True)
    c = ins.make_instance("t", 300, 20, 1000.0, 6, hotspot=True, traffic_sigma=1.5, marginal="capacity",
                          keep_geometry=True)
    for name in ("G", "lam", "q", "dev_xy", "rrh_xy", "shadow_db"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name
    assert not np.array_equal(a.G, c.G)


@pytest.mark.parametrize("marginal", ["uniform", "capacity"])
def test_marginals_positive_and_balanced(marginal):
    inst = ins.make_instance("t", 500, 37, 1000.0, 1, hotspot=False, traffic_sigma=1.0, marginal=marginal)
    assert inst.lam.shape == (500,) and inst.q.shape == (37,)
    assert (inst.lam > 0).all() and (inst.q > 0).all()
    assert inst.lam.sum() == pytest.approx(1.0, rel=1e-12)
    assert inst.q.sum() == pytest.approx(inst.lam.sum(), rel=1e-12)
    if marginal == "uniform":
        assert np.allclose(inst.q, inst.q[0], rtol=0, atol=0)
    else:  # kappa_j ~ U(0.5, 1.5): targets within a factor 3 of each other
        assert inst.q.max() / inst.q.min() <= 3.0


def test_positions_inside_the_area_and_rrh_grid():
    rng = np.random.Generator(np.random.PCG64(3))
    side = 2000.0
    dev = ins.devices_hotspot(4000, side, rng)
    assert dev.shape == (4000, 2) and (dev >= 0).all() and (dev <= side).all()
    rrh = ins.rrh_jittered_grid(30, side, rng)
    # r = floor(sqrt(30)) = 5 rows, ceil(30 / 5) = 6 columns; jitter keeps each RRH in its cell
    r, c = 5, 6
    col = np.floor(rrh[:, 0] / (side / c)).astype(int)
    row = np.floor(rrh[:, 1] / (side / r)).astype(int)
    k = np.arange(30)
    assert np.array_equal(col, k % c) and np.array_equal(row, k // c)


def test_path_gain_model():
    # one device, two RRHs at 100 m and at 5 m (clamped to 10 m), no shadowing:
    # G = 10^(-(30 + 35 log10 d)/10)
    dev = np.array([[0.0, 0.0]])
    rrh = np.array([[100.0, 0.0], [3.0, 4.0]])
    G = ins.path_gains(dev, rrh, np.zeros((1, 2), np.float32))
    want = [10 ** (-(30 + 35 * 2) / 10), 10 ** (-(30 + 35 * 1) / 10)]
    np.testing.assert_allclose(G[0], want, rtol=1e-13)
    # shadowing adds in dB
    G2 = ins.path_gains(dev, rrh, np.full((1, 2), 3.0, np.float32))
    np.testing.assert_allclose(G2[0], np.array(want) * 10 ** (-0.3), rtol=1e-13)


def test_noise_power():
    # -174 dBm/Hz + 10 log10(20 MHz) + 9 dB noise figure, in W
    want = 10 ** ((-174 + 10 * math.log10(20e6) + 9) / 10) / 1000
    assert ins.noise_power_w() == pytest.approx(want, rel=1e-12)


def test_ragged_batch_shapes():
    shapes = ins.config3_shapes(256, 0)
    assert len(shapes) == 256
    Is = np.array([s[0] for s in shapes])
    Js = np.array([s[1] for s in shapes])
    assert Is.min() >= 2000 and Is.max() <= 60000 and Js.min() >= 64 and Js.max() <= 1024
    assert len({s[2] for s in shapes}) == 256  # a seed per instance
    assert shapes == ins.config3_shapes(256, 0)


def test_blocked_instance_blocks_are_seeded_and_shaped():
    inst = ins.config4_blocked(0, I=20_000, J=64, block=8192)
    assert inst.nblocks == 3
    b0 = inst.gains_block(0)
    assert b0.shape == (8192, 64) and b0.dtype == np.float32
    assert inst.gains_block(2).shape == (20_000 - 2 * 8192, 64)
    assert np.array_equal(b0, inst.gains_block(0))
    assert not np.array_equal(b0[:100], inst.gains_block(1)[:100])
    assert inst.q.sum() == pytest.approx(inst.lam.sum(), rel=1e-12)


def test_mobile_cell_stays_inside_and_moves():
    cell = ins.serving_cell(500, 16, 7, side=1000.0)
    x0 = cell.dev_xy.copy()
    for _ in range(20):
        cell.advance(5.0)  # up to 150 m a step: several reflections
        assert (cell.dev_xy >= 0).all() and (cell.dev_xy <= cell.side).all()
    assert not np.array_equal(cell.dev_xy, x0)
    speed0 = np.hypot(*ins.serving_cell(500, 16, 7).vel.T)
    np.testing.assert_allclose(np.hypot(*cell.vel.T), speed0, rtol=1e-12)  # reflection keeps speed


def test_poisson_arrivals():
    t, cells = ins.poisson_arrivals(2000.0, 10.0, 64, seed=0)
    assert abs(len(t) - 20_000) < 5 * math.sqrt(20_000)
    assert (np.diff(t) >= 0).all() and t.min() >= 0 and t.max() <= 10.0
    assert cells.min() >= 0 and cells.max() < 64


def test_policy_cell_has_no_shadowing():
    cell = ins.policy_cell(200, 3)
    d = np.hypot(cell.dev_xy[:, None, 0].astype(np.float64) - cell.rrh_xy[None, :, 0],
                 cell.dev_xy[:, None, 1].astype(np.float64) - cell.rrh_xy[None, :, 1])
    want = 10 ** (-(30 + 35 * np.log10(np.maximum(d, 10.0))) / 10)
    np.testing.assert_allclose(cell.G, want, rtol=1e-6)
    assert cell.lam.sum() == pytest.approx(1.0, rel=1e-12)
