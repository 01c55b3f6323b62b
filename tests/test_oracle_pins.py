"""Pins for the FP64 oracle: closed forms, exact LPs, brute force and invariants.

None of these re-types the oracle's own formulas: each check reaches the answer
another way (a closed form, a different algorithm, a library LP, a theorem's
bound), so that a dropped term, a wrong sign, a swapped index or a transposed
operand in ``oracle/ot_oracle.c`` fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1805_01559_gb300 import instances as ins


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _entropy(x):
    x = np.asarray(x, dtype=np.float64)
    x = x / x.sum()
    x = x[x > 0]
    return float(-(x * np.log(x)).sum())


def _balanced(rng, I, J):
    p = rng.uniform(0.2, 1.0, I)
    q = rng.uniform(0.2, 1.0, J)
    p /= p.sum()
    q /= q.sum()
    return p, q


# ------------------------------------------------------------------------------- rates / cost
def test_rates_single_rrh_closed_form():
    # J = 1: nothing interferes, SINR = P G / N0 (Sec. II-A).
    G = np.array([[1e-9], [3e-12], [5e-7]])
    P = np.array([2.0])
    N0, W = 1e-12, 20e6
    R = oracle.rates(G, P, N0, W)
    want = W * np.log2(1.0 + P[0] * G[:, 0] / N0)
    np.testing.assert_allclose(R[:, 0], want, rtol=1e-14)


def test_rates_hand_example_two_rows():
    # Received powers (1, 1, 2) and no noise: SINR = 1/3, 1/3, 1 exactly.
    # Second row reversed to catch a transposed interference sum.
    G = np.array([[1.0, 0.5, 2.0 / 3.0], [2.0 / 3.0, 0.5, 1.0]])
    P = np.array([1.0, 2.0, 3.0])
    R = oracle.rates(G, P, 0.0, 1.0)
    np.testing.assert_allclose(R[0], [math.log2(4 / 3), math.log2(4 / 3), 1.0], rtol=1e-14)
    # row 2 received powers (2/3, 1, 3): SINR = 1/6, 3/11, 9/5
    np.testing.assert_allclose(R[1], [math.log2(7 / 6), math.log2(14 / 11), math.log2(14 / 5)],
                               rtol=1e-14)


def test_rates_low_sinr_limit():
    # For SINR s -> 0, log2(1+s) = s/ln2 * (1 - s/2 + ...): needs log1p, not log(1+s).
    G = np.array([[1e-20, 1.0]])
    P = np.array([1.0, 1.0])
    R = oracle.rates(G, P, 0.0, 1.0)
    s = 1e-20
    np.testing.assert_allclose(R[0, 0], s / math.log(2.0), rtol=1e-12)


def test_rates_symmetric_pair():
    # Equal received power from both RRHs: SINR = PG / (PG + N0) for both.
    G = np.full((1, 2), 1e-10)
    P = np.array([1.0, 1.0])
    N0 = 3e-11
    R = oracle.rates(G, P, N0, 1.0)
    s = 1e-10 / (1e-10 + 3e-11)
    np.testing.assert_allclose(R[0], [math.log2(1 + s)] * 2, rtol=1e-14)


def test_rates_total_form_equals_direct_sum():
    """The O(I J) total-minus-own interference gives the direct sum's rates (Sec. II-A), on the
    config-1 channel, on rows where one link carries nearly all of the received power, and on
    a single-RRH row (no interference: SINR = P G / N0)."""
    inst = ins.config1()
    G = inst.G[:200].astype(np.float64)
    R1 = oracle.rates(G, inst.P, inst.N0, inst.W_hz)
    R2 = oracle.rates_total(G, inst.P, inst.N0, inst.W_hz)
    np.testing.assert_allclose(R2, R1, rtol=1e-12)
    rng = _rng(17)
    Gd = rng.uniform(1e-12, 1e-10, (5, 9))
    Gd[np.arange(5), rng.integers(0, 9, 5)] = 1e-3  # dominant links, SINR ~ 1e6
    P = rng.uniform(0.5, 2.0, 9)
    np.testing.assert_allclose(oracle.rates_total(Gd, P, 1e-13, 2e7), oracle.rates(Gd, P, 1e-13, 2e7), rtol=1e-9)
    g1 = np.array([[3e-9]])
    np.testing.assert_allclose(oracle.rates_total(g1, [2.0], 1e-12, 1e6), 1e6 * np.log2(1 + 2.0 * 3e-9 / 1e-12),
                               rtol=1e-13)


def test_cost_closed_form_and_validation():
    np.testing.assert_allclose(oracle.cost(np.array([[2.0, 4.0]]), 0.5), [[1.0, 0.5]], rtol=0)
    with pytest.raises(ValueError):
        oracle.cost(np.array([[1.0, 0.0]]), 1.0)
    with pytest.raises(ValueError):
        oracle.cost(np.array([[1.0, -2.0]]), 1.0)


# ------------------------------------------------------------------------------------- median
@pytest.mark.parametrize("n", [1, 2, 7, 10, 1001, 1000])
def test_median_arange_closed_form(n):
    x = np.arange(1, n + 1, dtype=np.float64)
    _rng(n).shuffle(x)
    assert oracle.median(x) == (n + 1) / 2.0


def test_median_duplicates_and_library():
    assert oracle.median([3.0, 1.0, 3.0, 3.0]) == 3.0
    assert oracle.median([5.0, 5.0]) == 5.0
    rng = _rng(1)
    for n in (2, 3, 64, 999, 4096):
        x = rng.lognormal(0.0, 3.0, n)
        assert oracle.median(x) == np.median(x)
    with pytest.raises(ValueError):
        oracle.median([1.0, float("nan")])


# ----------------------------------------------------------------------------- Sinkhorn pins
@pytest.mark.parametrize("eps", [1e-3, 0.3, 50.0])
def test_single_rrh_gives_pi_equal_p(eps):
    # J = 1: the only feasible plan is pi = p (q = sum p), reached after one iteration.
    rng = _rng(2)
    C = rng.uniform(0, 10, (37, 1))
    p = rng.uniform(0.1, 1.0, 37)
    q = np.array([p.sum()])
    # FP64 rounding of (f + g - C)/eps is about (max C / eps) * 2^-52 relative.
    tol = max(1e-13, 40 * C.max() / eps * 2.0 ** -52)
    f, g, it, err = oracle.sinkhorn(C, p, q, eps, tol, 100)
    assert it == 1
    pi = oracle.plan(C, f, g, eps)
    np.testing.assert_allclose(pi[:, 0], p, rtol=tol)


@pytest.mark.parametrize("eps", [0.01, 1.0, 100.0])
def test_separable_cost_gives_product_plan(eps):
    # C_ij = u_i + v_j makes xi rank one, so one iteration gives pi = p q^T / sum(p).
    rng = _rng(3)
    I, J = 23, 9
    u, v = rng.uniform(0, 5, I), rng.uniform(0, 5, J)
    C = u[:, None] + v[None, :]
    p, q = _balanced(rng, I, J)
    f, g, it, err = oracle.sinkhorn(C, p * 3.0, q * 3.0, eps, 1e-13, 100)
    assert it == 1
    pi = oracle.plan(C, f, g, eps)
    np.testing.assert_allclose(pi, 3.0 * np.outer(p, q), rtol=1e-11)


def _two_by_two_closed_form(C, p, q, eps):
    # pi = [[x, p1-x], [q1-x, p2-q1+x]] and pi11 pi22 / (pi12 pi21) = exp(-(C11+C22-C12-C21)/eps).
    p1, p2 = p
    q1 = q[0]
    kap = math.exp(-(C[0, 0] + C[1, 1] - C[0, 1] - C[1, 0]) / eps)
    a = 1.0 - kap
    b = p2 - q1 + kap * (p1 + q1)
    c = -kap * p1 * q1
    lo, hi = max(0.0, q1 - p2), min(p1, q1)
    if abs(a) < 1e-15:
        roots = [-c / b]
    else:
        disc = math.sqrt(b * b - 4 * a * c)
        roots = [(-b + disc) / (2 * a), (-b - disc) / (2 * a)]
    x = [r for r in roots if lo - 1e-15 <= r <= hi + 1e-15]
    assert len(x) == 1
    x = x[0]
    return np.array([[x, p1 - x], [q1 - x, p2 - q1 + x]])


@pytest.mark.parametrize("eps", [0.05, 0.5, 5.0])
def test_two_by_two_closed_form(eps):
    rng = _rng(4)
    for _ in range(5):
        C = rng.uniform(0, 2, (2, 2))
        p, q = _balanced(rng, 2, 2)
        f, g, it, err = oracle.sinkhorn(C, p, q, eps, 1e-15, 100000)
        pi = oracle.plan(C, f, g, eps)
        np.testing.assert_allclose(pi, _two_by_two_closed_form(C, p, q, eps), rtol=1e-9, atol=1e-14)


def _alg1_scaling_domain(C, p, q, eps, tol, max_iter):
    """Algorithm 1 as printed: xi = exp(-C/eps), b = 1, a = p/(xi b), b = q/(xi^T a)."""
    xi = np.exp(-C / eps)
    b = np.ones(C.shape[1])
    k = 0
    while True:
        k += 1
        a = p / (xi @ b)
        b = q / (xi.T @ a)
        pi = a[:, None] * xi * b[None, :]
        err = np.abs(pi.sum(1) - p).sum()
        if err <= tol or k >= max_iter:
            return pi, k, err


@pytest.mark.parametrize("shape", [(7, 4), (4, 9), (31, 13)])
def test_log_domain_matches_printed_scaling_iteration(shape):
    # The oracle's log-domain updates must reproduce the printed a/b iteration iterate by iterate.
    rng = _rng(5)
    I, J = shape
    C = rng.uniform(0, 1, shape)
    p, q = _balanced(rng, I, J)
    eps = 0.2
    for k in (1, 2, 5, 17):
        f, g, it, err = oracle.sinkhorn(C, p, q, eps, 0.0, k)
        pi_ref, k_ref, err_ref = _alg1_scaling_domain(C, p, q, eps, 0.0, k)
        assert it == k == k_ref
        np.testing.assert_allclose(oracle.plan(C, f, g, eps), pi_ref, rtol=1e-12)
        np.testing.assert_allclose(err, err_ref, rtol=1e-8, atol=1e-16)
    f, g, it, err = oracle.sinkhorn(C, p, q, eps, 1e-9, 10000)
    _, k_ref, _ = _alg1_scaling_domain(C, p, q, eps, 1e-9, 10000)
    assert it == k_ref and err <= 1e-9


def test_warm_start_continues_the_iteration():
    rng = _rng(6)
    C = rng.uniform(0, 1, (12, 5))
    p, q = _balanced(rng, 12, 5)
    f6, g6, _, _ = oracle.sinkhorn(C, p, q, 0.1, 0.0, 6)
    f2, g2, _, _ = oracle.sinkhorn(C, p, q, 0.1, 0.0, 2)
    f4, g4, _, _ = oracle.sinkhorn(C, p, q, 0.1, 0.0, 4, g0=g2)
    np.testing.assert_allclose(f4, f6, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(g4, g6, rtol=1e-13, atol=1e-13)


def _lp_value(C, p, q):
    scipy_opt = pytest.importorskip("scipy.optimize")
    I, J = C.shape
    A_eq = np.zeros((I + J, I * J))
    for i in range(I):
        A_eq[i, i * J:(i + 1) * J] = 1.0
    for j in range(J):
        A_eq[I + j, j::J] = 1.0
    res = scipy_opt.linprog(C.ravel(), A_eq=A_eq, b_eq=np.concatenate([p, q]), bounds=(0, None),
                            method="highs")
    assert res.status == 0
    return res.fun, res.x.reshape(I, J)


def _lp_two_columns(C, p, q):
    # Exact LP with two RRHs: give RRH 0 the devices with the largest advantage C_i1 - C_i0.
    order = np.argsort(C[:, 0] - C[:, 1], kind="stable")
    room = q[0]
    val = 0.0
    for i in order:
        take = min(p[i], room)
        val += take * C[i, 0] + (p[i] - take) * C[i, 1]
        room -= take
    return val


def _lp_permutations(C):
    # I = J with uniform marginals: the LP optimum sits on a permutation (Birkhoff-von Neumann).
    n = C.shape[0]
    best = min(sum(C[i, s[i]] for i in range(n)) for s in itertools.permutations(range(n)))
    return best / n


def _reg_cost(C, p, q, eps, tol=1e-12, max_iter=500000):
    f, g, it, err = oracle.sinkhorn(C, p, q, eps, tol, max_iter)
    cost, rho, er, ec = oracle.finalize(C, f, g, p, q, eps)
    return cost, er, f, g


def test_lp_pins_agree_with_each_other():
    rng = _rng(7)
    C = rng.uniform(0, 1, (15, 2))
    p, q = _balanced(rng, 15, 2)
    assert _lp_two_columns(C, p, q) == pytest.approx(_lp_value(C, p, q)[0], rel=1e-9)
    C = rng.uniform(0, 1, (5, 5))
    u = np.full(5, 0.2)
    assert _lp_permutations(C) == pytest.approx(_lp_value(C, u, u)[0], rel=1e-9)


@pytest.mark.parametrize("case", ["highs", "two_columns", "permutations"])
def test_entropic_cost_within_entropy_bound_of_lp(case):
    # 0 <= <C, pi_eps> - OPT <= eps * min(H(p), H(q)) (joint entropy between max and sum of
    # the marginal entropies), and the gap closes as eps -> 0 (Sec. III-B, Prop. 4.1 cited there).
    rng = _rng(8)
    if case == "highs":
        C = rng.uniform(0, 1, (9, 4))
        p, q = _balanced(rng, 9, 4)
        opt = _lp_value(C, p, q)[0]
    elif case == "two_columns":
        C = rng.uniform(0, 1, (25, 2))
        p, q = _balanced(rng, 25, 2)
        opt = _lp_two_columns(C, p, q)
    else:
        C = rng.uniform(0, 1, (6, 6))
        p = q = np.full(6, 1 / 6)
        opt = _lp_permutations(C)
    bound_h = min(_entropy(p), _entropy(q))
    gaps = []
    for eps in (0.2, 0.05, 0.01):
        cost, er, _, _ = _reg_cost(C, p, q, eps)
        slack = 10 * er * C.max() + 1e-12
        gap = cost - opt
        assert -slack <= gap <= eps * bound_h + slack
        gaps.append(gap)
    assert gaps[0] >= gaps[1] >= gaps[2] - 1e-12


def test_small_eps_plan_approaches_lp_plan():
    rng = _rng(9)
    C = rng.uniform(0, 1, (6, 4))
    p, q = _balanced(rng, 6, 4)
    opt, x = _lp_value(C, p, q)
    f, g, it, err = oracle.sinkhorn(C, p, q, 2e-3, 1e-12, 500000)
    pi = oracle.plan(C, f, g, 2e-3)
    assert np.abs(pi - x).sum() < 2e-2


def test_marginals_after_convergence():
    rng = _rng(10)
    C = rng.uniform(0, 3, (40, 11))
    p, q = _balanced(rng, 40, 11)
    f, g, it, err = oracle.sinkhorn(C, p * 7, q * 7, 0.1, 1e-10, 100000)
    assert err <= 1e-10
    pi = oracle.plan(C, f, g, 0.1)
    # columns are exact after the b-update; rows within tol (unit-mass residual)
    np.testing.assert_allclose(pi.sum(0), 7 * q, rtol=1e-12)
    assert np.abs(pi.sum(1) - 7 * p).sum() / 7 <= 1e-10 * 1.0001


def test_dual_objective_never_decreases():
    # Each half-step is an exact block maximisation of the dual
    # D(f, g) = <p, f> + <q, g> - eps * sum exp((f_i + g_j - C_ij)/eps).
    rng = _rng(11)
    C = rng.uniform(0, 1, (20, 6))
    p, q = _balanced(rng, 20, 6)
    eps = 0.05

    def dual(f, g):
        return p @ f + q @ g - eps * np.exp((f[:, None] + g[None, :] - C) / eps).sum()

    g = np.zeros(6)
    f = np.full(20, -1e3)
    last = dual(f, g)
    for _ in range(30):
        f_new, g_new, _, _ = oracle.sinkhorn(C, p, q, eps, 0.0, 1, g0=g)
        d_half = dual(f_new, g)
        d_full = dual(f_new, g_new)
        assert d_half >= last - 1e-13
        assert d_full >= d_half - 1e-13
        last, f, g = d_full, f_new, g_new


def test_invariances():
    rng = _rng(12)
    I, J = 17, 6
    C = rng.uniform(0, 2, (I, J))
    p, q = _balanced(rng, I, J)
    eps = 0.1
    f, g, _, _ = oracle.sinkhorn(C, p, q, eps, 1e-13, 100000)
    pi = oracle.plan(C, f, g, eps)
    # (C, eps) -> (sC, s eps)
    f2, g2, _, _ = oracle.sinkhorn(4.0 * C, p, q, 4.0 * eps, 1e-13, 100000)
    np.testing.assert_allclose(oracle.plan(4.0 * C, f2, g2, 4.0 * eps), pi, rtol=1e-9, atol=1e-15)
    # C -> C + u_i + v_j
    u, v = rng.uniform(-3, 3, I), rng.uniform(-3, 3, J)
    C3 = C + u[:, None] + v[None, :]
    f3, g3, _, _ = oracle.sinkhorn(C3, p, q, eps, 1e-13, 100000)
    np.testing.assert_allclose(oracle.plan(C3, f3, g3, eps), pi, rtol=1e-8, atol=1e-15)
    # row permutation
    perm = rng.permutation(I)
    f4, g4, _, _ = oracle.sinkhorn(C[perm], p[perm], q, eps, 1e-13, 100000)
    np.testing.assert_allclose(oracle.plan(C[perm], f4, g4, eps), pi[perm], rtol=1e-9, atol=1e-15)


def test_cost_increases_with_eps():
    rng = _rng(13)
    C = rng.uniform(0, 1, (30, 7))
    p, q = _balanced(rng, 30, 7)
    costs = [_reg_cost(C, p, q, eps)[0] for eps in (0.01, 0.03, 0.1, 0.3, 1.0)]
    assert all(a <= b + 1e-12 for a, b in zip(costs, costs[1:]))


def test_iteration_cap_and_validation():
    rng = _rng(14)
    C = rng.uniform(0, 1, (8, 3))
    p, q = _balanced(rng, 8, 3)
    f, g, it, err = oracle.sinkhorn(C, p, q, 0.01, 0.0, 7)
    assert it == 7
    for bad in (dict(eps=0.0), dict(eps=-1.0), dict(tol=-1.0), dict(max_iter=0)):
        kw = dict(eps=0.1, tol=1e-6, max_iter=10)
        kw.update(bad)
        with pytest.raises(ValueError):
            oracle.sinkhorn(C, p, q, kw["eps"], kw["tol"], kw["max_iter"])
    p0 = p.copy()
    p0[2] = 0.0
    with pytest.raises(ValueError):
        oracle.sinkhorn(C, p0, q, 0.1, 1e-6, 10)


# --------------------------------------------------------------------------------- finalize
def test_finalize_on_product_plan():
    rng = _rng(15)
    I, J = 13, 5
    u, v = rng.uniform(0, 5, I), rng.uniform(0, 5, J)
    C = u[:, None] + v[None, :]
    p, q = _balanced(rng, I, J)
    eps = 0.7
    f, g, _, _ = oracle.sinkhorn(C, p, q, eps, 1e-14, 10)
    cost, rho, er, ec = oracle.finalize(C, f, g, p, q, eps)
    np.testing.assert_allclose(cost, p @ C @ q, rtol=1e-12)
    np.testing.assert_allclose(rho, q * (p @ C), rtol=1e-12)
    assert er < 1e-14 and ec < 1e-14


def test_finalize_residuals_of_a_perturbed_plan_with_mass_three():
    """Residuals are total absolute residuals per unit of mass (Sec. III-C; Eqs. (3)-(4)).

    A separable cost C_ij = u_i + v_j and potentials f_i = u_i + eps log(p_i (1 + d_i)),
    g_j = v_j + eps log(q_j / M) give the product plan pi_ij = p_i (1 + d_i) q_j / M with
    M = sum p = sum q = 3.  Its rows are p_i (1 + d_i) and its columns q_j (1 + sum_i p_i d_i / M),
    so the row and column L1 residuals divided by the mass are sum_i |p_i d_i| / M and
    |sum_i p_i d_i| / M; the cost and loads follow from the product form."""
    rng = _rng(16)
    I, J, M = 11, 6, 3.0
    u, v = rng.uniform(0, 4, I), rng.uniform(0, 4, J)
    C = u[:, None] + v[None, :]
    p, q = _balanced(rng, I, J)
    p, q = M * p, M * q
    d = rng.uniform(-0.2, 0.1, I)
    eps = 0.4
    f = u + eps * np.log(p * (1.0 + d))
    g = v + eps * np.log(q / M)
    cost, rho, er, ec = oracle.finalize(C, f, g, p, q, eps)
    P, Q = p * (1.0 + d), q / M
    np.testing.assert_allclose(er, np.abs(p * d).sum() / M, rtol=1e-12)
    np.testing.assert_allclose(ec, abs((p * d).sum()) / M, rtol=1e-12)
    assert er > 1e-3 and ec > 1e-3
    np.testing.assert_allclose(cost, P @ u + P.sum() * (Q @ v), rtol=1e-12)
    np.testing.assert_allclose(rho, Q * (P @ u + v * P.sum()), rtol=1e-12)


# ------------------------------------------------------------------------- maxSINR / Lemma 1
def test_maxsinr_brute_force_and_ties():
    rng = _rng(16)
    R = rng.uniform(0, 1, (50, 7))
    R[3, [1, 4]] = 2.0  # a tie: lowest index wins
    R[9, :] = 1.0       # all tied
    C = 1.0 / R
    lam = rng.uniform(0.1, 1, 50)
    assoc, Lam, tot = oracle.maxsinr(R, C, lam)
    np.testing.assert_array_equal(assoc, np.argmax(R, axis=1))
    assert assoc[3] == 1 and assoc[9] == 0
    np.testing.assert_allclose(Lam, np.bincount(assoc, weights=lam, minlength=7), rtol=1e-14)
    np.testing.assert_allclose(tot, (lam * C[np.arange(50), assoc]).sum(), rtol=1e-14)


def test_lemma1_bounds_on_config1_channel():
    # Lemma 1 (Sec. IV): with q = Lambda (the maxSINR traffic) and C = 1/(mu R), the OT optimum
    # equals the maxSINR total load sum_i lambda_i min_j C_ij.  The entropic plan's cost therefore
    # lies in [total, total + eps * min(H(p), H(q))] and shrinks toward it as eps decreases.
    inst = ins.config1()
    R = oracle.rates(inst.G, inst.P, inst.N0, inst.W_hz)
    C = oracle.cost(R, inst.mu)
    assoc, Lam, tot = oracle.maxsinr(R, C, inst.lam)
    keep = Lam > 0
    C, Lam = C[:, keep], Lam[keep]
    np.testing.assert_allclose(tot, (inst.lam * C.min(axis=1)).sum(), rtol=1e-12)
    scale = np.median(C.min(axis=1))
    gaps = []
    for rel in (3.0, 1.0, 0.5):
        eps = rel * scale
        cost, er, _, _ = _reg_cost(C, inst.lam, Lam, eps, tol=1e-9, max_iter=200000)
        slack = er * np.quantile(C.min(axis=1), 0.99) * 10
        assert tot - slack <= cost <= tot + eps * min(_entropy(inst.lam), _entropy(Lam)) + slack
        gaps.append(cost - tot)
    assert gaps[0] > gaps[1] > gaps[2]


# --------------------------------------------------------------------------------- Alg. 2
def test_adaptive_one_step_is_plain_sinkhorn_with_equal_split():
    rng = _rng(17)
    C = rng.uniform(0, 1, (20, 4))
    lam = rng.uniform(0.1, 1, 20)
    lam /= lam.sum()
    f, g, q, ml = oracle.adaptive(C, lam, 0.1, 1e-12, 10000, 1, 0.01)
    np.testing.assert_allclose(q, np.full(4, 0.25), rtol=1e-15)
    f2, g2, _, _ = oracle.sinkhorn(C, lam, np.full(4, 0.25), 0.1, 1e-12, 10000)
    np.testing.assert_allclose(f, f2, rtol=1e-14)
    cost, rho, _, _ = oracle.finalize(C, f2, g2, lam, np.full(4, 0.25), 0.1)
    assert ml[0] == pytest.approx(rho.max(), rel=1e-14)


def test_adaptive_moves_delta_off_the_most_loaded_rrh():
    rng = _rng(18)
    C = rng.uniform(0, 1, (30, 3))
    C[:, 0] *= 0.2  # RRH 0 is cheap for everyone: the equal split overloads it
    lam = np.full(30, 1 / 30)
    delta = 0.02
    f, g, q, ml = oracle.adaptive(C, lam, 0.05, 1e-12, 100000, 2, delta)
    np.testing.assert_allclose(q.sum(), 1.0, rtol=1e-14)
    f1, g1, _, _ = oracle.sinkhorn(C, lam, np.full(3, 1 / 3), 0.05, 1e-12, 100000)
    _, rho1, _, _ = oracle.finalize(C, f1, g1, lam, np.full(3, 1 / 3), 0.05)
    js = int(np.argmax(rho1))
    want = np.full(3, 1 / 3 + delta / 2)
    want[js] = 1 / 3 - delta
    np.testing.assert_allclose(q, want, rtol=1e-13)


def test_adaptive_trace_matches_its_own_steps():
    # the trace's j* is the argmax (lowest index on ties) of the same step's loads, its max
    # load is that entry, and replaying the q updates from the trace reproduces the final q
    rng = _rng(19)
    C = rng.uniform(0, 1, (40, 5))
    C[:, 1] *= 0.3
    lam = rng.uniform(0.5, 1.5, 40)
    delta = 0.01 * lam.sum()
    f, g, q, ml, js, rho = oracle.adaptive_trace(C, lam, 0.05, 1e-12, 100000, 6, delta)
    for s in range(6):
        assert js[s] == int(np.argmax(rho[s]))
        assert ml[s] == rho[s, js[s]]
    qq = np.full(5, lam.sum() / 5)
    for s in range(5):
        d = delta if delta < qq[js[s]] else 0.5 * qq[js[s]]
        qq = qq + d / 4
        qq[js[s]] -= d + d / 4
    np.testing.assert_allclose(q, qq, rtol=1e-13)
    # the final plan is the last solve's, with the q it used
    f2, g2, _, _ = oracle.sinkhorn(C, lam, q, 0.05, 1e-12, 100000, g0=None)
    _, rho2, _, _ = oracle.finalize(C, f2, g2, lam, q, 0.05)
    np.testing.assert_allclose(rho2, rho[-1], rtol=1e-9)


def test_adaptive_half_move_when_delta_exceeds_the_target():
    # delta larger than every target: each step halves the chosen RRH's target (mass kept)
    rng = _rng(20)
    C = rng.uniform(0, 1, (25, 3))
    lam = np.full(25, 0.04)
    _, _, q, _, js, _ = oracle.adaptive_trace(C, lam, 0.1, 1e-12, 100000, 2, 5.0)
    want = np.full(3, 1 / 3)
    want += (1 / 6) / 2
    want[js[0]] = 1 / 3 - 1 / 6
    np.testing.assert_allclose(q, want, rtol=1e-14)
    assert q.sum() == pytest.approx(1.0, rel=1e-15)


# ------------------------------------------------------------------ completion time (Sec. II-B)
def test_completion_time_hand_worked_assignment():
    # device 0 -> RRH 0, device 1 -> RRH 1 (hard association)
    C = np.array([[0.5, 2.0], [3.0, 0.25]])
    lam = np.array([0.4, 2.0])
    x = np.array([[0.4, 0.0], [0.0, 2.0]])
    T, rho = oracle.completion_time(C, x, lam)
    # rho_0 = 0.4 * 0.5 = 0.2, rho_1 = 2 * 0.25 = 0.5
    np.testing.assert_allclose(rho, [0.2, 0.5], rtol=1e-15)
    # T_0 = 0.5 / 0.8, T_1 = 0.25 / 0.5
    assert T == pytest.approx(0.5 * (0.625 + 0.5), rel=1e-15)


def test_completion_time_split_plan_and_overload():
    C = np.array([[1.0, 2.0], [0.5, 0.5]])
    lam = np.array([0.2, 0.4])
    x = np.array([[0.1, 0.1], [0.0, 0.4]])  # device 0 splits its time equally
    T, rho = oracle.completion_time(C, x, lam)
    np.testing.assert_allclose(rho, [0.1, 0.4], rtol=1e-15)  # 0.1 * 1; 0.1 * 2 + 0.4 * 0.5
    T0 = 0.5 * 1.0 / 0.9 + 0.5 * 2.0 / 0.6
    T1 = 1.0 * 0.5 / 0.6
    assert T == pytest.approx(0.5 * (T0 + T1), rel=1e-14)
    # RRH 1 overloaded: every device that uses it waits forever
    T, rho = oracle.completion_time(C * 4, x, lam)
    assert rho[1] >= 1.0 and math.isinf(T)
    # an overloaded RRH that nobody uses changes nothing for the others
    x2 = np.array([[0.2, 0.0], [0.4, 0.0]])
    C2 = np.array([[1.0, 50.0], [0.5, 50.0]])
    T, rho = oracle.completion_time(C2, x2, lam)
    assert rho[1] == 0.0 and T == pytest.approx(0.5 * (1.0 / 0.6 + 0.5 / 0.6), rel=1e-14)


def test_completion_time_of_maxsinr_against_brute_force():
    # the maxSINR association as a 0/1 plan, summed device by device in Python
    inst = ins.config1()
    I = 200
    R = oracle.rates(inst.G[:I], inst.P, inst.N0, inst.W_hz)
    C = oracle.cost(R, inst.mu)
    lam = inst.lam[:I] * 20.0  # enough traffic for visible queueing
    assoc, Lam, tot = oracle.maxsinr(R, C, lam)
    x = np.zeros_like(C)
    x[np.arange(I), assoc] = lam
    T, rho = oracle.completion_time(C, x, lam)
    rho_bf = np.zeros(C.shape[1])
    for i in range(I):
        rho_bf[assoc[i]] += lam[i] * C[i, assoc[i]]
    assert rho_bf.max() < 1.0
    np.testing.assert_allclose(rho, rho_bf, rtol=1e-13)
    T_bf = sum(C[i, assoc[i]] / (1.0 - rho_bf[assoc[i]]) for i in range(I)) / I
    assert T == pytest.approx(T_bf, rel=1e-13)
    assert rho.sum() == pytest.approx(tot, rel=1e-13)  # Lemma 1: total load of maxSINR


# ------------------------------------------------------------------- Euclidean cost (Sec. IV)
def test_euclid_cost_triangles():
    dev = np.array([[0.0, 0.0], [3.0, 4.0], [-6.0, 8.0]])
    rrh = np.array([[0.0, 0.0], [3.0, 0.0]])
    C = oracle.euclid_cost(dev, rrh)
    want = np.array([[0.0, 3.0], [5.0, 4.0], [10.0, math.hypot(9.0, 8.0)]])
    np.testing.assert_allclose(C, want, rtol=1e-15)
    # swapping the roles transposes the matrix
    np.testing.assert_allclose(oracle.euclid_cost(rrh, dev), C.T, rtol=0, atol=0)
