"""AV@R (Sec. "Risk measures"): four independent evaluations agree."""
import numpy as np
import pytest

from oracle import risk


@pytest.mark.parametrize("seed", range(12))
def test_avar_four_ways(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 7))
    Z = rng.standard_normal(n) * 3
    pi = rng.dirichlet(np.ones(n))
    for a in [1.0, 0.73, 0.5, 0.2, 0.05, 1e-3]:
        v_sort = risk.avar_sort(Z, pi, a)
        v_t = risk.avar_min_t(Z, pi, a)
        v_lp = risk.avar_lp(Z, pi, a)
        v_bf = risk.avar_bruteforce(Z, pi, a)
        assert abs(v_sort - v_bf) < 1e-12 * max(1, abs(v_bf))
        assert abs(v_t - v_bf) < 1e-12 * max(1, abs(v_bf))
        assert abs(v_lp - v_bf) < 1e-8 * max(1, abs(v_bf))


def test_avar_special_cases():
    Z = np.array([1.0, -2.0, 5.0, 0.5])
    pi = np.array([0.1, 0.2, 0.3, 0.4])
    assert abs(risk.avar_sort(Z, pi, 1.0) - pi @ Z) < 1e-14      # a = 1: expectation
    assert risk.avar_sort(Z, pi, 0.0) == 5.0                       # a = 0: maximum
    assert abs(risk.avar_lp(Z, pi, 0.0) - 5.0) < 1e-9
    assert abs(risk.avar_sort(Z, pi, 0.29) - 5.0) < 1e-12          # a <= pi_max: the max


def _path_costs(P, x, u):
    """Per leaf: absolute probability and the cost along its path (stage
    costs of every edge on the path plus the terminal cost)."""
    t = P.tree
    out = []
    for j in range(t.n):
        if t.children[j]:
            continue
        cost = float(x[j] @ P.QNmat(j) @ x[j])
        prob = 1.0
        c = j
        while c != 0:
            a = int(t.anc[c])
            cost += float(x[a] @ P.Qmat(c) @ x[a] + u[a] @ P.Rmat(c) @ u[a])
            prob *= t.prob[c]
            c = a
        out.append((prob, cost))
    return out


@pytest.mark.parametrize("seed", range(3))
def test_nested_value_special_cases_by_scenario_enumeration(seed):
    """The nested value of a trajectory (Eq. (original-problem)), which the
    convergence pins compare s^0 with: with a = 1 at every node it is the
    expected cost over the scenarios (leaf paths weighted by their absolute
    probabilities), with a = 0 the cost of the worst scenario."""
    from oracle.problem import Problem
    from paper_2212_01110_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    d = W.random_tree(10 + seed, N=3, max_branch=3, nx=3, nu=2)
    n = len(d["anc"])
    x = rng.standard_normal((n, 3))
    u = rng.standard_normal((n, 2))
    paths = _path_costs(Problem(d), x, u)
    d1 = dict(d, a=np.ones(n))
    v1, _ = risk.nested_value(Problem(d1), x, u)
    assert abs(v1 - sum(p * c for p, c in paths)) <= 1e-12 * max(1.0, abs(v1))
    d0 = dict(d, a=np.zeros(n))
    v0, _ = risk.nested_value(Problem(d0), x, u)
    assert abs(v0 - max(c for _, c in paths)) <= 1e-12 * max(1.0, abs(v0))
