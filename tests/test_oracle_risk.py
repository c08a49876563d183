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
