"""Oracle T: firmly nonexpansive in the M-metric (Sec. "The Chambolle-Pock
method"); prox_f pieces; fixed-point residual identities."""
import numpy as np
import pytest

from oracle.cp import CP, vanilla_cp
from oracle.problem import Problem
from paper_2212_01110_gb300 import workloads


@pytest.mark.parametrize("d", [workloads.small_binary(0),
                               workloads.random_tree(2, N=3, max_branch=3, nx=3, nu=2)])
def test_T_fne_in_M(d):
    P = Problem(d)
    cp = CP(P)
    rng = np.random.default_rng(0)
    n = cp.n_z + cp.n_eta
    for _ in range(10):
        v = rng.standard_normal(n) * 3
        w = rng.standard_normal(n) * 3
        Tv, Tw = cp.T(v, d["x0"]), cp.T(w, d["x0"])
        lhs = cp.inner_M(Tv - Tw, Tv - Tw)
        rhs = cp.inner_M(Tv - Tw, v - w)
        assert lhs <= rhs + 1e-10 * abs(rhs)
        assert cp.inner_M(v - w, v - w) > 0  # M positive definite for alpha ||L|| < 1


def test_prox_f_pieces():
    d = workloads.small_binary(1)
    P = Problem(d)
    cp = CP(P)
    rng = np.random.default_rng(1)
    z = rng.standard_normal(cp.n_z)
    zp = cp.prox_f(z, d["x0"])
    assert zp[0] == z[0] - cp.alpha                         # prox of alpha * s^0
    np.testing.assert_allclose(cp.prox_f(zp + 0.0, d["x0"])[1:], zp[1:], atol=1e-12)  # projections idempotent


def test_vanilla_cp_decreases_residual():
    d = workloads.small_binary(0)
    P = Problem(d)
    cp = CP(P)
    n = cp.n_z + cp.n_eta
    v, xi_a = vanilla_cp(cp, np.zeros(n), d["x0"], 50)
    v, xi_b = vanilla_cp(cp, v, d["x0"], 2000)
    assert xi_b < 1e-2 * xi_a
