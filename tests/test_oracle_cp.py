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


@pytest.mark.parametrize("d", [workloads.small_binary(0),
                               workloads.random_tree(2, N=3, max_branch=3, nx=3, nu=2),
                               workloads.risk_measures(workloads.small_binary(1, a=0.5), "tv", radius=0.3)])
def test_residual_certificate_inclusions(d):
    """The two quantities of the termination rule certify the pair
    (z+, eta+) = T(z, eta) (Sec. "The Chambolle-Pock method"):
      xi_p in d f(z+) + L* eta+,    xi_d in d g*(eta+) - L z+,
    with f = s^0 + indicator of S1 x S2 and g = indicator of S3.  Checked
    from the definitions, not from the prox formulas: the s^0 entry of
    xi_p - L* eta+ is 1; its z_1 part is orthogonal to the null space of the
    dynamics constraints (scipy's null_space of the constraint matrix); its
    z_2 part of every nonleaf node lies in the row space of the S2 matrix
    (its component in ker M, by pseudoinverse, vanishes); and
    w = xi_d + L z+ lies in S3 with eta+ in the normal cone of S3 at w,
    i.e. w = proj_S3(w + eta+)."""
    from scipy.linalg import null_space
    from oracle.cones import proj_S3, s2_matrix, z2_block
    P = Problem(d)
    cp = CP(P)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(cp.n_z + cp.n_eta) * 2
    Tv = cp.T(v, d["x0"])
    st = cp.stats(v, Tv)
    rz, re = cp.split(st["r"])
    zp, ep = cp.split(Tv)
    xi_p = rz / cp.alpha - cp.Lt @ re
    xi_d = re / cp.alpha - cp.L @ rz
    g = xi_p - cp.Lt @ ep
    lay = P.lay
    assert abs(g[lay.s0] - 1.0) < 1e-10
    sl = slice(cp.S1.off, cp.S1.off + cp.S1.n1)
    N = null_space(cp.S1.G.toarray())
    assert np.max(np.abs(N.T @ g[sl])) < 1e-9 * max(1.0, np.max(np.abs(g)))
    for i in P.tree.nonleaf:
        M = s2_matrix(P, i)
        gi = g[z2_block(P, i)]
        assert np.max(np.abs(gi - np.linalg.pinv(M) @ (M @ gi))) < 1e-9 * max(1.0, np.max(np.abs(gi)))
    w = xi_d + cp.L @ zp
    assert np.max(np.abs(proj_S3(w, P) - w)) < 1e-9 * max(1.0, np.max(np.abs(w)))
    assert np.max(np.abs(proj_S3(w + ep, P) - w)) < 1e-9 * max(1.0, np.max(np.abs(w)))
