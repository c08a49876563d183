"""Oracle proj_S1 (KKT solve) against the definition of a projection onto an
affine set: feasibility, idempotence, optimality, and a null-space method."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.problem import Problem
from oracle.s1 import S1Projector
from paper_2212_01110_gb300 import workloads


def simulate(P, x0, u_of):
    """A point of S1 built by running the dynamics x^c = A^c x^i + B^c u^i
    (Eq. (finite-horizon-evolution-2)) with given inputs."""
    t = P.tree
    x = np.zeros((t.n, P.nx))
    u = {}
    x[0] = x0
    for i in sorted(range(t.n), key=lambda k: t.stage[k]):
        if t.children[i]:
            u[i] = u_of(i)
            for c in t.children[i]:
                x[c] = P.A[c] @ x[i] + P.B[c] @ u[i]
    z1 = np.concatenate([x.ravel()] + [u[i] for i in t.nonleaf])
    return z1


CASES = [workloads.small_binary(0), workloads.with_tree(workloads.fig1_tree(), seed=2),
         workloads.random_tree(4, N=4, max_branch=3, nx=5, nu=2),
         workloads.random_tree(9, N=6, max_branch=2, nx=3, nu=3, chain_after=2)]


@pytest.mark.parametrize("d", CASES)
def test_projection_properties(d):
    P = Problem(d)
    S = S1Projector(P)
    rng = np.random.default_rng(1)
    x0 = d["x0"]
    zb = rng.standard_normal(S.n1) * 2
    z = S.project(zb, x0)
    h = S.rhs_h(x0)
    assert np.max(np.abs(S.G @ z - h)) < 1e-12 * max(1, np.max(np.abs(z)))
    np.testing.assert_allclose(S.project(z, x0), z, atol=1e-11)
    # optimality: zbar - P(zbar) is orthogonal to every feasible direction
    for _ in range(5):
        w = simulate(P, np.zeros(P.nx), lambda i: rng.standard_normal(P.nu))
        assert abs((zb - z) @ w) < 1e-10 * np.linalg.norm(zb - z) * np.linalg.norm(w)
    # a feasible point built by simulation is its own projection
    f = simulate(P, x0, lambda i: rng.standard_normal(P.nu))
    np.testing.assert_allclose(S.project(f, x0), f, atol=1e-10)


def test_nullspace_method():
    d = workloads.with_tree(workloads.fig1_tree(), seed=5, nx=2, nu=2)
    P = Problem(d)
    S = S1Projector(P)
    G = S.G.toarray()
    h = S.rhs_h(d["x0"])
    Z = sla.null_space(G)
    zp = np.linalg.lstsq(G, h, rcond=None)[0]
    rng = np.random.default_rng(3)
    zb = rng.standard_normal(S.n1)
    ref = zp + Z @ (Z.T @ (zb - zp))
    np.testing.assert_allclose(S.project(zb, d["x0"]), ref, atol=1e-12)
