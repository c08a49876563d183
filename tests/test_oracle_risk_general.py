"""The oracle with general conic risk measures (b, E, F, K) at the nonleaf
nodes (Sec. "Conic representation of risk measures"; S2 = ker [[E^T, -I, -I],
[F^T, 0, 0]], y in (K^i)* in S3), pinned by facts independent of the
assembly:
  * AV@R written in the general form gives the built-in AV@R's L, S2
    projection and solution;
  * the conic dual value (Eq. (dual_risk), an LP) of the two risk measures
    used equals their closed forms: lam E + (1 - lam) AV@R_a by sorting, the
    total-variation worst case by moving mass from the smallest to the
    largest outcome;
  * at convergence s^0 equals the nested value of the returned trajectory
    under the closed forms, and the trajectory satisfies the dynamics;
  * the total-variation ball of radius 0 is the expectation: tree LQR."""
import numpy as np
import pytest

from oracle import risk
from oracle.cones import proj_S2
from oracle.cp import CP
from oracle.linop import build_L
from oracle.lqr import tree_lqr
from oracle.problem import Problem
from oracle.spock import Settings, spock
from paper_2212_01110_gb300 import workloads

TIGHT = Settings(eps_abs=1e-10, eps_rel=1e-10, max_iter=40000)


def mean_avar(Z, pi, a, lam):
    return lam * float(pi @ Z) + (1 - lam) * risk.avar_sort(Z, pi, a)


def tv_worst(Z, pi, r):
    """max mu'Z over the simplex with ||mu - pi||_1 <= r: move
    d = min(r / 2, 1 - pi_top) from the smallest outcomes to the largest."""
    Z = np.asarray(Z, float)
    mu = np.array(pi, float)
    top = int(np.argmax(Z))
    d = min(r / 2.0, 1.0 - mu[top])
    left = d
    for k in np.argsort(Z, kind="stable"):
        if k == top or left <= 0:
            continue
        take = min(mu[k], left)
        mu[k] -= take
        left -= take
    mu[top] += d - left
    return float(mu @ Z)


def _closed_form(P, kind, lam=0.5, radius=0.3):
    t = P.tree

    def rho(i, Z):
        pi = t.prob[t.children[i]]
        return mean_avar(Z, pi, P.a[i], lam) if kind == "mean_avar" else tv_worst(Z, pi, radius)
    return rho


def test_avar_in_general_form_is_the_builtin():
    d = workloads.with_tree(workloads.fig1_tree(), seed=4, nx=3, nu=2, a=0.3)
    d["a"] = np.linspace(0.2, 0.8, len(d["anc"]))
    Pb, Pg = Problem(d), Problem(workloads.risk_measures(d, "avar"))
    assert Pg.general_risk
    np.testing.assert_array_equal(build_L(Pg).toarray(), build_L(Pb).toarray())
    z = np.random.default_rng(0).standard_normal(Pb.lay.n_z)
    np.testing.assert_allclose(proj_S2(z, Pg), proj_S2(z, Pb), atol=1e-12)
    rb = spock(CP(Pb), d["x0"], s=TIGHT)
    rg = spock(CP(Pg), d["x0"], s=TIGHT)
    assert rb.status == rg.status == "converged"
    assert abs(rb.v[0] - rg.v[0]) <= 1e-9 * max(1.0, abs(rb.v[0]))


@pytest.mark.parametrize("seed", range(6))
def test_conic_values_equal_closed_forms(seed):
    rng = np.random.default_rng(seed)
    m = 2 + seed % 4
    pi = rng.dirichlet(np.ones(m))
    Z = rng.standard_normal(m) * 3
    a = float(rng.uniform(0.1, 0.9))
    d = dict(anc=np.array([-1] + [0] * m, np.int32), prob=np.concatenate([[1.0], pi]), a=np.full(m + 1, a))
    for kind, ref in (("mean_avar", mean_avar(Z, pi, a, 0.4)), ("tv", tv_worst(Z, pi, 0.25))):
        r = workloads.risk_measures(d, kind, lam=0.4, radius=0.25)["risk"][0]
        val = risk.conic_lp(Z, np.asarray(r["b"]), np.asarray(r["E"]), np.asarray(r["F"]), r["kp"])
        assert abs(val - ref) <= 1e-9 * max(1.0, abs(ref)), (kind, val, ref)


@pytest.mark.parametrize("kind,seed", [("mean_avar", 0), ("tv", 1), ("tv", 2)])
def test_solution_attains_the_nested_value(kind, seed):
    base = workloads.small_binary(seed, a=0.5)
    d = workloads.risk_measures(base, kind, lam=0.5, radius=0.3)
    P = Problem(d)
    res = spock(CP(P), d["x0"], s=TIGHT)
    assert res.status == "converged"
    x, u = risk.trajectory(P, res.v[: P.lay.n_z])
    t = P.tree
    np.testing.assert_allclose(x[0], d["x0"], atol=1e-8)
    for c in t.nonroot:
        p = int(t.anc[c])
        np.testing.assert_allclose(x[c], P.A[c] @ x[p] + P.B[c] @ u[p], atol=1e-7)
    val, _ = risk.nested_value(P, x, u, risk=_closed_form(P, kind))
    assert abs(val - res.v[0]) <= 1e-6 * max(1.0, abs(val))


def test_tv_radius_zero_is_the_expectation():
    base = workloads.random_tree(6, N=3, max_branch=3, nx=3, nu=2, a_range=(1.0, 1.0))
    n = len(base["anc"])
    big = 1e6
    base = dict(base)
    base["xmin"], base["xmax"] = -big * np.ones((n, base["nx"])), big * np.ones((n, base["nx"]))
    base["umin"], base["umax"] = -big * np.ones((n, base["nu"])), big * np.ones((n, base["nu"]))
    d = workloads.risk_measures(base, "tv", radius=0.0)
    P = Problem(d)
    res = spock(CP(P), d["x0"], s=TIGHT)
    assert res.status == "converged"
    V, x, u = tree_lqr(P, d["x0"])
    assert abs(res.v[0] - V) <= 1e-7 * max(1.0, abs(V))


def test_norm_with_risk_measures_matches_power_iteration():
    """||L|| from the column-group blocks, with the (y, s) blocks of general
    b vectors (total variation: ny = 3m + 2), against a power iteration."""
    from oracle.linop import norm_L_blocks, norm_L_power
    d = workloads.risk_measures(workloads.general_random(workloads.small_binary(3), seed=4), "tv", radius=0.4)
    P = Problem(d)
    ref = norm_L_power(build_L(P), iters=20000)
    assert abs(norm_L_blocks(P) - ref) <= 1e-7 * ref


def test_expectation_as_a_conic_risk_measure_is_tree_lqr():
    """The expectation written as a conic risk measure with ambiguity set
    {pi}: b = (pi, -pi), E = [I; -I], K = R^2m_+ (mu <= pi and mu >= pi), no F.
    With loose constraints the solve is the tree LQR."""
    base = workloads.small_binary(2, a=0.5)
    n = len(base["anc"])
    big = 1e6
    base = dict(base)
    base["xmin"], base["xmax"] = -big * np.ones((n, base["nx"])), big * np.ones((n, base["nx"]))
    base["umin"], base["umax"] = -big * np.ones((n, base["nu"])), big * np.ones((n, base["nu"]))
    kids = [[c for c in range(1, n) if base["anc"][c] == i] for i in range(n)]
    risk = [None] * n
    for i in range(n):
        if kids[i]:
            pi = np.asarray(base["prob"])[kids[i]]
            m = len(pi)
            risk[i] = dict(b=np.concatenate([pi, -pi]), E=np.vstack([np.eye(m), -np.eye(m)]),
                           F=np.zeros((2 * m, 0)), kp=2 * m)
    d = dict(base, risk=risk)
    P = Problem(d)
    res = spock(CP(P), d["x0"], s=TIGHT)
    assert res.status == "converged"
    V, _, _ = tree_lqr(Problem(dict(base, a=np.ones(n))), d["x0"])
    assert abs(res.v[0] - V) <= 1e-7 * max(1.0, abs(V))
