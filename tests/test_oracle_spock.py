"""Oracle SPOCK (Algorithm 3) pinned by closed forms and brute force:
tree LQR for a = 1 with inactive constraints, a one-step problem solved by
golden section, the nested AV@R value of the returned trajectory (Eq.
(original-problem)), Anderson's multi-secant property."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import risk
from oracle.cp import CP, vanilla_cp
from oracle.lqr import tree_lqr
from oracle.problem import Problem
from oracle.spock import Anderson, Settings, spock
from paper_2212_01110_gb300 import workloads

TIGHT = Settings(eps_abs=1e-10, eps_rel=1e-10, max_iter=20000)


def _solve(d, s=TIGHT):
    P = Problem(d)
    cp = CP(P)
    res = spock(cp, d["x0"], s=s)
    return P, cp, res


@pytest.mark.parametrize("d", [
    workloads.small_binary(0, a=1.0),
    workloads.with_tree(workloads.fig1_tree(), seed=4, nx=3, nu=2, a=1.0),
    workloads.random_tree(6, N=3, max_branch=3, nx=3, nu=2, a_range=(1.0, 1.0)),
    workloads.random_tree(7, N=5, max_branch=1, nx=3, nu=2, a_range=(1.0, 1.0)),  # single-child chain: deterministic LQR
])
def test_tree_lqr_closed_form(d):
    d = dict(d)
    n = len(d["anc"])
    big = 1e6
    d["xmin"], d["xmax"] = -big * np.ones((n, d["nx"])), big * np.ones((n, d["nx"]))
    d["umin"], d["umax"] = -big * np.ones((n, d["nu"])), big * np.ones((n, d["nu"]))
    P, cp, res = _solve(d)
    assert res.status == "converged"
    V, x, u = tree_lqr(P, d["x0"])
    s0 = res.v[0]
    assert abs(s0 - V) <= 1e-7 * max(1.0, abs(V))
    xs, us = risk.trajectory(P, res.v[: cp.n_z])
    np.testing.assert_allclose(us[0], u[0], atol=1e-6)
    np.testing.assert_allclose(xs, x, atol=1e-6)


@pytest.mark.parametrize("seed", range(4))
def test_one_step_bruteforce(seed):
    """N = 1, nx = nu = 1, 2-3 children, constraints possibly active:
    V(u) = AV@R_a over children of Q x0^2 + R u^2 + Q_N (A x0 + B u)^2 on the
    feasible interval of u, minimised by golden section."""
    rng = np.random.default_rng(seed)
    m = 2 + seed % 2
    anc = np.array([-1] + [0] * m, np.int32)
    d = workloads.with_tree(anc, seed=seed, nx=1, nu=1, a=float(rng.uniform(0.2, 0.9)), box=(5.0, 0.6))
    d["x0"] = np.array([1.5])
    d["A"][1:, 0, 0] = rng.uniform(0.8, 1.3, size=m)
    d["B"][1:, 0, 0] = rng.uniform(0.5, 1.5, size=m)
    P, cp, res = _solve(d)
    assert res.status == "converged"
    x0 = d["x0"][0]
    lo, hi = d["umin"][0, 0], d["umax"][0, 0]
    for c in range(1, m + 1):  # leaf box |A x0 + B u| <= 5
        a_, b_ = d["A"][c, 0, 0], d["B"][c, 0, 0]
        lo = max(lo, (-5 - a_ * x0) / b_)
        hi = min(hi, (5 - a_ * x0) / b_)

    def V(u):
        Z = [d["Q"][c, 0] * x0 ** 2 + d["R"][c, 0] * u ** 2 + d["QN"][c, 0] * (d["A"][c, 0, 0] * x0 + d["B"][c, 0, 0] * u) ** 2
             for c in range(1, m + 1)]
        return risk.avar_sort(np.array(Z), d["prob"][1:], d["a"][0])

    grid = np.linspace(lo, hi, 2001)
    k = int(np.argmin([V(g) for g in grid]))
    br = minimize_scalar(V, bounds=(grid[max(k - 1, 0)], grid[min(k + 1, 2000)]), method="bounded",
                         options={"xatol": 1e-12})
    assert abs(res.v[0] - br.fun) < 1e-7 * max(1, abs(br.fun))
    assert abs(res.v[P.lay.u[0][0]] - br.x) < 1e-5


@pytest.mark.parametrize("d", [workloads.small_binary(0), workloads.small_binary(3, a=0.2),
                               workloads.random_tree(8, N=3, max_branch=3, nx=3, nu=2, a_range=(0.0, 1.0))])
def test_nested_value_and_kkt(d):
    """At convergence: s^0 equals the nested AV@R cost of the returned
    trajectory; dynamics hold exactly; L z lies (almost) in S3."""
    from oracle.cones import proj_S3
    P, cp, res = _solve(d)
    assert res.status == "converged"
    z = res.v[: cp.n_z]
    x, u = risk.trajectory(P, z)
    V, _ = risk.nested_value(P, x, u)
    assert abs(z[0] - V) <= 1e-7 * max(1.0, abs(V))
    S = cp.S1
    assert np.max(np.abs(S.G @ z[1:1 + S.n1] - S.rhs_h(d["x0"]))) < 1e-10
    Lz = cp.L @ z
    assert np.max(np.abs(proj_S3(Lz, P) - Lz)) < 1e-7
    # the same problem solved by vanilla CP reaches the same cost
    v, xi = vanilla_cp(cp, np.zeros(cp.n_z + cp.n_eta), d["x0"], 20000)
    assert abs(v[0] - z[0]) < 1e-5 * max(1, abs(z[0]))


def test_anderson_multisecant():
    """d = -c - (M^P - M^R) gamma satisfies the multi-secant condition: for
    c equal to a stored column of M^R, d is minus the matching column of M^P."""
    rng = np.random.default_rng(0)
    aa = Anderson(3)
    for _ in range(5):
        aa.push(rng.standard_normal(20), rng.standard_normal(20))
    MP = np.column_stack(list(aa.P))
    MR = np.column_stack(list(aa.R))
    for j in range(3):
        np.testing.assert_allclose(aa.direction(MR[:, j]), -MP[:, j], atol=1e-12)
    c = rng.standard_normal(20)
    d = aa.direction(c)
    gamma = np.linalg.lstsq(MR, c, rcond=None)[0]
    assert np.max(np.abs(MR.T @ (MR @ gamma - c))) < 1e-12  # normal equations of the LS
    np.testing.assert_allclose(d, -c - (MP - MR) @ gamma)


def test_forced_replay_reproduces():
    d = workloads.small_binary(0)
    P = Problem(d)
    cp = CP(P)
    s = Settings(max_iter=40)
    r1 = spock(cp, d["x0"], s=s)
    r2 = spock(cp, d["x0"], s=s, forced=r1.trace)
    assert r1.trace == r2.trace
    np.testing.assert_array_equal(r1.v, r2.v)


@pytest.mark.parametrize("x0v,ub", [(0.1, 1.5), (0.5, 0.6)])
def test_scaled_inputs_are_the_same_problem(x0v, ub):
    """The change of input u' = sqrt(10) u used by the Table 1 study (R = I,
    B / sqrt(10), input box times sqrt(10)) leaves the problem unchanged: the
    same optimal value, and the same inputs after scaling back."""
    from oracle.risk import trajectory
    from oracle.table1_study import scaled_inputs
    d = workloads.datacenter(N=2, nx=3)
    d["x0"] = np.full(3, x0v)
    d["umin"][:] = -ub
    d["umax"][:] = ub
    res = []
    for prob in (d, scaled_inputs(d)):
        P = Problem(prob)
        r = spock(CP(P), prob["x0"], s=Settings(eps_abs=1e-10, eps_rel=1e-10, max_iter=30000))
        assert r.status == "converged"
        res.append((r.v[0], trajectory(P, r.v[:P.lay.n_z])[1]))
    (v1, u1), (v2, u2) = res
    assert abs(v1 - v2) <= 1e-8 * max(1.0, abs(v1))
    np.testing.assert_allclose(u2 / np.sqrt(10.0), u1, atol=1e-6)
