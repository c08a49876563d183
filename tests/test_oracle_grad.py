"""Oracle envelope gradient of V* against finite differences: of the closed-
form tree LQR cost (a = 1, inactive constraints; no solver error in the
reference), and of oracle solves on a one-step problem with active
constraints."""
import numpy as np
import pytest

from oracle.cp import CP
from oracle.grad import envelope_gradient
from oracle.lqr import tree_lqr
from oracle.problem import Problem
from oracle.spock import Settings, spock
from paper_2212_01110_gb300 import workloads

TIGHT = Settings(eps_abs=1e-12, eps_rel=1e-12, max_iter=100000, memory=5)


def _unconstrained_a1(d):
    d = dict(d)
    n = len(d["anc"])
    big = 1e6
    d["xmin"], d["xmax"] = -big * np.ones((n, d["nx"])), big * np.ones((n, d["nx"]))
    d["umin"], d["umax"] = -big * np.ones((n, d["nu"])), big * np.ones((n, d["nu"]))
    d["a"] = np.ones(n)
    return d


def _fd(f, d, key, idx, h=1e-6):
    dp, dm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d.items()}, \
             {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d.items()}
    dp[key][idx] += h
    dm[key][idx] -= h
    return (f(dp) - f(dm)) / (2 * h)


@pytest.mark.parametrize("d0", [workloads.small_binary(2, nx=2, nu=2),
                                workloads.with_tree(workloads.fig1_tree(), seed=3, nx=2, nu=1)])
def test_envelope_gradient_vs_lqr_closed_form(d0):
    d = _unconstrained_a1(d0)
    P = Problem(d)
    cp = CP(P)
    res = spock(cp, d["x0"], s=TIGHT)
    assert res.status == "converged"
    z, eta = res.v[:cp.n_z], res.v[cp.n_z:]
    g = envelope_gradient(cp, z, eta)
    assert g["kkt_residual"] < 1e-8
    V = lambda dd: tree_lqr(Problem(dd), dd["x0"])[0]
    # x0: exact closed form 2 P^0 x0
    for k in range(d["nx"]):
        assert abs(g["x0"][k] - _fd(V, d, "x0", (k,))) < 1e-6
    rng = np.random.default_rng(0)
    for key in ("A", "B", "Q", "R", "QN"):
        for _ in range(4):
            node = int(rng.integers(1, len(d["anc"])))
            if key == "QN" and node not in P.tree.leaves:
                node = P.tree.leaves[0]
            shape = g[key].shape[1:]
            idx = (node,) + tuple(int(rng.integers(0, s)) for s in shape)
            fd = _fd(V, d, key, idx)
            assert abs(g[key][idx] - fd) < 1e-6 * max(1, abs(fd)), (key, idx, g[key][idx], fd)


def test_envelope_gradient_active_constraints_fd():
    """One-step problem with the input box active and AV@R a < 1: gradient
    against central differences of tight oracle solves."""
    anc = np.array([-1, 0, 0, 0], np.int32)
    d = workloads.with_tree(anc, seed=5, nx=2, nu=1, a=0.4, box=(5.0, 0.3))
    d["x0"] = np.array([1.2, -0.7])
    P = Problem(d)
    cp = CP(P)
    res = spock(cp, d["x0"], s=TIGHT)
    z, eta = res.v[:cp.n_z], res.v[cp.n_z:]
    g = envelope_gradient(cp, z, eta)

    def V(dd):
        c = CP(Problem(dd))
        return spock(c, dd["x0"], s=TIGHT).v[0]

    for key, idx in (("x0", (0,)), ("x0", (1,)), ("A", (2, 0, 1)), ("B", (1, 1, 0)), ("Q", (3, 0)),
                     ("R", (2, 0)), ("QN", (1, 1))):
        fd = _fd(V, d, key, idx, h=1e-5)
        assert abs(g[key][idx] - fd) < 1e-5 * max(1, abs(fd)), (key, idx, g[key][idx], fd)
