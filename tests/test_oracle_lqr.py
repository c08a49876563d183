"""The tree-LQR closed form (oracle/lqr.py), which several oracle pins use
as their reference, pinned by brute force: with a = 1 the risk is the
expectation (Sec. "Risk measures": the ambiguity set of AV@R_1 is {pi}), so
with no active constraint the problem is the equality-constrained quadratic
program
    min  sum_{nonroot c} pi^c (x^a' Q^c x^a + u^a' R^c u^a) + sum_{leaves j} pi^j x^j' Q_N^j x^j
    s.t. x^0 = x0,  x^c = A^c x^a + B^c u^a   (a = anc(c)),
with pi the absolute node probabilities.  Its KKT system is assembled here
densely and solved directly; the optimal value, every input and every state
must equal the recursion's."""
import numpy as np
import pytest

from oracle.lqr import tree_lqr
from oracle.problem import Problem
from paper_2212_01110_gb300 import workloads as W


def _brute_force(P, x0):
    t = P.tree
    n, nx, nu = t.n, P.nx, P.nu
    nonleaf = [i for i in range(n) if t.children[i]]
    uix = {i: k for k, i in enumerate(nonleaf)}
    nv = n * nx + len(nonleaf) * nu
    xs = lambda i: slice(i * nx, (i + 1) * nx)
    us = lambda i: slice(n * nx + uix[i] * nu, n * nx + (uix[i] + 1) * nu)
    pi = np.ones(n)
    for c in sorted(range(1, n), key=lambda k: t.stage[k]):   # ancestors first
        pi[c] = pi[t.anc[c]] * t.prob[c]
    H = np.zeros((nv, nv))
    for c in range(1, n):
        a = int(t.anc[c])
        H[xs(a), xs(a)] += pi[c] * P.Qmat(c)
        H[us(a), us(a)] += pi[c] * P.Rmat(c)
    for j in range(n):
        if not t.children[j]:
            H[xs(j), xs(j)] += pi[j] * P.QNmat(j)
    rows = []
    rhs = []
    G0 = np.zeros((nx, nv))
    G0[:, xs(0)] = np.eye(nx)
    rows.append(G0)
    rhs.append(x0)
    for c in range(1, n):
        a = int(t.anc[c])
        Gc = np.zeros((nx, nv))
        Gc[:, xs(c)] = np.eye(nx)
        Gc[:, xs(a)] -= P.A[c]
        Gc[:, us(a)] -= P.B[c]
        rows.append(Gc)
        rhs.append(np.zeros(nx))
    G = np.vstack(rows)
    h = np.concatenate(rhs)
    m = G.shape[0]
    K = np.block([[2 * H, G.T], [G, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([np.zeros(nv), h]))
    v = sol[:nv]
    x = np.array([v[xs(i)] for i in range(n)])
    u = {i: v[us(i)] for i in nonleaf}
    return float(v @ H @ v), x, u


@pytest.mark.parametrize("make", [
    lambda: W.small_binary(0, a=1.0),
    lambda: W.with_tree(W.fig1_tree(), seed=3, nx=3, nu=2, a=1.0),
    lambda: W.random_tree(4, N=4, max_branch=3, nx=3, nu=2, a_range=(1.0, 1.0)),
    lambda: W.general_random(W.random_tree(6, N=3, max_branch=3, nx=3, nu=4, a_range=(1.0, 1.0)), seed=2),
])
def test_tree_lqr_is_the_expected_cost_qp(make):
    d = make()
    P = Problem(d)
    V, x, u = tree_lqr(P, d["x0"])
    Vb, xb, ub = _brute_force(P, d["x0"])
    assert abs(V - Vb) <= 1e-10 * max(1.0, abs(Vb))
    scale = max(1.0, float(np.max(np.abs(xb))))
    np.testing.assert_allclose(x, xb, rtol=0, atol=1e-10 * scale)
    for i, ui in ub.items():
        np.testing.assert_allclose(u[i], ui, rtol=0, atol=1e-10 * scale)
