"""Risk measures (Sec. "Risk measures", "Conic representation of risk
measures", "Conditional risk mappings") and the nested value of Eq.
(original-problem) at a given trajectory.  Oracle (test infrastructure only).

Reading: in the definition of AV@R_a the minimisation variable t is a
scalar (the paper's "t in R^n" is garbled); a = 0 is the maximum.

Pins (tests/test_oracle_risk.py): the sort closed form, the min-over-t
formula, the conic dual LP (scipy linprog) and a brute-force enumeration of
the vertices of the ambiguity set agree.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import linprog


def avar_sort(Z, pi, a):
    """max over mu in A_a = {sum mu = 1, 0 <= mu <= pi / a}: put as much mass
    as allowed on the largest costs first."""
    Z = np.asarray(Z, float)
    pi = np.asarray(pi, float)
    if a == 0:
        return float(np.max(Z))
    cap = pi / a
    order = np.argsort(-Z, kind="stable")
    left = 1.0
    val = 0.0
    for i in order:
        take = min(cap[i], left)
        val += take * Z[i]
        left -= take
        if left <= 0:
            break
    return float(val)


def avar_min_t(Z, pi, a):
    """min_t { t + E^pi[Z - t]_+ / a }; the piecewise-linear convex function
    attains its minimum at one of the Z_i."""
    Z = np.asarray(Z, float)
    pi = np.asarray(pi, float)
    if a == 0:
        return float(np.max(Z))
    return float(min(t + pi @ np.maximum(Z - t, 0.0) / a for t in Z))


def avar_lp(Z, pi, a):
    """Conic dual: min { y^T b : E^T y = Z, y in K* } with b = (pi, 0, 1),
    E = [aI, -I, 1]^T, K* = R^{2n}_+ x R."""
    Z = np.asarray(Z, float)
    n = Z.size
    b = np.concatenate([pi, np.zeros(n), [1.0]])
    E = np.vstack([a * np.eye(n), -np.eye(n), np.ones((1, n))])
    bounds = [(0, None)] * (2 * n) + [(None, None)]
    res = linprog(b, A_eq=E.T, b_eq=Z, bounds=bounds, method="highs")
    assert res.status == 0, res.message
    return float(res.fun)


def avar_bruteforce(Z, pi, a):
    """Enumerate the vertices of A_a: every mu_i at 0 or at its cap pi_i/a,
    except at most one free coordinate fixed by sum mu = 1."""
    Z = np.asarray(Z, float)
    pi = np.asarray(pi, float)
    n = Z.size
    cap = pi / a if a > 0 else np.full(n, np.inf)
    best = -np.inf
    for free in range(n):
        others = [i for i in range(n) if i != free]
        for pattern in itertools.product((0, 1), repeat=n - 1):
            mu = np.zeros(n)
            ok = True
            for i, at_cap in zip(others, pattern):
                if at_cap:
                    if not np.isfinite(cap[i]):
                        ok = False
                        break
                    mu[i] = cap[i]
            if not ok:
                continue
            mu[free] = 1.0 - mu.sum()
            if mu[free] < -1e-12 or mu[free] > cap[free] + 1e-12:
                continue
            best = max(best, float(mu @ Z))
    return best


def conic_lp(Z, b, E, F, kp):
    """rho[Z] of the conic representation, Eq. (dual_risk):
    min { y^T b : E^T y = Z, F^T y = 0, y in K* }, K* = R^kp_+ x R^(ny - kp)
    (scipy linprog, a library primitive)."""
    Z = np.asarray(Z, float)
    ny = b.size
    A_eq = E.T if F.shape[1] == 0 else np.vstack([E.T, F.T])
    b_eq = Z if F.shape[1] == 0 else np.concatenate([Z, np.zeros(F.shape[1])])
    bounds = [(0, None)] * kp + [(None, None)] * (ny - kp)
    res = linprog(b, A_eq=A_eq, b_eq=b_eq, bounds=bounds, method="highs")
    assert res.status == 0, res.message
    return float(res.fun)


def nested_value(P, x, u, avar=avar_sort, risk=None):
    """Nested risk-averse cost of Eq. (original-problem) of a given
    trajectory, by backward recursion over the tree:
      W^j = x^jT Q_N^j x^j at leaves,
      W^i = rho^i[ (x^iT Q^c x^i + u^iT R^c u^i + W^c)_{c in ch(i)} ]
    with rho^i = AV@R_{a^i} over the conditional probabilities of the
    children, or risk(i, Z) when given.  x: [n, nx], u: dict or [n, nu]
    (nonleaf rows used)."""
    t = P.tree
    W = np.zeros(t.n)
    for i in sorted(range(t.n), key=lambda k: -t.stage[k]):
        if not t.children[i]:
            W[i] = float(x[i] @ P.QNmat(i) @ x[i])
        else:
            ch = t.children[i]
            Z = np.array([x[i] @ P.Qmat(c) @ x[i] + u[i] @ P.Rmat(c) @ u[i] + W[c] for c in ch])
            W[i] = risk(i, Z) if risk is not None else avar(Z, t.prob[ch], P.a[i])
    return float(W[0]), W


def trajectory(P, z):
    """(x [n, nx], u [n, nu]) from a z-shaped vector (u rows of leaves 0)."""
    lay = P.lay
    x = z[lay.x]
    u = np.zeros((P.tree.n, P.nu))
    for i in P.tree.nonleaf:
        u[i] = z[lay.u[i]]
    return x, u
