"""Closed forms used to pin the oracle.  Oracle (test infrastructure only).

tree_lqr: with AV@R parameter a = 1 the ambiguity set is {pi} (the risk is
the expectation) and with inactive constraints the RAOCP is a stochastic
LQ problem on the tree, solved by the probability-weighted Riccati
recursion (dynamic programming, textbook):
  P^j = Q_N^j at leaves; for nonleaf i with children c (conditional p^c):
  H = sum p^c A^cT P^c B^c,  S = sum p^c (R^c + B^cT P^c B^c),
  P^i = sum p^c (Q^c + A^cT P^c A^c) - H S^-1 H^T,  u^i = -S^-1 H^T x^i,
  optimal cost x^0T P^0 x^0.  Q, R, Q_N enter as matrices (diagonal or dense).
"""
from __future__ import annotations

import numpy as np


def tree_lqr(P, x0):
    t = P.tree
    Pm = [None] * t.n
    K = [None] * t.n
    for i in sorted(range(t.n), key=lambda k: -t.stage[k]):
        if not t.children[i]:
            Pm[i] = P.QNmat(i)
            continue
        nx, nu = P.nx, P.nu
        H = np.zeros((nx, nu))
        S = np.zeros((nu, nu))
        G = np.zeros((nx, nx))
        for c in t.children[i]:
            p = t.prob[c]
            A, B, Pc = P.A[c], P.B[c], Pm[c]
            H += p * A.T @ Pc @ B
            S += p * (P.Rmat(c) + B.T @ Pc @ B)
            G += p * (P.Qmat(c) + A.T @ Pc @ A)
        K[i] = -np.linalg.solve(S, H.T)
        Pm[i] = G - H @ np.linalg.solve(S, H.T)
    # forward simulation of the optimal policy
    x = np.zeros((t.n, P.nx))
    u = np.zeros((t.n, P.nu))
    x[0] = x0
    for i in sorted(range(t.n), key=lambda k: t.stage[k]):
        if t.children[i]:
            u[i] = K[i] @ x[i]
            for c in t.children[i]:
                x[c] = P.A[c] @ x[i] + P.B[c] @ u[i]
    return float(x0 @ Pm[0] @ x0), x, u
