"""Scenario tree (Sec. "Scenario trees"): nodes, ancestors, children, stages,
probabilities.  Oracle (test infrastructure only).

Pinned by tests/test_oracle_tree.py against the 9-node tree drawn in Fig. 1
(tests/golden/fig1_tree.json).
"""
from __future__ import annotations

import numpy as np


class TreeError(ValueError):
    pass


class Tree:
    """Tree given by ancestors ``anc`` (anc[0] = -1) and *conditional*
    probabilities ``prob`` (prob[i] = pi^i / pi^anc(i), prob[0] = 1).

    The paper requires every leaf at stage N (nodes(N)); children are kept in
    increasing node id.
    """

    def __init__(self, anc, prob=None, tol=1e-9):
        anc = np.asarray(anc, dtype=np.int64)
        n = int(anc.size)
        if n < 2:
            raise TreeError("a scenario tree needs a root and at least one child")
        if anc[0] != -1:
            raise TreeError("node 0 must be the root (anc[0] = -1)")
        if np.any(anc[1:] < 0) or np.any(anc[1:] >= n):
            raise TreeError("ancestor out of range")
        self.n = n
        self.anc = anc
        self.children = [[] for _ in range(n)]
        for i in range(1, n):
            self.children[int(anc[i])].append(i)
        # stages by walking up (detects cycles)
        stage = np.full(n, -1, dtype=np.int64)
        stage[0] = 0
        for i in range(1, n):
            path = []
            j = i
            while stage[j] < 0:
                path.append(j)
                j = int(anc[j])
                if len(path) > n:
                    raise TreeError("cycle in ancestor array")
            s = stage[j]
            for k in reversed(path):
                s += 1
                stage[k] = s
        self.stage = stage
        self.leaves = [i for i in range(n) if not self.children[i]]
        self.nonleaf = [i for i in range(n) if self.children[i]]
        self.nonroot = list(range(1, n))
        depths = {int(stage[j]) for j in self.leaves}
        if len(depths) != 1:
            raise TreeError("all leaves must lie at the same stage N")
        self.N = depths.pop()
        if prob is None:
            prob = np.zeros(n)
            prob[0] = 1.0
            for i in self.nonleaf:
                for c in self.children[i]:
                    prob[c] = 1.0 / len(self.children[i])
        prob = np.asarray(prob, dtype=np.float64)
        if prob.shape != (n,):
            raise TreeError("prob must have one entry per node")
        for i in self.nonleaf:
            p = prob[self.children[i]]
            if np.any(p <= 0) or abs(p.sum() - 1.0) > tol:
                raise TreeError(f"children probabilities of node {i} must be positive and sum to 1")
        self.prob = prob
        # absolute probabilities pi^i (Sec. "Scenario trees")
        pi = np.zeros(n)
        pi[0] = 1.0
        for i in np.argsort(stage, kind="stable"):
            if i:
                pi[i] = pi[anc[i]] * prob[i]
        self.pi = pi

    def nodes(self, t):
        """nodes(t): the nodes at stage t."""
        return [i for i in range(self.n) if self.stage[i] == t]

    def sibling_index(self, c):
        """Position of nonroot node c among the children of anc(c)."""
        return self.children[int(self.anc[c])].index(c)
