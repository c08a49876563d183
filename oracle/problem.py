"""RAOCP data and the layout of z and eta (Sec. "Operator splitting").
Oracle (test infrastructure only).

z   = (s^0, z_1, z_2), z_1 = (x^i for every node, u^i for every nonleaf node),
      z_2 = (y^i, tau^[i], s^[i]) for every nonleaf node i, children of i in
      increasing id.  y^i has 2 m_i + 1 entries for AV@R over m_i children
      (E = [aI, -I, 1]^T, Sec. "Conic representation of risk measures").
eta = ((y^i, s^i - b^iT y^i, x^i, u^i) for nonleaf i,
       (Q^i^1/2 x^anc(i), R^i^1/2 u^anc(i), tau^i/2, tau^i/2) for nonroot i,
       (x^j, Q_N^j^1/2 x^j, s^j/2, s^j/2) for leaf j)
with the box constraints Gamma = I of Eq. (constraints).

The index maps below are an interface: the CUDA library documents the same
ordering for its z and eta buffers.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .tree import Tree


@dataclass
class Layout:
    n_z: int
    n_eta: int
    s0: int
    x: np.ndarray          # [n, nx] index of x^i entries in z
    u: dict                # nonleaf i -> index array (nu,)
    y: dict                # nonleaf i -> (2m+1,)
    tau: dict              # nonroot c -> index of tau^c in z
    s: dict                # node -> index of s^i in z (root -> s0)
    e_y: dict              # nonleaf i -> eta indices of y block
    e_sb: dict             # nonleaf i -> eta index of s^i - b^T y^i
    e_x: dict              # nonleaf i -> eta indices (nx,)
    e_u: dict              # nonleaf i -> (nu,)
    e_qx: dict             # nonroot c -> (nx,)   Q^c^1/2 x^anc(c)
    e_ru: dict             # nonroot c -> (nu,)   R^c^1/2 u^anc(c)
    e_t: dict              # nonroot c -> (2,)    tau^c/2, tau^c/2
    e_lx: dict             # leaf j -> (nx,)      x^j (terminal box)
    e_qn: dict             # leaf j -> (nx,)      Q_N^1/2 x^j
    e_ls: dict             # leaf j -> (2,)       s^j/2, s^j/2


def build_layout(tree: Tree, nx: int, nu: int) -> Layout:
    n = tree.n
    pos = 0
    s0 = pos
    pos += 1
    x = np.arange(pos, pos + n * nx).reshape(n, nx)
    pos += n * nx
    u = {}
    for i in tree.nonleaf:
        u[i] = np.arange(pos, pos + nu)
        pos += nu
    y, tau, s = {}, {}, {0: s0}
    for i in tree.nonleaf:
        m = len(tree.children[i])
        y[i] = np.arange(pos, pos + 2 * m + 1)
        pos += 2 * m + 1
        for k, c in enumerate(tree.children[i]):
            tau[c] = pos + k
        pos += m
        for k, c in enumerate(tree.children[i]):
            s[c] = pos + k
        pos += m
    n_z = pos
    pos = 0
    e_y, e_sb, e_x, e_u = {}, {}, {}, {}
    for i in tree.nonleaf:
        m = len(tree.children[i])
        e_y[i] = np.arange(pos, pos + 2 * m + 1)
        pos += 2 * m + 1
        e_sb[i] = pos
        pos += 1
        e_x[i] = np.arange(pos, pos + nx)
        pos += nx
        e_u[i] = np.arange(pos, pos + nu)
        pos += nu
    e_qx, e_ru, e_t = {}, {}, {}
    for c in tree.nonroot:
        e_qx[c] = np.arange(pos, pos + nx)
        pos += nx
        e_ru[c] = np.arange(pos, pos + nu)
        pos += nu
        e_t[c] = np.arange(pos, pos + 2)
        pos += 2
    e_lx, e_qn, e_ls = {}, {}, {}
    for j in tree.leaves:
        e_lx[j] = np.arange(pos, pos + nx)
        pos += nx
        e_qn[j] = np.arange(pos, pos + nx)
        pos += nx
        e_ls[j] = np.arange(pos, pos + 2)
        pos += 2
    return Layout(n_z, pos, s0, x, u, y, tau, s, e_y, e_sb, e_x, e_u,
                  e_qx, e_ru, e_t, e_lx, e_qn, e_ls)


class Problem:
    """A RAOCP with diagonal quadratic costs and box constraints.

    Arrays follow the workload dict convention: per-node A, B of the edge
    into the node, diagonal Q, R (edge into the node), Q_N (leaves), AV@R
    parameter a (nonleaf), box bounds on x (all nodes) and u (nonleaf).
    """

    def __init__(self, d):
        self.tree = Tree(d["anc"], d["prob"])
        self.nx = int(d["nx"])
        self.nu = int(d["nu"])
        n, nx, nu = self.tree.n, self.nx, self.nu
        self.A = np.asarray(d["A"], float).reshape(n, nx, nx)
        self.B = np.asarray(d["B"], float).reshape(n, nx, nu)
        self.Q = np.asarray(d["Q"], float).reshape(n, nx)
        self.R = np.asarray(d["R"], float).reshape(n, nu)
        self.QN = np.asarray(d["QN"], float).reshape(n, nx)
        self.a = np.asarray(d["a"], float).reshape(n)
        self.xmin = np.asarray(d["xmin"], float).reshape(n, nx)
        self.xmax = np.asarray(d["xmax"], float).reshape(n, nx)
        self.umin = np.asarray(d["umin"], float).reshape(n, nu)
        self.umax = np.asarray(d["umax"], float).reshape(n, nu)
        self.lay = build_layout(self.tree, nx, nu)

    def b(self, i):
        """b^i = (p^ch(i), 0_m, 1) for AV@R (Sec. "Conic representation of
        risk measures"), with conditional child probabilities."""
        ch = self.tree.children[i]
        m = len(ch)
        return np.concatenate([self.tree.prob[ch], np.zeros(m), [1.0]])

    def E(self, i):
        """E^i = [a I, -I, 1]^T, shape (2m+1, m)."""
        m = len(self.tree.children[i])
        return np.vstack([self.a[i] * np.eye(m), -np.eye(m), np.ones((1, m))])
