"""RAOCP data and the layout of z and eta (Sec. "Operator splitting").
Oracle (test infrastructure only).

z   = (s^0, z_1, z_2), z_1 = (x^i for every node, u^i for every nonleaf node),
      z_2 = (y^i, tau^[i], s^[i]) for every nonleaf node i, children of i in
      increasing id.  y^i has 2 m_i + 1 entries for AV@R over m_i children
      (E = [aI, -I, 1]^T, Sec. "Conic representation of risk measures").
eta = ((y^i, s^i - b^iT y^i, Gamma_x^i x^i + Gamma_u^i u^i) for nonleaf i,
       (Q^i^1/2 x^anc(i), R^i^1/2 u^anc(i), tau^i/2, tau^i/2) for nonroot i,
       (Gamma_N^j x^j, Q_N^j^1/2 x^j, s^j/2, s^j/2) for leaf j)
(definition of L).  Two forms of the data:
  * box form: Gamma = I (the constraint rows are x^i, u^i and x^j) with C^i,
    C_N^j boxes, diagonal Q, R, Q_N given by their diagonals;
  * general form (Eq. (constraints) with polyhedral C): constraint matrices
    Gamma_x^i (nc x nx), Gamma_u^i (nc x nu), Gamma_N^j (ncN x nx) with C^i,
    C_N^j boxes [cmin, cmax] of nc / ncN rows, and/or dense symmetric
    positive definite Q, R, Q_N.  The square roots in L are the upper
    Cholesky factors F (F^T F = Q): any factor with F^T F = Q gives the same
    cost x'Qx = ||F x||^2, so the choice is a reading of the paper's
    notation Q^1/2; the library documents the same factor.
With Gamma = I and diagonal costs both forms give the same L.

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
    e_c: dict              # nonleaf i -> (nc,)   Gamma_x x^i + Gamma_u u^i
    e_lc: dict             # leaf j -> (ncN,)     Gamma_N x^j


def build_layout(tree: Tree, nx: int, nu: int, nc: int | None = None, ncN: int | None = None,
                 ny: dict | None = None) -> Layout:
    """Index maps of z and eta.  ``nc`` / ``ncN`` (constraint rows per nonleaf
    / leaf node) default to the box form's nx + nu / nx; in the box form the
    constraint rows are also split into e_x, e_u (nonleaf) and e_lx (leaf).
    ``ny`` (nonleaf node -> rows of y^i) defaults to AV@R's 2 m + 1."""
    box = nc is None and ncN is None
    nyof = (lambda i: 2 * len(tree.children[i]) + 1) if ny is None else (lambda i: int(ny[i]))
    nc = nx + nu if nc is None else int(nc)
    ncN = nx if ncN is None else int(ncN)
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
        y[i] = np.arange(pos, pos + nyof(i))
        pos += nyof(i)
        for k, c in enumerate(tree.children[i]):
            tau[c] = pos + k
        pos += m
        for k, c in enumerate(tree.children[i]):
            s[c] = pos + k
        pos += m
    n_z = pos
    pos = 0
    e_y, e_sb, e_x, e_u, e_c = {}, {}, {}, {}, {}
    for i in tree.nonleaf:
        e_y[i] = np.arange(pos, pos + nyof(i))
        pos += nyof(i)
        e_sb[i] = pos
        pos += 1
        e_c[i] = np.arange(pos, pos + nc)
        if box:
            e_x[i] = e_c[i][:nx]
            e_u[i] = e_c[i][nx:]
        pos += nc
    e_qx, e_ru, e_t = {}, {}, {}
    for c in tree.nonroot:
        e_qx[c] = np.arange(pos, pos + nx)
        pos += nx
        e_ru[c] = np.arange(pos, pos + nu)
        pos += nu
        e_t[c] = np.arange(pos, pos + 2)
        pos += 2
    e_lx, e_qn, e_ls, e_lc = {}, {}, {}, {}
    for j in tree.leaves:
        e_lc[j] = np.arange(pos, pos + ncN)
        if box:
            e_lx[j] = e_lc[j]
        pos += ncN
        e_qn[j] = np.arange(pos, pos + nx)
        pos += nx
        e_ls[j] = np.arange(pos, pos + 2)
        pos += 2
    return Layout(n_z, pos, s0, x, u, y, tau, s, e_y, e_sb, e_x, e_u,
                  e_qx, e_ru, e_t, e_lx, e_qn, e_ls, e_c, e_lc)


class Problem:
    """A RAOCP with quadratic costs and polyhedral constraints.

    Arrays follow the workload dict convention: per-node A, B of the edge
    into the node, Q, R (edge into the node), Q_N (leaves), AV@R parameter a
    (nonleaf).  Q, R, Q_N are diagonals ([n][nx]) or, when given as [n][nx][nx]
    arrays, dense symmetric positive definite matrices (``dense_cost``).
    Constraints: box bounds xmin/xmax (all nodes) and umin/umax (nonleaf), or,
    when the dict has "Gx", the general form: Gx [n][nc][nx], Gu [n][nc][nu],
    cmin/cmax [n][nc] (nonleaf), GN [n][ncN][nx], cNmin/cNmax [n][ncN] (leaves).
    """

    def __init__(self, d):
        self.tree = Tree(d["anc"], d["prob"])
        self.nx = int(d["nx"])
        self.nu = int(d["nu"])
        n, nx, nu = self.tree.n, self.nx, self.nu
        self.A = np.asarray(d["A"], float).reshape(n, nx, nx)
        self.B = np.asarray(d["B"], float).reshape(n, nx, nu)
        self.dense_cost = np.asarray(d["Q"]).ndim == 3
        if self.dense_cost:
            self.Q = np.asarray(d["Q"], float).reshape(n, nx, nx)
            self.R = np.asarray(d["R"], float).reshape(n, nu, nu)
            self.QN = np.asarray(d["QN"], float).reshape(n, nx, nx)
        else:
            self.Q = np.asarray(d["Q"], float).reshape(n, nx)
            self.R = np.asarray(d["R"], float).reshape(n, nu)
            self.QN = np.asarray(d["QN"], float).reshape(n, nx)
        self.a = np.asarray(d["a"], float).reshape(n)
        # coherent risk measures in conic form (b, E, F, K) per nonleaf node,
        # K = R^kp_+ x {0}^(ny - kp) (Sec. "Conic representation of risk
        # measures"); absent: AV@R with parameter a
        self.general_risk = d.get("risk") is not None
        self.risk = {}
        if self.general_risk:
            for i in self.tree.nonleaf:
                r = d["risk"][i]
                m = len(self.tree.children[i])
                b = np.asarray(r["b"], float).reshape(-1)
                E = np.asarray(r["E"], float).reshape(b.size, m)
                F = np.asarray(r.get("F", np.zeros((b.size, 0))), float).reshape(b.size, -1)
                self.risk[i] = (b, E, F, int(r["kp"]))
        ny = {i: self.risk[i][0].size for i in self.tree.nonleaf} if self.general_risk else None
        self.general = "Gx" in d
        if self.general:
            self.Gx = np.asarray(d["Gx"], float)
            self.nc = self.Gx.shape[1]
            self.Gx = self.Gx.reshape(n, self.nc, nx)
            self.Gu = np.asarray(d["Gu"], float).reshape(n, self.nc, nu)
            self.cmin = np.asarray(d["cmin"], float).reshape(n, self.nc)
            self.cmax = np.asarray(d["cmax"], float).reshape(n, self.nc)
            self.GN = np.asarray(d["GN"], float)
            self.ncN = self.GN.shape[1]
            self.GN = self.GN.reshape(n, self.ncN, nx)
            self.cNmin = np.asarray(d["cNmin"], float).reshape(n, self.ncN)
            self.cNmax = np.asarray(d["cNmax"], float).reshape(n, self.ncN)
            self.lay = build_layout(self.tree, nx, nu, self.nc, self.ncN, ny=ny)
        else:
            self.xmin = np.asarray(d["xmin"], float).reshape(n, nx)
            self.xmax = np.asarray(d["xmax"], float).reshape(n, nx)
            self.umin = np.asarray(d["umin"], float).reshape(n, nu)
            self.umax = np.asarray(d["umax"], float).reshape(n, nu)
            self.nc, self.ncN = nx + nu, nx
            self.lay = build_layout(self.tree, nx, nu, ny=ny)

    # -- cost matrices and their square roots (definition of L) ---------------
    def _mat(self, M, i):
        return M[i] if self.dense_cost else np.diag(M[i])

    def Qmat(self, i):
        return self._mat(self.Q, i)

    def Rmat(self, i):
        return self._mat(self.R, i)

    def QNmat(self, i):
        return self._mat(self.QN, i)

    def _half(self, M, i):
        """F with F^T F = M^i: sqrt of the diagonal, or the upper Cholesky
        factor (numpy's lower factor, transposed) of a dense matrix."""
        if self.dense_cost:
            return np.linalg.cholesky(M[i]).T
        return np.diag(np.sqrt(M[i]))

    def Qhalf(self, i):
        return self._half(self.Q, i)

    def Rhalf(self, i):
        return self._half(self.R, i)

    def QNhalf(self, i):
        return self._half(self.QN, i)

    def require_box_diag(self, what):
        """Parts of the oracle written for the box form with diagonal costs
        and AV@R."""
        if self.general or self.dense_cost or self.general_risk:
            raise NotImplementedError(what + ": box constraints, diagonal costs and AV@R only")

    def b(self, i):
        """b^i of the conic representation (Sec. "Conic representation of
        risk measures"); AV@R: (p^ch(i), 0_m, 1) with conditional child
        probabilities."""
        if self.general_risk:
            return self.risk[i][0]
        ch = self.tree.children[i]
        m = len(ch)
        return np.concatenate([self.tree.prob[ch], np.zeros(m), [1.0]])

    def E(self, i):
        """E^i; AV@R: [a I, -I, 1]^T, shape (2m+1, m)."""
        if self.general_risk:
            return self.risk[i][1]
        m = len(self.tree.children[i])
        return np.vstack([self.a[i] * np.eye(m), -np.eye(m), np.ones((1, m))])

    def F(self, i):
        """F^i (ny x n_nu); AV@R: no columns."""
        if self.general_risk:
            return self.risk[i][2]
        return np.zeros((2 * len(self.tree.children[i]) + 1, 0))

    def kp(self, i):
        """Rows of y^i in the orthant part of K^i (the rest: the zero cone);
        (K^i)* = R^kp_+ x R^(ny - kp).  AV@R: 2 m."""
        if self.general_risk:
            return self.risk[i][3]
        return 2 * len(self.tree.children[i])
