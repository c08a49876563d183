"""Implicit differentiation of the CP fixed point (adjoint method) for the
gradient of a linear function phi(z*) = <g, z*> of the solution with
respect to the problem data.  Oracle (test infrastructure only).

At a fixed point v* = T(v*) of the operator T of Eq.
(chambolle-pock-operator), dv* = J dv* + T_theta dtheta with J the Jacobian
of T in v, so
    d phi / d theta = w^T T_theta,   w = J^T w + (g, 0),
i.e. w solves (I - J^T) w = (g, 0).  With zbar = z - alpha L* eta and
wbar = eta + alpha L (2 z+ - z) the points where the two proximal operators
are evaluated (Sec. "Proximal operator of f", Eq. (prox:g)):
    J (dz, deta) = (A (dz - alpha L* deta),  B (deta + alpha L (2 dz+ - dz)))
where A is the Jacobian of prox_{alpha f} (identity on s^0, the projection
on the null space of the dynamics on z_1, proj_S2 on z_2) and
B = I - D(wbar / alpha) the Jacobian of prox_{alpha g*}, D the Jacobian of
proj_S3 (block diagonal: 0/1 on boxes and orthants, the SOC projection's
Jacobian on the cones).  A and B are symmetric, and
    J^T (wz, weta) = (p - alpha L* q,  q - alpha L p),
    q = B weta,  p = A (wz + 2 alpha L* q).
Here (I - J^T) w = (g, 0) is solved by GMRES on that linear map (a library
primitive); the CUDA path iterates the fixed point instead.

Derivatives of T in the data, with r = wz + 2 alpha L* q, p1 the z_1 part of
A r, and mu, nu the multipliers of the dynamics constraints G z_1 = h in
  G^T mu = r_1 - p1,          G^T nu = -alpha (L* eta*)_1
(the projection of zbar lands on z*, so zbar - z* = -alpha L* eta*):
  d phi / d x0    = mu^0,
  d phi / d A^c   = nu^c (p1_x^anc(c))^T + mu^c (x*^anc(c))^T,
  d phi / d B^c   = nu^c (p1_u^anc(c))^T + mu^c (u*^anc(c))^T,
  d phi / d Q^c_kk = alpha (q_{c,Qx,k} x*^anc_k - eta*_{c,Qx,k} p_{x^anc,k}) / (2 sqrt(Q^c_kk)),
and likewise R^c (rows R^1/2 u^anc) and Q_N^j (rows Q_N^1/2 x^j).  For
phi = s^0 (the optimal cost) the result equals the envelope gradient of
oracle/grad.py.

Pins (tests/test_oracle_adjoint.py): equality with the envelope gradient
for phi = s^0, and central finite differences of oracle solves for phi = a
component of the first input u^0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .cones import s2_matrix, z2_block
from .cp import CP


def dproj_soc(w):
    """Jacobian of the projection on SOC = {(v, t): ||v|| <= t} at w."""
    w = np.asarray(w, float)
    v, t = w[:-1], w[-1]
    n = w.size
    nv = float(np.linalg.norm(v))
    if nv <= t:
        return np.eye(n)
    if nv <= -t:
        return np.zeros((n, n))
    vh = v / nv
    J = np.zeros((n, n))
    J[:-1, :-1] = 0.5 * ((1.0 + t / nv) * np.eye(n - 1) - (t / nv) * np.outer(vh, vh))
    J[:-1, -1] = 0.5 * vh
    J[-1, :-1] = 0.5 * vh
    J[-1, -1] = 0.5
    return J


def jac_proj_S3(y, P):
    """Jacobian of proj_S3 at y (eta-shaped), as a sparse block-diagonal
    matrix (blocks follow Eq. (S3-def) with the readings of oracle/cones.py)."""
    t, lay = P.tree, P.lay
    n = lay.n_eta
    rows, cols, vals = [], [], []

    def diag(idx, d):
        for i, v in zip(np.atleast_1d(idx), np.atleast_1d(d)):
            if v != 0.0:
                rows.append(int(i)); cols.append(int(i)); vals.append(float(v))

    def block(idx, Jb):
        idx = np.asarray(idx, int)
        for a in range(idx.size):
            for b in range(idx.size):
                if Jb[a, b] != 0.0:
                    rows.append(int(idx[a])); cols.append(int(idx[b])); vals.append(float(Jb[a, b]))

    for i in t.nonleaf:
        m = len(t.children[i])
        ey = lay.e_y[i]
        diag(ey[:2 * m], (y[ey[:2 * m]] > 0).astype(float))
        diag(ey[2 * m], 1.0)
        diag(lay.e_sb[i], float(y[lay.e_sb[i]] > 0))
        ex, eu = lay.e_x[i], lay.e_u[i]
        diag(ex, ((y[ex] > P.xmin[i]) & (y[ex] < P.xmax[i])).astype(float))
        diag(eu, ((y[eu] > P.umin[i]) & (y[eu] < P.umax[i])).astype(float))
    sh_nr = np.zeros(P.nx + P.nu + 2)
    sh_nr[-2:] = (0.5, -0.5)
    for c in t.nonroot:
        idx = np.concatenate([lay.e_qx[c], lay.e_ru[c], lay.e_t[c]])
        block(idx, dproj_soc(y[idx] - sh_nr))
    sh_lf = np.zeros(P.nx + 2)
    sh_lf[-2:] = (0.5, -0.5)
    for j in t.leaves:
        ex = lay.e_lx[j]
        diag(ex, ((y[ex] > P.xmin[j]) & (y[ex] < P.xmax[j])).astype(float))
        idx = np.concatenate([lay.e_qn[j], lay.e_ls[j]])
        block(idx, dproj_soc(y[idx] - sh_lf))
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


class Linearisation:
    """J^T and the data derivatives at a converged pair (z*, eta*) = T(v*)."""

    def __init__(self, cp: CP, z, eta):
        self.cp = cp
        P = cp.P
        P.require_box_diag("Linearisation")
        self.P = P
        self.z = np.asarray(z, float)
        self.eta = np.asarray(eta, float)
        a = cp.alpha
        self.wbar = self.eta + a * (cp.L @ self.z)
        self.D = jac_proj_S3(self.wbar / a, P)
        S = cp.S1
        self.off, self.n1 = S.off, S.n1
        self.S2 = [(z2_block(P, i), s2_matrix(P, i)) for i in P.tree.nonleaf]

    def A(self, r):
        """Jacobian of prox_{alpha f}: identity on s^0, projection on the null
        space of the dynamics on z_1 (homogeneous KKT solve), proj_S2 on z_2."""
        out = np.array(r, float, copy=True)
        sl = slice(self.off, self.off + self.n1)
        out[sl] = self.cp.S1.project(r[sl], np.zeros(self.P.nx))
        for idx, M in self.S2:
            out[idx] = r[idx] - np.linalg.pinv(M) @ (M @ r[idx])
        return out

    def B(self, x):
        return x - self.D @ x

    def JT(self, w):
        cp, a = self.cp, self.cp.alpha
        wz, we = w[:cp.n_z], w[cp.n_z:]
        q = self.B(we)
        t = cp.Lt @ q
        r = wz + 2 * a * t
        p = self.A(r)
        return np.concatenate([p - a * t, q - a * (cp.L @ p)]), (q, r, p)

    def solve(self, g, tol=1e-13, maxiter=20000):
        """w with (I - J^T) w = (g, 0) by GMRES."""
        n = self.cp.n_z + self.cp.n_eta
        op = spla.LinearOperator((n, n), matvec=lambda w: w - self.JT(w)[0], dtype=float)
        rhs = np.concatenate([np.asarray(g, float), np.zeros(self.cp.n_eta)])
        w, info = spla.gmres(op, rhs, rtol=tol, atol=0.0, restart=200, maxiter=maxiter)
        res = float(np.max(np.abs(op @ w - rhs)))
        return w, info, res

    def gradients(self, w):
        cp, P, a = self.cp, self.P, self.cp.alpha
        t, lay, nx, nu = P.tree, P.lay, P.nx, P.nu
        _, (q, r, p) = self.JT(w)
        S = cp.S1
        G = S.G.T.tocsr()
        sl = slice(self.off, self.off + self.n1)
        p1 = p[sl]
        y = r[sl] - p1
        mu = spla.lsqr(G, y, atol=1e-15, btol=1e-15, iter_lim=100000)[0].reshape(t.n, nx)
        lt = cp.Lt @ self.eta
        nu_ = spla.lsqr(G, -a * lt[sl], atol=1e-15, btol=1e-15, iter_lim=100000)[0].reshape(t.n, nx)
        z, eta = self.z, self.eta
        pfull = p
        out = {"x0": mu[0].copy(), "A": np.zeros((t.n, nx, nx)), "B": np.zeros((t.n, nx, nu)),
               "Q": np.zeros((t.n, nx)), "R": np.zeros((t.n, nu)), "QN": np.zeros((t.n, nx))}
        for c in t.nonroot:
            pa = int(t.anc[c])
            out["A"][c] = np.outer(nu_[c], pfull[lay.x[pa]]) + np.outer(mu[c], z[lay.x[pa]])
            out["B"][c] = np.outer(nu_[c], pfull[lay.u[pa]]) + np.outer(mu[c], z[lay.u[pa]])
            out["Q"][c] = a * (q[lay.e_qx[c]] * z[lay.x[pa]] - eta[lay.e_qx[c]] * pfull[lay.x[pa]]) \
                / (2.0 * np.sqrt(P.Q[c]))
            out["R"][c] = a * (q[lay.e_ru[c]] * z[lay.u[pa]] - eta[lay.e_ru[c]] * pfull[lay.u[pa]]) \
                / (2.0 * np.sqrt(P.R[c]))
        for j in t.leaves:
            out["QN"][j] = a * (q[lay.e_qn[j]] * z[lay.x[j]] - eta[lay.e_qn[j]] * pfull[lay.x[j]]) \
                / (2.0 * np.sqrt(P.QN[j]))
        return out


def adjoint_gradient(cp: CP, z, eta, g=None, tol=1e-13):
    """Gradient of phi(z*) = <g, z*> (default g = e_{s^0}: the optimal cost)
    with respect to x0, A, B and the diagonals of Q, R, Q_N, at a converged
    pair (z*, eta*)."""
    lin = Linearisation(cp, z, eta)
    if g is None:
        g = np.zeros(cp.n_z)
        g[cp.P.lay.s0] = 1.0
    w, info, res = lin.solve(g, tol=tol)
    out = lin.gradients(w)
    out["gmres_info"] = info
    out["adjoint_residual"] = res
    out["w"] = w
    return out
