"""Gradient of the optimal risk-averse cost V* = s^0* with respect to the
problem data, from a converged primal-dual pair (z*, eta*).  Oracle (test
infrastructure only).

Write the splitting of Sec. "Operator splitting" as the saddle problem
  min_z max_{lambda, mu, eta}  s^0 + lambda^T (G z_1 - h) + mu^T M z_2
                               + <eta, L z> - g*(eta)
where G z_1 = h are the dynamics of S1 (x^0 = x; x^c - A^c x^anc - B^c u^anc
= 0), M z_2 = 0 the kernel of S2, and the last two terms the conjugate form
of g(Lz) (Eq. (g)).  At a saddle point the z-stationarity gives
  G^T lambda = -(L* eta*)_{z_1}
and, by the envelope theorem, dV*/dtheta is the partial derivative of the
Lagrangian at the saddle point:
  dV*/dx        = -lambda^0,
  dV*/dA^c      = -lambda^c (x^anc(c))^T,     dV*/dB^c = -lambda^c (u^anc(c))^T,
  dV*/dQ^c_kk   = eta*_{c, Q x, k} x^anc(c)_k / (2 sqrt(Q^c_kk)),
  dV*/dR^c_jj   = eta*_{c, R u, j} u^anc(c)_j / (2 sqrt(R^c_jj)),
  dV*/dQ_N^j_kk = eta*_{j, Q_N x, k} x^j_k / (2 sqrt(Q_N^j_kk))
(the square roots enter through the rows of L).  Here lambda is obtained
with a sparse least-squares solve of G^T lambda = -(L* eta*)_{z_1}
(consistent at a solution), not with the tree recursion the CUDA path uses.

Pinned (tests/test_oracle_grad.py) by the gradient of the closed-form tree
LQR cost (a = 1, inactive constraints) computed by central finite
differences of the closed form itself, and by finite differences of
oracle solves on small constrained problems.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .cp import CP


def envelope_gradient(cp: CP, z, eta):
    P = cp.P
    P.require_box_diag("envelope_gradient")
    t, lay, nx, nu = P.tree, P.lay, P.nx, P.nu
    w = cp.Lt @ eta
    S = cp.S1
    rhs = -w[S.off:S.off + S.n1]
    lam = spla.lsqr(S.G.T.tocsr(), rhs, atol=1e-15, btol=1e-15, iter_lim=100000)[0]
    n = t.n
    lam_nodes = lam.reshape(n, nx)        # row block 0: x^0 = x; row block c: node c
    g = {"x0": -lam_nodes[0].copy(),
         "A": np.zeros((n, nx, nx)), "B": np.zeros((n, nx, nu)),
         "Q": np.zeros((n, nx)), "R": np.zeros((n, nu)), "QN": np.zeros((n, nx))}
    for c in t.nonroot:
        p = int(t.anc[c])
        xp, up = z[lay.x[p]], z[lay.u[p]]
        g["A"][c] = -np.outer(lam_nodes[c], xp)
        g["B"][c] = -np.outer(lam_nodes[c], up)
        g["Q"][c] = eta[lay.e_qx[c]] * xp / (2.0 * np.sqrt(P.Q[c]))
        g["R"][c] = eta[lay.e_ru[c]] * up / (2.0 * np.sqrt(P.R[c]))
    for j in t.leaves:
        xj = z[lay.x[j]]
        g["QN"][j] = eta[lay.e_qn[j]] * xj / (2.0 * np.sqrt(P.QN[j]))
    # u-rows of G^T lambda = -(L* eta)_{z_1}: residual of the consistency check
    resid = S.G.T @ lam - rhs
    g["kkt_residual"] = float(np.max(np.abs(resid))) if resid.size else 0.0
    return g
