"""The linear operator L of Sec. "Operator splitting" as an explicit sparse
matrix, its adjoint L* = L^T (definition in Sec. "Notation"), and ||L||, for
the box form and the general form (polyhedral constraints Gamma, dense cost
matrices) of oracle/problem.py.  Oracle (test infrastructure only).

Pins (tests/test_oracle_linop.py): the rows of L encode the epigraph and
AV@R constraints of Eq. (min-s0-v1) -- checked on constructed points,
independent of how L is assembled; the closed-form block norm (remark after
the definition of L: block-diagonal after a column permutation) agrees with
a power iteration on L^T L.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .problem import Problem


def build_L(P: Problem) -> sp.csr_matrix:
    """Assemble L row by row following the definition of eta."""
    t, lay = P.tree, P.lay
    rows, cols, vals = [], [], []

    def put(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for i in t.nonleaf:
        b = P.b(i)
        # (y^i, s^i - b^iT y^i, Gamma_x x^i + Gamma_u u^i) with Gamma = I
        for r, c in zip(lay.e_y[i], lay.y[i]):
            put(r, c, 1.0)
        put(lay.e_sb[i], lay.s[i], 1.0)
        for k, c in enumerate(lay.y[i]):
            put(lay.e_sb[i], c, -b[k])
        if P.general:
            for r in range(P.nc):
                for k in range(P.nx):
                    if P.Gx[i, r, k] != 0.0:
                        put(lay.e_c[i][r], lay.x[i][k], P.Gx[i, r, k])
                for k in range(P.nu):
                    if P.Gu[i, r, k] != 0.0:
                        put(lay.e_c[i][r], lay.u[i][k], P.Gu[i, r, k])
        else:
            for k in range(P.nx):
                put(lay.e_x[i][k], lay.x[i][k], 1.0)
            for k in range(P.nu):
                put(lay.e_u[i][k], lay.u[i][k], 1.0)

    def put_block(erows, zcols, F):
        for r in range(F.shape[0]):
            for k in range(F.shape[1]):
                if F[r, k] != 0.0:
                    put(erows[r], zcols[k], F[r, k])

    for c in t.nonroot:
        p = int(t.anc[c])
        # (Q^c^1/2 x^anc(c), R^c^1/2 u^anc(c), tau^c/2, tau^c/2)
        if P.dense_cost:
            put_block(lay.e_qx[c], lay.x[p], P.Qhalf(c))
            put_block(lay.e_ru[c], lay.u[p], P.Rhalf(c))
        else:
            for k in range(P.nx):
                put(lay.e_qx[c][k], lay.x[p][k], np.sqrt(P.Q[c, k]))
            for k in range(P.nu):
                put(lay.e_ru[c][k], lay.u[p][k], np.sqrt(P.R[c, k]))
        put(lay.e_t[c][0], lay.tau[c], 0.5)
        put(lay.e_t[c][1], lay.tau[c], 0.5)
    for j in t.leaves:
        # (Gamma_N x^j, (Q_N^1/2 x^j, s^j/2, s^j/2))
        if P.general:
            put_block(lay.e_lc[j], lay.x[j], P.GN[j])
        else:
            for k in range(P.nx):
                put(lay.e_lx[j][k], lay.x[j][k], 1.0)
        if P.dense_cost:
            put_block(lay.e_qn[j], lay.x[j], P.QNhalf(j))
        else:
            for k in range(P.nx):
                put(lay.e_qn[j][k], lay.x[j][k], np.sqrt(P.QN[j, k]))
        put(lay.e_ls[j][0], lay.s[j], 0.5)
        put(lay.e_ls[j][1], lay.s[j], 0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(lay.n_eta, lay.n_z))


def norm_L_blocks(P: Problem) -> float:
    """||L|| as the largest norm of the blocks of L after grouping columns by
    the rows they touch (remark after the definition of L).

    Column groups and their blocks (diagonal Q, R, Q_N, box Gamma = I):
      * x^i_k of nonleaf i: rows (box row, sqrt(Q^c_kk) for each child c)
        -> squared norm 1 + sum_c Q^c_kk;  u^i_k likewise with R;
      * x^j_k of leaf j: 1 + Q_N^j_kk;
      * tau^c, s^j (leaf): column (1/2, 1/2) -> 1/2;
      * (y^i, s^i) of nonleaf i against rows (y^i, s^i - b^T y^i): the matrix
        [[I, 0], [-b^T, 1]] whose largest singular value squared is
        (2 + beta^2 + beta sqrt(beta^2 + 4)) / 2 with beta = ||b^i||.
    """
    t = P.tree
    if P.general or P.dense_cost:
        return norm_L_blocks_general(P)
    best = 0.5
    for i in t.nonleaf:
        ch = t.children[i]
        best = max(best, float(np.max(1.0 + P.Q[ch].sum(axis=0))))
        best = max(best, float(np.max(1.0 + P.R[ch].sum(axis=0))))
        beta2 = float(np.dot(P.b(i), P.b(i)))
        beta = np.sqrt(beta2)
        best = max(best, (2.0 + beta2 + beta * np.sqrt(beta2 + 4.0)) / 2.0)
    for j in t.leaves:
        best = max(best, float(np.max(1.0 + P.QN[j])))
    return float(np.sqrt(best))


def norm_L_blocks_general(P: Problem) -> float:
    """||L|| by the same column grouping for the general form: the block of
    the columns (x^i, u^i) of nonleaf i stacks Gamma^i = [Gamma_x^i, Gamma_u^i]
    and, per child c, blockdiag(Q^c^1/2, R^c^1/2); its squared norm is the
    largest eigenvalue of Gamma^iT Gamma^i + sum_c blockdiag(Q^c, R^c)
    (F^T F = Q for the factor in L).  Leaf x^j: Gamma_N^jT Gamma_N^j + Q_N^j.
    The (y, s), tau and leaf-s blocks are those of the box form."""
    t, nx, nu = P.tree, P.nx, P.nu
    best = 0.5
    for i in t.nonleaf:
        if P.general:
            G = np.hstack([P.Gx[i], P.Gu[i]])
            M = G.T @ G
        else:
            M = np.eye(nx + nu)
        for c in t.children[i]:
            M[:nx, :nx] += P.Qmat(c)
            M[nx:, nx:] += P.Rmat(c)
        best = max(best, float(np.linalg.eigvalsh(M)[-1]))
        beta2 = float(np.dot(P.b(i), P.b(i)))
        beta = np.sqrt(beta2)
        best = max(best, (2.0 + beta2 + beta * np.sqrt(beta2 + 4.0)) / 2.0)
    for j in t.leaves:
        M = (P.GN[j].T @ P.GN[j]) if P.general else np.eye(nx)
        best = max(best, float(np.linalg.eigvalsh(M + P.QNmat(j))[-1]))
    return float(np.sqrt(best))


def norm_L_power(L: sp.spmatrix, iters=2000, seed=0) -> float:
    """||L|| by power iteration on L^T L (check of norm_L_blocks)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(L.shape[1])
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = L.T @ (L @ v)
        lam_new = float(np.linalg.norm(w))
        v = w / lam_new
        if abs(lam_new - lam) <= 1e-15 * lam_new:
            lam = lam_new
            break
        lam = lam_new
    return float(np.sqrt(lam))
