"""Projection onto the tree dynamics S1 (Sec. "Projection on S1") by a direct
KKT solve.  Oracle (test infrastructure only).

proj_S1(zbar_1) minimises 1/2 ||z_1 - zbar_1||^2 subject to G z_1 = h, where
the rows of G are x^0 = x (initial state) and x^c - A^c x^anc(c) - B^c
u^anc(c) = 0 for every nonroot c.  Its KKT system
    [ I  G^T ] [ z_1    ]   [ zbar_1 ]
    [ G  0   ] [ lambda ] = [ h      ]
is factored once (sparse LU, a library primitive) and solved per call, with
one step of iterative refinement.  This replaces the Riccati recursion of
Algorithms 1-2, which only the CUDA path uses.

Pins (tests/test_oracle_s1.py): exact feasibility, idempotence, optimality
(zbar - P(zbar) orthogonal to the null space of G, checked with
independently simulated feasible directions), and agreement with a
null-space-basis projection on tiny trees.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .problem import Problem


class S1Projector:
    def __init__(self, P: Problem):
        self.P = P
        t, nx, nu = P.tree, P.nx, P.nu
        lay = P.lay
        # z_1 occupies z[1 : 1 + n nx + |nonleaf| nu] (x block then u block)
        self.off = 1
        self.n1 = t.n * nx + len(t.nonleaf) * nu
        xi = lambda i: lay.x[i] - self.off
        ui = lambda i: lay.u[i] - self.off
        rows, cols, vals = [], [], []
        for k in range(nx):
            rows.append(k)
            cols.append(xi(0)[k])
            vals.append(1.0)
        r0 = nx
        for c in t.nonroot:
            p = int(t.anc[c])
            for k in range(nx):
                r = r0 + k
                rows.append(r)
                cols.append(xi(c)[k])
                vals.append(1.0)
                for j in range(nx):
                    if P.A[c, k, j] != 0.0:
                        rows.append(r)
                        cols.append(xi(p)[j])
                        vals.append(-P.A[c, k, j])
                for j in range(nu):
                    if P.B[c, k, j] != 0.0:
                        rows.append(r)
                        cols.append(ui(p)[j])
                        vals.append(-P.B[c, k, j])
            r0 += nx
        self.m = r0
        self.G = sp.csr_matrix((vals, (rows, cols)), shape=(self.m, self.n1))
        kkt = sp.bmat([[sp.identity(self.n1), self.G.T], [self.G, None]], format="csc")
        self.kkt = kkt
        self.lu = spla.splu(kkt)

    def rhs_h(self, x0):
        h = np.zeros(self.m)
        h[: self.P.nx] = x0
        return h

    def project(self, zbar1, x0):
        rhs = np.concatenate([zbar1, self.rhs_h(x0)])
        sol = self.lu.solve(rhs)
        sol = sol + self.lu.solve(rhs - self.kkt @ sol)
        return sol[: self.n1]

    def project_z(self, z, x0):
        """Apply proj_S1 to the z_1 part of a z-shaped vector."""
        out = np.array(z, dtype=float, copy=True)
        sl = slice(self.off, self.off + self.n1)
        out[sl] = self.project(z[sl], x0)
        return out
