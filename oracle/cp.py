"""Chambolle-Pock operator T (Eq. (chambolle-pock-operator)), residual
R = id - T, the termination quantities xi_p, xi_d, xi and the M-metric
(Sec. "The Chambolle-Pock method"), prox of f (Sec. "Proximal operator of
f").  Oracle (test infrastructure only).

Reading: the CP step is alpha = 0.99 / ||L|| unless given (the paper only
asks 0 < alpha ||L|| < 1).

Pins (tests/test_oracle_cp.py): firm nonexpansiveness of T in the M-norm on
random pairs, and -- through the SPOCK solve -- the converged solution
against closed forms and brute force (tests/test_oracle_spock.py).
"""
from __future__ import annotations

import numpy as np

from .cones import proj_S2, prox_gconj
from .linop import build_L, norm_L_blocks
from .problem import Problem
from .s1 import S1Projector


class CP:
    def __init__(self, P: Problem, alpha=None):
        self.P = P
        self.L = build_L(P)
        self.Lt = self.L.T.tocsr()
        self.normL = norm_L_blocks(P)
        self.alpha = 0.99 / self.normL if alpha is None else float(alpha)
        self.S1 = S1Projector(P)
        self.n_z = P.lay.n_z
        self.n_eta = P.lay.n_eta
        self.n_L = 0  # applications of L (counted like the paper's Fig. 1 x-axis)

    # -- operators -----------------------------------------------------------
    def apply_L(self, z):
        self.n_L += 1
        return self.L @ z

    def apply_Lt(self, eta):
        return self.Lt @ eta

    def prox_f(self, z, x0):
        """prox_{alpha f}: s^0 - alpha, proj_S1 on z_1, proj_S2 on z_2 (the
        separable sum of Eq. (f))."""
        out = self.S1.project_z(z, x0)
        out = proj_S2(out, self.P)
        out[self.P.lay.s0] = z[self.P.lay.s0] - self.alpha
        return out

    def prox_gconj(self, eta):
        return prox_gconj(eta, self.alpha, self.P)

    def T(self, v, x0):
        """T(z, eta) = (prox_{alpha f}(z - alpha L* eta),
                        prox_{alpha g*}(eta + alpha L (2 z+ - z)))."""
        z, eta = v[: self.n_z], v[self.n_z:]
        zp = self.prox_f(z - self.alpha * self.apply_Lt(eta), x0)
        etap = self.prox_gconj(eta + self.alpha * self.apply_L(2.0 * zp - z))
        return np.concatenate([zp, etap])

    # -- residual quantities -------------------------------------------------
    def split(self, v):
        return v[: self.n_z], v[self.n_z:]

    def stats(self, v, Tv):
        """r = v - T(v); xi_p = r_z / alpha - L* r_eta; xi_d = r_eta / alpha -
        L r_z; xi = max(||xi_p||_inf, ||xi_d||_inf); omega = ||r||_M."""
        r = v - Tv
        rz, re = self.split(r)
        Lrz = self.apply_L(rz)
        Ltre = self.apply_Lt(re)
        xi_p = rz / self.alpha - Ltre
        xi_d = re / self.alpha - Lrz
        xi = max(np.max(np.abs(xi_p)), np.max(np.abs(xi_d)))
        om2 = float(rz @ (rz - self.alpha * Ltre) + re @ (re - self.alpha * Lrz))
        return dict(r=r, xi=float(xi), omega=float(np.sqrt(max(om2, 0.0))), omega2=om2)

    def inner_M(self, a, b):
        """<a, M b> with M(z, eta) = (z - alpha L* eta, eta - alpha L z)."""
        az, ae = self.split(a)
        bz, be = self.split(b)
        return float(az @ (bz - self.alpha * self.apply_Lt(be)) + ae @ (be - self.alpha * self.apply_L(bz)))

    def norm_M(self, a):
        return float(np.sqrt(max(self.inner_M(a, a), 0.0)))


def vanilla_cp(cp: CP, v0, x0, k):
    """k iterations v <- T(v) (Eq. (chambolle-pock-operator)).  Returns the
    last iterate T(v_{k-1}) and xi of the pair (v_{k-1}, T(v_{k-1}))."""
    v = np.array(v0, dtype=float, copy=True)
    xi = float("nan")
    for it in range(k):
        Tv = cp.T(v, x0)
        if it == k - 1:
            xi = cp.stats(v, Tv)["xi"]
        v = Tv
    return v, xi
