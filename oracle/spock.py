"""SPOCK: SuperMann with Chambolle-Pock and Anderson directions
(Algorithm 3, Sec. "SuperMann", Sec. "Anderson's acceleration").
Oracle (test infrastructure only).

Readings of the paper (each also listed in the design notes):
  * Order of steps: per iteration r = v - T(v) and omega = ||r||_M are
    available first, then the termination test on xi(r), then the Anderson
    update with (v, c = r), then K0 / line search.  After a K1 step the
    residual of the trial point is reused.
  * rho = omega~^2 - coef * <r~, v~ - v>_M with coef = 1: the factor 2 alpha
    printed in Algorithm 3 is SuperMann's averagedness 1/2 for a firmly
    nonexpansive T (not the CP step), so 2 * 1/2 = 1.
  * The line search is capped at ``max_backtracks``; at the cap tau = 0 is
    taken, which makes K2 the plain relaxed step v - lambda r.
  * Anderson memory m = number of stored difference columns; with no column
    yet, d = -c.  gamma is the least-squares solution (numpy lstsq).
  * SuperMann parameters are not printed in the paper (they are deferred to
    the SuperMann paper); defaults c0 = c1 = c2 = 0.99, beta = 0.5,
    sigma = 0.1, lambda = 1, m = 3.
  * The returned point is T(v) at termination, the pair the certificate xi
    is about.

``forced`` replays a branch trace (one entry per iteration, as produced in
``trace``) instead of taking decisions; fixed-iteration comparisons use it so
that a near-tie decided differently in other floating-point arithmetic does
not change the path.

Parity of the branch logic is pinned only indirectly (converged solutions
against closed forms / brute force, tests/test_oracle_spock.py); the
iteration counts printed in the paper cannot be reproduced without its
SuperMann parameters ("parity unpinned" for those counts).
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass, field

import numpy as np

from .cp import CP


@dataclass
class Settings:
    eps_abs: float = 1e-6
    eps_rel: float = 1e-6
    memory: int = 3
    c0: float = 0.99
    c1: float = 0.99
    c2: float = 0.99
    beta: float = 0.5
    sigma: float = 0.1
    lam: float = 1.0
    rho_coef: float = 1.0
    max_iter: int = 100000
    max_backtracks: int = 30


@dataclass
class Result:
    v: np.ndarray            # T(v^(k)) at termination (or the last iterate)
    v_iter: np.ndarray       # v^(k)
    status: str
    k: int
    xi: float
    xi0: float
    trace: list = field(default_factory=list)
    n_T: int = 0
    xi_hist: list = field(default_factory=list)


class Anderson:
    """Buffers M^P (differences of v) and M^R (differences of c), memory m."""

    def __init__(self, m):
        self.m = m
        self.P = deque()
        self.R = deque()
        self.v_prev = None
        self.c_prev = None

    def push(self, v, c):
        if self.v_prev is not None and self.m > 0:
            self.P.append(v - self.v_prev)
            self.R.append(c - self.c_prev)
            if len(self.P) > self.m:
                self.P.popleft()
                self.R.popleft()
        self.v_prev = v.copy()
        self.c_prev = c.copy()

    def direction(self, c):
        """d = -c - (M^P - M^R) gamma, gamma = argmin ||M^R gamma - c||."""
        if not self.P:
            return -c
        MP = np.column_stack(list(self.P))
        MR = np.column_stack(list(self.R))
        gamma = np.linalg.lstsq(MR, c, rcond=None)[0]
        return -c - (MP - MR) @ gamma


def spock(cp: CP, x0, v0=None, s: Settings = None, forced=None):
    s = s or Settings()
    n = cp.n_z + cp.n_eta
    v = np.zeros(n) if v0 is None else np.array(v0, dtype=float, copy=True)
    nT = 0

    def R_eval(w):
        nonlocal nT
        nT += 1
        Tw = cp.T(w, x0)
        st = cp.stats(w, Tw)
        st["Tv"] = Tw
        return st

    cur = R_eval(v)
    zeta = cur["omega"]
    omega_safe = zeta
    xi0 = cur["xi"]
    tol = max(s.eps_abs, s.eps_rel * xi0)
    aa = Anderson(s.memory)
    trace = []
    xi_hist = [cur["xi"]]
    k = 0
    status = "max_iter"
    while True:
        if cur["xi"] <= tol:
            status = "converged"
            break
        if k >= s.max_iter or (forced is not None and k >= len(forced)):
            break
        r, omega = cur["r"], cur["omega"]
        aa.push(v, r)
        d = aa.direction(r)
        want = forced[k] if forced is not None else None
        if (want is None and omega <= s.c0 * zeta) or (want is not None and want[0] == "K0"):
            v = v + d
            zeta = omega
            cur = R_eval(v)
            trace.append(("K0", 0))
        else:
            tau = 1.0
            nb = 0
            while True:
                capped = (want is None and nb >= s.max_backtracks) or (want is not None and want[0] == "CAP" and nb >= want[1])
                if capped:
                    # tau = 0: v~ = v, r~ = r, rho = omega^2 -> relaxed step
                    rho = omega * omega
                    v = v - s.lam * r
                    cur = R_eval(v)
                    trace.append(("CAP", nb))
                    break
                vt = v + tau * d
                new = R_eval(vt)
                om_t = new["omega"]
                k1 = omega <= omega_safe and om_t <= s.c1 * omega
                if want is not None:
                    k1 = want[0] == "K1" and nb == want[1]
                if k1:
                    v = vt
                    omega_safe = om_t + s.c2 ** k
                    cur = new
                    trace.append(("K1", nb))
                    break
                rho = om_t ** 2 - s.rho_coef * cp.inner_M(new["r"], vt - v)
                k2 = rho >= s.sigma * om_t * omega
                if want is not None:
                    k2 = want[0] == "K2" and nb == want[1]
                if k2:
                    v = v - s.lam * rho / (om_t ** 2) * new["r"]
                    cur = R_eval(v)
                    trace.append(("K2", nb))
                    break
                tau *= s.beta
                nb += 1
        k += 1
        xi_hist.append(cur["xi"])
    return Result(v=cur["Tv"], v_iter=v, status=status, k=k, xi=cur["xi"], xi0=xi0,
                  trace=trace, n_T=nT, xi_hist=xi_hist)
