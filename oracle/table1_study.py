"""SPOCK iteration counts on the data-center system of the paper's numerical
section (Eq. (dynamics-example); Table 1: nx = nu = 50, x0 = 0.1 * 1,
tolerance 1e-3, AV@R_0.95, two disturbance values with probabilities 0.3 and
0.7), computed with the oracle alone.  Oracle (test infrastructure only): a
study of how the method behaves on the paper's own workload; the CUDA path is
not involved.

    python -m oracle.table1_study            # a few minutes on one core
    python -m oracle.table1_study --sweep    # plus the SuperMann parameter sweep
    python -m oracle.table1_study --fig1     # the Fig. 1 setting instead (about a minute)

Prints, for horizons N = 3 and 6:
  * the problem as printed (R = 10 I): ||L||, and the iterations with
    Anderson memory 3 and 10;
  * the same problem in the scaled input u' = sqrt(10) u (R = I, B / sqrt(10),
    input box times sqrt(10)): an equivalent problem with the same optimal
    value (the cost rows R^1/2 u = u' and the dynamics B u = (B / sqrt(10)) u'
    are unchanged), but ||L|| drops from sqrt(1 + sum_c R^c) = sqrt(21) (the
    input columns of a node with two children) to 1.81 (the (y, s) block of
    the AV@R rows), so the step alpha = 0.99 / ||L|| grows 2.5 times; the
    iterations with memory 3 and 10;
  * the cost s^0 of both forms at termination (equal up to the accuracy the
    tolerance, a bound on the residual xi, allows: about 1e-2 here);
and with --sweep the best of 108 SuperMann parameter combinations (memory
3/5/10, lambda 1/1.5/1.9, sigma 0.1/1e-2/1e-4, c0 = c1 = c2 0.99/0.9,
beta 0.5/0.8) on the printed problem at N = 3.  The paper reports 105 (N = 3)
and 128 (N = 6) iterations without printing its SuperMann parameters.

With --fig1: the setting of Fig. 1 (N = 7, nx = nu = 5, tolerance 1e-5),
printed and in scaled inputs, vanilla CP iterations and SPOCK iterations /
evaluations of T to the tolerance (Fig. 1 plots xi against calls of L: 3,159
for CP and 571 for SPOCK, with no statement of how calls are counted).
"""
from __future__ import annotations

import itertools
import sys

import numpy as np

from oracle.cp import CP
from oracle.problem import Problem
from oracle.spock import Settings, spock

TOL = 1e-3
TABLE1 = {3: 105, 6: 128}   # iterations printed in Table 1


def printed(N):
    from paper_2212_01110_gb300 import workloads as W
    return W.datacenter(N=N, nx=50)


def scaled_inputs(d, r=10.0):
    """The change of input u' = sqrt(r) u: R = r I becomes I, B becomes
    B / sqrt(r) and the input box is multiplied by sqrt(r)."""
    sc = np.sqrt(r)
    e = dict(d)
    e["B"] = np.asarray(d["B"]) / sc
    e["R"] = np.asarray(d["R"]) / r
    e["umin"], e["umax"] = np.asarray(d["umin"]) * sc, np.asarray(d["umax"]) * sc
    return e


def iterations(d, memory, **kw):
    cp = CP(Problem(d))
    res = spock(cp, d["x0"], s=Settings(eps_abs=TOL, eps_rel=TOL, max_iter=5000, memory=memory, **kw))
    return cp.normL, res


def main(sweep=False):
    for N in (3, 6):
        d = printed(N)
        e = scaled_inputs(d)
        for name, prob in (("printed (R = 10 I)", d), ("scaled inputs (R = I)", e)):
            for m in (3, 10):
                nL, res = iterations(prob, m)
                print(f"N = {N:2d}  {name:22s} ||L|| = {nL:.3f}  memory {m:2d}: {res.k:4d} iterations "
                      f"({res.n_T} T, {res.status}), s0 = {res.v[0]:.6f}   [Table 1: {TABLE1[N]}]", flush=True)
    if sweep:
        d = printed(3)
        cp = CP(Problem(d))
        rows = []
        for mem, lam, sig, c0, beta in itertools.product((3, 5, 10), (1.0, 1.5, 1.9), (0.1, 1e-2, 1e-4),
                                                         (0.99, 0.9), (0.5, 0.8)):
            s = Settings(eps_abs=TOL, eps_rel=TOL, max_iter=5000, memory=mem, lam=lam, sigma=sig,
                         c0=c0, c1=c0, c2=c0, beta=beta)
            r = spock(cp, d["x0"], s=s)
            rows.append((r.k, mem, lam, sig, c0, beta, r.status))
        rows.sort()
        print(f"SuperMann sweep at N = 3 (printed problem), {len(rows)} combinations; best five "
              "(iterations, memory, lambda, sigma, c, beta, status):")
        for row in rows[:5]:
            print("  ", row)


def fig1():
    from paper_2212_01110_gb300 import workloads as W
    d = W.datacenter(N=7, nx=5)
    tol = 1e-5
    for name, prob in (("printed (R = 10 I)", d), ("scaled inputs (R = I)", scaled_inputs(d))):
        cp = CP(Problem(prob))
        v = np.zeros(cp.n_z + cp.n_eta)
        xi0 = None
        k = 0
        for k in range(1, 20001):   # vanilla CP: v <- T(v) until xi <= max(tol, tol xi0)
            Tv = cp.T(v, prob["x0"])
            xi = cp.stats(v, Tv)["xi"]
            xi0 = xi if xi0 is None else xi0
            if xi <= max(tol, tol * xi0):
                break
            v = Tv
        r = spock(cp, prob["x0"], s=Settings(eps_abs=tol, eps_rel=tol, max_iter=20000))
        print(f"Fig. 1 setting, {name:22s} ||L|| = {cp.normL:.3f}: vanilla CP {k} evaluations of T; "
              f"SPOCK {r.k} iterations, {r.n_T} evaluations of T ({r.status})", flush=True)


if __name__ == "__main__":
    if "--fig1" in sys.argv:
        fig1()
    else:
        main(sweep="--sweep" in sys.argv)
