"""Convergence of vanilla CP and SPOCK on small members of the large-tree
family (branching 4, Dirichlet(1) child probabilities floored at 1e-3,
AV@R parameter U(0.1, 0.9), Haar-orthogonal A scaled to 0.95), computed
with the oracle alone.  Oracle (test infrastructure only): a study that
documents how the method itself behaves on that workload; the CUDA path is
not involved.

    python -m oracle.convergence_study            # about 10 minutes on one core

Prints, for the 85-node member (branching 4 for 2 stages, N = 6, nx = 10,
nu = 4): xi of vanilla CP every 1,000 iterations up to 20,000; SPOCK with
Anderson memory 3 and 10 up to 20,000 iterations; and the variants with the
boxes removed, with a = 1, and with uniform child probabilities; the
components of the residual that remain largest after 8,000 CP iterations;
finally SPOCK (memory 5) to 1e-6 on a 31-node member (branching 3 for 2
stages, N = 4, nx = 10, nu = 4) with the Dirichlet child probabilities and
with uniform ones.

    python -m oracle.convergence_study --batch   # about 15 minutes

instead runs SPOCK (memory 3, at most 10,000 iterations) on the six smallest
and the median-size instance of the batched workload (512 instances, seed 0).
"""
from __future__ import annotations

import sys
from collections import Counter

import numpy as np

from oracle.cp import CP
from oracle.problem import Problem
from oracle.spock import Settings, spock


def member(variant="", small=False):
    from paper_2212_01110_gb300 import workloads as W
    if small:
        d = W.large_tree(seed=0, branching_stages=2, branch=3, N=4, nx=10, nu=4)
    else:
        d = W.large_tree(seed=0, branching_stages=2, N=6, nx=10, nu=4)
    if "nobox" in variant:
        for k in ("xmin", "umin"):
            d[k][:] = -1e3
        for k in ("xmax", "umax"):
            d[k][:] = 1e3
    if "a1" in variant:
        d["a"][:] = 1.0
    if "uniform" in variant:
        d["prob"] = W._conditional_probs(None, d["anc"], "uniform")
    return d


def cp_history(d, iters, every):
    cp = CP(Problem(d))
    v = np.zeros(cp.n_z + cp.n_eta)
    hist = []
    for k in range(iters):
        Tv = cp.T(v, d["x0"])
        if k % every == 0 or k == iters - 1:
            st = cp.stats(v, Tv)
            hist.append((k, st["xi"], st["omega"]))
        v = Tv
    return cp, v, hist


def largest_residual_components(cp, v, d, count=8):
    """Names of the primal / dual residual entries that dominate xi."""
    lay = cp.P.lay
    zname = {lay.s0: "s0"}
    for i, ix in lay.y.items():
        for k, j in enumerate(ix):
            zname[int(j)] = f"y^{i}[{k}]"
    for c, j in lay.tau.items():
        zname[int(j)] = f"tau^{c}"
    for c, j in lay.s.items():
        if c:
            zname[int(j)] = f"s^{c}"
    Tv = cp.T(v, d["x0"])
    r = v - Tv
    xp = r[: cp.n_z] / cp.alpha - cp.Lt @ r[cp.n_z:]
    return [(zname.get(int(j), f"z[{j}]"), float(xp[j]), float(v[j])) for j in np.argsort(-np.abs(xp))[:count]]


def main(quick=False):
    iters = 4000 if quick else 20000
    every = iters // 20
    for variant in ("", "nobox", "a1", "uniform"):
        d = member(variant)
        cp, v, hist = cp_history(d, iters if variant == "" else iters // 2, every)
        print(f"vanilla CP {variant or 'as drawn'}: " + ", ".join(f"{k}: {xi:.2e}" for k, xi, _ in hist), flush=True)
        if variant == "":
            print("largest primal residual entries (name, xi_p, value):", largest_residual_components(cp, v, d))
    d = member()
    cp = CP(Problem(d))
    for m in (3, 10):
        r = spock(cp, d["x0"], s=Settings(memory=m, max_iter=iters))
        h = r.xi_hist
        print(f"SPOCK m={m}: status {r.status}, {r.k} iterations, {r.n_T} evaluations of T, "
              f"branches {dict(Counter(t[0] for t in r.trace))}, xi every {len(h) // 10}: "
              + ", ".join(f"{h[k]:.1e}" for k in range(0, len(h), max(1, len(h) // 10))), flush=True)
    for variant in ("", "uniform"):
        d = member(variant, small=True)
        r = spock(CP(Problem(d)), d["x0"], s=Settings(memory=5, max_iter=iters))
        print(f"SPOCK m=5 on the 31-node member, {variant or 'Dirichlet'} probabilities: status {r.status}, "
              f"{r.k} iterations, branches {dict(Counter(t[0] for t in r.trace))}", flush=True)


def batch_members():
    from paper_2212_01110_gb300 import workloads as W
    ds = W.batch_instances(seed=0, count=512)
    order = sorted(range(len(ds)), key=lambda i: len(ds[i]["anc"]) * (ds[i]["nx"] + ds[i]["nu"]))
    for i in order[:6] + [order[len(order) // 2]]:
        d = ds[i]
        cp = CP(Problem(d))
        r = spock(cp, d["x0"], s=Settings(max_iter=10000))
        h = r.xi_hist
        print(f"instance {i}: {len(d['anc'])} nodes, nx {d['nx']}, nu {d['nu']}, ||L|| {cp.normL:.2f}: "
              f"{r.status} after {r.k} iterations, branches {dict(Counter(t[0] for t in r.trace))}, xi "
              + ", ".join(f"{h[k]:.1e}" for k in range(0, len(h), max(1, len(h) // 8))), flush=True)


if __name__ == "__main__":
    if "--batch" in sys.argv:
        batch_members()
    else:
        main(quick="--quick" in sys.argv)
