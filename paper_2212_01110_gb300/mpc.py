"""Closed-loop model predictive control with warm starts (the paper's
closed-loop simulation: successive RAOCPs solved for successive initial
states, each solve started from the previous step's primal and dual
vectors).

Every solve runs in the library (spock_solve_dev); this module only steps
the plant between solves: the realised disturbance of a step is one child of
the root, drawn with its conditional probability, and the plant moves with
that child's dynamics, x+ = A^c x + B^c u^0 (the dynamics are the same at
every stage of the paper's scenario trees, so the root's children describe
the plant).
"""
from __future__ import annotations

import numpy as np


def closed_loop(spock, d, steps=20, seed=0, tol=1e-3, precision=0, memory=3, warm=True, device=None,
                max_iter=100000):
    """Runs ``steps`` MPC steps from d["x0"].  Returns one record per step:
    iterations, evaluations of T, device time of the solve (ms), the applied
    input u^0 and the state.  ``warm=False`` cold-starts every solve."""
    import torch
    dev = device or torch.device("cuda:0")
    P = spock.Problem(d)
    try:
        anc = np.asarray(d["anc"])
        children = np.flatnonzero(anc == 0)
        probs = np.asarray(d["prob"])[children]
        probs = probs / probs.sum()
        A = np.asarray(d["A"]).reshape(len(anc), P.nx, P.nx)
        B = np.asarray(d["B"]).reshape(len(anc), P.nx, P.nu)
        umin, umax = np.asarray(d["umin"]).reshape(len(anc), P.nu)[0], np.asarray(d["umax"]).reshape(len(anc), P.nu)[0]
        xmin, xmax = np.asarray(d["xmin"]).reshape(len(anc), P.nx)[0], np.asarray(d["xmax"]).reshape(len(anc), P.nx)[0]
        rng = np.random.default_rng(seed)
        x = np.array(d["x0"], dtype=np.float64)
        z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
        e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
        u_slice = slice(1 + len(anc) * P.nx, 1 + len(anc) * P.nx + P.nu)   # u of the root (user layout)
        st = spock.spock_default_settings(eps_abs=tol, eps_rel=tol, memory=memory, precision=precision,
                                          max_iter=max_iter)
        out = []
        for k in range(steps):
            x0 = torch.tensor(x, dtype=torch.float64, device=dev)
            info = spock.spock_solve_dev(P.handle, x0, st, z, e, 1 if (warm and k > 0) else 0)
            u0 = z[u_slice].cpu().numpy()
            # the solution meets its box up to the tolerance: apply the clipped input
            u0 = np.clip(u0, umin, umax)
            out.append({"step": k, "iterations": info.iterations, "n_T": info.n_T, "ms": info.solve_ms,
                        "status": info.status, "xi": info.xi, "u0": u0.copy(), "x": x.copy()})
            c = children[rng.choice(len(children), p=probs)]
            x = A[c] @ x + B[c] @ u0
            # the predicted child state meets its box up to the solve tolerance;
            # clipping absorbs that tolerance so the next problem stays feasible
            x = np.clip(x, xmin, xmax)
        return out
    finally:
        P.close()
