"""torch.autograd.Function around spock_solve_dev / spock_grad_dev: the
optimal risk-averse cost V*(x0, Q, R, Q_N, A, B) of a problem on a fixed
tree, differentiable in those arguments.

Forward: build the problem from the (detached) data, solve to the given
tolerance on the GPU, return s^0.  Backward: the envelope gradient of the
library (spock_grad_dev) at the returned primal-dual pair, scaled by the
incoming gradient.  Marshalling only: every step runs in libspock.
"""
from __future__ import annotations

import numpy as np
import torch

from . import spock


class SpockValue(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, Q, R, QN, A, B, static, settings):
        d = dict(static)
        for k, t in (("Q", Q), ("R", R), ("QN", QN), ("A", A), ("B", B)):
            d[k] = t.detach().double().cpu().numpy()
        d["x0"] = x0.detach().double().cpu().numpy()
        P = spock.Problem(d)
        dev = x0.device
        xd = x0.detach().double().to(dev).contiguous()
        z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
        e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
        info = spock.spock_solve_dev(P.handle, xd, settings, z, e, 0)
        ctx.P, ctx.z, ctx.e, ctx.info = P, z, e, info
        ctx.precision = int(settings.precision)
        ctx.shapes = (x0.shape, Q.shape, R.shape, QN.shape, A.shape, B.shape)
        ctx.dtypes = (x0.dtype, Q.dtype, R.dtype, QN.dtype, A.dtype, B.dtype)
        return z[0].detach().clone().to(x0.dtype)

    @staticmethod
    def backward(ctx, gout):
        P, dev = ctx.P, ctx.z.device
        n = P.n_nodes
        gx0 = torch.zeros(P.nx, dtype=torch.float64, device=dev)
        gA = torch.zeros(n, P.nx, P.nx, dtype=torch.float64, device=dev)
        gB = torch.zeros(n, P.nx, P.nu, dtype=torch.float64, device=dev)
        gQ = torch.zeros(n, P.nx, dtype=torch.float64, device=dev)
        gR = torch.zeros(n, P.nu, dtype=torch.float64, device=dev)
        gQN = torch.zeros(n, P.nx, dtype=torch.float64, device=dev)
        spock.spock_grad_dev(P.handle, ctx.z, ctx.e, ctx.precision, gx0, gA, gB, gQ, gR, gQN)
        s = gout.to(torch.float64)
        outs = []
        for g, shp, dt in zip((gx0, gQ, gR, gQN, gA, gB), ctx.shapes, ctx.dtypes):
            outs.append((s * g).reshape(shp).to(dt))
        P.close()
        return (*outs, None, None)


def optimal_cost(d, x0, Q, R, QN, A, B, settings=None):
    """V*(x0, Q, R, Q_N, A, B) for the tree, probabilities, AV@R parameters
    and boxes of the workload dict d (other entries of d are ignored)."""
    static = {k: d[k] for k in ("anc", "prob", "nx", "nu", "a", "xmin", "xmax", "umin", "umax")}
    st = settings if settings is not None else spock.spock_default_settings(eps_abs=1e-10, eps_rel=1e-10,
                                                                              memory=5, max_iter=200000)
    return SpockValue.apply(x0, Q, R, QN, A, B, static, st)
