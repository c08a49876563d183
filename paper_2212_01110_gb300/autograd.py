"""torch.autograd.Functions around spock_solve_dev and the library's
gradients, on a fixed tree:
  SpockValue   the optimal risk-averse cost V*(x0, Q, R, Q_N, A, B);
               backward: the envelope gradient (spock_grad_dev) at the
               returned primal-dual pair;
  SpockPolicy  (V*, u^0*): the optimal cost and the first input of the
               solution (the MPC control law) as functions of the data;
               backward: one adjoint solve of the CP fixed point
               (spock_adjoint_dev) for the incoming gradient
               g = dL/dV* e_{s^0} + sum_j dL/du^0_j e_{u^0_j}.
Forward: build the problem from the (detached) data, solve to the given
tolerance on the GPU.  Marshalling only: every step runs in libspock.
"""
from __future__ import annotations

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


def _solve(x0, Q, R, QN, A, B, static, settings):
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
    return P, z, e, info


class SpockPolicy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, Q, R, QN, A, B, static, settings, adj_iter, adj_tol):
        P, z, e, info = _solve(x0, Q, R, QN, A, B, static, settings)
        ctx.P, ctx.z, ctx.e, ctx.info = P, z, e, info
        ctx.adj = (int(adj_iter), float(adj_tol))
        ctx.u0 = 1 + P.n_nodes * P.nx        # u of the root in the z layout
        ctx.shapes = (x0.shape, Q.shape, R.shape, QN.shape, A.shape, B.shape)
        ctx.dtypes = (x0.dtype, Q.dtype, R.dtype, QN.dtype, A.dtype, B.dtype)
        v = z[0].detach().clone().to(x0.dtype)
        u0 = z[ctx.u0:ctx.u0 + P.nu].detach().clone().to(x0.dtype)
        return v, u0

    @staticmethod
    def backward(ctx, gv, gu):
        P, dev = ctx.P, ctx.z.device
        n = P.n_nodes
        g = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
        if gv is not None:
            g[0] = gv.to(torch.float64)
        if gu is not None:
            g[ctx.u0:ctx.u0 + P.nu] = gu.to(torch.float64)
        outs = [torch.zeros(P.nx, dtype=torch.float64, device=dev),
                torch.zeros(n, P.nx, P.nx, dtype=torch.float64, device=dev),
                torch.zeros(n, P.nx, P.nu, dtype=torch.float64, device=dev),
                torch.zeros(n, P.nx, dtype=torch.float64, device=dev),
                torch.zeros(n, P.nu, dtype=torch.float64, device=dev),
                torch.zeros(n, P.nx, dtype=torch.float64, device=dev)]
        gx0, gA, gB, gQ, gR, gQN = outs
        spock.spock_adjoint_dev(P.handle, ctx.z, ctx.e, g, ctx.adj[0], ctx.adj[1], gx0, gA, gB, gQ, gR, gQN)
        res = [t.reshape(shp).to(dt) for t, shp, dt in zip((gx0, gQ, gR, gQN, gA, gB), ctx.shapes, ctx.dtypes)]
        P.close()
        return (*res, None, None, None, None)


def policy(d, x0, Q, R, QN, A, B, settings=None, adj_iter=200000, adj_tol=1e-11):
    """(V*, u^0*) for the tree, probabilities, AV@R parameters and boxes of
    the workload dict d, differentiable in x0, Q, R, Q_N, A, B by the adjoint
    of the CP fixed point."""
    static = {k: d[k] for k in ("anc", "prob", "nx", "nu", "a", "xmin", "xmax", "umin", "umax")}
    st = settings if settings is not None else spock.spock_default_settings(eps_abs=1e-11, eps_rel=1e-11,
                                                                              memory=5, max_iter=200000)
    return SpockPolicy.apply(x0, Q, R, QN, A, B, static, st, adj_iter, adj_tol)
