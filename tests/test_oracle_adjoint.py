"""Adjoint (implicit differentiation of the CP fixed point) in the oracle:
for phi = s^0 (the optimal cost) it must equal the envelope gradient, itself
pinned by the closed-form tree LQR and finite differences; for phi = a
component of the first input u^0 (a solution component, which the envelope
theorem does not give) it must match central finite differences of solves
to 1e-12 in x0, in diag Q and in A."""
import numpy as np
import pytest

from oracle.adjoint import adjoint_gradient, dproj_soc
from oracle.cones import proj_soc
from oracle.cp import CP
from oracle.grad import envelope_gradient
from oracle.problem import Problem
from oracle.spock import Settings, spock
from paper_2212_01110_gb300 import workloads as W

TIGHT = Settings(eps_abs=1e-12, eps_rel=1e-12, memory=5, max_iter=100000)


def _solve(d):
    cp = CP(Problem(d))
    r = spock(cp, d["x0"], s=TIGHT)
    assert r.status == "converged"
    return cp, r.v[:cp.n_z], r.v[cp.n_z:]


def test_soc_jacobian_matches_finite_differences():
    rng = np.random.default_rng(0)
    for _ in range(20):
        w = rng.standard_normal(5)
        J = dproj_soc(w)
        h = 1e-7
        Jfd = np.column_stack([(proj_soc(w + h * e) - proj_soc(w - h * e)) / (2 * h) for e in np.eye(5)])
        assert np.max(np.abs(J - Jfd)) < 1e-6


@pytest.mark.parametrize("name", ["binary_N3", "fig1"])
def test_cost_gradient_equals_envelope_gradient(name):
    d = W.small_binary(0) if name == "binary_N3" else W.with_tree(W.fig1_tree(), seed=1, nx=3, nu=2)
    cp, z, e = _solve(d)
    env = envelope_gradient(cp, z, e)
    adj = adjoint_gradient(cp, z, e)
    assert adj["gmres_info"] == 0 and adj["adjoint_residual"] < 1e-10
    for k in ("x0", "A", "B", "Q", "R", "QN"):
        scale = max(1.0, float(np.max(np.abs(env[k]))))
        assert np.max(np.abs(adj[k] - env[k])) < 1e-8 * scale, k


def test_first_input_sensitivity_matches_finite_differences():
    d = W.small_binary(0)
    cp, z, e = _solve(d)
    lay = cp.P.lay
    j = int(lay.u[0][0])          # phi = u^0_0
    g = np.zeros(cp.n_z)
    g[j] = 1.0
    adj = adjoint_gradient(cp, z, e, g=g)
    rng = np.random.default_rng(3)
    h = 1e-4                      # u^0 is piecewise smooth in the data: central differences on one piece

    def u0(dd):
        _, zz, _ = _solve(dd)
        return zz[j]

    dx = rng.standard_normal(d["nx"])
    fd = (u0(dict(d, x0=d["x0"] + h * dx)) - u0(dict(d, x0=d["x0"] - h * dx))) / (2 * h)
    assert abs(float(adj["x0"] @ dx) - fd) < 1e-5 * max(1.0, abs(fd))
    dq = rng.standard_normal(d["Q"].shape)
    dq[0] = 0.0
    fdq = (u0(dict(d, Q=d["Q"] + h * dq)) - u0(dict(d, Q=d["Q"] - h * dq))) / (2 * h)
    assert abs(float(np.sum(adj["Q"] * dq)) - fdq) < 1e-5 * max(1.0, abs(fdq))
    dA = np.zeros_like(d["A"])
    dA[1:] = rng.standard_normal(d["A"][1:].shape)
    fda = (u0(dict(d, A=d["A"] + h * dA)) - u0(dict(d, A=d["A"] - h * dA))) / (2 * h)
    assert abs(float(np.sum(adj["A"] * dA)) - fda) < 1e-5 * max(1.0, abs(fda))
