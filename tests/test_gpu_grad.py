"""Gradient of the optimal cost through the C-ABI (spock_grad_dev) and the
torch.autograd.Function: against the oracle's envelope gradient at the same
converged pair, against finite differences of the closed-form tree-LQR cost
(a = 1, inactive constraints), and FP32 against FP64."""
import numpy as np
import pytest

from oracle.cp import CP
from oracle.grad import envelope_gradient
from oracle.lqr import tree_lqr
from oracle.problem import Problem as OProblem
from oracle.spock import Settings as OSettings, spock as ospock
from paper_2212_01110_gb300 import workloads as W

pytestmark = pytest.mark.gpu
KEYS = ("x0", "A", "B", "Q", "R", "QN")


def _gpu_grad(gp, z, e, precision=0):
    import torch
    from paper_2212_01110_gb300 import spock
    dev = z.device
    n, nx, nu = gp.n_nodes, gp.nx, gp.nu
    out = {"x0": torch.zeros(nx, dtype=torch.float64, device=dev),
           "A": torch.zeros(n, nx, nx, dtype=torch.float64, device=dev),
           "B": torch.zeros(n, nx, nu, dtype=torch.float64, device=dev),
           "Q": torch.zeros(n, nx, dtype=torch.float64, device=dev),
           "R": torch.zeros(n, nu, dtype=torch.float64, device=dev),
           "QN": torch.zeros(n, nx, dtype=torch.float64, device=dev)}
    spock.spock_grad_dev(gp.handle, z, e, precision, out["x0"], out["A"], out["B"], out["Q"], out["R"], out["QN"])
    return {k: v.cpu().numpy() for k, v in out.items()}


def _unconstrained_a1(d):
    d = dict(d)
    n = len(d["anc"])
    d["xmin"], d["xmax"] = -1e6 * np.ones((n, d["nx"])), 1e6 * np.ones((n, d["nx"]))
    d["umin"], d["umax"] = -1e6 * np.ones((n, d["nu"])), 1e6 * np.ones((n, d["nu"]))
    d["a"] = np.ones(n)
    return d


@pytest.mark.parametrize("d", [W.small_binary(0), W.with_tree(W.fig1_tree(), seed=2, nx=3, nu=2, a=0.4),
                               W.random_tree(3, N=4, max_branch=3, nx=4, nu=3),
                               W.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2)])
def test_grad_matches_oracle_at_same_pair(d):
    """Both evaluate the envelope formula at the oracle's converged pair; they
    differ only in how the dynamics multipliers are obtained (tree recursion
    on the x-rows vs least squares on all rows), which agree at a saddle
    point up to the pair's KKT residual."""
    import torch
    from paper_2212_01110_gb300 import spock
    op = OProblem(d)
    cp = CP(op)
    res = ospock(cp, d["x0"], s=OSettings(eps_abs=1e-12, eps_rel=1e-12, memory=5, max_iter=100000))
    assert res.status == "converged"
    z, eta = res.v[:cp.n_z], res.v[cp.n_z:]
    ref = envelope_gradient(cp, z, eta)
    gp = spock.Problem(d)
    dev = torch.device("cuda:0")
    got = _gpu_grad(gp, torch.tensor(z, device=dev), torch.tensor(eta, device=dev))
    for k in KEYS:
        scale = max(1.0, float(np.max(np.abs(ref[k]))))
        assert np.max(np.abs(got[k] - ref[k])) < 1e-8 * scale, k


def test_grad_vs_lqr_closed_form_fd():
    import torch
    from paper_2212_01110_gb300 import spock
    d = _unconstrained_a1(W.small_binary(1, nx=3, nu=2))
    gp = spock.Problem(d)
    dev = torch.device("cuda:0")
    x0 = torch.tensor(d["x0"], device=dev)
    z = torch.zeros(gp.n_z, dtype=torch.float64, device=dev)
    e = torch.zeros(gp.n_eta, dtype=torch.float64, device=dev)
    info = spock.spock_solve_dev(gp.handle, x0, spock.spock_default_settings(eps_abs=1e-12, eps_rel=1e-12, memory=5,
                                                                             max_iter=200000), z, e, 0)
    assert info.status == 0
    g = _gpu_grad(gp, z, e)
    V = lambda dd: tree_lqr(OProblem(dd), dd["x0"])[0]
    h = 1e-6
    rng = np.random.default_rng(0)
    for key in KEYS:
        for _ in range(4):
            shape = g[key].shape
            if key == "x0":
                idx = (int(rng.integers(0, shape[0])),)
            else:
                node = int(rng.integers(1, len(d["anc"])))
                if key == "QN":
                    node = int(rng.integers(7, 15))
                idx = (node,) + tuple(int(rng.integers(0, s)) for s in shape[1:])
            dp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d.items()}
            dm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d.items()}
            dp[key][idx] += h
            dm[key][idx] -= h
            fd = (V(dp) - V(dm)) / (2 * h)
            assert abs(g[key][idx] - fd) < 1e-5 * max(1, abs(fd)), (key, idx, g[key][idx], fd)


def test_autograd_function():
    import torch
    from paper_2212_01110_gb300 import autograd as AG
    d = W.with_tree(W.fig1_tree(), seed=7, nx=2, nu=2, a=0.5, box=(5.0, 0.4))
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev, requires_grad=True)
    x0, Q, R, QN, A, B = t(d["x0"]), t(d["Q"]), t(d["R"]), t(d["QN"]), t(d["A"]), t(d["B"])
    V = AG.optimal_cost(d, x0, Q, R, QN, A, B)
    V.backward()
    # directional finite difference of the same function (solve tolerance 1e-10)
    rng = np.random.default_rng(3)
    dirs = [rng.standard_normal(a.shape) for a in (d["x0"], d["Q"], d["R"], d["QN"], d["A"], d["B"])]
    dirs[1] *= 0.1
    dirs[2] *= 0.1
    dirs[3] *= 0.1
    h = 1e-5

    def Vat(s):
        args = [torch.tensor(a + s * dv, dtype=torch.float64, device=dev)
                for a, dv in zip((d["x0"], d["Q"], d["R"], d["QN"], d["A"], d["B"]), dirs)]
        return float(AG.optimal_cost(d, *args).item())

    fd = (Vat(h) - Vat(-h)) / (2 * h)
    an = sum(float((g.grad.cpu().numpy() * dv).sum()) for g, dv in zip((x0, Q, R, QN, A, B), dirs))
    assert abs(an - fd) < 1e-4 * max(1, abs(fd)), (an, fd)


def test_grad_fp32_vs_fp64():
    import torch
    from paper_2212_01110_gb300 import spock
    d = W.small_binary(0)
    gp = spock.Problem(d)
    dev = torch.device("cuda:0")
    x0 = torch.tensor(d["x0"], device=dev)
    z = torch.zeros(gp.n_z, dtype=torch.float64, device=dev)
    e = torch.zeros(gp.n_eta, dtype=torch.float64, device=dev)
    spock.spock_solve_dev(gp.handle, x0, spock.spock_default_settings(eps_abs=1e-10, eps_rel=1e-10, memory=5,
                                                                      max_iter=200000), z, e, 0)
    g64 = _gpu_grad(gp, z, e, 0)
    g32 = _gpu_grad(gp, z, e, 1)
    for k in KEYS:
        scale = max(1.0, float(np.max(np.abs(g64[k]))))
        assert np.max(np.abs(g32[k] - g64[k])) < 1e-4 * scale, k
