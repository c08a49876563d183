"""spock_adjoint_dev (implicit differentiation of the CP fixed point through
the C-ABI): for phi = s^0 it equals the envelope gradient of spock_grad_dev;
for phi = a component of the first input u^0 it equals the oracle's adjoint
(GMRES on the same linearisation) at the same converged pair."""
import numpy as np
import pytest

from oracle.adjoint import adjoint_gradient
from paper_2212_01110_gb300 import workloads as W
from tests.gpu_common import Pair

pytestmark = pytest.mark.gpu
KEYS = ("x0", "A", "B", "Q", "R", "QN")


def _solved(d, tol=1e-12):
    import torch
    from paper_2212_01110_gb300 import spock
    pair = Pair(d)
    s = spock.spock_default_settings(alpha=pair.alpha, eps_abs=tol, eps_rel=tol, memory=5, max_iter=200000)
    z = pair.t(np.zeros(pair.gp.n_z))
    e = pair.t(np.zeros(pair.gp.n_eta))
    info = spock.spock_solve_dev(pair.gp.handle, pair.x0, s, z, e, 0)
    assert info.status == spock.SPOCK_OK
    return pair, z, e


def _outs(pair):
    import torch
    n, nx, nu = pair.op.tree.n, pair.op.nx, pair.op.nu
    shapes = [(nx,), (n, nx, nx), (n, nx, nu), (n, nx), (n, nu), (n, nx)]
    return [torch.zeros(sh, dtype=torch.float64, device=pair.dev) for sh in shapes]


@pytest.mark.parametrize("name", ["binary_N3", "datacenter_N6", "chains_uniform"])
def test_cost_gradient_equals_envelope_gradient(name):
    from paper_2212_01110_gb300 import spock
    d = {"binary_N3": W.small_binary(0), "datacenter_N6": W.datacenter(N=6, nx=3),
         "chains_uniform": W.large_tree(2, branching_stages=2, branch=3, N=5, nx=6, nu=3, probs="uniform")}[name]
    pair, z, e = _solved(d)
    env = _outs(pair)
    spock.spock_grad_dev(pair.gp.handle, z, e, spock.SPOCK_FP64, *env)
    adj = _outs(pair)
    rc, its, res = spock.spock_adjoint_dev(pair.gp.handle, z, e, None, 200000, 1e-12, *adj)
    print(f"{name}: adjoint {its} iterations, relative change {res:.1e}")
    assert rc == spock.SPOCK_OK
    for k, a, b in zip(KEYS, adj, env):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        scale = max(1.0, float(np.max(np.abs(b))))
        assert np.max(np.abs(a - b)) < 1e-8 * scale, (k, np.max(np.abs(a - b)))


def test_first_input_sensitivity_equals_oracle_adjoint():
    from paper_2212_01110_gb300 import spock
    pair, z, e = _solved(W.small_binary(0))
    zh, eh = z.cpu().numpy(), e.cpu().numpy()
    j = int(pair.op.lay.u[0][0])
    g = np.zeros(pair.gp.n_z)
    g[j] = 1.0
    adj = _outs(pair)
    rc, its, res = spock.spock_adjoint_dev(pair.gp.handle, z, e, pair.t(g), 200000, 1e-12, *adj)
    assert rc == spock.SPOCK_OK
    ref = adjoint_gradient(pair.cp, zh, eh, g=g)
    assert ref["gmres_info"] == 0
    for k, a in zip(KEYS, adj):
        a = a.cpu().numpy()
        scale = max(1.0, float(np.max(np.abs(ref[k]))))
        assert np.max(np.abs(a - ref[k])) < 1e-8 * scale, (k, np.max(np.abs(a - ref[k])))


def test_rejects_bad_arguments():
    from paper_2212_01110_gb300 import spock
    pair, z, e = _solved(W.small_binary(0), tol=1e-6)
    with pytest.raises(spock.SpockError):
        spock.spock_adjoint_dev(pair.gp.handle, z, e, None, 0, 1e-10)


def test_policy_autograd_matches_finite_differences():
    """SpockPolicy: d u^0_0 / d x0 along a random direction through
    torch.autograd (one adjoint solve) against central differences of GPU
    solves (h = 1e-4: u^0 is piecewise smooth, one piece around x0)."""
    import torch
    from paper_2212_01110_gb300 import autograd as AG
    d = W.small_binary(0)
    dev = torch.device("cuda:0")
    args = {k: torch.tensor(d[k], dtype=torch.float64, device=dev) for k in ("Q", "R", "QN", "A", "B")}
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev, requires_grad=True)
    v, u0 = AG.policy(d, x0, args["Q"], args["R"], args["QN"], args["A"], args["B"])
    u0[0].backward()
    rng = np.random.default_rng(4)
    dx = rng.standard_normal(d["nx"])
    h = 1e-4
    up = AG.policy(d, torch.tensor(d["x0"] + h * dx, device=dev), args["Q"], args["R"], args["QN"], args["A"],
                   args["B"])[1][0].item()
    um = AG.policy(d, torch.tensor(d["x0"] - h * dx, device=dev), args["Q"], args["R"], args["QN"], args["A"],
                   args["B"])[1][0].item()
    fd = (up - um) / (2 * h)
    an = float(x0.grad.cpu().numpy() @ dx)
    assert abs(an - fd) < 1e-5 * max(1.0, abs(fd)), (an, fd)
