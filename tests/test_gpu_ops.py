"""CUDA operators through the C-ABI against the oracle, element by element:
L, L* (definition of L), prox_{alpha g*} (Eq. (prox:g)), prox_{alpha f}
(Algorithm 2 vs a KKT solve), and T (Eq. (chambolle-pock-operator))."""
import numpy as np
import pytest

from tests.gpu_common import RTOL, Pair, cases, rel_err

pytestmark = pytest.mark.gpu
CASES = cases()


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    return Pair(CASES[request.param])


def test_apply_L_and_adjoint(pair):
    import torch
    from paper_2212_01110_gb300 import spock
    rng = np.random.default_rng(0)
    z = rng.standard_normal(pair.gp.n_z)
    w = rng.standard_normal(pair.gp.n_eta)
    out = torch.empty(pair.gp.n_eta, dtype=torch.float64, device=pair.dev)
    spock.spock_apply_L_dev(pair.gp.handle, pair.t(z), out)
    ref = pair.cp.L @ z
    assert rel_err(out.cpu().numpy(), ref) < RTOL
    outz = torch.empty(pair.gp.n_z, dtype=torch.float64, device=pair.dev)
    spock.spock_apply_Lt_dev(pair.gp.handle, pair.t(w), outz)
    assert rel_err(outz.cpu().numpy(), pair.cp.Lt @ w) < RTOL
    # adjoint identity of the CUDA pair itself
    lhs = float(out.cpu().numpy() @ w)
    rhs = float(z @ outz.cpu().numpy())
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs)) * 10


@pytest.mark.parametrize("alpha_scale", [1.0, 0.3])
def test_prox_gconj(pair, alpha_scale):
    import torch
    from paper_2212_01110_gb300 import spock
    from oracle.cones import prox_gconj
    alpha = pair.alpha * alpha_scale
    rng = np.random.default_rng(1)
    eta = 3 * rng.standard_normal(pair.gp.n_eta)
    out = torch.empty_like(pair.t(eta))
    spock.spock_prox_gconj_dev(pair.gp.handle, alpha, pair.t(eta), out)
    assert rel_err(out.cpu().numpy(), prox_gconj(eta, alpha, pair.op)) < RTOL


@pytest.fixture(params=["auto", "grp", "tma", "direct"])
def kernels(request, monkeypatch):
    """Every Riccati kernel family: the default per-pass choice, three warps
    per chain, one warp per chain with bulk-copy staging, direct loads."""
    monkeypatch.setenv("SPOCK_RICCATI_KERNELS", request.param)
    return request.param


def test_prox_f(pair, kernels):
    import torch
    from paper_2212_01110_gb300 import spock
    rng = np.random.default_rng(2)
    z = 2 * rng.standard_normal(pair.gp.n_z)
    out = torch.empty_like(pair.t(z))
    spock.spock_prox_f_dev(pair.gp.handle, pair.x0, pair.alpha, pair.t(z), out)
    ref = pair.cp.prox_f(z, pair.d["x0"])
    assert rel_err(out.cpu().numpy(), ref) < RTOL


def test_T(pair, kernels):
    import torch
    from paper_2212_01110_gb300 import spock
    rng = np.random.default_rng(3)
    z = rng.standard_normal(pair.gp.n_z)
    eta = rng.standard_normal(pair.gp.n_eta)
    zo = torch.empty_like(pair.t(z))
    eo = torch.empty_like(pair.t(eta))
    spock.spock_T_dev(pair.gp.handle, pair.x0, pair.alpha, pair.t(z), pair.t(eta), zo, eo)
    ref = pair.cp.T(np.concatenate([z, eta]), pair.d["x0"])
    got = np.concatenate([zo.cpu().numpy(), eo.cpu().numpy()])
    assert rel_err(got, ref) < RTOL
