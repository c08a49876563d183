"""The 62,805-node tree (branching 4 for 6 stages then chains, N = 20,
nx = 50, nu = 20: the benchmark's workload, 4.62 M primal and 9.29 M dual
variables) at full size, in the launch configuration of the benchmark's
solves, against riccati_cpu (the oracle's C++ CP operator, Algorithms 1-2
as printed; pinned against the Python oracle at 1e-12): one evaluation of
T through spock_cp_step_dev (the kernels of the solve's evaluation of T,
statistics included) in FP64 at 1e-10 and in FP32 at the FP32 tolerance,
the residual xi of that pair, and prox_{alpha f} and T through the
operator-level entry points at 1e-10.  Every output element is compared."""
import os

import numpy as np
import pytest

from tests.gpu_common import RTOL, rel_err

pytestmark = pytest.mark.gpu
TOL_FP32_T = 2e-6   # as tests/test_gpu_fp32.py: 33 unit roundoffs of FP32


@pytest.fixture(scope="module")
def big():
    import torch
    from oracle.riccati_cpu import RiccatiCPU
    from paper_2212_01110_gb300 import spock, workloads
    d = workloads.large_tree(seed=0, branching_stages=6, branch=4, N=20, nx=50, nu=20)
    try:
        threads = len(os.sched_getaffinity(0))
    except Exception:
        threads = os.cpu_count() or 1
    rc = RiccatiCPU(d, threads=threads)
    P = spock.Problem(d)
    assert (P.n_z, P.n_eta) == (rc.n_z, rc.n_eta) == (4624356, 9292336)
    rng = np.random.default_rng(21)
    z = rng.standard_normal(P.n_z)
    e = rng.standard_normal(P.n_eta)
    alpha = 0.99 / P.norm_L
    ref_z, ref_e = rc.T(z, e, alpha)
    ref = np.concatenate([ref_z, ref_e])
    yield dict(d=d, rc=rc, P=P, z=z, e=e, alpha=alpha, ref=ref, dev=torch.device("cuda:0"))
    P.close()
    rc.close()


def _cp1(big, precision):
    import torch
    from paper_2212_01110_gb300 import spock
    dev = big["dev"]
    x0 = torch.tensor(big["d"]["x0"], dtype=torch.float64, device=dev)
    z = torch.tensor(big["z"], dtype=torch.float64, device=dev)
    e = torch.tensor(big["e"], dtype=torch.float64, device=dev)
    xi = spock.spock_cp_step_dev(big["P"].handle, x0, 1, big["alpha"], precision, z, e)
    got = np.concatenate([z.cpu().numpy(), e.cpu().numpy()])
    del z, e
    torch.cuda.empty_cache()
    return got, xi


def _xi(big, Tv):
    """xi of the pair (v, T(v)) computed on the host from riccati_cpu's L, L*."""
    rc, a = big["rc"], big["alpha"]
    nz = rc.n_z
    r = np.concatenate([big["z"], big["e"]]) - Tv
    xp = r[:nz] / a - rc.apply_Lt(r[nz:])
    xd = r[nz:] / a - rc.apply_L(r[:nz])
    return max(np.max(np.abs(xp)), np.max(np.abs(xd)))


def test_T_fp64_in_the_solve_configuration(big):
    from paper_2212_01110_gb300 import spock
    got, xi = _cp1(big, spock.SPOCK_FP64)
    err = rel_err(got, big["ref"])
    print(f"62,805-node tree, FP64 T: max rel. error {err:.2e}")
    assert err < RTOL
    xi_ref = _xi(big, big["ref"])
    assert abs(xi - xi_ref) < 1e-8 * max(1.0, xi_ref)


def test_T_fp32_in_the_solve_configuration(big):
    from paper_2212_01110_gb300 import spock
    got, xi = _cp1(big, spock.SPOCK_FP32)
    err = rel_err(got, big["ref"])
    print(f"62,805-node tree, FP32 T: max rel. error {err:.2e} (tolerance {TOL_FP32_T:.0e})")
    assert err < TOL_FP32_T


def test_operator_entry_points(big):
    import torch
    from paper_2212_01110_gb300 import spock
    dev = big["dev"]
    P = big["P"]
    x0 = torch.tensor(big["d"]["x0"], dtype=torch.float64, device=dev)
    z = torch.tensor(big["z"], dtype=torch.float64, device=dev)
    e = torch.tensor(big["e"], dtype=torch.float64, device=dev)
    zo = torch.empty_like(z)
    spock.spock_prox_f_dev(P.handle, x0, big["alpha"], z, zo)
    assert rel_err(zo.cpu().numpy(), big["rc"].prox_f(big["z"], big["alpha"])) < RTOL
    eo = torch.empty_like(e)
    spock.spock_T_dev(P.handle, x0, big["alpha"], z, e, zo, eo)
    got = np.concatenate([zo.cpu().numpy(), eo.cpu().numpy()])
    assert rel_err(got, big["ref"]) < RTOL
