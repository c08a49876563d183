"""riccati_cpu (plain C++ FP64, Algorithms 1-2 as printed, OpenMP over the
nodes of a stage) against the Python oracle (explicit sparse L, KKT
projection on S1, pseudoinverse projection on S2): every part of T and T
itself to 1e-12 relative, with 1 and 3 threads.  This pins the C++ checker
that the large-tree parity tests and the CPU baseline use."""
import numpy as np
import pytest

from oracle.cones import prox_gconj
from oracle.cp import CP
from oracle.problem import Problem
from oracle.riccati_cpu import RiccatiCPU
from paper_2212_01110_gb300 import workloads as W

TOL = 1e-12


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


CASES = {
    "binary_N3": lambda: W.small_binary(0),
    "fig1": lambda: W.with_tree(W.fig1_tree(), seed=1, nx=3, nu=2),
    "ragged": lambda: W.random_tree(3, N=4, max_branch=3, nx=4, nu=3),
    "chains": lambda: W.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2),
    "wide_50_20": lambda: W.large_tree(0, branching_stages=2, branch=3, N=5, nx=50, nu=20),
    "datacenter": lambda: W.datacenter(N=4, nx=6),
    "root_17_2": lambda: W.with_tree(W.tree_from_branching([17, 2])[0], seed=10, nx=4, nu=2, a=0.3),
    "nu_gt_nx": lambda: W.random_tree(9, N=3, max_branch=4, nx=2, nu=5),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    d = CASES[request.param]()
    cp = CP(Problem(d))
    return d, cp


@pytest.mark.parametrize("threads", [1, 3])
def test_parts_and_T_match_python_oracle(pair, threads):
    d, cp = pair
    rc = RiccatiCPU(d, threads=threads)
    assert (rc.n_z, rc.n_eta) == (cp.n_z, cp.n_eta)
    rng = np.random.default_rng(7)
    z = rng.standard_normal(cp.n_z)
    e = 2 * rng.standard_normal(cp.n_eta)
    assert _rel(rc.apply_L(z), cp.L @ z) < TOL
    assert _rel(rc.apply_Lt(e), cp.Lt @ e) < TOL
    assert _rel(rc.prox_f(z, cp.alpha), cp.prox_f(z, d["x0"])) < TOL
    assert _rel(rc.prox_gconj(e, cp.alpha), prox_gconj(e, cp.alpha, cp.P)) < TOL
    zo, eo = rc.T(z, e, cp.alpha)
    ref = cp.T(np.concatenate([z, e]), d["x0"])
    assert _rel(np.concatenate([zo, eo]), ref) < TOL
    rc.close()


def test_riccati_projection_is_a_projection_on_a_larger_tree():
    """Algorithm 2 on a 309-node tree of the large-tree family (nx = 50,
    nu = 20): agreement with the KKT projection and idempotence."""
    d = W.large_tree(1, branching_stages=2, branch=4, N=20, nx=50, nu=20)
    cp = CP(Problem(d))
    rc = RiccatiCPU(d, threads=2)
    z = np.random.default_rng(3).standard_normal(cp.n_z)
    p1 = rc.prox_f(z, 0.0)
    assert _rel(p1, cp.prox_f(z, d["x0"]) + np.eye(1, cp.n_z, 0)[0] * cp.alpha) < TOL
    assert _rel(rc.prox_f(p1, 0.0), p1) < TOL
