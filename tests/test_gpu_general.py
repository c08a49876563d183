"""The general form on the GPU (spock_problem_create_general and the dense-cost
flag of spock_problem_create) against the oracle's general form, element by
element: ||L|| (an upper bound within 1e-8), L, L*, prox_{alpha g*}, prox_f,
T (FP64, 1e-10), CP iterates in FP64 and FP32, converged solutions, and the
entry points that reject general problems.

The cases span the kernels' lane layouts (constraint rows nc up to 104: one,
three and five register slots per lane), diagonal and dense costs, a tree
whose root has 40 children, chains below branching stages, and a problem
written in scrambled coordinates (x' = T x, u' = S u per node) whose optimal
value is that of a box-form problem."""
import numpy as np
import pytest

from oracle.cp import CP, vanilla_cp
from oracle.problem import Problem as OProblem
from oracle.spock import Settings as OSettings, spock as ospock
from tests.gpu_common import RTOL, rel_err

pytestmark = pytest.mark.gpu


def _dense_box(d, seed):
    """Box-form constraints with dense cost matrices (SPOCK_DENSE_COST)."""
    from paper_2212_01110_gb300 import workloads as W
    g = W.general_random(d, seed=seed, dense=True)
    out = dict(d)
    out["Q"], out["R"], out["QN"] = g["Q"], g["R"], g["QN"]
    return out


def general_cases():
    from paper_2212_01110_gb300 import workloads as W
    return {
        "dense_box_binary": _dense_box(W.small_binary(0), 1),
        "poly_ragged": W.general_random(W.random_tree(3, N=4, max_branch=3, nx=4, nu=3), seed=1),
        "poly_binary": W.general_random(W.small_binary(0), seed=3),
        "poly_diag_chains": W.general_random(W.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2),
                                             seed=2, dense=False),
        "transform_fig1": W.general_transform(W.with_tree(W.fig1_tree(), seed=1, nx=3, nu=2), seed=3)[0],
        "poly_wide_50_20": W.general_random(W.large_tree(0, branching_stages=2, branch=3, N=5, nx=50, nu=20),
                                            seed=4, extra_rows=10, extra_leaf_rows=6),
        "poly_nc104": W.general_random(W.random_tree(7, N=3, max_branch=2, nx=60, nu=30, stable=True), seed=5,
                                       extra_rows=14, extra_leaf_rows=3),
        "poly_root_40": W.general_random(W.with_tree(W.tree_from_branching([40, 1])[0], seed=9, nx=3, nu=2),
                                         seed=6),
        # more inputs than states (R^1/2 blocks larger than Q^1/2; nu > 32)
        "poly_nu_gt_nx": W.general_random(W.random_tree(9, N=3, max_branch=4, nx=2, nu=5), seed=7),
        "poly_wide_20_50": W.general_random(W.large_tree(1, branching_stages=2, branch=3, N=5, nx=20, nu=50),
                                            seed=8, extra_rows=6, extra_leaf_rows=4),
        # conic risk measures (b, E, F, K): total variation (n_nu = m, zero-cone
        # row), mean-AV@R, AV@R in general form on a 30-child root
        # (z_2 block of 121 entries: four lane slots)
        "risk_tv_binary1": W.risk_measures(W.small_binary(1, a=0.5), "tv", radius=0.3),
        "risk_mean_avar_binary0": W.risk_measures(W.small_binary(0, a=0.5), "mean_avar", lam=0.5),
        "risk_tv_poly_ragged": W.risk_measures(
            W.general_random(W.random_tree(3, N=4, max_branch=3, nx=4, nu=3), seed=1), "tv", radius=0.2),
        "risk_avar_root_30": W.risk_measures(W.with_tree(W.tree_from_branching([30, 1])[0], seed=9, nx=3, nu=2),
                                             "avar"),
        "risk_tv_root_17": W.risk_measures(W.with_tree(W.tree_from_branching([17, 2])[0], seed=10, nx=4, nu=2,
                                                       a=0.3), "tv", radius=0.5),
    }


CASES = general_cases()


class GPair:
    def __init__(self, d):
        import torch
        from paper_2212_01110_gb300 import spock
        self.d = d
        self.op = OProblem(d)
        assert self.op.general or self.op.dense_cost or self.op.general_risk
        self.cp = CP(self.op)
        self.gp = spock.Problem(d)
        assert (self.gp.n_z, self.gp.n_eta) == (self.op.lay.n_z, self.op.lay.n_eta)
        self.alpha = self.cp.alpha
        self.dev = torch.device("cuda:0")
        self.x0 = torch.tensor(d["x0"], dtype=torch.float64, device=self.dev)

    def t(self, a):
        import torch
        return torch.tensor(np.asarray(a, float), dtype=torch.float64, device=self.dev)


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    return GPair(CASES[request.param])


def test_norm_L_is_a_tight_upper_bound(pair):
    """The library certifies an upper bound of each block's eigenvalue
    (power iteration, then Cholesky of sigma I - M); it may exceed the exact
    value by a few parts in 1e9 (up to 1e-6 when the power iteration stops
    early), which only shortens alpha = 0.99 / ||L|| as much."""
    ref = pair.cp.normL
    assert pair.gp.norm_L >= ref * (1 - 1e-12)
    assert pair.gp.norm_L <= ref * (1 + 1e-6)


def test_apply_L_and_adjoint(pair):
    import torch
    from paper_2212_01110_gb300 import spock
    rng = np.random.default_rng(0)
    z = rng.standard_normal(pair.gp.n_z)
    w = rng.standard_normal(pair.gp.n_eta)
    out = torch.empty(pair.gp.n_eta, dtype=torch.float64, device=pair.dev)
    spock.spock_apply_L_dev(pair.gp.handle, pair.t(z), out)
    assert rel_err(out.cpu().numpy(), pair.cp.L @ z) < RTOL
    outz = torch.empty(pair.gp.n_z, dtype=torch.float64, device=pair.dev)
    spock.spock_apply_Lt_dev(pair.gp.handle, pair.t(w), outz)
    assert rel_err(outz.cpu().numpy(), pair.cp.Lt @ w) < RTOL
    lhs = float(out.cpu().numpy() @ w)
    rhs = float(z @ outz.cpu().numpy())
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


@pytest.mark.parametrize("alpha_scale", [1.0, 0.3])
def test_prox_gconj(pair, alpha_scale):
    import torch
    from paper_2212_01110_gb300 import spock
    from oracle.cones import prox_gconj
    alpha = pair.alpha * alpha_scale
    eta = 3 * np.random.default_rng(1).standard_normal(pair.gp.n_eta)
    out = torch.empty_like(pair.t(eta))
    spock.spock_prox_gconj_dev(pair.gp.handle, alpha, pair.t(eta), out)
    assert rel_err(out.cpu().numpy(), prox_gconj(eta, alpha, pair.op)) < RTOL


def test_prox_f(pair):
    import torch
    from paper_2212_01110_gb300 import spock
    z = 2 * np.random.default_rng(2).standard_normal(pair.gp.n_z)
    out = torch.empty_like(pair.t(z))
    spock.spock_prox_f_dev(pair.gp.handle, pair.x0, pair.alpha, pair.t(z), out)
    assert rel_err(out.cpu().numpy(), pair.cp.prox_f(z, pair.d["x0"])) < RTOL


def test_T(pair):
    import torch
    from paper_2212_01110_gb300 import spock
    rng = np.random.default_rng(3)
    z = rng.standard_normal(pair.gp.n_z)
    eta = rng.standard_normal(pair.gp.n_eta)
    zo = torch.empty_like(pair.t(z))
    eo = torch.empty_like(pair.t(eta))
    spock.spock_T_dev(pair.gp.handle, pair.x0, pair.alpha, pair.t(z), pair.t(eta), zo, eo)
    ref = pair.cp.T(np.concatenate([z, eta]), pair.d["x0"])
    assert rel_err(np.concatenate([zo.cpu().numpy(), eo.cpu().numpy()]), ref) < RTOL


@pytest.mark.parametrize("k", [1, 25])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cp_steps(pair, k, prec):
    """k CP iterations through the solve path's kernels (the fused dual
    kernel with statistics): FP64 at 1e-10; FP32 at the tolerances of the box
    form's FP32 parity (2e-6 for one T, 5e-6 after 25), whose argument --
    unit roundoff 6e-8, dot products of at most 130 terms, T nonexpansive --
    holds for the matrix rows as well."""
    from paper_2212_01110_gb300 import spock
    rng = np.random.default_rng(40 + k)
    z0 = rng.standard_normal(pair.gp.n_z)
    e0 = rng.standard_normal(pair.gp.n_eta)
    z, e = pair.t(z0), pair.t(e0)
    p = spock.SPOCK_FP64 if prec == "fp64" else spock.SPOCK_FP32
    xi = spock.spock_cp_step_dev(pair.gp.handle, pair.x0, k, pair.alpha, p, z, e)
    ref, xi_ref = vanilla_cp(pair.cp, np.concatenate([z0, e0]), pair.d["x0"], k)
    got = np.concatenate([z.cpu().numpy(), e.cpu().numpy()])
    tol = RTOL if prec == "fp64" else {1: 2e-6, 25: 5e-6}[k]
    assert rel_err(got, ref) < tol
    if prec == "fp64":
        assert abs(xi - xi_ref) <= 1e-9 * max(1.0, xi_ref)


@pytest.mark.parametrize("name", ["poly_binary", "dense_box_binary", "transform_fig1", "risk_tv_binary1",
                                  "risk_mean_avar_binary0"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_matches_oracle(name, prec):
    """Converged solutions (graph driver; the single-block solve does not
    take the general form), certified at xi <= eps = 1e-6 (FP32: by the FP64
    tail): the optimal value against the oracle's (solved to 1e-9) at 10 eps
    relative, the tolerance the box form's converged solves use (a pair
    certified at eps has a cost within O(eps) of the optimum)."""
    from paper_2212_01110_gb300 import spock
    pair = GPair(CASES[name])
    p = spock.SPOCK_FP64 if prec == "fp64" else spock.SPOCK_FP32
    s = spock.spock_default_settings(alpha=pair.alpha, precision=p, memory=5, max_iter=60000)
    z = np.zeros(pair.gp.n_z)
    e = np.zeros(pair.gp.n_eta)
    info = spock.spock_solve(pair.gp.handle, pair.d["x0"], s, z, e, 0)
    assert info.status == spock.SPOCK_OK
    assert info.n_launches > 1
    ref = ospock(pair.cp, pair.d["x0"], s=OSettings(eps_abs=1e-9, eps_rel=1e-9, memory=5, max_iter=60000))
    assert ref.status == "converged"
    assert abs(z[0] - ref.v[0]) <= 1e-5 * max(1.0, abs(ref.v[0]))


def test_scrambled_coordinates_solve_to_the_box_value():
    """The general problem written in per-node coordinates x' = T x, u' = S u
    of a box-form problem has the box problem's optimal value: the GPU solves
    of both agree to 1e-6."""
    from paper_2212_01110_gb300 import spock, workloads as W
    d = W.random_tree(21, N=3, max_branch=3, nx=3, nu=2, a_range=(0.5, 0.5), box=(1.2, 0.25))
    g, T, S = W.general_transform(d, seed=0)
    vals = []
    for dd in (d, g):
        P = spock.Problem(dd)
        s = spock.spock_default_settings(eps_abs=1e-9, eps_rel=1e-9, memory=5, max_iter=60000)
        z = np.zeros(P.n_z)
        e = np.zeros(P.n_eta)
        info = spock.spock_solve(P.handle, dd["x0"], s, z, e, 0)
        assert info.status == spock.SPOCK_OK
        vals.append(z[0])
        P.close()
    assert abs(vals[0] - vals[1]) <= 1e-6 * max(1.0, abs(vals[0]))


def test_avar_in_general_form_solves_like_the_box_form():
    """AV@R given as a conic risk measure (the general kernels, S2 by the
    dense projector) and the built-in AV@R (box-form kernels, closed-form
    S2) reach the same optimal value."""
    from paper_2212_01110_gb300 import spock, workloads as W
    d = W.random_tree(3, N=3, max_branch=3, nx=3, nu=2, a_range=(0.2, 0.8))
    vals = []
    for dd in (d, W.risk_measures(d, "avar")):
        P = spock.Problem(dd)
        s = spock.spock_default_settings(eps_abs=1e-9, eps_rel=1e-9, memory=5, max_iter=60000)
        z = np.zeros(P.n_z)
        e = np.zeros(P.n_eta)
        info = spock.spock_solve(P.handle, dd["x0"], s, z, e, 0)
        assert info.status == spock.SPOCK_OK
        vals.append(z[0])
        P.close()
    assert abs(vals[0] - vals[1]) <= 1e-7 * max(1.0, abs(vals[0]))


def test_general_problems_rejected_where_unsupported():
    import torch
    from paper_2212_01110_gb300 import spock
    pair = GPair(CASES["poly_ragged"])
    n, nx, nu = pair.op.tree.n, pair.op.nx, pair.op.nu
    z = torch.zeros(pair.gp.n_z, dtype=torch.float64, device=pair.dev)
    e = torch.zeros(pair.gp.n_eta, dtype=torch.float64, device=pair.dev)
    g = torch.zeros(nx, dtype=torch.float64, device=pair.dev)
    with pytest.raises(spock.SpockError) as ei:
        spock.spock_grad_dev(pair.gp.handle, z, e, spock.SPOCK_FP64, g, None, None, None, None, None)
    assert ei.value.code == spock.SPOCK_ERR_UNSUPPORTED
    with pytest.raises(spock.SpockError) as ei:
        spock.spock_adjoint_dev(pair.gp.handle, z, e, None, 10, 1e-8, g)
    assert ei.value.code == spock.SPOCK_ERR_UNSUPPORTED
    with pytest.raises(spock.SpockError) as ei:
        spock.spock_batch_create([pair.gp.handle])
    assert ei.value.code == spock.SPOCK_ERR_UNSUPPORTED


def test_invalid_general_inputs():
    """Non-positive-definite cost matrix, crossed bounds, bad row counts."""
    from paper_2212_01110_gb300 import spock, workloads as W
    base = W.general_random(W.random_tree(3, N=2, max_branch=2, nx=3, nu=2), seed=1)
    bad = dict(base)
    bad["Q"] = base["Q"].copy()
    bad["Q"][1] = -np.eye(3)
    with pytest.raises(spock.SpockError) as ei:
        spock.Problem(bad)
    assert ei.value.code == spock.SPOCK_ERR_NOT_POSDEF
    bad = dict(base)
    bad["cmin"] = base["cmin"].copy()
    bad["cmin"][0, 0] = base["cmax"][0, 0] + 1.0
    with pytest.raises(spock.SpockError) as ei:
        spock.Problem(bad)
    assert ei.value.code == spock.SPOCK_ERR_INVALID_ARG
    bad = W.risk_measures(W.small_binary(0), "tv")   # F without full column rank
    bad["risk"] = [None if r is None else dict(r, F=np.zeros_like(r["F"])) for r in bad["risk"]]
    with pytest.raises(spock.SpockError) as ei:
        spock.Problem(bad)
    assert ei.value.code == spock.SPOCK_ERR_INVALID_ARG
    bad = dict(base)
    bad["Gx"] = np.zeros((len(base["anc"]), 0, 3))
    bad["Gu"] = np.zeros((len(base["anc"]), 0, 2))
    with pytest.raises(spock.SpockError) as ei:
        spock.Problem(bad)
    assert ei.value.code == spock.SPOCK_ERR_INVALID_ARG


def test_general_kernels_at_launch_scale_equal_the_box_kernels():
    """The 17,749-node tree (branching 4 for 6 stages, then 4,096 chains;
    nx = 50, nu = 20) written twice: in the box form and in the general form
    with Gamma = I and the diagonal costs as dense matrices.  The two define
    the same L, so one evaluation of T (FP64) and one CP step through the
    solve path's kernels with statistics (FP64 and FP32) agree element by
    element: the general kernels at the benchmark's launch shapes (many
    blocks per SM, every node of a stage in flight) against the box-form
    kernels, which are parity-tested against the oracle and riccati_cpu."""
    import torch
    from paper_2212_01110_gb300 import spock, workloads as W
    d = W.large_tree(seed=0, branching_stages=6, N=9)
    n, nx, nu = len(d["anc"]), d["nx"], d["nu"]
    g = dict(d)
    g["Q"] = np.zeros((n, nx, nx))
    g["R"] = np.zeros((n, nu, nu))
    g["QN"] = np.zeros((n, nx, nx))
    idx_x, idx_u = np.arange(nx), np.arange(nu)
    g["Q"][:, idx_x, idx_x] = d["Q"]
    g["R"][:, idx_u, idx_u] = d["R"]
    g["QN"][:, idx_x, idx_x] = d["QN"]
    Pb, Pg = spock.Problem(d), spock.Problem(g)   # Q dense: SPOCK_DENSE_COST, boxes as Gamma = I
    assert (Pb.n_z, Pb.n_eta) == (Pg.n_z, Pg.n_eta)
    assert Pb.norm_L * (1 - 1e-12) <= Pg.norm_L <= Pb.norm_L * (1 + 1e-6)
    dev = torch.device("cuda:0")
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
    alpha = 0.99 / Pg.norm_L
    rng = np.random.default_rng(5)
    z0 = torch.tensor(rng.standard_normal(Pb.n_z), dtype=torch.float64, device=dev)
    e0 = torch.tensor(rng.standard_normal(Pb.n_eta), dtype=torch.float64, device=dev)
    outs = []
    for P in (Pb, Pg):
        zo, eo = torch.empty_like(z0), torch.empty_like(e0)
        spock.spock_T_dev(P.handle, x0, alpha, z0, e0, zo, eo)
        outs.append(torch.cat([zo, eo]).cpu().numpy())
    assert rel_err(outs[1], outs[0]) < 1e-12
    for prec, tol in ((spock.SPOCK_FP64, 1e-12), (spock.SPOCK_FP32, 2e-6)):
        res = []
        for P in (Pb, Pg):
            z, e = z0.clone(), e0.clone()
            xi = spock.spock_cp_step_dev(P.handle, x0, 1, alpha, prec, z, e)
            res.append((torch.cat([z, e]).cpu().numpy(), xi))
        assert rel_err(res[1][0], res[0][0]) < tol
        assert abs(res[1][1] - res[0][1]) <= 1e3 * tol * max(1.0, res[0][1])
    Pb.close()
    Pg.close()
