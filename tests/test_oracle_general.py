"""The oracle's general form (polyhedral constraints Gamma of Eq.
(constraints), dense Q^1/2, R^1/2, Q_N^1/2 in L) pinned by facts that do not
depend on how it is assembled:
  * with Gamma = I and diagonal matrices it gives the box form's L, ||L||
    and prox_{alpha g*} exactly;
  * ||L|| from the column-group blocks equals a power iteration on L^T L;
  * a = 1 with loose constraints: the tree LQR recursion with dense Q, R, Q_N;
  * invariance under per-node coordinate changes x' = T x, u' = S u: the
    transformed problem (dense costs, Gamma = T^-1, S^-1) has the same value
    and the transformed solution, also with AV@R a < 1 and active boxes;
  * a = 1 with coupled constraints that are active at the solution: the
    quadratic program solved by enumerating active sets (brute force)."""
import itertools

import numpy as np
import pytest

from oracle import risk
from oracle.cones import prox_gconj
from oracle.cp import CP
from oracle.linop import build_L, norm_L_blocks, norm_L_power
from oracle.lqr import tree_lqr
from oracle.problem import Problem
from oracle.spock import Settings, spock
from paper_2212_01110_gb300 import workloads

TIGHT = Settings(eps_abs=1e-10, eps_rel=1e-10, max_iter=40000)


def _identity_general(d):
    n, nx, nu = len(d["anc"]), d["nx"], d["nu"]
    g = dict(d)
    for k in ("xmin", "xmax", "umin", "umax"):
        g.pop(k)
    Gx = np.zeros((n, nx + nu, nx))
    Gu = np.zeros((n, nx + nu, nu))
    Gx[:, :nx] = np.eye(nx)
    Gu[:, nx:] = np.eye(nu)
    g.update(Gx=Gx, Gu=Gu, cmin=np.concatenate([d["xmin"], d["umin"]], 1),
             cmax=np.concatenate([d["xmax"], d["umax"]], 1),
             GN=np.repeat(np.eye(nx)[None], n, 0), cNmin=d["xmin"].copy(), cNmax=d["xmax"].copy())
    g["Q"] = np.stack([np.diag(q) for q in d["Q"]])
    g["R"] = np.stack([np.diag(r) for r in d["R"]])
    g["QN"] = np.stack([np.diag(q) for q in d["QN"]])
    return g


def test_identity_general_is_the_box_form():
    d = workloads.random_tree(3, N=3, max_branch=3, nx=4, nu=2)
    Pb, Pg = Problem(d), Problem(_identity_general(d))
    assert Pg.general and Pg.dense_cost
    assert Pg.lay.n_eta == Pb.lay.n_eta and Pg.lay.n_z == Pb.lay.n_z
    Lb, Lg = build_L(Pb).toarray(), build_L(Pg).toarray()
    np.testing.assert_allclose(Lg, Lb, rtol=1e-15, atol=0)
    assert abs(norm_L_blocks(Pg) - norm_L_blocks(Pb)) <= 1e-13 * norm_L_blocks(Pb)
    eta = np.random.default_rng(0).standard_normal(Pb.lay.n_eta) * 3
    np.testing.assert_array_equal(prox_gconj(eta, 0.3, Pg), prox_gconj(eta, 0.3, Pb))


@pytest.mark.parametrize("seed", [0, 1])
def test_general_norm_matches_power_iteration(seed):
    d = workloads.general_random(workloads.random_tree(seed, N=3, max_branch=3, nx=4, nu=3), seed=seed)
    P = Problem(d)
    L = build_L(P)
    assert abs(norm_L_blocks(P) - norm_L_power(L, iters=20000)) <= 1e-7 * norm_L_blocks(P)


def test_general_factors_are_cholesky():
    d = workloads.general_random(workloads.random_tree(2, N=2, max_branch=2, nx=5, nu=3), seed=2)
    P = Problem(d)
    for c in range(1, P.tree.n):
        F = P.Qhalf(c)
        assert np.allclose(np.tril(F, -1), 0.0)
        np.testing.assert_allclose(F.T @ F, P.Q[c], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed,base", [
    (0, workloads.random_tree(6, N=3, max_branch=3, nx=3, nu=2, a_range=(1.0, 1.0))),
    (1, workloads.small_binary(0, a=1.0)),
    (2, workloads.with_tree(workloads.fig1_tree(), seed=4, nx=3, nu=2, a=1.0)),
])
def test_dense_lqr_closed_form(seed, base):
    d = workloads.general_random(base, seed=seed, bound=1e6)
    for k in ("cmin", "cNmin"):
        d[k] = np.full_like(d[k], -1e6)
    for k in ("cmax", "cNmax"):
        d[k] = np.full_like(d[k], 1e6)
    P = Problem(d)
    res = spock(CP(P), d["x0"], s=TIGHT)
    assert res.status == "converged"
    V, x, u = tree_lqr(P, d["x0"])
    assert abs(res.v[0] - V) <= 1e-7 * max(1.0, abs(V))
    xs, us = risk.trajectory(P, res.v[: P.lay.n_z])
    np.testing.assert_allclose(xs, x, atol=1e-6)
    np.testing.assert_allclose(us[0], u[0], atol=1e-6)


@pytest.mark.parametrize("seed,a", [(0, 0.5), (1, 0.2), (2, 1.0)])
def test_coordinate_change_invariance(seed, a):
    d = workloads.random_tree(20 + seed, N=3, max_branch=3, nx=3, nu=2, a_range=(a, a), box=(1.2, 0.25))
    g, T, S = workloads.general_transform(d, seed=seed)
    Pd, Pg = Problem(d), Problem(g)
    rd = spock(CP(Pd), d["x0"], s=TIGHT)
    rg = spock(CP(Pg), g["x0"], s=TIGHT)
    assert rd.status == "converged" and rg.status == "converged"
    assert abs(rg.v[0] - rd.v[0]) <= 1e-7 * max(1.0, abs(rd.v[0]))
    xd, ud = risk.trajectory(Pd, rd.v[: Pd.lay.n_z])
    xg, ug = risk.trajectory(Pg, rg.v[: Pg.lay.n_z])
    # AV@R with a < 1 leaves the controls below zero-weight children free, so
    # compare what is unique: mapped back to the original coordinates the
    # solution is feasible there and attains the optimal nested value
    t = Pd.tree
    xb = np.stack([np.linalg.solve(T[i], xg[i]) for i in range(t.n)])
    ub = np.zeros_like(ud)
    for i in t.nonleaf:
        ub[i] = np.linalg.solve(S[i], ug[i])
    np.testing.assert_allclose(xb[0], d["x0"], atol=1e-9)
    for c in t.nonroot:
        p = int(t.anc[c])
        np.testing.assert_allclose(xb[c], d["A"][c] @ xb[p] + d["B"][c] @ ub[p], atol=1e-8)
    assert np.all(xb <= d["xmax"] + 1e-7) and np.all(xb >= d["xmin"] - 1e-7)
    assert np.all(ub[t.nonleaf] <= d["umax"][t.nonleaf] + 1e-7)
    assert np.all(ub[t.nonleaf] >= d["umin"][t.nonleaf] - 1e-7)
    val, _ = risk.nested_value(Pd, xb, ub)
    assert abs(val - rd.v[0]) <= 1e-6 * max(1.0, abs(rd.v[0]))
    if a == 1.0:   # strictly convex: the solution itself is unique
        np.testing.assert_allclose(xb, xd, atol=1e-6)
    # some box constraints are active in the original coordinates
    act = max(np.max(np.abs(ud[t.nonleaf])) / 0.25, np.max(np.abs(xd)) / 1.2)
    assert act > 1.0 - 1e-6


def _qp_bruteforce(P, x0, cand):
    """min sum_c pi^c (x^p'Q^c x^p + u^p'R^c u^p) + sum_j pi^j x^j'Q_N x^j
    subject to the dynamics, x^0 = x0 and the constraint rows, by enumerating
    which rows in ``cand`` (pairs (kind, node, row)) are at their lower or
    upper bound; every other row must come out strictly inside."""
    t, nx, nu = P.tree, P.nx, P.nu
    lay = P.lay
    nz = lay.n_z
    ix = lambda i: lay.x[i]
    iu = lambda i: lay.u[i]
    pi = np.ones(t.n)
    for i in sorted(range(t.n), key=lambda k: t.stage[k]):
        if i > 0:
            pi[i] = pi[int(t.anc[i])] * t.prob[i]
    H = np.zeros((nz, nz))
    for c in t.nonroot:
        p = int(t.anc[c])
        H[np.ix_(ix(p), ix(p))] += 2 * pi[c] * P.Qmat(c)
        H[np.ix_(iu(p), iu(p))] += 2 * pi[c] * P.Rmat(c)
    for j in t.leaves:
        H[np.ix_(ix(j), ix(j))] += 2 * pi[j] * P.QNmat(j)
    Eq, e = [], []
    for k in range(nx):
        r = np.zeros(nz); r[ix(0)[k]] = 1; Eq.append(r); e.append(x0[k])
    for c in t.nonroot:
        p = int(t.anc[c])
        for k in range(nx):
            r = np.zeros(nz)
            r[ix(c)[k]] = 1
            r[ix(p)] -= P.A[c][k]
            r[iu(p)] -= P.B[c][k]
            Eq.append(r); e.append(0.0)
    rows, lo, hi, keys = [], [], [], []
    for i in t.nonleaf:
        for q in range(P.nc):
            r = np.zeros(nz); r[ix(i)] = P.Gx[i, q]; r[iu(i)] = P.Gu[i, q]
            rows.append(r); lo.append(P.cmin[i, q]); hi.append(P.cmax[i, q]); keys.append(("n", i, q))
    for j in t.leaves:
        for q in range(P.ncN):
            r = np.zeros(nz); r[ix(j)] = P.GN[j, q]
            rows.append(r); lo.append(P.cNmin[j, q]); hi.append(P.cNmax[j, q]); keys.append(("l", j, q))
    rows, lo, hi = np.array(rows), np.array(lo), np.array(hi)
    cidx = [keys.index(c) for c in cand]
    # variables not in the problem (s, y, tau) are pinned to zero
    used = np.zeros(nz, bool)
    for i in range(t.n):
        used[ix(i)] = True
    for i in t.nonleaf:
        used[iu(i)] = True
    for k in np.where(~used)[0]:
        r = np.zeros(nz); r[k] = 1; Eq.append(r); e.append(0.0)
    Eq, e = np.array(Eq), np.array(e)
    best = None
    for pattern in itertools.product((0, -1, 1), repeat=len(cidx)):
        act = [(cidx[k], s) for k, s in enumerate(pattern) if s != 0]
        Aeq = np.vstack([Eq] + [rows[q][None] for q, _ in act]) if act else Eq
        beq = np.concatenate([e, [lo[q] if s < 0 else hi[q] for q, s in act]])
        m = Aeq.shape[0]
        K = np.block([[H, Aeq.T], [Aeq, np.zeros((m, m))]])
        sol = np.linalg.lstsq(K, np.concatenate([np.zeros(nz), beq]), rcond=None)[0]
        w, lam = sol[:nz], sol[nz:]
        if np.max(np.abs(Aeq @ w - beq)) > 1e-9:
            continue
        v = rows @ w
        if np.any(v < lo - 1e-9) or np.any(v > hi + 1e-9):
            continue
        # KKT sign of the multipliers of active rows (H w + A^T lam = 0)
        ok = all((lam[len(e) + k] <= 1e-9) if s < 0 else (lam[len(e) + k] >= -1e-9)
                 for k, (q, s) in enumerate(act))
        if not ok:
            continue
        val = 0.5 * w @ H @ w
        if best is None or val < best[0] - 1e-12:
            best = (val, w)
    return best


@pytest.mark.parametrize("seed", [0, 4, 6])
def test_coupled_constraints_bruteforce(seed):
    """a = 1 (expectation), N = 2, coupled rows x_1 + u <= c at the root and
    x_1 + x_2 <= c at the leaves, tight enough to be active."""
    rng = np.random.default_rng(seed)
    anc = np.array([-1, 0, 0, 1, 2], np.int32)
    d = workloads.with_tree(anc, seed=seed, nx=2, nu=1, a=1.0, box=(50.0, 50.0))
    d["x0"] = np.array([1.0, -0.5])
    g = workloads.general_random(d, seed=seed, extra_rows=1, extra_leaf_rows=1, bound=50.0)
    g["Gx"][:, 3, :] = [1.0, 0.0]
    g["Gu"][:, 3, :] = [1.0]
    g["cmin"][:, 3], g["cmax"][:, 3] = -50.0, -0.3 - 0.2 * rng.uniform()
    g["GN"][:, 2, :] = [1.0, 1.0]
    g["cNmin"][:, 2], g["cNmax"][:, 2] = 0.2 + 0.2 * rng.uniform(), 50.0
    P = Problem(g)
    res = spock(CP(P), g["x0"], s=TIGHT)
    assert res.status == "converged"
    cand = [("n", i, 3) for i in (0, 1, 2)] + [("l", j, 2) for j in (3, 4)]
    val, w = _qp_bruteforce(P, g["x0"], cand)
    assert abs(res.v[0] - val) <= 1e-7 * max(1.0, abs(val))
    xs, us = risk.trajectory(P, res.v[: P.lay.n_z])
    xb, ub = risk.trajectory(P, w)
    np.testing.assert_allclose(xs, xb, atol=1e-5)
    np.testing.assert_allclose(us[P.tree.nonleaf], ub[P.tree.nonleaf], atol=1e-5)
    # the coupled rows decide the solution: at least two are active
    act = sum(abs(P.Gx[i, 3] @ xb[i] + P.Gu[i, 3] @ ub[i] - P.cmax[i, 3]) < 1e-7 for i in (0, 1, 2))
    act += sum(abs(P.GN[j, 2] @ xb[j] - P.cNmin[j, 2]) < 1e-7 for j in (3, 4))
    assert act >= 2
