"""Oracle projections: SOC by Moreau and brute force, prox_{alpha g*} by its
optimality condition over sampled points of S3, proj_S2 kernel property."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import cones
from oracle.problem import Problem
from paper_2212_01110_gb300 import workloads


@pytest.mark.parametrize("seed", range(20))
def test_soc_moreau(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(2, 9))
    w = rng.standard_normal(d) * 2
    p = cones.proj_soc(w)
    q = -cones.proj_soc(-w)          # projection on the polar cone -SOC
    np.testing.assert_allclose(p + q, w, atol=1e-14)
    assert abs(p @ q) < 1e-13
    assert np.linalg.norm(p[:-1]) <= p[-1] + 1e-14


def _soc_bruteforce(w):
    """Nearest point of SOC_2 / SOC_3 by searching the boundary rays
    (grid over the angle, golden-section refinement), plus 0 and w."""
    d = w.size
    cands = [np.zeros(d)]
    if np.linalg.norm(w[:-1]) <= w[-1]:
        cands.append(w.copy())

    def ray(theta):
        if d == 2:
            r = np.array([np.sign(np.cos(theta)) or 1.0, 1.0])
        else:
            r = np.array([np.cos(theta), np.sin(theta), 1.0])
        s = max(0.0, w @ r) / (r @ r)
        return s * r

    if d == 2:
        cands += [ray(0.0), ray(np.pi)]
    else:
        grid = np.linspace(0, 2 * np.pi, 721)
        f = [np.linalg.norm(ray(th) - w) for th in grid]
        k = int(np.argmin(f))
        res = minimize_scalar(lambda th: np.linalg.norm(ray(th) - w),
                              bounds=(grid[max(k - 1, 0)], grid[min(k + 1, 720)]),
                              method="bounded", options={"xatol": 1e-12})
        cands.append(ray(res.x))
    return min(cands, key=lambda c: np.linalg.norm(c - w))


@pytest.mark.parametrize("seed", range(30))
def test_soc_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    for d in (2, 3):
        w = rng.standard_normal(d) * 2
        p = cones.proj_soc(w)
        b = _soc_bruteforce(w)
        assert np.linalg.norm(p - w) <= np.linalg.norm(b - w) + 1e-12
        np.testing.assert_allclose(p, b, atol=1e-6)  # angle found to ~sqrt(machine eps)


def _sample_S3(P, rng, k):
    """Random points of S3 (block by block, Eq. (S3-def))."""
    lay, t = P.lay, P.tree
    pts = []
    for _ in range(k):
        s = np.zeros(lay.n_eta)
        for i in t.nonleaf:
            m = len(t.children[i])
            ey = lay.e_y[i]
            s[ey[:2 * m]] = np.abs(rng.standard_normal(2 * m)) * rng.choice([0.0, 1.0, 10.0])
            s[ey[2 * m]] = rng.standard_normal() * 10
            s[lay.e_sb[i]] = abs(rng.standard_normal()) * rng.choice([0.0, 1.0, 10.0])
            s[lay.e_x[i]] = rng.uniform(P.xmin[i], P.xmax[i])
            s[lay.e_u[i]] = rng.uniform(P.umin[i], P.umax[i])
        for c in t.nonroot:
            idx = np.concatenate([lay.e_qx[c], lay.e_ru[c], lay.e_t[c]])
            v = rng.standard_normal(idx.size - 1) * rng.choice([0.0, 1.0, 10.0])
            tt = np.linalg.norm(v) * (1 + rng.choice([0.0, 0.5]))
            w = np.concatenate([v, [tt]])
            w[-2:] += (0.5, -0.5)
            s[idx] = w
        for j in t.leaves:
            s[lay.e_lx[j]] = rng.uniform(P.xmin[j], P.xmax[j])
            idx = np.concatenate([lay.e_qn[j], lay.e_ls[j]])
            v = rng.standard_normal(idx.size - 1) * rng.choice([0.0, 1.0, 10.0])
            w = np.concatenate([v, [np.linalg.norm(v)]])
            w[-2:] += (0.5, -0.5)
            s[idx] = w
        pts.append(s)
    return pts


def _prox_opt_violation(P, eta, etap, alpha, pts):
    """Optimality of eta+ = prox_{alpha g*}(eta), g* the support function of
    S3: p = (eta - eta+)/alpha must lie in S3 (checked by projecting) and
    <eta+, s - p> <= 0 for every s in S3."""
    p = (eta - etap) / alpha
    dist = np.linalg.norm(cones.proj_S3(p, P) - p)
    worst = max(float(etap @ (s - p)) for s in pts)
    return dist, worst


@pytest.mark.parametrize("alpha", [1.0, 0.37, 2.5])
def test_prox_gconj_optimality(alpha):
    P = Problem(workloads.with_tree(workloads.fig1_tree(), seed=3, nx=3, nu=2))
    rng = np.random.default_rng(7)
    pts = _sample_S3(P, rng, 300)
    for trial in range(5):
        eta = rng.standard_normal(P.lay.n_eta) * 3
        etap = cones.prox_gconj(eta, alpha, P)
        dist, worst = _prox_opt_violation(P, eta, etap, alpha, pts)
        assert dist < 1e-12
        assert worst < 1e-9


def test_prox_gconj_literal_formula_is_wrong():
    """Planted mistake: the formula printed as eta - proj_S3(eta/alpha) (no
    alpha factor) violates the optimality condition for alpha != 1 -- the
    reason for the reading eta - alpha proj_S3(eta/alpha)."""
    P = Problem(workloads.with_tree(workloads.fig1_tree(), seed=3, nx=3, nu=2))
    rng = np.random.default_rng(8)
    pts = _sample_S3(P, rng, 300)
    alpha = 0.37
    eta = rng.standard_normal(P.lay.n_eta) * 3
    etap = eta - cones.proj_S3(eta / alpha, P)
    dist, worst = _prox_opt_violation(P, eta, etap, alpha, pts)
    assert dist > 1e-3 or worst > 1e-3


@pytest.mark.parametrize("seed", range(6))
def test_proj_S2(seed):
    P = Problem(workloads.random_tree(seed, N=3, max_branch=4, nx=2, nu=1))
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(P.lay.n_z)
    pz = cones.proj_S2(z, P)
    for i in P.tree.nonleaf:
        idx = cones.z2_block(P, i)
        M = cones.s2_matrix(P, i)
        assert np.max(np.abs(M @ pz[idx])) < 1e-13
        # z - P z in range(M^T): least-squares residual is zero
        diff = z[idx] - pz[idx]
        coef = np.linalg.lstsq(M.T, diff, rcond=None)[0]
        assert np.max(np.abs(M.T @ coef - diff)) < 1e-12
    np.testing.assert_allclose(cones.proj_S2(pz, P), pz, atol=1e-13)
