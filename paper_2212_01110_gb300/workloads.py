"""Seeded synthetic RAOCP instances (inputs only, no solver arithmetic).

Every generator returns a plain dict of numpy arrays in *user* node order
(which here is already stage-major breadth-first order):

    anc     int32[n]        ancestor of each node, anc[0] = -1
    prob    float64[n]      conditional probability of reaching node i from
                            anc(i); prob[0] = 1
    nx, nu  int
    A       float64[n,nx,nx]  dynamics of the edge into node i (A[0] unused)
    B       float64[n,nx,nu]
    Q       float64[n,nx]   diagonal of Q^i, cost weight on the edge into i
    R       float64[n,nu]   diagonal of R^i
    QN      float64[n,nx]   diagonal of the terminal weight (read at leaves)
    a       float64[n]      AV@R parameter of each nonleaf node, in [0, 1]
    xmin, xmax float64[n,nx]; umin, umax float64[n,nu]   box constraints
    x0      float64[nx]     initial state

General form (polyhedral constraints, dense costs; ``general_*`` below):
    Q, R, QN  float64[n,nx,nx] / [n,nu,nu] / [n,nx,nx]  dense SPD matrices
    Gx, Gu    float64[n,nc,nx], [n,nc,nu]   constraint matrices of nonleaf nodes
    cmin, cmax float64[n,nc]                bounds of Gx x + Gu u (nonleaf)
    GN        float64[n,ncN,nx]             terminal constraint matrices (leaves)
    cNmin, cNmax float64[n,ncN]             bounds of GN x (leaves)
(no xmin/xmax/umin/umax).

The tree shapes, distributions and sizes follow the workloads described for
SPOCK (scenario trees with stage-wise branching, Sec. "Scenario trees"; the
data-center system of Eq. (dynamics-example)).  Random draws use
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# tree shapes
# ----------------------------------------------------------------------------

def tree_from_branching(branching):
    """Stage-wise branching factors -> (anc, stage).

    ``branching[t]`` is the number of children of every node at stage t, so
    the horizon is N = len(branching) and leaves sit at stage N.  Nodes are
    numbered breadth first, children of a node contiguous.
    """
    anc = [-1]
    stage = [0]
    frontier = [0]
    for t, b in enumerate(branching):
        nxt = []
        for parent in frontier:
            for _ in range(int(b)):
                anc.append(parent)
                stage.append(t + 1)
                nxt.append(len(anc) - 1)
        frontier = nxt
    return np.asarray(anc, np.int32), np.asarray(stage, np.int32)


def _children_counts(anc):
    n = len(anc)
    cnt = np.zeros(n, np.int64)
    np.add.at(cnt, anc[1:], 1)
    return cnt


def _conditional_probs(rng, anc, kind):
    """Conditional child probabilities; kind in {'uniform', 'dirichlet'} or a
    fixed tuple used for every parent with that many children."""
    n = len(anc)
    prob = np.zeros(n)
    prob[0] = 1.0
    cnt = _children_counts(anc)
    start = 1
    # children are contiguous in breadth-first numbering
    for parent in range(n):
        m = int(cnt[parent])
        if m == 0:
            continue
        idx = np.arange(start, start + m)
        assert np.all(anc[idx] == parent)
        if m == 1:
            p = np.ones(1)
        elif isinstance(kind, tuple):
            p = np.asarray(kind, float)
            assert len(p) == m
        elif kind == "uniform":
            p = np.full(m, 1.0 / m)
        elif kind == "dirichlet":
            p = rng.dirichlet(np.ones(m))
            p = np.maximum(p, 1e-3)
            p = p / p.sum()
        else:
            raise ValueError(kind)
        prob[idx] = p
        start += m
    return prob


def _haar_orthogonal(rng, count, n):
    g = rng.standard_normal((count, n, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diagonal(r, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return q * d[:, None, :]


def _box(n, dim, lim):
    lo = np.full((n, dim), -float(lim))
    return lo, -lo


def _draw_x0(rng, nx, xlim):
    while True:
        x0 = rng.standard_normal(nx)
        if np.max(np.abs(x0)) <= xlim:
            return x0


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def small_binary(seed=0, N=3, nx=3, nu=2, a=0.5):
    """Binary tree of horizon N (N=3: 15 nodes, 8 leaves), uniform child
    probabilities, A = I + 0.1 N(0,1), B ~ N(0,1), Q = I, R = 0.1 I, Q_N = I,
    AV@R parameter ``a`` at every nonleaf node, |x| <= 5, |u| <= 1,
    x0 ~ N(0,1) redrawn until inside the box."""
    rng = np.random.default_rng(seed)
    anc, _ = tree_from_branching([2] * N)
    n = len(anc)
    prob = _conditional_probs(rng, anc, "uniform")
    A = np.eye(nx)[None] + 0.1 * rng.standard_normal((n, nx, nx))
    B = rng.standard_normal((n, nx, nu))
    A[0] = 0.0
    B[0] = 0.0
    Q = np.ones((n, nx))
    R = np.full((n, nu), 0.1)
    QN = np.ones((n, nx))
    av = np.full(n, float(a))
    xmin, xmax = _box(n, nx, 5.0)
    umin, umax = _box(n, nu, 1.0)
    x0 = _draw_x0(rng, nx, 5.0)
    return dict(anc=anc, prob=prob, nx=nx, nu=nu, A=A, B=B, Q=Q, R=R, QN=QN,
                a=av, xmin=xmin, xmax=xmax, umin=umin, umax=umax, x0=x0)


def large_tree(seed=0, branching_stages=6, branch=4, N=20, nx=50, nu=20,
               xlim=5.0, ulim=1.0, probs="dirichlet", rho=0.95):
    """Branching ``branch`` for the first ``branching_stages`` stages, then one
    child per node, horizon N (defaults: 62,805 nodes, 58,709 nonleaf, 4,096
    scenarios, about 4.3 M state/input variables).  A = rho U with U
    Haar-orthogonal (spectral radius rho, default 0.95), B ~ N(0, 1/nx), Q = diag U(0.5, 2),
    R = 0.1 I, Q_N = I, AV@R parameter U(0.1, 0.9) per nonleaf node,
    Dirichlet(1) child probabilities (``probs="uniform"``: 1/branch; the draws
    of the other data do not change), |x| <= xlim, |u| <= ulim,
    x0 ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    branching = [branch] * branching_stages + [1] * (N - branching_stages)
    anc, _ = tree_from_branching(branching)
    n = len(anc)
    prob = _conditional_probs(rng, anc, "dirichlet")
    if probs == "uniform":
        prob = _conditional_probs(None, anc, "uniform")
    A = float(rho) * _haar_orthogonal(rng, n, nx)
    B = rng.standard_normal((n, nx, nu)) / np.sqrt(nx)
    A[0] = 0.0
    B[0] = 0.0
    Q = rng.uniform(0.5, 2.0, size=(n, nx))
    R = np.full((n, nu), 0.1)
    QN = np.ones((n, nx))
    av = rng.uniform(0.1, 0.9, size=n)
    xmin, xmax = _box(n, nx, xlim)
    umin, umax = _box(n, nu, ulim)
    x0 = _draw_x0(rng, nx, xlim)
    return dict(anc=anc, prob=prob, nx=nx, nu=nu, A=A, B=B, Q=Q, R=R, QN=QN,
                a=av, xmin=xmin, xmax=xmax, umin=umin, umax=umax, x0=x0)


def random_tree(seed=0, N=3, max_branch=3, nx=4, nu=2, chain_after=None,
                a_range=(0.0, 1.0), box=(5.0, 1.0), stable=False):
    """Ragged random tree: every nonleaf node draws its own number of
    children in 1..max_branch (optionally one child from stage
    ``chain_after`` on); Dirichlet child probabilities; Gaussian data."""
    rng = np.random.default_rng(seed)
    anc = [-1]
    frontier = [0]
    for t in range(N):
        nxt = []
        for parent in frontier:
            m = 1 if (chain_after is not None and t >= chain_after) else int(rng.integers(1, max_branch + 1))
            for _ in range(m):
                anc.append(parent)
                nxt.append(len(anc) - 1)
        frontier = nxt
    anc = np.asarray(anc, np.int32)
    n = len(anc)
    prob = _conditional_probs(rng, anc, "dirichlet")
    if stable:
        A = 0.95 * _haar_orthogonal(rng, n, nx)
    else:
        A = np.eye(nx)[None] + 0.1 * rng.standard_normal((n, nx, nx))
    B = rng.standard_normal((n, nx, nu)) / np.sqrt(nx)
    A[0] = 0.0
    B[0] = 0.0
    Q = rng.uniform(0.5, 2.0, size=(n, nx))
    R = rng.uniform(0.05, 0.5, size=(n, nu))
    QN = rng.uniform(0.5, 2.0, size=(n, nx))
    av = rng.uniform(a_range[0], a_range[1], size=n)
    xmin, xmax = _box(n, nx, box[0])
    umin, umax = _box(n, nu, box[1])
    x0 = _draw_x0(rng, nx, box[0])
    return dict(anc=anc, prob=prob, nx=nx, nu=nu, A=A, B=B, Q=Q, R=R, QN=QN,
                a=av, xmin=xmin, xmax=xmax, umin=umin, umax=umax, x0=x0)


def datacenter(N=7, nx=5, nu=None, d=2, probs=(0.3, 0.7), a=0.95):
    """The data-center thermal system of Eq. (dynamics-example): tridiagonal
    A(w) with diagonal 1 + (w-1)/d (1 + (j-1)/nx) and off-diagonals 0.01,
    B = I, d disturbance values with conditional probabilities ``probs``,
    Q = Q_N = I, R = 10 I, |x| <= 1, |u| <= 1.5, AV@R_a at every node,
    x0 = 0.1 * 1."""
    nu = nx if nu is None else nu
    anc, _ = tree_from_branching([d] * N)
    n = len(anc)
    prob = _conditional_probs(None, anc, tuple(probs))
    A = np.zeros((n, nx, nx))
    B = np.zeros((n, nx, nu))
    cnt = _children_counts(anc)
    # child index w (1-based) within its sibling group
    w_of = np.zeros(n, np.int64)
    start = 1
    for parent in range(n):
        for w in range(int(cnt[parent])):
            w_of[start + w] = w + 1
        start += int(cnt[parent])
    j = np.arange(1, nx + 1)
    for i in range(1, n):
        w = w_of[i]
        Ai = np.diag(1.0 + (w - 1) / d * (1.0 + (j - 1) / nx))
        Ai += np.diag(np.full(nx - 1, 0.01), 1) + np.diag(np.full(nx - 1, 0.01), -1)
        A[i] = Ai
        B[i] = np.eye(nx, nu)
    Q = np.ones((n, nx))
    R = np.full((n, nu), 10.0)
    QN = np.ones((n, nx))
    av = np.full(n, float(a))
    xmin, xmax = _box(n, nx, 1.0)
    umin, umax = _box(n, nu, 1.5)
    x0 = np.full(nx, 0.1)
    return dict(anc=anc, prob=prob, nx=nx, nu=nu, A=A, B=B, Q=Q, R=R, QN=QN,
                a=av, xmin=xmin, xmax=xmax, umin=umin, umax=umax, x0=x0)


def fig1_tree():
    """The 9-node scenario tree drawn in Fig. 1 (node 1 has children {3,4},
    node 2 has children {5,6,7,8})."""
    return np.asarray([-1, 0, 0, 1, 1, 2, 2, 2, 2], np.int32)


def with_tree(anc, seed=0, nx=3, nu=2, a=0.5, box=(5.0, 1.0)):
    """Gaussian data (as ``small_binary``) on a given tree."""
    rng = np.random.default_rng(seed)
    anc = np.asarray(anc, np.int32)
    n = len(anc)
    prob = _conditional_probs(rng, anc, "dirichlet")
    A = np.eye(nx)[None] + 0.1 * rng.standard_normal((n, nx, nx))
    B = rng.standard_normal((n, nx, nu))
    A[0] = 0.0
    B[0] = 0.0
    Q = rng.uniform(0.5, 2.0, size=(n, nx))
    R = rng.uniform(0.05, 0.5, size=(n, nu))
    QN = rng.uniform(0.5, 2.0, size=(n, nx))
    av = np.full(n, float(a))
    xmin, xmax = _box(n, nx, box[0])
    umin, umax = _box(n, nu, box[1])
    x0 = _draw_x0(rng, nx, box[0])
    return dict(anc=anc, prob=prob, nx=nx, nu=nu, A=A, B=B, Q=Q, R=R, QN=QN,
                a=av, xmin=xmin, xmax=xmax, umin=umin, umax=umax, x0=x0)


def random_vectors(n_z, n_eta, seed=0, scale=1.0):
    """Seeded test points (z, eta) for operator-level comparisons."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(n_z), scale * rng.standard_normal(n_eta)


def batch_instances(seed=0, count=512, max_scenarios=64, probs="uniform"):
    """Heterogeneous batch: per instance a branching factor b ~ U{2,3,4},
    horizon N ~ U{5..15}, nx ~ U{10..30}, nu ~ U{4..10}; the tree branches
    for the first floor(log_b max_scenarios) stages and then has one child
    per node (scenario cap: full trees of branching 4 and horizon 15 would
    have 1.4e9 nodes).  Data as ``large_tree`` (A = 0.95 x Haar-orthogonal,
    B ~ N(0, 1/nx), Q = diag U(0.5, 2), R = 0.1 I, Q_N = I, AV@R a ~ U(0.1, 0.9),
    |x| <= 5, |u| <= 1, x0 ~ N(0, 1)) with uniform child probabilities by
    default (the batched workload states the cost, AV@R and box distributions
    but not the probabilities)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        b = int(rng.integers(2, 5))
        N = int(rng.integers(5, 16))
        nx = int(rng.integers(10, 31))
        nu = int(rng.integers(4, 11))
        stages = 0
        while b ** (stages + 1) <= max_scenarios:
            stages += 1
        stages = min(stages, N)
        out.append(large_tree(seed=1000 * seed + i, branching_stages=stages, branch=b, N=N, nx=nx, nu=nu,
                              probs=probs))
    return out


# ----------------------------------------------------------------------------
# general form: polyhedral constraints and dense cost matrices
# ----------------------------------------------------------------------------

def _scaled_orthogonal(rng, count, n):
    """count matrices U diag(s), U Haar-orthogonal, s ~ U(0.5, 2): random
    well-conditioned coordinate changes."""
    return _haar_orthogonal(rng, count, n) * rng.uniform(0.5, 2.0, size=(count, 1, n))


def general_transform(d, seed=0):
    """The same problem as the box-form instance ``d`` in new coordinates
    x'^i = T^i x^i, u'^i = S^i u^i with per-node random T^i, S^i (scaled
    orthogonal).  Returns (d', T, S): dynamics A'^c = T^c A^c T^p^-1,
    B'^c = T^c B^c S^p^-1 (p the ancestor), dense costs Q'^c = T^p^-T Q^c T^p^-1,
    R'^c = S^p^-T R^c S^p^-1, Q_N'^j = T^j^-T Q_N^j T^j^-1, constraint rows
    Gx = [T^i^-1; 0], Gu = [0; S^i^-1] with the box bounds of d, GN = T^j^-1,
    x0' = T^0 x0.  Its solution is (T^i x^i, S^i u^i) and its optimal value
    that of d."""
    rng = np.random.default_rng(seed)
    anc = np.asarray(d["anc"])
    n, nx, nu = len(anc), int(d["nx"]), int(d["nu"])
    T = _scaled_orthogonal(rng, n, nx)
    S = _scaled_orthogonal(rng, n, nu)
    Ti, Si = np.linalg.inv(T), np.linalg.inv(S)
    A = np.zeros((n, nx, nx))
    B = np.zeros((n, nx, nu))
    Q = np.zeros((n, nx, nx))
    R = np.zeros((n, nu, nu))
    QN = np.zeros((n, nx, nx))
    for c in range(n):
        QN[c] = Ti[c].T @ np.diag(d["QN"][c]) @ Ti[c]
        if c == 0:
            Q[c], R[c] = np.eye(nx), np.eye(nu)
            continue
        p = int(anc[c])
        A[c] = T[c] @ d["A"][c] @ Ti[p]
        B[c] = T[c] @ d["B"][c] @ Si[p]
        Q[c] = Ti[p].T @ np.diag(d["Q"][c]) @ Ti[p]
        R[c] = Si[p].T @ np.diag(d["R"][c]) @ Si[p]
    Q = 0.5 * (Q + Q.transpose(0, 2, 1))
    R = 0.5 * (R + R.transpose(0, 2, 1))
    QN = 0.5 * (QN + QN.transpose(0, 2, 1))
    Gx = np.zeros((n, nx + nu, nx))
    Gu = np.zeros((n, nx + nu, nu))
    Gx[:, :nx, :] = Ti
    Gu[:, nx:, :] = Si
    cmin = np.concatenate([d["xmin"], d["umin"]], axis=1)
    cmax = np.concatenate([d["xmax"], d["umax"]], axis=1)
    out = dict(anc=d["anc"], prob=d["prob"], nx=nx, nu=nu, A=A, B=B, Q=Q, R=R, QN=QN, a=d["a"],
               Gx=Gx, Gu=Gu, cmin=cmin, cmax=cmax, GN=Ti.copy(), cNmin=d["xmin"].copy(),
               cNmax=d["xmax"].copy(), x0=T[0] @ d["x0"])
    return out, T, S


def general_random(d, seed=0, extra_rows=4, extra_leaf_rows=2, bound=3.0, dense=True):
    """General-form data on the tree and dynamics of ``d``: dense SPD costs
    Q^i = D (0.5 I + M M^T / nx) D with M ~ N(0, 1), D the square root of the
    diagonal of d's Q^i (R, Q_N alike), and constraint rows: the box rows of d
    (Gamma = I) followed by ``extra_rows`` coupled rows g^T (x, u) in
    [-bound, bound], g ~ N(0, 1/(nx + nu)) (leaves: ``extra_leaf_rows`` rows
    on x).  With ``dense=False`` the costs stay diagonal."""
    rng = np.random.default_rng(seed)
    n, nx, nu = len(d["anc"]), int(d["nx"]), int(d["nu"])

    def spd(diag, dim):
        M = rng.standard_normal((n, dim, dim))
        core = 0.5 * np.eye(dim)[None] + M @ M.transpose(0, 2, 1) / dim
        Dh = np.sqrt(np.asarray(diag))
        out = Dh[:, :, None] * core * Dh[:, None, :]
        return 0.5 * (out + out.transpose(0, 2, 1))

    out = dict(anc=d["anc"], prob=d["prob"], nx=nx, nu=nu, A=d["A"], B=d["B"], a=d["a"], x0=d["x0"])
    if dense:
        out["Q"], out["R"], out["QN"] = spd(d["Q"], nx), spd(d["R"], nu), spd(d["QN"], nx)
    else:
        out["Q"], out["R"], out["QN"] = d["Q"], d["R"], d["QN"]
    nc, ncN = nx + nu + extra_rows, nx + extra_leaf_rows
    Gx = np.zeros((n, nc, nx))
    Gu = np.zeros((n, nc, nu))
    Gx[:, :nx, :] = np.eye(nx)
    Gu[:, nx:nx + nu, :] = np.eye(nu)
    g = rng.standard_normal((n, extra_rows, nx + nu)) / np.sqrt(nx + nu)
    Gx[:, nx + nu:, :] = g[:, :, :nx]
    Gu[:, nx + nu:, :] = g[:, :, nx:]
    cmin = np.concatenate([d["xmin"], d["umin"], np.full((n, extra_rows), -bound)], axis=1)
    cmax = np.concatenate([d["xmax"], d["umax"], np.full((n, extra_rows), bound)], axis=1)
    GN = np.zeros((n, ncN, nx))
    GN[:, :nx, :] = np.eye(nx)
    GN[:, nx:, :] = rng.standard_normal((n, extra_leaf_rows, nx)) / np.sqrt(nx)
    cNmin = np.concatenate([d["xmin"], np.full((n, extra_leaf_rows), -bound)], axis=1)
    cNmax = np.concatenate([d["xmax"], np.full((n, extra_leaf_rows), bound)], axis=1)
    out.update(Gx=Gx, Gu=Gu, cmin=cmin, cmax=cmax, GN=GN, cNmin=cNmin, cNmax=cNmax)
    return out


# ----------------------------------------------------------------------------
# coherent risk measures in conic form (b, E, F, K), K = R^kp_+ x {0}^(ny-kp)
# ----------------------------------------------------------------------------

def risk_measures(d, kind="mean_avar", lam=0.5, radius=0.3):
    """The instance ``d`` with a conic risk measure at every nonleaf node
    (key "risk": per node None or dict(b, E, F, kp)), children's conditional
    probabilities pi = d["prob"], AV@R parameter a = d["a"]:
      "avar":      AV@R_a written in the general form, b = (pi, 0, 1),
                   E = [a I, -I, 1]^T, kp = 2m;
      "mean_avar": lam E^pi + (1 - lam) AV@R_a, ambiguity set
                   {mu : sum mu = 1, lam pi <= mu <= lam pi + (1 - lam) pi / a}:
                   b = (pi (lam + (1 - lam) / a), -lam pi, 1), E = [I, -I, 1]^T,
                   kp = 2m (needs a > 0);
      "tv":        worst case over the total-variation ball
                   {mu in simplex : ||mu - pi||_1 <= radius}, with nu >= |mu - pi|:
                   rows (pi - mu + nu, -pi + mu + nu, radius - 1'nu, mu >= 0 | 1 - 1'mu = 0),
                   n_nu = m, kp = 3m + 1, ny = 3m + 2."""
    anc = np.asarray(d["anc"])
    n = len(anc)
    kids = [[] for _ in range(n)]
    for c in range(1, n):
        kids[int(anc[c])].append(c)
    risk = [None] * n
    for i in range(n):
        ch = kids[i]
        m = len(ch)
        if m == 0:
            continue
        pi = np.asarray(d["prob"], float)[ch]
        a = float(d["a"][i])
        I, one = np.eye(m), np.ones((1, m))
        if kind == "avar":
            b = np.concatenate([pi, np.zeros(m), [1.0]])
            E = np.vstack([a * I, -I, one])
            risk[i] = dict(b=b, E=E, F=np.zeros((2 * m + 1, 0)), kp=2 * m)
        elif kind == "mean_avar":
            if a <= 0:
                raise ValueError("mean_avar needs a > 0")
            b = np.concatenate([pi * (lam + (1.0 - lam) / a), -lam * pi, [1.0]])
            E = np.vstack([I, -I, one])
            risk[i] = dict(b=b, E=E, F=np.zeros((2 * m + 1, 0)), kp=2 * m)
        elif kind == "tv":
            Z = np.zeros((m, m))
            b = np.concatenate([pi, -pi, [radius], np.zeros(m), [1.0]])
            E = np.vstack([I, -I, np.zeros((1, m)), -I, one])
            F = np.vstack([-I, -I, one, Z, np.zeros((1, m))])
            risk[i] = dict(b=b, E=E, F=F, kp=3 * m + 1)
        else:
            raise ValueError(kind)
    out = dict(d)
    out["risk"] = risk
    return out
