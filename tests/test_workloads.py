"""The seeded input generators (paper_2212_01110_gb300/workloads.py) produce
the stated recipes: the same seed gives the same arrays and another seed
different ones; tree sizes, probability vectors, spectra, cost and AV@R
ranges, boxes and x0 as the recipes say (the large scenario tree of the
benchmark, the batched workload with its scenario cap, the small binary
tree, the data-center system of Eq. (dynamics-example))."""
import numpy as np
import pytest

from paper_2212_01110_gb300 import workloads as W

KEYS = ("anc", "prob", "A", "B", "Q", "R", "QN", "a", "xmin", "xmax", "umin", "umax", "x0")


def _same(d1, d2):
    return all(np.array_equal(np.asarray(d1[k]), np.asarray(d2[k])) for k in KEYS)


def _children(anc):
    return np.bincount(np.asarray(anc)[1:], minlength=len(anc))


def _check_probs(d):
    anc, prob = np.asarray(d["anc"]), np.asarray(d["prob"])
    for i in np.flatnonzero(_children(anc)):
        p = prob[anc == i]
        assert np.all(p > 0) and abs(p.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("make", [
    lambda s: W.small_binary(s),
    lambda s: W.large_tree(s, branching_stages=2, N=6, nx=10, nu=4),
    lambda s: W.random_tree(s, N=3, max_branch=3, nx=3, nu=2),
    lambda s: W.batch_instances(seed=s, count=3)[2],
])
def test_seeded_and_deterministic(make):
    assert _same(make(0), make(0))
    assert not _same(make(0), make(1))


def test_large_tree_recipe():
    d = W.large_tree(seed=0, branching_stages=3, branch=4, N=6, nx=12, nu=5)
    anc, n, nx, nu = np.asarray(d["anc"]), len(d["anc"]), d["nx"], d["nu"]
    ch = _children(anc)
    assert n == 1 + 4 + 16 + 64 * 4 and int(np.sum(ch == 0)) == 64
    _check_probs(d)
    assert np.min(np.asarray(d["prob"])[1:]) >= 1e-3 / 1.004   # Dirichlet(1), floored at 1e-3, renormalised
    A = np.asarray(d["A"])
    for c in range(1, n):   # 0.95 x orthogonal: every singular value 0.95
        np.testing.assert_allclose(np.linalg.svd(A[c], compute_uv=False), 0.95, atol=1e-12)
    assert np.all((d["Q"][1:] >= 0.5) & (d["Q"][1:] <= 2.0))
    assert np.all(d["R"] == 0.1) and np.all(d["QN"] == 1.0)
    nl = np.flatnonzero(ch)
    assert np.all((d["a"][nl] >= 0.1) & (d["a"][nl] <= 0.9))
    assert np.all(d["xmax"] == 5.0) and np.all(d["xmin"] == -5.0)
    assert np.all(d["umax"] == 1.0) and np.all(d["umin"] == -1.0)
    assert np.max(np.abs(d["x0"])) <= 5.0 and d["x0"].shape == (nx,)
    assert np.asarray(d["B"]).shape == (n, nx, nu)
    u = W.large_tree(seed=0, branching_stages=3, branch=4, N=6, nx=12, nu=5, probs="uniform")
    np.testing.assert_array_equal(np.asarray(u["prob"])[1:5], 0.25)
    np.testing.assert_array_equal(u["A"], d["A"])   # the other draws do not change


def test_benchmark_tree_size():
    anc, _ = W.tree_from_branching([4] * 6 + [1] * 14)
    ch = _children(anc)
    assert (len(anc), int(np.sum(ch > 0)), int(np.sum(ch == 0))) == (62805, 58709, 4096)


def test_batch_recipe():
    ds = W.batch_instances(seed=0, count=64)
    for d in ds:
        anc = np.asarray(d["anc"])
        ch = _children(anc)
        leaves = int(np.sum(ch == 0))
        b = int(ch[0])
        assert b in (2, 3, 4) and leaves <= 64
        assert 10 <= d["nx"] <= 30 and 4 <= d["nu"] <= 10
        depth = np.zeros(len(anc), int)
        for i in range(1, len(anc)):
            depth[i] = depth[anc[i]] + 1
        N = int(depth.max())
        assert 5 <= N <= 15
        # branching for floor(log_b 64) stages (at most N), then one child
        stages = min(int(np.floor(np.log(64) / np.log(b) + 1e-9)), N)
        assert leaves == b ** stages
        _check_probs(d)
        nl = np.flatnonzero(ch)
        for i in nl:   # uniform child probabilities by default
            p = np.asarray(d["prob"])[anc == i]
            np.testing.assert_allclose(p, 1.0 / len(p))


def test_small_binary_recipe():
    d = W.small_binary(0)
    assert len(d["anc"]) == 15 and int(np.sum(_children(d["anc"]) == 0)) == 8
    _check_probs(d)
    assert np.all(d["Q"] == 1.0) and np.all(d["R"] == 0.1) and np.all(d["QN"] == 1.0)
    assert np.all(d["a"] == 0.5) and np.max(np.abs(d["x0"])) <= 5.0


def test_datacenter_system():
    """Eq. (dynamics-example): A(w) tridiagonal with off-diagonals 0.01 and
    diagonal growing with the disturbance index w and the state index j,
    B = I; Q = Q_N = I, R = 10 I; boxes 1 and 1.5; x0 = 0.1 * 1; children
    with probabilities 0.3, 0.7."""
    d = W.datacenter(N=3, nx=4)
    anc = np.asarray(d["anc"])
    A = np.asarray(d["A"])
    kids = np.flatnonzero(anc == 0)
    np.testing.assert_allclose(np.asarray(d["prob"])[kids], [0.3, 0.7])
    for w, c in enumerate(kids, start=1):
        Ac = A[c]
        np.testing.assert_allclose(np.diag(Ac, 1), 0.01)
        np.testing.assert_allclose(np.diag(Ac, -1), 0.01)
        assert np.count_nonzero(np.triu(Ac, 2)) == 0 and np.count_nonzero(np.tril(Ac, -2)) == 0
        # A_jj(w) = 1 + (w - 1)/d (1 + (j - 1)/nx), d = 2 disturbance values
        j = np.arange(1, 5)
        np.testing.assert_allclose(np.diag(Ac), 1.0 + (w - 1) / 2.0 * (1.0 + (j - 1) / 4.0), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(np.asarray(d["B"])[1], np.eye(4))
    assert np.all(d["Q"] == 1.0) and np.all(d["QN"] == 1.0) and np.all(d["R"] == 10.0)
    assert np.all(d["xmax"] == 1.0) and np.all(d["umax"] == 1.5)
    np.testing.assert_array_equal(d["x0"], 0.1)
    assert np.all(np.asarray(d["a"]) == 0.95)
