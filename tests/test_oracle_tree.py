"""Oracle tree against the tree drawn in Fig. 1 and basic validation."""
import json
import os

import pytest

from oracle.tree import Tree, TreeError
from oracle.problem import Problem
from paper_2212_01110_gb300 import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fig1_tree.json")


def test_fig1_tree_structure():
    g = json.load(open(GOLD))
    t = Tree(g["anc"])
    for k, v in g["children"].items():
        assert t.children[int(k)] == v
    for s, nodes in enumerate(g["stages"]):
        assert t.nodes(s) == nodes
    assert t.N == g["N"]
    assert t.leaves == g["leaves"]
    assert t.nonleaf == g["nonleaf"]
    # uniform conditional probabilities -> absolute probabilities per stage sum to 1
    for s in range(t.N + 1):
        assert abs(t.pi[t.nodes(s)].sum() - 1.0) < 1e-15


@pytest.mark.parametrize("anc", [[0, 0], [-1, 5], [-1, 0, 0, 1], [-1, 2, 1]])
def test_bad_trees(anc):
    with pytest.raises(TreeError):
        Tree(anc)


def test_bad_probabilities():
    with pytest.raises(TreeError):
        Tree([-1, 0, 0], [1.0, 0.3, 0.3])


def test_sizes_formula():
    # n_z = 1 + nx n + nu |nonleaf| + 4 E + |nonleaf|
    # n_eta = (2E + |nonleaf|) + |nonleaf| (1 + nx + nu) + E (nx + nu + 2) + |leaves| (2 nx + 2)
    for d in [workloads.small_binary(0), workloads.with_tree(workloads.fig1_tree(), nx=2, nu=3),
              workloads.random_tree(3, N=4, max_branch=3)]:
        P = Problem(d)
        t = P.tree
        n, nl, E, lv = t.n, len(t.nonleaf), t.n - 1, len(t.leaves)
        nx, nu = P.nx, P.nu
        assert P.lay.n_z == 1 + nx * n + nu * nl + 4 * E + nl
        assert P.lay.n_eta == (2 * E + nl) + nl * (1 + nx + nu) + E * (nx + nu + 2) + lv * (2 * nx + 2)
    P = Problem(workloads.small_binary(0))
    assert (P.lay.n_z, P.lay.n_eta) == (123, 239)
