"""Helpers shared by the GPU parity tests: build the oracle and the CUDA
problem from the same seeded workload, compare element by element."""
import numpy as np

from oracle.cp import CP
from oracle.problem import Problem as OProblem

RTOL = 1e-10   # FP64 parity: relative to max(1, |reference|_inf)


def rel_err(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b))))) if b.size else 0.0


class Pair:
    def __init__(self, d):
        import torch
        from paper_2212_01110_gb300 import spock
        self.d = d
        self.op = OProblem(d)
        self.cp = CP(self.op)
        self.gp = spock.Problem(d)
        assert (self.gp.n_z, self.gp.n_eta) == (self.op.lay.n_z, self.op.lay.n_eta)
        assert abs(self.gp.norm_L - self.cp.normL) < 1e-12 * self.cp.normL
        self.alpha = self.cp.alpha
        self.dev = torch.device("cuda:0")
        self.x0 = torch.tensor(d["x0"], dtype=torch.float64, device=self.dev)

    def t(self, a):
        import torch
        return torch.tensor(np.asarray(a, float), dtype=torch.float64, device=self.dev)


# trees spanning the code paths: full branching (no chain region), chains
# below branching stages, a pure chain (every node one child), ragged
# branching, the tree of Fig. 1, and state/input sizes crossing 32/64/96 lanes
def cases():
    from paper_2212_01110_gb300 import workloads as W
    return {
        "binary_N3": W.small_binary(0),
        "fig1": W.with_tree(W.fig1_tree(), seed=1, nx=3, nu=2),
        "ragged": W.random_tree(3, N=4, max_branch=3, nx=4, nu=3),
        "chains": W.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2),
        "pure_chain": W.random_tree(5, N=5, max_branch=1, nx=3, nu=2),
        "nx1_nu1": W.random_tree(6, N=3, max_branch=2, nx=1, nu=1),
        "wide_50_20": W.large_tree(0, branching_stages=2, branch=3, N=5, nx=50, nu=20),
        "wide_100_28": W.random_tree(7, N=3, max_branch=2, nx=100, nu=28, stable=True),
        "a0_a1": W.random_tree(8, N=3, max_branch=3, nx=3, nu=2, a_range=(0.0, 0.0)),
        # nodes with more than 16 and more than 32 children: the y block
        # (2m + 1 entries) and the children of a node span several warp chunks
        "root_40": W.with_tree(W.tree_from_branching([40, 1])[0], seed=9, nx=3, nu=2),
        "root_17_2": W.with_tree(W.tree_from_branching([17, 2])[0], seed=10, nx=4, nu=2, a=0.3),
        # the paper's system on a 127-node tree: above the single-block size,
        # so solves run the graph-driven kernels
        "datacenter_N6": W.datacenter(N=6, nx=3),
        # the large tree's launch shapes: 1,024 chains of 3 nonleaf nodes below
        # 5 stages with 4 children (4,437 nodes), nx = 50, nu = 20 -- many blocks
        # per SM for the direct kernels, several chains per block in the
        # persistent loops of the staged kernels
        "chains_1024_50_20": W.large_tree(3, branching_stages=5, branch=4, N=8, nx=50, nu=20),
        # more inputs than states: nu > nx, and nu > 32 with chains below two
        # branching stages (the input-indexed loops and slots of every kernel)
        "nu_gt_nx": W.random_tree(9, N=3, max_branch=4, nx=2, nu=5),
        "wide_20_50": W.large_tree(1, branching_stages=2, branch=3, N=5, nx=20, nu=50),
        # horizon 1: a root and one leaf (a chain of one step), a root and
        # five leaves (one branching stage, no chain region)
        "two_nodes": W.with_tree(W.tree_from_branching([1])[0], seed=11, nx=3, nu=2),
        "N1_star": W.with_tree(W.tree_from_branching([5])[0], seed=12, nx=3, nu=2),
    }
