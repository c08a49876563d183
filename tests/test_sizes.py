"""Sizes quoted for the 62,805-node scenario tree (branching 4 for 6 stages,
then one child, N = 20, nx = 50, nu = 20): node counts of the generator's
tree, the lengths of z and eta from the oracle's layout against the counting
formulas of the problem statement (Sec. "Operator splitting": per nonleaf
node x, u, the z_2 block of 4m + 1 entries; eta blocks per nonleaf, nonroot
and leaf node), and the algorithmic bytes per chain launch used by bench.py."""
import numpy as np

import bench
from oracle.problem import build_layout
from oracle.tree import Tree
from paper_2212_01110_gb300 import workloads as W


def test_large_tree_sizes():
    anc, _ = W.tree_from_branching([4] * 6 + [1] * 14)
    n = len(anc)
    children = np.bincount(anc[1:], minlength=n)
    nl = int(np.sum(children > 0))
    leaves = n - nl
    assert (n, nl, leaves) == (62805, 58709, 4096)
    prob = np.ones(n)
    for i in range(n):
        if children[i]:
            prob[anc == i] = 1.0 / children[i]
    nx, nu = 50, 20
    lay = build_layout(Tree(anc, prob), nx, nu)
    E = n - 1
    n_z = 1 + nx * n + nu * nl + 4 * E + nl
    n_eta = (2 * E + nl) + nl * (1 + nx + nu) + E * (nx + nu + 2) + leaves * (2 * nx + 2)
    assert (lay.n_z, lay.n_eta) == (n_z, n_eta) == (4624356, 9292336)


def test_chain_launch_bytes():
    d = {"nx": 50, "nu": 20}
    # per chain node: [Abar | B] 50x70, K and W^T 2x20x50, Rt^-1 20x20, xbar, ubar, d; per chain two x vectors
    assert bench.bytes_bwd_chain(d, 4096, 14, 8) == 2751201280
    assert bench.bytes_bwd_chain(d, 4096, 14, 4) == 1375600640
    assert bench.flops_bwd_chain(d, 4096, 14) == 676659200.0
    assert bench.bytes_fwd_chain(d, 4096, 14, 4) == 1053655040


def test_clock_summary_parses_nvidia_smi_rows(tmp_path):
    """The clocks record of the timed region: median SM clock under load, the
    maximum clock, and every throttle reason seen Active in any sample (rows
    as nvidia-smi --format=csv,noheader,nounits writes them; a malformed row
    is skipped)."""
    rows = [
        "0, 2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1201.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    c = bench.Clocks(0)
    c.path = str(path)
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    rows[0] = rows[0].replace("Not Active, Not Active, Not Active, Not Active",
                              "Active, Not Active, Active, Not Active")
    path.write_text("\n".join(rows) + "\n")
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.Clocks(0).summary()["reasons"] == ["unavailable"]
