"""Oracle L against the constraints it must encode (Eq. (min-s0-v1), Eq.
(S3-def)) and ||L|| closed form vs power iteration."""
import numpy as np
import pytest

from oracle.linop import build_L, norm_L_blocks, norm_L_power
from oracle.problem import Problem
from paper_2212_01110_gb300 import workloads


def in_translated_soc(w, tol=0.0):
    """(v, t) - (0, 1/2, -1/2) in SOC  <=>  ||v'|| <= t' (t' last coordinate)."""
    s = np.zeros_like(w)
    s[-2:] = (0.5, -0.5)
    v = w - s
    return np.linalg.norm(v[:-1]) <= v[-1] + tol


def problems():
    return [Problem(workloads.small_binary(0)),
            Problem(workloads.with_tree(workloads.fig1_tree(), seed=1, nx=3, nu=2)),
            Problem(workloads.random_tree(5, N=3, max_branch=3, nx=4, nu=3))]


@pytest.mark.parametrize("P", problems())
def test_epigraph_rows(P):
    """Nonroot block of L z lies in SOC + (0,1/2,-1/2) iff x'Qx + u'Ru <= tau;
    leaf block iff x'Q_N x <= s; nonleaf row s - b'y >= 0 iff y'b <= s."""
    rng = np.random.default_rng(0)
    L = build_L(P)
    lay, t = P.lay, P.tree
    for sign in (+1, -1):
        z = rng.standard_normal(lay.n_z)
        for c in t.nonroot:
            p = t.anc[c]
            x, u = z[lay.x[p]], z[lay.u[p]]
            ell = x @ (P.Q[c] * x) + u @ (P.R[c] * u)
            z[lay.tau[c]] = ell + sign * 0.1
        for j in t.leaves:
            x = z[lay.x[j]]
            z[lay.s[j]] = x @ (P.QN[j] * x) + sign * 0.1
        eta = L @ z
        for c in t.nonroot:
            idx = np.concatenate([lay.e_qx[c], lay.e_ru[c], lay.e_t[c]])
            assert in_translated_soc(eta[idx]) == (sign > 0)
        for j in t.leaves:
            idx = np.concatenate([lay.e_qn[j], lay.e_ls[j]])
            assert in_translated_soc(eta[idx]) == (sign > 0)
        for i in t.nonleaf:
            y = z[lay.y[i]]
            assert (eta[lay.e_sb[i]] >= 0) == (y @ P.b(i) <= z[lay.s[i]])
            np.testing.assert_array_equal(eta[lay.e_x[i]], z[lay.x[i]])
            np.testing.assert_array_equal(eta[lay.e_u[i]], z[lay.u[i]])
            np.testing.assert_array_equal(eta[lay.e_y[i]], y)


@pytest.mark.parametrize("P", problems() + [Problem(workloads.datacenter(N=3, nx=4))])
def test_norm_blocks_vs_power(P):
    L = build_L(P)
    assert abs(norm_L_blocks(P) - norm_L_power(L)) < 1e-9 * norm_L_blocks(P)


def test_norm_independent_of_horizon():
    """||L|| does not grow with N (remark after the definition of L)."""
    vals = [norm_L_blocks(Problem(workloads.datacenter(N=N, nx=3))) for N in (2, 4, 6)]
    assert max(vals) - min(vals) < 1e-14
