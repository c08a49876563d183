"""Entry points of the C-ABI beyond the solve: trees from absolute
probabilities (Sec. "Scenario trees"), the host-buffer batch solve and
gradient, and the count of applications of L reported by a solve (the
x-axis of Fig. 1)."""
import numpy as np
import pytest

from paper_2212_01110_gb300 import workloads as W
from tests.gpu_common import rel_err

pytestmark = pytest.mark.gpu


def _absolute(anc, prob):
    pi = np.ones(len(anc))
    for i in range(1, len(anc)):   # parents precede children in these trees
        pi[i] = pi[anc[i]] * prob[i]
    return pi


def test_tree_from_absolute_probabilities_gives_the_same_operator():
    import torch
    from paper_2212_01110_gb300 import spock
    d = W.random_tree(3, N=4, max_branch=3, nx=4, nu=3)
    dev = torch.device("cuda:0")
    t_abs = spock.spock_tree_create_abs(d["anc"], _absolute(d["anc"], d["prob"]))
    p_abs = spock.spock_problem_create(t_abs, d)
    P = spock.Problem(d)
    nz, ne, nl, _ = spock.spock_problem_info(p_abs)
    assert (nz, ne) == (P.n_z, P.n_eta) and abs(nl - P.norm_L) <= 1e-14 * P.norm_L
    rng = np.random.default_rng(5)
    z = torch.tensor(rng.standard_normal(nz), dtype=torch.float64, device=dev)
    e = torch.tensor(rng.standard_normal(ne), dtype=torch.float64, device=dev)
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
    outs = []
    for h in (p_abs, P.handle):
        zo, eo = torch.empty_like(z), torch.empty_like(e)
        spock.spock_T_dev(h, x0, 0.0, z, e, zo, eo)
        outs.append(torch.cat([zo, eo]).cpu().numpy())
    # p = pi^c / pi^anc(c) reproduces the conditional probabilities to rounding
    assert rel_err(outs[0], outs[1]) < 1e-13
    spock.spock_free(p_abs)
    spock.spock_free(t_abs)
    bad = _absolute(d["anc"], d["prob"])
    bad[1] *= 1.5   # children of the root no longer carry the root's probability
    with pytest.raises(spock.SpockError) as ex:
        spock.spock_tree_create_abs(d["anc"], bad)
    assert ex.value.code == -1


def test_host_buffer_batch_solve_equals_device_buffer_batch_solve():
    import torch
    from paper_2212_01110_gb300 import spock
    dev = torch.device("cuda:0")
    ds = [W.small_binary(0), W.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2), W.datacenter(N=3, nx=4)]
    probs = [spock.Problem(d) for d in ds]
    s = spock.spock_default_settings(max_iter=40, eps_abs=1e-14, eps_rel=1e-14)
    b1 = spock.spock_batch_create([p.handle for p in probs])
    zs = [np.zeros(p.n_z) for p in probs]
    es = [np.zeros(p.n_eta) for p in probs]
    infos = spock.spock_batch_solve(b1, [d["x0"] for d in ds], s, zs, es, 0)
    spock.spock_free(b1)
    b2 = spock.spock_batch_create([p.handle for p in probs])
    zd = [torch.zeros(p.n_z, dtype=torch.float64, device=dev) for p in probs]
    ed = [torch.zeros(p.n_eta, dtype=torch.float64, device=dev) for p in probs]
    x0d = [torch.tensor(d["x0"], dtype=torch.float64, device=dev) for d in ds]
    infos_d = spock.spock_batch_solve_dev(b2, x0d, s, zd, ed, 0)
    spock.spock_free(b2)
    for i in range(len(ds)):
        assert infos[i].n_T == infos_d[i].n_T and infos[i].n_L == 2 * infos[i].n_T
        got = np.concatenate([zs[i], es[i]])
        ref = torch.cat([zd[i], ed[i]]).cpu().numpy()
        assert rel_err(got, ref) < 1e-13


def test_host_buffer_gradient_equals_device_gradient():
    import torch
    from paper_2212_01110_gb300 import spock
    dev = torch.device("cuda:0")
    d = W.small_binary(0)
    P = spock.Problem(d)
    n, nx, nu = len(d["anc"]), d["nx"], d["nu"]
    z = np.zeros(P.n_z)
    e = np.zeros(P.n_eta)
    info = spock.spock_solve(P.handle, d["x0"], None, z, e, 0)
    assert info.status == spock.SPOCK_OK and info.n_L == 2 * info.n_T
    shapes = [(nx,), (n, nx, nx), (n, nx, nu), (n, nx), (n, nu), (n, nx)]
    host = [np.zeros(sh) for sh in shapes]
    spock.spock_grad(P.handle, z, e, spock.SPOCK_FP64, *host)
    devo = [torch.zeros(sh, dtype=torch.float64, device=dev) for sh in shapes]
    spock.spock_grad_dev(P.handle, torch.tensor(z, device=dev), torch.tensor(e, device=dev), spock.SPOCK_FP64,
                         *devo)
    for h, g in zip(host, devo):
        assert np.array_equal(h, g.cpu().numpy())
    # a NULL output is skipped
    g_x0 = np.zeros(nx)
    spock.spock_grad(P.handle, z, e, spock.SPOCK_FP64, g_x0)
    assert np.array_equal(g_x0, host[0])


def test_cp_counts_of_L_match_between_cp_and_spock():
    """Vanilla CP applies L twice per iteration (the dual update and the
    residual); SPOCK reports the same per evaluation of T."""
    import torch
    from paper_2212_01110_gb300 import spock
    d = W.datacenter(N=3, nx=3)
    P = spock.Problem(d)
    dev = torch.device("cuda:0")
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
    z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
    e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
    info = spock.spock_solve_dev(P.handle, x0, spock.spock_default_settings(eps_abs=1e-5, eps_rel=1e-5), z, e, 0)
    assert info.status == spock.SPOCK_OK and info.n_L == 2 * info.n_T > 0


def test_fp64_fma_rate_is_plausible():
    """The measured FP64 FMA throughput (the ALU roofline of the FP64 path):
    positive and within the range of current GPUs (0.1 to 100 TFLOP/s)."""
    from paper_2212_01110_gb300 import spock
    v = spock.spock_fp64_fma_rate(2000)
    assert 0.1 < v < 100.0
    with pytest.raises(spock.SpockError):
        spock.spock_fp64_fma_rate(0)


def test_problem_clones_share_data_and_solve_alike():
    """spock_problem_clone: a clone solves exactly as its base; a batch of
    clones (one family, different x0) equals the batch of independent
    problems built from the same data; the base may be freed first."""
    import torch
    from paper_2212_01110_gb300 import spock
    dev = torch.device("cuda:0")
    d = W.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2)
    base = spock.Problem(d)
    clones = [base.clone() for _ in range(3)]
    rng = np.random.default_rng(9)
    x0s = [torch.tensor(np.clip(d["x0"] + 0.3 * rng.standard_normal(d["nx"]), -5, 5), dtype=torch.float64,
                        device=dev) for _ in range(3)]
    s = spock.spock_default_settings(max_iter=60, eps_abs=1e-14, eps_rel=1e-14)
    # a clone against its base, same x0
    z1, e1 = torch.zeros(base.n_z, dtype=torch.float64, device=dev), torch.zeros(base.n_eta, dtype=torch.float64,
                                                                                 device=dev)
    z2, e2 = torch.zeros_like(z1), torch.zeros_like(e1)
    spock.spock_solve_dev(base.handle, x0s[0], s, z1, e1, 0)
    spock.spock_solve_dev(clones[0].handle, x0s[0], s, z2, e2, 0)
    assert torch.equal(z1, z2) and torch.equal(e1, e2)
    # batch of clones vs batch of independent problems with the same data
    indep = [spock.Problem(d) for _ in range(3)]
    outs = []
    for probs in (clones, indep):
        b = spock.spock_batch_create([p.handle for p in probs])
        zs = [torch.zeros(base.n_z, dtype=torch.float64, device=dev) for _ in probs]
        es = [torch.zeros(base.n_eta, dtype=torch.float64, device=dev) for _ in probs]
        spock.spock_batch_solve_dev(b, x0s, s, zs, es, 0)
        spock.spock_free(b)
        outs.append([torch.cat([z, e]).cpu().numpy() for z, e in zip(zs, es)])
    for a, b_ in zip(*outs):
        assert np.array_equal(a, b_)
    # freeing the base first keeps the clones usable
    base.close()
    z3, e3 = torch.zeros_like(z1), torch.zeros_like(e1)
    spock.spock_solve_dev(clones[1].handle, x0s[0], s, z3, e3, 0)
    assert torch.equal(z3, z1)
    for c in clones:
        c.close()
