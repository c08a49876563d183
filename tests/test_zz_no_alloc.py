"""spock_prox_f_noalloc_dev: prox_{alpha f} for callers that cannot allocate
device memory while they run.  It must return what spock_prox_f_dev returns
(same tolerance as the other parity tests) on consecutive calls -- the fixed
scratch array keeps the previous call's contents -- and must reject problems
whose scratch does not fit the fixed array.  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def test_noalloc_matches_prox_f_on_consecutive_calls():
    import torch
    from paper_2212_01110_gb300 import build
    build.build()
    from paper_2212_01110_gb300 import spock, workloads
    dev = torch.device("cuda:0")
    for d in (workloads.small_binary(0), workloads.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2),
              workloads.large_tree(1, branching_stages=2, branch=3, N=5, nx=50, nu=20)):
        P = spock.Problem(d)
        x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
        alpha = 0.99 / P.norm_L
        rng = np.random.default_rng(11)
        for call in range(2):   # two calls in a row share the scratch array
            z = torch.tensor(3 * rng.standard_normal(P.n_z), dtype=torch.float64, device=dev)
            ref = torch.empty_like(z)
            out = torch.full_like(z, float("nan"))
            spock.spock_prox_f_dev(P.handle, x0, alpha, z, ref)
            spock.spock_prox_f_noalloc_dev(P.handle, x0, alpha, z, out)
            torch.cuda.synchronize()
            assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < RTOL, call
        P.close()


def test_noalloc_allocates_nothing():
    """On a fresh problem, after one warm-up call (which loads the kernels'
    code), further calls leave the device's free memory unchanged; only then
    is the result compared with spock_prox_f_dev."""
    import torch
    from paper_2212_01110_gb300 import build
    build.build()
    from paper_2212_01110_gb300 import spock, workloads
    dev = torch.device("cuda:0")
    d = workloads.large_tree(2, branching_stages=2, branch=3, N=5, nx=50, nu=20)
    P = spock.Problem(d)
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
    alpha = 0.99 / P.norm_L
    z = torch.tensor(np.random.default_rng(12).standard_normal(P.n_z), dtype=torch.float64, device=dev)
    out = torch.empty_like(z)
    ref = torch.empty_like(z)
    torch.cuda.synchronize()
    spock.spock_prox_f_noalloc_dev(P.handle, x0, alpha, z, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        spock.spock_prox_f_noalloc_dev(P.handle, x0, alpha, z, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    spock.spock_prox_f_dev(P.handle, x0, alpha, z, ref)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < RTOL
    P.close()


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    import torch
    from paper_2212_01110_gb300 import build
    build.build()
    from paper_2212_01110_gb300 import spock, workloads
    d = workloads.small_binary(0, N=10, nx=100, nu=28)   # 2047 nodes: about 1.08 M doubles of scratch
    P = spock.Problem(d)
    dev = torch.device("cuda:0")
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
    z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
    out = torch.zeros_like(z)
    with pytest.raises(spock.SpockError) as e:
        spock.spock_prox_f_noalloc_dev(P.handle, x0, 0.1, z, out)
    assert e.value.code == -1 and "too large" in str(e.value)
    P.close()
