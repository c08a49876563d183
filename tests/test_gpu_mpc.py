"""Closed-loop MPC with warm starts (the paper's closed-loop simulation):
every solve converges, warm starts from the previous step's primal and dual
vectors take fewer iterations in total than cold starts, and the
trajectory obeys the state box."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_started_closed_loop():
    from paper_2212_01110_gb300 import mpc, spock, workloads
    d = workloads.datacenter(N=5, nx=6)
    warm = mpc.closed_loop(spock, d, steps=10, seed=3, tol=1e-3, warm=True)
    cold = mpc.closed_loop(spock, d, steps=10, seed=3, tol=1e-3, warm=False)
    assert all(r["status"] == spock.SPOCK_OK for r in warm + cold)
    it_w = sum(r["iterations"] for r in warm[1:])
    it_c = sum(r["iterations"] for r in cold[1:])
    print(f"closed loop, 9 steps after the first: warm {it_w} iterations, cold {it_c}")
    assert it_w < it_c
    # same realisations (same seed) and solutions within the tolerance: the
    # first inputs agree, the states stay in the box
    assert np.allclose(warm[0]["u0"], cold[0]["u0"], atol=1e-6)
    xs = np.array([r["x"] for r in warm])
    assert np.all(np.abs(xs) <= 1.0 + 1e-12)
