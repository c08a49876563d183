"""Replica aggregation of bench.py on world size 2 (gloo, CPU): the job's
time is the slowest rank's and its work the sum over ranks; each rank draws
its own seeded instance."""
import os
import socket
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2212_01110_gb300 import workloads
        ms, units = bench.replica_reduce(10.0 * (rank + 1), 100 + rank, None)
        x0 = workloads.large_tree(seed=rank, branching_stages=1, branch=2, N=3, nx=3, nu=2)["x0"]
        q.put((rank, ms, units, x0.tolist()))
    finally:
        dist.destroy_process_group()


def test_replica_reduce_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, _ in res:
        assert ms == 20.0          # max over ranks
        assert units == 201.0      # sum over ranks
    assert not np.allclose(res[0][3], res[1][3])   # seed = rank: distinct instances


def test_replica_reduce_single_process():
    import bench
    assert bench.replica_reduce(3.5, 7, None) == (3.5, 7.0)


def test_cpu_baseline_leg_runs_on_the_host():
    """bench.py's CPU baseline (the oracle's C++ operator) on a small tree of
    the benchmark family: the fields the bench line reports."""
    import bench
    from paper_2212_01110_gb300 import workloads
    cores, model = bench.host_cpu()
    assert cores >= 1 and isinstance(model, str)
    d = workloads.large_tree(seed=0, branching_stages=1, branch=4, N=6, nx=5, nu=2)
    out = bench.cpu_baseline(d, seconds=0.2, threads=2)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] == 2
    assert out["one_thread"]["value"] > 0 and out["nproc"] == cores


def test_reference_arm_line():
    """bench.py --impl reference prints one JSON line with the contract's
    keys (the oracle's C++ operator on the host cores, on the benchmark's
    own tree); under a multi-rank launch only rank 0 prints."""
    import json
    import subprocess
    root = os.path.dirname(HERE)
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=root, capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    r1 = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                        cwd=root, capture_output=True, text=True, timeout=120,
                        env=dict(env, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1"))
    assert r1.returncode == 0 and not r1.stdout.strip()
