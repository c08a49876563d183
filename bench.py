"""Benchmark: SPOCK on the 62,805-node scenario tree on one GB300.

Workload: branching 4 for 6 stages then chains, N = 20, nx = 50, nu = 20
(4.62 M primal / 9.29 M dual variables), seeded synthetic data, inputs
resident in HBM.  One step = one SPOCK iteration (Algorithm 3: residual
r = v - T(v), termination test, Anderson update and direction, K0 or the
SuperMann line search with its extra T evaluations); K steps are timed as one
cold-start solve capped at K iterations.  value = CP operator evaluations per
second over the timed steps ("CP iters/s").  A separate cold-start solve,
capped by a time budget, reports the time to the 1e-6 residual.  The FP64
path is the headline (the problem is stated in double precision); the FP32
operator path (FP64 residual and Anderson least squares) is reported in the
same line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own seeded instance (replicas,
weak scaling, no collective on the data path); the timed region is bracketed
by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "time-to-1e-6 residual and CP iters/s (FP64 vs FP32/batched); % HBM peak"
WORKLOAD = dict(branching_stages=6, branch=4, N=20, nx=50, nu=20)


def measured_peaks():
    try:
        return json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# DRAM bytes (read + write) per chain node of one launch of the backward
# chain kernel (k_bwd_chain<double> / k_bwd_chain_tma<float>), from ncu
# captures on the 17,749-node tree (branching 4 for 6 stages, N = 9: 4,096
# chains of 3 nonleaf nodes, nx = 50, nu = 20), scaled by the chain nodes of
# the measured tree (each chain node's factors are read once).  Valid for the
# kernels as captured (None: not captured since the kernel last changed);
# remeasure after changing them.
NCU_TRAFFIC_PER_CHAIN_NODE = {"fp64": 594.511104e6 / (4096 * 3), "fp32": 296.087040e6 / (4096 * 3)}
NCU_CHAIN_SHAPE = (50, 20)   # nx, nu of the capture



def replica_reduce(ms, units, dev=None):
    """Whole-job figures of the replicas: the slowest rank's time and the
    units (CP evaluations) summed over ranks.  Identity at world size 1."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(prefix="spock_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def bytes_bwd_chain(d, n_chains, chain_len, elt):
    """Algorithmic bytes of one launch of the Riccati backward chain kernel:
    per chain node [Abar|B] (nx (nx+nu)), K, W^T (2 nu nx), Rt^-1 (nu^2),
    xbar and ubar reads (nx + nu), d write (nu); per chain the leaf's xbar
    (nx) and the q of its top node (nx)."""
    nx, nu = d["nx"], d["nu"]
    per_node = nx * (nx + nu) + 2 * nu * nx + nu * nu + nx + 2 * nu
    return elt * (n_chains * chain_len * per_node + n_chains * 2 * nx)


def flops_bwd_chain(d, n_chains, chain_len):
    nx, nu = d["nx"], d["nu"]
    return 2.0 * n_chains * chain_len * (nx * (nx + nu) + nu * nu + 2 * nu * nx)


def bytes_fwd_chain(d, n_chains, chain_len, elt):
    nx, nu = d["nx"], d["nu"]
    per_node = (nx + nu) * nx + nx * nu + nu + nx + nu   # Gf, K^T, d read, x and u writes
    return elt * (n_chains * chain_len * per_node + n_chains * nx)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2212_01110_gb300 import build
    build.build()
    from paper_2212_01110_gb300 import spock, workloads

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    t0 = time.time()
    wl = dict(WORKLOAD, branching_stages=args.branching_stages, N=args.horizon)
    d = workloads.large_tree(seed=rank, **wl)
    gen_s = time.time() - t0
    P = spock.Problem(d)
    n = len(d["anc"])
    nl = n - int(np.sum(np.bincount(d["anc"][1:], minlength=n) == 0))
    n_chains, chain_len = 4 ** wl["branching_stages"], wl["N"] - wl["branching_stages"]
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
    z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
    e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # the FP64 ALU roofline, measured here (spock_fp64_fma_rate: the best of
    # 8 / 16 independent FMA chains per thread and 4 / 8 blocks per SM)
    fp64_peak = max(spock.spock_fp64_fma_rate(20000) for _ in range(2))

    def settings(prec, profile, max_iter):
        return spock.spock_default_settings(precision=prec, memory=args.memory, max_iter=max_iter,
                                            profile=int(profile))

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(prec):
        infos = []
        spock.spock_solve_dev(P.handle, x0, settings(prec, False, args.warmup), z, e, 0)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local_rank) as clk:
            ev0.record(st)
            infos.append(spock.spock_solve_dev(P.handle, x0, settings(prec, True, args.steps), z, e, 0))
            ev1.record(st)
            torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        nT = sum(i.n_T for i in infos)
        ms, nT_all = replica_reduce(ev0.elapsed_time(ev1), nT, dev)
        return ms, nT, nT_all, infos, clk.summary()

    def traffic(prec):
        per = NCU_TRAFFIC_PER_CHAIN_NODE["fp64" if prec == spock.SPOCK_FP64 else "fp32"]
        if per is None or (d["nx"], d["nu"]) != NCU_CHAIN_SHAPE:
            return None
        return round(per * n_chains * chain_len)

    def roofline(infos, prec):
        elt = 8 if prec == spock.SPOCK_FP64 else 4
        timed_T = sum(i.n_timed for i in infos)
        t_bwd = sum(i.t_group_ms[1] for i in infos) / max(timed_T, 1)
        t_fwd = sum(i.t_group_ms[4] for i in infos) / max(timed_T, 1)
        bb = bytes_bwd_chain(d, n_chains, chain_len, elt)
        fl = flops_bwd_chain(d, n_chains, chain_len)
        groups = {g: sum(i.t_group_ms[k] for i in infos) / max(timed_T, 1)
                  for k, g in enumerate(spock.Info.GROUPS)}
        if prec == spock.SPOCK_FP64:
            ach = fl / (t_bwd * 1e-3) / 1e12
            r = {"kernel": "k_bwd_chain<double>", "bound": "alu", "achieved": round(ach, 4),
                 "peak": round(fp64_peak, 4), "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4),
                 "peak_source": "measured in this run by spock_fp64_fma_rate (FP64 FMA throughput kernels, "
                                "best over 8 / 16 chains per thread and 4 / 8 blocks per SM, best of 2 calls)",
                 "traffic": traffic(prec), "algorithmic_bytes": bb, "algorithmic_flops": fl,
                 "hbm_achieved_gbs": round(bb / (t_bwd * 1e-3) / 1e9, 1),
                 "hbm_frac_of_measured": round(bb / (t_bwd * 1e-3) / 1e9 / hbm, 4),
                 "avg_launch_ms": round(t_bwd, 4)}
        else:
            ach = bb / (t_bwd * 1e-3) / 1e9
            r = {"kernel": "k_bwd_chain<float>", "bound": "hbm", "achieved": round(ach, 1), "peak": hbm,
                 "unit": "GB/s", "frac": round(ach / hbm, 4), "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                 "traffic": traffic(prec), "algorithmic_bytes": bb, "avg_launch_ms": round(t_bwd, 4)}
        fb = bytes_fwd_chain(d, n_chains, chain_len, elt)
        r["fwd_chain"] = {"avg_launch_ms": round(t_fwd, 4), "algorithmic_bytes": fb,
                          "achieved_gbs": round(fb / (t_fwd * 1e-3) / 1e9, 1) if t_fwd > 0 else None}
        r["per_T_group_ms"] = {k: round(v, 4) for k, v in groups.items()}
        return r

    def time_to_tol(prec, ms_per_iter):
        """Cold-start solve to xi <= 1e-6, capped by the time budget."""
        cap = max(10, int(args.tol_budget_s * 1e3 / max(ms_per_iter, 1e-3)))
        inf = spock.spock_solve_dev(P.handle, x0, settings(prec, False, cap), z, e, 0)
        return {"seconds": round(inf.solve_ms * 1e-3, 3), "iterations": inf.iterations, "n_T": inf.n_T,
                "xi": inf.xi, "xi0": inf.xi0, "tol": max(1e-6, 1e-6 * inf.xi0),
                "status": "converged" if inf.status == 0 else f"not reached within the {args.tol_budget_s:.0f} s cap",
                "K0_K1_K2": [inf.n_K0, inf.n_K1, inf.n_K2]}

    out = {}
    precs = [spock.SPOCK_FP64, spock.SPOCK_FP32] if args.precision == "both" else \
        [spock.SPOCK_FP64 if args.precision == "fp64" else spock.SPOCK_FP32]
    for prec in precs:
        ms, nT, nT_all, infos, clk = timed(prec)
        i0 = infos[0]
        out[prec] = dict(
            value=nT_all / (ms * 1e-3), ms_per_step=ms / max(i0.iterations, 1), n_T=nT, infos=infos, clocks=clk,
            iterations=i0.iterations, n_T_steps=i0.n_T, branches=[i0.n_K0, i0.n_K1, i0.n_K2, i0.n_cap],
            gpu_launches=sum(i.n_launches for i in infos), roofline=roofline(infos, prec))
        if args.tol_budget_s > 0:
            out[prec]["time_to_tol"] = time_to_tol(prec, out[prec]["ms_per_step"])

    # end to end through the host-buffer entry point (pinned host memory)
    head = precs[0]
    zh = torch.zeros(P.n_z, dtype=torch.float64).pin_memory().numpy()
    eh = torch.zeros(P.n_eta, dtype=torch.float64).pin_memory().numpy()
    x0h = torch.tensor(d["x0"], dtype=torch.float64).pin_memory().numpy()
    spock.spock_solve(P.handle, x0h, settings(head, False, args.warmup), zh, eh, 0)
    barrier()
    t0 = time.perf_counter()
    inf = spock.spock_solve(P.handle, x0h, settings(head, False, args.steps), zh, eh, 0)
    nT_e2e = inf.n_T
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s, nT_e2e = replica_reduce(e2e_s, nT_e2e, dev)
    e2e = {"value": nT_e2e / e2e_s, "unit": "CP iters/s", "h2d_bytes_per_step": 8 * P.nx / args.steps,
           "d2h_bytes_per_step": 8 * (P.n_z + P.n_eta) / args.steps, "ms_per_step": 1e3 * e2e_s / args.steps,
           "api": "spock_solve: host buffers (pinned), x0 copied in and (z, eta) copied out inside the timed "
                  "call, K iterations from a cold start"}

    def section(name, fn):
        t_s = time.time()
        res = fn()
        print(f"[bench] {name}: {time.time() - t_s:.1f} s", file=sys.stderr, flush=True)
        return res

    paper = section("paper workload", lambda: paper_workload(args, spock, workloads, dev)) \
        if (rank == 0 and args.paper_workload) else None
    mpc_res = section("closed loop", lambda: closed_loop_workload(args, spock, workloads, dev)) \
        if (rank == 0 and args.mpc_realisations > 0) else None
    small = section("small tree", lambda: small_workload(args, spock, workloads, dev)) if rank == 0 else None
    batch = section("batch", lambda: batch_workload(args, spock, workloads, dev, seed=rank)) if args.batch > 0 else None
    family = section("family batch", lambda: family_workload(args, spock, workloads, dev, seed=rank)) \
        if args.families > 0 else None
    grad = section("gradient", lambda: grad_workload(args, spock, workloads, dev)) \
        if (rank == 0 and args.grad_instances > 0) else None
    general = section("general form", lambda: general_workload(args, spock, workloads, dev)) \
        if (rank == 0 and args.general) else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = section("cpu baseline", lambda: cpu_baseline(d, seconds=args.cpu_seconds))

    if rank == 0:
        h = out[head]
        line = {
            "metric": METRIC, "value": round(h["value"], 2), "unit": "CP iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(h["ms_per_step"], 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head == spock.SPOCK_FP64 else "f32", "data": "synthetic (seeded, rank = seed)",
            "config": {"workload": f"large scenario tree: branching 4 for {wl['branching_stages']} stages then 1, "
                                   f"N={wl['N']} ({n:,} nodes, {n_chains:,} scenarios), nx=50, nu=20, AV@R a~U(0.1,0.9), "
                                   "box |x|<=5 |u|<=1",
                       "n_z": P.n_z, "n_eta": P.n_eta, "nodes": n, "nonleaf": nl,
                       "step": "one SPOCK iteration (Anderson m=%d), K steps = one cold-start solve capped "
                               "at K iterations" % args.memory,
                       "l2": "inputs larger than L2 (chain factors %.2f GB FP64 / %.2f GB FP32 per T)" % (
                           (bytes_bwd_chain(d, n_chains, wl["N"] - wl["branching_stages"], 8)
                            + bytes_fwd_chain(d, n_chains, wl["N"] - wl["branching_stages"], 8)) / 1e9,
                           (bytes_bwd_chain(d, n_chains, wl["N"] - wl["branching_stages"], 4)
                            + bytes_fwd_chain(d, n_chains, wl["N"] - wl["branching_stages"], 4)) / 1e9),
                       "parallelism": f"replicas x{world}"},
            "time_to_tol": h.get("time_to_tol"), "iterations": h["iterations"], "n_T_steps": h["n_T_steps"],
            "branches_K0_K1_K2_cap": h["branches"], "roofline": h["roofline"], "clocks": h["clocks"], "gpu_launches": h["gpu_launches"], "e2e": e2e,
            "setup": {"instance_generation_s": round(gen_s, 2), "factor_seconds_alg1_fp64_host": round(P.factor_seconds, 3)},
        }
        for prec, nm in ((spock.SPOCK_FP32, "fp32"), (spock.SPOCK_FP64, "fp64")):
            if prec in out and prec != head:
                o = out[prec]
                tt, tf = o.get("time_to_tol"), out.get(spock.SPOCK_FP64, {}).get("time_to_tol")
                line[nm] = {"value": round(o["value"], 2), "unit": "CP iters/s",
                            "ms_per_step": round(o["ms_per_step"], 3), "time_to_tol": tt,
                            "iterations": o["iterations"], "n_T_steps": o["n_T_steps"],
                            "branches_K0_K1_K2_cap": o["branches"], "roofline": o["roofline"],
                            "clocks": o["clocks"], "gpu_launches": o["gpu_launches"],
                            "speedup_vs_fp64_per_step": round(out[spock.SPOCK_FP64]["ms_per_step"] / o["ms_per_step"], 3)
                            if spock.SPOCK_FP64 in out else None,
                            "speedup_vs_fp64_time_to_tol": round(tf["seconds"] / tt["seconds"], 3)
                            if (tt and tf and tt["status"] == "converged" and tf["status"] == "converged") else None}
        if paper:
            line["paper_workload"] = paper
        if small:
            line["small_tree"] = small
        if mpc_res:
            line["closed_loop_mpc"] = mpc_res
        if batch:
            line["batch"] = batch
        if family:
            line["family_batch"] = family
        if grad:
            line["gradient"] = grad
        if general:
            line["general_form"] = general
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)


def small_workload(args, spock, workloads, dev):
    """The 15-node binary tree (N = 3, nx = 3, nu = 2): time to the
    1e-6 residual in FP64 (Anderson m = 3; the captured graph reused, so
    the second solve is timed), and the FP32 iteration with FP64 factors,
    residual, Anderson m = 5 and FP64 certification/tail: its optimal cost
    and trajectory against a tight FP64 solve (1e-11) of the same problem."""
    import torch
    d = workloads.small_binary(0)
    P = spock.Problem(d)
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)

    def solve(prec, mem, tol):
        z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
        e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
        st = spock.spock_default_settings(precision=prec, memory=mem, eps_abs=tol, eps_rel=tol, max_iter=100000)
        inf = spock.spock_solve_dev(P.handle, x0, st, z, e, 0)
        return z, inf

    solve(spock.SPOCK_FP64, 3, 1e-6)
    _, inf = solve(spock.SPOCK_FP64, 3, 1e-6)
    out = {"nodes": len(d["anc"]), "n_z": P.n_z, "n_eta": P.n_eta,
           "fp64_to_1e-6": {"ms": round(inf.solve_ms, 3), "iterations": inf.iterations, "n_T": inf.n_T,
                            "T_per_s": round(inf.n_T / (inf.solve_ms * 1e-3), 1),
                            "status": "converged" if inf.status == 0 else "max_iter"}}
    zr, _ = solve(spock.SPOCK_FP64, 5, 1e-11)
    solve(spock.SPOCK_FP32, 5, 1e-6)
    z32, inf32 = solve(spock.SPOCK_FP32, 5, 1e-6)
    n, nx, nu = len(d["anc"]), d["nx"], d["nu"]
    nl = n - int(np.sum(np.bincount(d["anc"][1:], minlength=n) == 0))
    a, b = z32.cpu().numpy(), zr.cpu().numpy()
    xs = slice(1, 1 + n * nx)
    us = slice(1 + n * nx, 1 + n * nx + nl * nu)
    out["fp32_fp64tail_m5"] = {
        "ms": round(inf32.solve_ms, 3), "iterations": inf32.iterations, "fp64_iterations": inf32.fp64_iterations,
        "certified": bool(inf32.certified), "xi": inf32.xi,
        "cost_abs_err": abs(a[0] - b[0]), "cost_rel_err": abs(a[0] - b[0]) / max(abs(b[0]), 1e-300),
        "x_max_err": float(np.max(np.abs(a[xs] - b[xs]))), "u_max_err": float(np.max(np.abs(a[us] - b[us]))),
        "reference": "FP64 solve of the same problem to 1e-11 (the FP64 path is parity-tested against the oracle)"}
    P.close()
    return out


def paper_workload(args, spock, workloads, dev):
    """Time to tolerance on the paper's own system (data-center thermal model
    of Eq. (dynamics-example): d = 2 disturbances, full binary tree,
    nx = nu = 50, x0 = 0.1): horizon 15 at tolerance 1e-3 (the largest case
    of Fig. 2, where the paper reports 151.5 s for its sequential CPU solver,
    hardware not stated -- context only), and horizon 12 at 1e-6 in FP64 and
    in FP32 with FP64 certification/tail.  Cold starts, Anderson memory m."""
    import torch
    out = {"fig1": fig1_comparison(args, spock, workloads, dev), "table1": table1_iterations(args, spock, workloads, dev)}
    for N, tol, key in ((15, 1e-3, "fig2_N15_tol1e-3"), (12, 1e-6, "N12_tol1e-6")):
        d = workloads.datacenter(N=N, nx=50)
        P = spock.Problem(d)
        x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
        z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
        e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
        res = {"nodes": len(d["anc"]), "n_z": P.n_z, "n_eta": P.n_eta, "tol": tol}
        for prec, nm in ((spock.SPOCK_FP64, "fp64"), (spock.SPOCK_FP32, "fp32_fp64tail")):
            st = spock.spock_default_settings(precision=prec, eps_abs=tol, eps_rel=tol, memory=args.memory,
                                              max_iter=args.paper_max_iter)
            inf = spock.spock_solve_dev(P.handle, x0, st, z, e, 0)
            res[nm] = {"seconds": round(inf.solve_ms * 1e-3, 3), "iterations": inf.iterations, "n_T": inf.n_T,
                       "xi": inf.xi, "status": "converged" if inf.status == 0 else "max_iter",
                       "fp64_iterations": inf.fp64_iterations}
        a, b = res["fp64"], res["fp32_fp64tail"]
        if a["status"] == "converged" and b["status"] == "converged":
            res["speedup_fp32_vs_fp64"] = round(a["seconds"] / b["seconds"], 3)
        if N == 15:
            res["paper_context"] = {"seconds": 151.5, "iterations": 105, "solver": "sequential Julia, CPU, hardware "
                                    "not stated; SuperMann parameters not printed (Fig. 2, Table 1)"}
        out[key] = res
        P.close()
        del P, z, e
        torch.cuda.empty_cache()
    return out


def fig1_comparison(args, spock, workloads, dev):
    """Fig. 1 of the paper: the data-center system with N = 7, nx = nu = 5,
    x0 = 0.1, tolerances 1e-5: applications of L until termination for
    vanilla CP and for SPOCK (Anderson m = 3).  Vanilla CP runs as
    spock_cp_step_dev calls of 10 iterations, its residual read after each
    call (so its count is exact to 10 iterations)."""
    import torch
    d = workloads.datacenter(N=7, nx=5)
    P = spock.Problem(d)
    x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
    z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
    e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
    tol = 1e-5
    st = spock.spock_default_settings(eps_abs=tol, eps_rel=tol, memory=3)
    inf = spock.spock_solve_dev(P.handle, x0, st, z, e, 0)
    out = {"nodes": len(d["anc"]), "tol": tol,
           "spock": {"iterations": inf.iterations, "n_T": inf.n_T, "n_L": inf.n_L,
                     "status": "converged" if inf.status == 0 else "max_iter",
                     "K0_K1_K2": [inf.n_K0, inf.n_K1, inf.n_K2]}}
    z.zero_()
    e.zero_()
    xi0 = spock.spock_cp_step_dev(P.handle, x0, 1, 0.0, spock.SPOCK_FP64, z, e)
    target = max(tol, tol * xi0)
    k, xi = 1, xi0
    while xi > target and k < 200000:
        xi = spock.spock_cp_step_dev(P.handle, x0, 10, 0.0, spock.SPOCK_FP64, z, e)
        k += 10
    out["vanilla_cp"] = {"iterations": k, "n_L": 2 * k, "xi": xi,
                         "status": "converged" if xi <= target else "max_iter"}
    out["ratio_L_calls"] = round(out["vanilla_cp"]["n_L"] / max(inf.n_L, 1), 2)
    out["paper"] = {"spock_L_calls": 571, "cp_L_calls": 3159, "ratio": round(3159 / 571, 2),
                    "note": "the paper does not say how it counts calls of L; here two per evaluation of T (L z "
                            "and L z+), for both methods"}
    P.close()
    return out


def table1_iterations(args, spock, workloads, dev):
    """Table 1 of the paper: SPOCK iterations to tolerance 1e-3 on the
    data-center system with nx = nu = 50, x0 = 0.1, horizons 3..15 (FP64,
    Anderson m = 3, cold starts)."""
    import torch
    rows = {}
    for N in (3, 6, 9, 12, 15):
        d = workloads.datacenter(N=N, nx=50)
        P = spock.Problem(d)
        x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
        z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
        e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
        st = spock.spock_default_settings(eps_abs=1e-3, eps_rel=1e-3, memory=3, max_iter=args.paper_max_iter)
        inf = spock.spock_solve_dev(P.handle, x0, st, z, e, 0)
        rows[str(N)] = {"nodes": len(d["anc"]), "iterations": inf.iterations, "n_T": inf.n_T,
                        "seconds": round(inf.solve_ms * 1e-3, 4),
                        "status": "converged" if inf.status == 0 else "max_iter"}
        P.close()
        del P, z, e
        torch.cuda.empty_cache()
    return {"rows": rows, "paper_iterations": {"3": 105, "6": 128, "9": 110, "12": 109, "15": 105}}


def closed_loop_workload(args, spock, workloads, dev):
    """The paper's closed-loop simulation: data-center system, N = 10,
    nx = nu = 20 (2,047 nodes), tolerance 1e-3, 20 MPC steps from
    x0 = 0.1, each solve warm-started from the previous step's primal and
    dual vectors; args.mpc_realisations random disturbance sequences (the
    paper uses 15).  Per step: mean device time and iterations over the
    realisations, warm and cold."""
    from paper_2212_01110_gb300 import mpc
    d = workloads.datacenter(N=10, nx=20)
    res = {}
    for mode in ("warm", "cold"):
        runs = [mpc.closed_loop(spock, d, steps=20, seed=s, tol=1e-3, warm=(mode == "warm"), device=dev)
                for s in range(args.mpc_realisations)]
        ms = np.array([[r["ms"] for r in run] for run in runs])
        it = np.array([[r["iterations"] for r in run] for run in runs])
        res[mode] = {"mean_ms_per_step": [round(float(v), 3) for v in ms.mean(axis=0)],
                     "mean_iterations_per_step": [round(float(v), 1) for v in it.mean(axis=0)],
                     "converged": int(sum(r["status"] == 0 for run in runs for r in run)),
                     "solves": int(ms.size)}
    w, c = res["warm"], res["cold"]
    res.update({"nodes": len(d["anc"]), "realisations": args.mpc_realisations, "steps": 20, "tol": 1e-3,
                "mean_ms_steps_2_20": {"warm": round(float(np.mean(w["mean_ms_per_step"][1:])), 3),
                                       "cold": round(float(np.mean(c["mean_ms_per_step"][1:])), 3)}})
    return res


def batch_workload(args, spock, workloads, dev, seed=0):
    """Batched SPOCK: args.batch heterogeneous instances (branching 2-4,
    N 5-15, nx 10-30, nu 4-10, scenario cap 64; data as the large tree with
    uniform child probabilities) in
    one spock_batch_solve_dev call -- every kernel of a round launched once
    for the whole batch, rounds replayed from a CUDA graph.  A warm-up solve
    (autotuning, capture) is excluded; the timed solve runs args.batch_iter
    SPOCK iterations per instance from a cold start, FP32 (FP64
    residual/Anderson) and FP64; then every instance from a cold start to the
    1e-6 residual (time for all to reach it)."""
    import torch
    t0 = time.time()
    ds = workloads.batch_instances(seed=seed, count=args.batch)
    probs = [spock.Problem(d) for d in ds]
    setup = time.time() - t0
    b = spock.spock_batch_create([p.handle for p in probs])
    x0s = [torch.tensor(d["x0"], dtype=torch.float64, device=dev) for d in ds]
    zs = [torch.zeros(p.n_z, dtype=torch.float64, device=dev) for p in probs]
    es = [torch.zeros(p.n_eta, dtype=torch.float64, device=dev) for p in probs]
    out = {"instances": len(ds), "nodes_total": int(sum(len(d["anc"]) for d in ds)),
           "variables_total": int(sum(p.n_z + p.n_eta for p in probs)), "setup_s": round(setup, 1),
           "iterations_per_instance": args.batch_iter}
    for prec, nm in ((spock.SPOCK_FP32, "fp32"), (spock.SPOCK_FP64, "fp64")):
        st = spock.spock_default_settings(precision=prec, max_iter=args.batch_iter, memory=args.memory, fp64_tail=0)
        spock.spock_batch_solve_dev(b, x0s, st, zs, es, 0)   # warm-up: autotune + capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = spock.spock_batch_solve_dev(b, x0s, st, zs, es, 0)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        nT = sum(i.n_T for i in infos)
        out[nm] = {"value": round(nT / infos[0].solve_ms * 1e3, 1), "unit": "instance CP iters/s",
                   "device_ms": round(infos[0].solve_ms, 2), "wall_ms": round(wall * 1e3, 2), "n_T_total": nT,
                   "converged": sum(1 for i in infos if i.status == 0),
                   "median_xi": float(np.median([i.xi for i in infos])),
                   "mode": "persistent (one launch, one block per instance)" if infos[0].n_launches == 1
                           else "work-list kernels, %d launches" % infos[0].n_launches}
        if args.batch_tol_iter > 0 and prec == spock.SPOCK_FP32:
            # every instance from a cold start to xi <= 1e-6 (iteration cap per
            # instance); the batched form is the FP32 one
            st = spock.spock_default_settings(precision=prec, max_iter=args.batch_tol_iter, memory=args.memory,
                                              fp64_tail=0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            infos = spock.spock_batch_solve_dev(b, x0s, st, zs, es, 0)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            its = [i.iterations for i in infos]
            out[nm]["to_tol_1e-6"] = {
                "device_ms": round(infos[0].solve_ms, 2), "wall_ms": round(wall * 1e3, 2),
                "converged": sum(1 for i in infos if i.status == 0), "instances": len(infos),
                "iterations_median_max": [int(np.median(its)), int(max(its))],
                "n_T_total": int(sum(i.n_T for i in infos)), "max_iter": args.batch_tol_iter,
                "xi_over_tol_max": float(max(i.xi / max(1e-6, 1e-6 * i.xi0) for i in infos))}
    spock.spock_free(b)
    for p in probs:
        p.close()
    torch.cuda.empty_cache()
    return out


def family_workload(args, spock, workloads, dev, seed=0):
    """Batched family form: 64 families of 8 instances that share tree and
    data and differ in x0 (the members are spock_problem_clone's of the
    family's problem, so a launch reads a family's factors from HBM once and
    from L2 for the other members).  Families drawn as the batched workload;
    x0 ~ N(0, 1) per member.  Same measurement as the independent batch:
    args.batch_iter SPOCK iterations per instance from a cold start."""
    import torch
    ds = workloads.batch_instances(seed=seed + 17, count=args.families)
    rng = np.random.default_rng(seed + 5)
    bases = [spock.Problem(d) for d in ds]
    members, x0s = [], []
    for P, d in zip(bases, ds):
        fam = [P] + [P.clone() for _ in range(args.family_size - 1)]
        for m in fam:
            members.append(m)
            x0s.append(torch.tensor(np.clip(rng.standard_normal(d["nx"]), -5, 5), dtype=torch.float64, device=dev))
    b = spock.spock_batch_create([m.handle for m in members])
    zs = [torch.zeros(m.n_z, dtype=torch.float64, device=dev) for m in members]
    es = [torch.zeros(m.n_eta, dtype=torch.float64, device=dev) for m in members]
    out = {"families": len(bases), "members": args.family_size, "instances": len(members),
           "nodes_total": int(sum(len(d["anc"]) for d in ds)) * args.family_size,
           "iterations_per_instance": args.batch_iter}
    for prec, nm in ((spock.SPOCK_FP32, "fp32"), (spock.SPOCK_FP64, "fp64")):
        st = spock.spock_default_settings(precision=prec, max_iter=args.batch_iter, memory=args.memory, fp64_tail=0)
        spock.spock_batch_solve_dev(b, x0s, st, zs, es, 0)   # warm-up: autotune + capture
        torch.cuda.synchronize()
        infos = spock.spock_batch_solve_dev(b, x0s, st, zs, es, 0)
        torch.cuda.synchronize()
        nT = sum(i.n_T for i in infos)
        out[nm] = {"value": round(nT / infos[0].solve_ms * 1e3, 1), "unit": "instance CP iters/s",
                   "device_ms": round(infos[0].solve_ms, 2), "n_T_total": nT}
    spock.spock_free(b)
    for m in members:
        m.close()
    torch.cuda.empty_cache()
    return out


def grad_workload(args, spock, workloads, dev):
    """Gradients of the optimal cost on 64 instances of the tree with
    branching 3 for 4 stages, N = 10 (607 nodes), nx = 20, nu = 8, data as
    the large tree with uniform child probabilities and dynamics of spectral
    radius 0.5 (the workload states neither; with 0.95 the method does not
    reach 1e-6 on this tree within 20,000 iterations).  One batched FP64
    solve (tolerance 1e-6, at most args.grad_iter iterations per instance),
    then per instance the envelope gradient (spock_grad_dev, FP64 and FP32),
    timed with CUDA events against the solve time per instance, and the
    adjoint of the CP fixed point (spock_adjoint_dev, FP64) at instance 0's
    solution to the solve's tolerance.  Finite-difference check on instance
    0: central differences with h = 1e-6 along random directions of x0,
    diag Q, diag R, A and B, from solves to xi <= 1e-12 (perturbed solves
    warm-started from the base solution), against both gradients (adjoint
    solved to 1e-11 there)."""
    import torch
    cnt = args.grad_instances
    ds = [workloads.large_tree(seed=s, branching_stages=4, branch=3, N=10, nx=20, nu=8, probs="uniform", rho=0.5)
          for s in range(cnt)]
    probs = [spock.Problem(d) for d in ds]
    b = spock.spock_batch_create([p.handle for p in probs])
    x0s = [torch.tensor(d["x0"], dtype=torch.float64, device=dev) for d in ds]
    zs = [torch.zeros(p.n_z, dtype=torch.float64, device=dev) for p in probs]
    es = [torch.zeros(p.n_eta, dtype=torch.float64, device=dev) for p in probs]
    warm = spock.spock_default_settings(precision=spock.SPOCK_FP64, memory=5, max_iter=50)
    spock.spock_batch_solve_dev(b, x0s, warm, zs, es, 0)
    for z, e in zip(zs, es):
        z.zero_()
        e.zero_()
    st = spock.spock_default_settings(precision=spock.SPOCK_FP64, memory=5, max_iter=args.grad_iter)
    torch.cuda.synchronize()
    infos = spock.spock_batch_solve_dev(b, x0s, st, zs, es, 0)
    torch.cuda.synchronize()
    batch_ms = infos[0].solve_ms
    its = [i.iterations for i in infos]
    out = {"instances": cnt, "nodes": len(ds[0]["anc"]), "n_z": probs[0].n_z, "n_eta": probs[0].n_eta,
           "dynamics": "A = 0.5 x Haar-orthogonal, B ~ N(0, 1/nx), uniform child probabilities",
           "solve": {"tol": 1e-6, "max_iter": args.grad_iter, "batch_ms": round(batch_ms, 2),
                     "ms_per_instance": round(batch_ms / cnt, 3),
                     "converged": sum(1 for i in infos if i.status == 0),
                     "iterations_median_max": [int(np.median(its)), int(max(its))],
                     "median_xi": float(np.median([i.xi for i in infos])),
                     "mode": "persistent (one launch, one block per instance)" if infos[0].n_launches == 1
                             else "work-list kernels, %d launches" % infos[0].n_launches}}
    n, nx, nu = len(ds[0]["anc"]), ds[0]["nx"], ds[0]["nu"]

    def grads():
        return [torch.zeros(nx, dtype=torch.float64, device=dev),
                torch.zeros(n, nx, nx, dtype=torch.float64, device=dev),
                torch.zeros(n, nx, nu, dtype=torch.float64, device=dev),
                torch.zeros(n, nx, dtype=torch.float64, device=dev),
                torch.zeros(n, nu, dtype=torch.float64, device=dev),
                torch.zeros(n, nx, dtype=torch.float64, device=dev)]

    g = grads()
    cur = torch.cuda.current_stream()
    per_inst = batch_ms / cnt
    for prec, nm in ((spock.SPOCK_FP64, "fp64"), (spock.SPOCK_FP32, "fp32")):
        for i in range(min(3, cnt)):   # warm-up
            spock.spock_grad_dev(probs[i].handle, zs[i], es[i], prec, *g)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(cur)
        for i in range(cnt):
            spock.spock_grad_dev(probs[i].handle, zs[i], es[i], prec, *g)
        ev1.record(cur)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / cnt
        out[f"grad_ms_{nm}"] = round(ms, 4)
        out[f"grad_over_solve_{nm}"] = round(ms / per_inst, 5)
    # adjoint of the fixed point (phi = s^0) at the first instance's solution,
    # to the solve's own tolerance
    ga = grads()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, it, res = spock.spock_adjoint_dev(probs[0].handle, zs[0], es[0], None, 10000, 1e-6, *ga)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    out["adjoint_fp64"] = {"instance": 0, "ms": round(ms, 3), "applications_of_JT": it, "tol": 1e-6,
                           "residual": res, "over_solve": round(ms / per_inst, 4)}
    spock.spock_free(b)
    for p in probs:
        p.close()
    # finite-difference checks on instance 0 of the workload (solves to 1e-12)
    d = ds[0]
    P = spock.Problem(d)
    tight = spock.spock_default_settings(precision=spock.SPOCK_FP64, eps_abs=1e-12, eps_rel=1e-12, memory=5,
                                         max_iter=args.grad_fd_iter)

    def solve(PP, x0, start=None):
        """Solve to 1e-12; perturbed problems start from the base solution."""
        z = torch.zeros(PP.n_z, dtype=torch.float64, device=dev)
        e = torch.zeros(PP.n_eta, dtype=torch.float64, device=dev)
        if start is not None:
            z.copy_(start[0])
            e.copy_(start[1])
        inf = spock.spock_solve_dev(PP.handle, torch.tensor(x0, dtype=torch.float64, device=dev), tight, z, e,
                                    0 if start is None else 1)
        return z, e, inf

    tight_base = tight
    tight = spock.spock_default_settings(precision=spock.SPOCK_FP64, eps_abs=1e-12, eps_rel=1e-12, memory=5,
                                         max_iter=args.grad_base_iter)
    t_fd = time.perf_counter()
    z, e, inf0 = solve(P, d["x0"])
    tight = tight_base
    base = (z.clone(), e.clone())
    t_base = time.perf_counter() - t_fd
    print(f"[bench]   gradient: base solve to 1e-12 {t_base:.1f} s, "
          f"{inf0.iterations} iterations", file=sys.stderr, flush=True)
    ge = grads()
    spock.spock_grad_dev(P.handle, z, e, spock.SPOCK_FP64, *ge)
    ga = grads()
    torch.cuda.synchronize()
    t_adj = time.perf_counter()
    rc, ait, ares = spock.spock_adjoint_dev(P.handle, z, e, None, 100000, 1e-11, *ga)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t_adj
    ge = [t.cpu().numpy() for t in ge]
    ga = [t.cpu().numpy() for t in ga]
    out["adjoint_vs_envelope"] = {"max_rel_diff": max(float(np.max(np.abs(a - b_)) / max(np.max(np.abs(b_)), 1e-300))
                                                      for a, b_ in zip(ga, ge)),
                                  "adjoint_applications_of_JT": ait, "adjoint_residual": ares,
                                  "adjoint_s": round(t_adj, 2), "base_solve_s": round(t_base, 1)}
    rng = np.random.default_rng(7)
    h = 1e-6
    checks = {}
    conv = [inf0.status == 0]
    dirv = rng.standard_normal(nx)
    dirv /= np.linalg.norm(dirv)
    zp_, _, infp = solve(P, d["x0"] + h * dirv, base)
    zm_, _, infm = solve(P, d["x0"] - h * dirv, base)
    conv += [infp.status == 0, infm.status == 0]
    fd_its = [infp.iterations, infm.iterations]
    fd_xi = [infp.xi, infm.xi]
    checks["x0"] = ((float(zp_[0].item()) - float(zm_[0].item())) / (2 * h), float(ge[0] @ dirv),
                    float(ga[0] @ dirv))
    P.close()
    # data directions: Q, R relative per entry; A, B absolute; all nonroot nodes
    for key, gi, rel in (("Q", 3, True), ("R", 4, True), ("A", 1, False), ("B", 2, False)):
        dq = rng.standard_normal(d[key].shape)
        dq[0] = 0.0
        scale = d[key] if rel else 1.0
        an_e = float(np.sum(ge[gi] * dq * scale))
        an_a = float(np.sum(ga[gi] * dq * scale))
        vals = []
        for sgn in (1.0, -1.0):
            dd = dict(d)
            dd[key] = d[key] + sgn * h * dq * scale
            PP = spock.Problem(dd)
            zz, _, inf_ = solve(PP, d["x0"], base)
            vals.append(float(zz[0].item()))
            conv.append(inf_.status == 0)
            fd_its.append(inf_.iterations)
            fd_xi.append(inf_.xi)
            PP.close()
        checks[key] = ((vals[0] - vals[1]) / (2 * h), an_e, an_a)
    out["fd_check"] = {
        "tree": "instance 0 of the workload (607 nodes)", "h": h, "solve_tol": 1e-12,
        "directions": "x0: unit N(0, 1); Q, R: X <- X (1 + h dX); A, B: X <- X + h dX; dX ~ N(0, 1) per entry",
        "converged": all(conv), "base_iterations": inf0.iterations, "base_xi": inf0.xi,
        "perturbed_solve_iterations": fd_its, "perturbed_xi_max": max(fd_xi),
        **{k: {"central_fd": fd, "envelope": ae, "adjoint": aa,
               "rel_err_envelope": abs(ae - fd) / max(abs(fd), 1e-12),
               "rel_err_adjoint": abs(aa - fd) / max(abs(fd), 1e-12)} for k, (fd, ae, aa) in checks.items()}}
    torch.cuda.empty_cache()
    return out


def general_workload(args, spock, workloads, dev):
    """The general form: polyhedral constraints, dense cost matrices and
    conic risk measures.  (1) T evaluations per second through
    spock_cp_step_dev (50 CP steps, CUDA events, FP64 and FP32) on a tree
    with the large tree's launch shapes at smaller size -- branching 4 for
    5 stages then chains, N = 9 (5,461 nodes), nx = 50, nu = 20 -- in the box
    form and in the general form (dense Q, R, Q_N; nc = 80 constraint rows:
    the box rows and 10 coupled rows; ncN = 56), with the bytes of the
    per-node matrices of L that one T reads (column-major copies once in the
    dual update, transposed copies in the dual update's L* r_eta and in the
    prox-f preparation).  (2) Solves to 1e-6 of the 15-node binary tree with
    AV@R, the mean-AV@R mixture and the total-variation worst case."""
    import torch
    base = workloads.large_tree(seed=1, branching_stages=5, branch=4, N=9)
    gen = workloads.general_random(base, seed=1, extra_rows=10, extra_leaf_rows=6)
    n, nl = len(base["anc"]), int(np.sum(np.bincount(base["anc"][1:], minlength=len(base["anc"])) > 0))
    nx, nu = base["nx"], base["nu"]
    nc, ncN = gen["Gx"].shape[1], gen["GN"].shape[1]
    pad = lambda k: (k + 3) // 4 * 4
    # entries of the per-node matrices (one layout): Gamma, Q^1/2, R^1/2 of
    # the edge into each nonroot node, Gamma_N and Q_N^1/2 at leaves
    ent_c = nl * (nx + nu) * pad(nc) + (n - 1) * (nx * pad(nx) + nu * pad(nu)) + (n - nl) * (
        nx * pad(ncN) + nx * pad(nx))
    ent_t = nl * nc * pad(nx + nu) + (n - 1) * (nx * pad(nx) + nu * pad(nu)) + (n - nl) * (
        ncN * pad(nx) + nx * pad(nx))
    out = {"nodes": n, "nx": nx, "nu": nu, "nc": nc, "ncN": ncN, "steps": 50}
    K = 50
    for nm, d in (("box", base), ("general", gen)):
        P = spock.Problem(d)
        x0 = torch.tensor(d["x0"], dtype=torch.float64, device=dev)
        alpha = 0.99 / P.norm_L
        r = {"norm_L": P.norm_L}
        for prec, pn in ((spock.SPOCK_FP64, "fp64"), (spock.SPOCK_FP32, "fp32")):
            z = torch.zeros(P.n_z, dtype=torch.float64, device=dev)
            e = torch.zeros(P.n_eta, dtype=torch.float64, device=dev)
            spock.spock_cp_step_dev(P.handle, x0, 3, alpha, prec, z, e)   # warm-up
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            cur = torch.cuda.current_stream()
            torch.cuda.synchronize()
            ev0.record(cur)
            spock.spock_cp_step_dev(P.handle, x0, K, alpha, prec, z, e)
            ev1.record(cur)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / K
            r[pn] = {"ms_per_T": round(ms, 4), "T_per_s": round(1e3 / ms, 1)}
            if nm == "general":
                elt = 8 if prec == spock.SPOCK_FP64 else 4
                mb = elt * (ent_c + 2 * ent_t)
                r[pn]["L_matrix_bytes_per_T"] = mb
        out[nm] = r
        P.close()
    for pn in ("fp64", "fp32"):
        out["general"][pn]["added_ms_per_T"] = round(out["general"][pn]["ms_per_T"] - out["box"][pn]["ms_per_T"], 4)
    # risk measures on the 15-node binary tree
    risks = {}
    for kind in ("avar", "mean_avar", "tv"):
        d = workloads.risk_measures(workloads.small_binary(0, a=0.5), kind, lam=0.5, radius=0.3)
        P = spock.Problem(d)
        s = spock.spock_default_settings(memory=5, max_iter=20000)
        z = np.zeros(P.n_z)
        e = np.zeros(P.n_eta)
        t0 = time.perf_counter()
        info = spock.spock_solve(P.handle, d["x0"], s, z, e, 0)
        risks[kind] = {"ms": round((time.perf_counter() - t0) * 1e3, 2), "iterations": info.iterations,
                       "status": "converged" if info.status == 0 else "max_iter", "cost": float(z[0]),
                       "n_z": P.n_z, "n_eta": P.n_eta}
        P.close()
    out["risk_measures_binary_N3"] = risks
    return out


def host_cpu():
    """Cores this process may use and the CPU model of the host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "Model name", "CPU part"):
            hits = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith(key)]
            if hits:
                model = hits[0] if key != "CPU part" else f"Arm CPU part {hits[0]}"
                break
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model or "unknown"


def cpu_baseline(d, seconds=10.0, threads=None):
    """The oracle's C++ CP operator (riccati_cpu: plain FP64, Algorithms 1-2
    as printed, OpenMP over the nodes of a stage) timed on the same
    62,805-node tree: evaluations of T from v = 0 for about ``seconds`` at
    one thread and at all host cores (Algorithm 1 excluded, as for the GPU)."""
    from oracle.riccati_cpu import RiccatiCPU
    cores, model = host_cpu()
    threads = threads or cores
    t0 = time.perf_counter()
    rc = RiccatiCPU(d, threads=threads)
    setup_s = time.perf_counter() - t0
    alpha = 0.3   # any step: the cost of T does not depend on it
    z, e = np.zeros(rc.n_z), np.zeros(rc.n_eta)
    out = (np.empty(rc.n_z), np.empty(rc.n_eta))
    rates = {}
    for th in sorted({1, threads}):
        rc.set_threads(th)
        rc.T(z, e, alpha, out=out)
        k, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < seconds / 2 or k < 2:
            rc.T(z, e, alpha, out=out)
            k += 1
        rates[th] = (k, time.perf_counter() - t0)
    rc.close()
    k, dt = rates[threads]
    k1, dt1 = rates[1]
    return {"value": k / dt, "unit": "CP iters/s", "cores": threads, "kind": "oracle",
            "cpu_model": model, "nproc": cores,
            "one_thread": {"value": k1 / dt1, "evaluations": k1, "seconds": round(dt1, 2)},
            "sample": f"{k} evaluations of T in {dt:.1f} s on the full {len(d['anc']):,}-node tree (the "
                      f"timed workload itself), riccati_cpu (C++ FP64, Algorithms 1-2 as printed, OpenMP "
                      f"over the nodes of a stage) on {threads} threads; Algorithm 1 ({setup_s:.1f} s) "
                      "not timed"}


def run_reference(args, rank, world):
    """The oracle's C++ CP operator on the host cores, one evaluation of T of
    the full tree per step."""
    if rank != 0:
        return
    from oracle.riccati_cpu import RiccatiCPU
    from paper_2212_01110_gb300 import workloads
    d = workloads.large_tree(seed=0, **WORKLOAD)
    cores, model = host_cpu()
    rc = RiccatiCPU(d, threads=cores)
    z, e = np.zeros(rc.n_z), np.zeros(rc.n_eta)
    out = (np.empty(rc.n_z), np.empty(rc.n_eta))
    for _ in range(args.warmup):
        rc.T(z, e, 0.3, out=out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rc.T(z, e, 0.3, out=out)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "CP iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": "large scenario tree: branching 4 for 6 stages then 1, N=20 (62,805 nodes), "
                                   "nx=50, nu=20",
                       "step": "one evaluation of the CP operator T on the host cores"},
            "cpu_baseline": {"value": v, "unit": "CP iters/s", "cores": cores, "kind": "oracle", "cpu_model": model,
                             "sample": f"{args.steps} evaluations of T on the full tree, riccati_cpu (C++ FP64, "
                                       f"Algorithms 1-2 as printed, OpenMP over the nodes of a stage), {cores} threads"},
            "e2e": {"value": v, "unit": "CP iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    rc.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["fp64", "fp32", "both"])
    ap.add_argument("--memory", type=int, default=3)
    ap.add_argument("--tol-budget-s", type=float, default=15.0,
                    help="time budget of the time-to-1e-6 solve per precision (0 skips it)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paper-workload", type=int, default=1,
                    help="also time SPOCK to tolerance on the paper's data-center system (1) or not (0)")
    ap.add_argument("--paper-max-iter", type=int, default=20000)
    ap.add_argument("--mpc-realisations", type=int, default=3,
                    help="disturbance sequences of the closed-loop MPC measurement (0 skips it; the paper uses 15)")
    ap.add_argument("--batch", type=int, default=512, help="instances of the batched measurement (0 skips it)")
    ap.add_argument("--batch-iter", type=int, default=50)
    ap.add_argument("--families", type=int, default=64, help="families of the family-form batch (0 skips it)")
    ap.add_argument("--general", type=int, default=1, help="general-form measurement (0 skips it)")
    ap.add_argument("--family-size", type=int, default=8, help="instances per family (x0 differs)")
    ap.add_argument("--batch-tol-iter", type=int, default=10000,
                    help="iteration cap of the batched time-to-1e-6 solve (0 skips it)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched measurement and print it (profiling aid, not a bench line)")
    ap.add_argument("--grad-instances", type=int, default=64,
                    help="instances of the gradient measurement (0 skips it)")
    ap.add_argument("--grad-iter", type=int, default=20000,
                    help="iteration cap per instance of the gradient workload's solve")
    ap.add_argument("--grad-base-iter", type=int, default=250000,
                    help="iteration cap of the finite-difference check's base solve to 1e-12")
    ap.add_argument("--grad-fd-iter", type=int, default=30000,
                    help="iteration cap of the 1e-12 solves of the finite-difference check")
    ap.add_argument("--horizon", type=int, default=20,
                    help="horizon N of the tree (20 = the 62,805-node tree; shorter chains for profiling)")
    ap.add_argument("--branching-stages", type=int, default=6,
                    help="stages with 4 children (6 = the 62,805-node tree; smaller trees for profiling)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.batch_only:   # profiling aid: the batched measurement alone
        import torch
        from paper_2212_01110_gb300 import build
        build.build()
        from paper_2212_01110_gb300 import spock, workloads
        torch.cuda.set_device(local_rank)
        print(json.dumps({"batch": batch_workload(args, spock, workloads, torch.device("cuda", local_rank))}))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
