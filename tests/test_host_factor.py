"""Host logic of the offline factorisation (csrc/factor.cpp, Algorithm 1 in
FP64 with W^i = sum_c Abar^cT P^c B^c precomputed) on the CPU: a small C++
driver built with g++ runs build_tree and riccati_factor on seeded trees and
prints the stored blocks ([Abar^c | B^c] per nonroot node; K^i, K^i + W^iT
and Rtilde^-1 per nonleaf node).  The test applies them the way the online
pass of Algorithm 2 does -- backward: d^i = Rtilde^-1 (ubar^i - sum_c B^cT
q^c), q^i = (K + W^T)^T d^i - K^T ubar^i - xbar^i + sum_c Abar^cT q^c (leaves
q = -xbar); forward: u^i = K^i x^i + d^i, x^c = Abar^c x^i + B^c d^i -- and
compares the result with the oracle's projection on S1 by a KKT solve
(Sec. "Projection on S1") for random (xbar, ubar, x0).  Every stored entry
enters that projection, so a wrong K, W, Abar or Rtilde^-1 fails it.  The
threaded factorisation (nodes of a stage spread over host threads) must give
the one-thread result bit for bit."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.problem import Problem
from oracle.s1 import S1Projector
from paper_2212_01110_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
SANITIZE = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g"]
CSRC = os.path.join(HERE, "..", "paper_2212_01110_gb300", "csrc")
INC = os.path.join(HERE, "..", "include")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include "spock_internal.h"
namespace spock {
static std::string g_err;
void set_error(const std::string& m) { g_err = m; }
int fail(int code, const std::string& m) { g_err = m; return code; }
}
using namespace spock;
static std::vector<double> rd(FILE* f, size_t n) { std::vector<double> v(n); for (auto& x : v) if (fscanf(f, "%lf", &x) != 1) exit(3); return v; }
static void pr(const char* k, const std::vector<double>& v) { printf("\"%s\": [", k); for (size_t i = 0; i < v.size(); ++i) printf(i ? ",%.17g" : "%.17g", v[i]); printf("],\n"); }
static void pri(const char* k, const std::vector<int32_t>& v) { printf("\"%s\": [", k); for (size_t i = 0; i < v.size(); ++i) printf(i ? ",%d" : "%d", v[i]); printf("],\n"); }
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "r");
  int n, nx, nu, threads;
  if (fscanf(f, "%d %d %d %d", &n, &nx, &nu, &threads) != 4) return 2;
  std::vector<int32_t> anc(n);
  for (auto& a : anc) if (fscanf(f, "%d", &a) != 1) return 3;
  auto prob = rd(f, n);
  auto A = rd(f, (size_t)n * nx * nx), B = rd(f, (size_t)n * nx * nu);
  Tree t;
  if (build_tree(n, anc.data(), prob.data(), t) != SPOCK_OK) { printf("tree error\n"); return 5; }
  std::vector<double> Ai((size_t)n * nx * nx), Bi((size_t)n * nx * nu);
  for (int32_t k = 1; k < n; ++k) {
    const int32_t u = t.user_of[k];
    std::memcpy(&Ai[(size_t)k * nx * nx], &A[(size_t)u * nx * nx], sizeof(double) * nx * nx);
    std::memcpy(&Bi[(size_t)k * nx * nu], &B[(size_t)u * nx * nu], sizeof(double) * nx * nu);
  }
  std::vector<double> Gb, NB;
  const bool ok = riccati_factor(t, nx, nu, Ai, Bi, Gb, NB, threads);
  printf("{\"ok\": %d,\n", ok ? 1 : 0);
  pri("user_of", t.user_of); pri("ch_begin", t.ch_begin); pri("ch_count", t.ch_count);
  pr("Gb", Gb); pr("NB", NB);
  printf("\"n_nonleaf\": %d}\n", t.n_nonleaf);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    cuda_inc = next((p for p in ("/usr/local/cuda/include", "/usr/include") if
                     os.path.exists(os.path.join(p, "cuda_runtime.h"))), None)
    if cuda_inc is None:
        pytest.skip("cuda_runtime.h not available")
    d = tmp_path_factory.mktemp("hostfactor")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    cmd = [gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", INC, "-I", cuda_inc, str(src),
           os.path.join(CSRC, "factor.cpp"), os.path.join(CSRC, "tree.cpp"), "-o", str(exe), "-lpthread"]
    # address and undefined-behaviour sanitizers where the toolchain has them:
    # an out-of-bounds write in the host code fails the run
    r = subprocess.run(cmd[:1] + SANITIZE + cmd[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def _factor(driver, d, threads, tmp_path):
    n, nx, nu = len(d["anc"]), d["nx"], d["nu"]
    parts = [f"{n} {nx} {nu} {threads}", " ".join(map(str, np.asarray(d["anc"], int)))]
    for k in ("prob", "A", "B"):
        parts.append(" ".join(repr(float(v)) for v in np.asarray(d[k], float).ravel()))
    inp = tmp_path / f"in{threads}.txt"
    inp.write_text("\n".join(parts) + "\n")
    r = subprocess.run([driver, str(inp)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = json.loads(r.stdout)
    assert out["ok"] == 1
    return out


def _project_with_factors(out, nx, nu, xbar, ubar, x0):
    """The online pass with the stored blocks, internal numbering."""
    user_of = out["user_of"]
    n, nl = len(user_of), out["n_nonleaf"]
    ncol = nx + nu
    Gb = np.array(out["Gb"]).reshape(n - 1, nx, ncol)
    NB = np.array(out["NB"]).reshape(nl, 2 * nu * nx + nu * nu)
    K = NB[:, :nu * nx].reshape(nl, nu, nx)
    C = NB[:, nu * nx:2 * nu * nx].reshape(nl, nu, nx)
    Ri = NB[:, 2 * nu * nx:].reshape(nl, nu, nu)
    kids = [range(out["ch_begin"][k], out["ch_begin"][k] + out["ch_count"][k]) for k in range(nl)]
    xb = np.array([xbar[user_of[k]] for k in range(n)])
    ub = np.array([ubar[user_of[k]] for k in range(nl)])
    q = np.zeros((n, nx))
    dd = np.zeros((nl, nu))
    q[nl:] = -xb[nl:]
    for k in reversed(range(nl)):   # children have larger internal ids
        sB = sum(Gb[c - 1][:, nx:].T @ q[c] for c in kids[k])
        sA = sum(Gb[c - 1][:, :nx].T @ q[c] for c in kids[k])
        dd[k] = Ri[k] @ (ub[k] - sB)
        q[k] = C[k].T @ dd[k] - K[k].T @ ub[k] - xb[k] + sA
    x = np.zeros((n, nx))
    u = np.zeros((nl, nu))
    x[0] = x0
    for k in range(nl):
        u[k] = K[k] @ x[k] + dd[k]
        for c in kids[k]:
            x[c] = Gb[c - 1][:, :nx] @ x[k] + Gb[c - 1][:, nx:] @ dd[k]
    xu = np.zeros((n, nx))
    uu = np.zeros((n, nu))
    for k in range(n):
        xu[user_of[k]] = x[k]
        if k < nl:
            uu[user_of[k]] = u[k]
    return xu, uu


CASES = {
    "binary_N3": lambda: W.small_binary(0),
    "fig1": lambda: W.with_tree(W.fig1_tree(), seed=2, nx=3, nu=2),
    "ragged": lambda: W.random_tree(5, N=4, max_branch=3, nx=4, nu=3),
    "chains": lambda: W.random_tree(7, N=6, max_branch=3, nx=3, nu=2, chain_after=2),
    "wide_nu_gt_nx": lambda: W.random_tree(9, N=3, max_branch=4, nx=2, nu=5),
    "branch4_stage3": lambda: W.large_tree(seed=3, branching_stages=3, branch=4, N=4, nx=6, nu=3),
    "two_nodes": lambda: W.with_tree(W.tree_from_branching([1])[0], seed=11, nx=3, nu=2),
    "N1_star": lambda: W.with_tree(W.tree_from_branching([5])[0], seed=12, nx=3, nu=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_factors_give_the_s1_projection(driver, tmp_path, name):
    d = CASES[name]()
    nx, nu = d["nx"], d["nu"]
    out = _factor(driver, d, 1, tmp_path)
    P = Problem(d)
    S1 = S1Projector(P)
    lay = P.lay
    rng = np.random.default_rng(11)
    n = len(d["anc"])
    nonleaf = set(P.tree.nonleaf)
    for _ in range(3):
        xbar = rng.standard_normal((n, nx))
        ubar = rng.standard_normal((n, nu))
        x0 = rng.standard_normal(nx)
        z = np.zeros(lay.n_z)
        for i in range(n):
            z[lay.x[i]] = xbar[i]
            if i in nonleaf:
                z[lay.u[i]] = ubar[i]
        ref = S1.project_z(z, x0)
        x, u = _project_with_factors(out, nx, nu, xbar, ubar, x0)
        scale = max(1.0, np.max(np.abs(ref)))
        for i in range(n):
            np.testing.assert_allclose(x[i], ref[lay.x[i]], rtol=0, atol=1e-10 * scale)
            if i in nonleaf:
                np.testing.assert_allclose(u[i], ref[lay.u[i]], rtol=0, atol=1e-10 * scale)


def test_threaded_factorisation_is_bitwise_the_serial_one(driver, tmp_path):
    d = CASES["branch4_stage3"]()   # 64 nodes at stage 3, 16 at stage 2: several threads per stage
    one = _factor(driver, d, 1, tmp_path)
    four = _factor(driver, d, 4, tmp_path)
    assert one["Gb"] == four["Gb"] and one["NB"] == four["NB"]


@pytest.mark.parametrize("anc,prob", [
    ([0, 0, 0], [1.0, 0.5, 0.5]),            # root's ancestor is not -1
    ([-1, 3, 0], [1.0, 0.5, 0.5]),           # ancestor out of range
    ([-1, -2, 0], [1.0, 0.5, 0.5]),          # negative ancestor below the root
    ([-1, 2, 1], [1.0, 1.0, 1.0]),           # cycle not reachable from the root
    ([-1, 0, 0, 1], [1.0, 0.5, 0.5, 1.0]),   # leaves at different stages
    ([-1, 0, 0], [1.0, 0.5, 0.4]),           # child probabilities do not sum to 1
    ([-1, 0, 0], [1.0, 1.5, -0.5]),          # a negative probability
    ([-1, 0, 0], [1.0, float("nan"), 0.5]),  # NaN probability
])
def test_invalid_trees_are_rejected_cleanly(driver, tmp_path, anc, prob):
    """build_tree turns every malformed ancestor array or probability
    vector into an error return, with no out-of-bounds access on the way
    (the driver runs under the sanitizers)."""
    n, nx, nu = len(anc), 1, 1
    parts = [f"{n} {nx} {nu} 1", " ".join(map(str, anc)), " ".join(repr(float(p)) for p in prob),
             " ".join(["0.5"] * (n * nx * nx)), " ".join(["1.0"] * (n * nx * nu))]
    inp = tmp_path / "bad.txt"
    inp.write_text("\n".join(parts) + "\n")
    r = subprocess.run([driver, str(inp)], capture_output=True, text=True)
    assert r.returncode == 5 and "tree error" in r.stdout, (r.returncode, r.stdout, r.stderr[-1500:])


def test_threaded_factorisation_has_no_data_race(tmp_path):
    """The factorisation with four host threads per stage, built with the
    thread sanitizer: no data race is reported."""
    gxx = shutil.which("g++")
    cuda_inc = next((p for p in ("/usr/local/cuda/include", "/usr/include") if
                     os.path.exists(os.path.join(p, "cuda_runtime.h"))), None)
    if not gxx or cuda_inc is None:
        pytest.skip("g++ or cuda_runtime.h not available")
    src = tmp_path / "driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "driver_tsan"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-I", CSRC, "-I", INC, "-I", cuda_inc,
                        str(src), os.path.join(CSRC, "factor.cpp"), os.path.join(CSRC, "tree.cpp"), "-o", str(exe),
                        "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("thread sanitizer unavailable: " + r.stderr[-200:])
    d = CASES["branch4_stage3"]()
    out = _factor(str(exe), d, 4, tmp_path)   # fails on a sanitizer report (non-zero exit)
    ref = _factor(str(exe), d, 1, tmp_path)
    assert out["Gb"] == ref["Gb"] and out["NB"] == ref["NB"]
