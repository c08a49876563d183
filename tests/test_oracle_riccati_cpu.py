"""riccati_cpu (plain C++ FP64, Algorithms 1-2 as printed, OpenMP over the
nodes of a stage) against the Python oracle (explicit sparse L, KKT
projection on S1, pseudoinverse projection on S2): every part of T and T
itself to 1e-12 relative, with 1 and 3 threads.  This pins the C++ checker
that the large-tree parity tests and the CPU baseline use."""
import numpy as np
import pytest

from oracle.cones import prox_gconj
from oracle.cp import CP
from oracle.problem import Problem
from oracle.riccati_cpu import RiccatiCPU
from paper_2212_01110_gb300 import workloads as W

TOL = 1e-12


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


CASES = {
    "binary_N3": lambda: W.small_binary(0),
    "fig1": lambda: W.with_tree(W.fig1_tree(), seed=1, nx=3, nu=2),
    "ragged": lambda: W.random_tree(3, N=4, max_branch=3, nx=4, nu=3),
    "chains": lambda: W.random_tree(4, N=6, max_branch=3, nx=5, nu=2, chain_after=2),
    "wide_50_20": lambda: W.large_tree(0, branching_stages=2, branch=3, N=5, nx=50, nu=20),
    "datacenter": lambda: W.datacenter(N=4, nx=6),
    "root_17_2": lambda: W.with_tree(W.tree_from_branching([17, 2])[0], seed=10, nx=4, nu=2, a=0.3),
    "nu_gt_nx": lambda: W.random_tree(9, N=3, max_branch=4, nx=2, nu=5),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    d = CASES[request.param]()
    cp = CP(Problem(d))
    return d, cp


@pytest.mark.parametrize("threads", [1, 3])
def test_parts_and_T_match_python_oracle(pair, threads):
    d, cp = pair
    rc = RiccatiCPU(d, threads=threads)
    assert (rc.n_z, rc.n_eta) == (cp.n_z, cp.n_eta)
    rng = np.random.default_rng(7)
    z = rng.standard_normal(cp.n_z)
    e = 2 * rng.standard_normal(cp.n_eta)
    assert _rel(rc.apply_L(z), cp.L @ z) < TOL
    assert _rel(rc.apply_Lt(e), cp.Lt @ e) < TOL
    assert _rel(rc.prox_f(z, cp.alpha), cp.prox_f(z, d["x0"])) < TOL
    assert _rel(rc.prox_gconj(e, cp.alpha), prox_gconj(e, cp.alpha, cp.P)) < TOL
    zo, eo = rc.T(z, e, cp.alpha)
    ref = cp.T(np.concatenate([z, e]), d["x0"])
    assert _rel(np.concatenate([zo, eo]), ref) < TOL
    rc.close()


def test_riccati_projection_is_a_projection_on_a_larger_tree():
    """Algorithm 2 on a 309-node tree of the large-tree family (nx = 50,
    nu = 20): agreement with the KKT projection and idempotence."""
    d = W.large_tree(1, branching_stages=2, branch=4, N=20, nx=50, nu=20)
    cp = CP(Problem(d))
    rc = RiccatiCPU(d, threads=2)
    z = np.random.default_rng(3).standard_normal(cp.n_z)
    p1 = rc.prox_f(z, 0.0)
    assert _rel(p1, cp.prox_f(z, d["x0"]) + np.eye(1, cp.n_z, 0)[0] * cp.alpha) < TOL
    assert _rel(rc.prox_f(p1, 0.0), p1) < TOL


SAN_DRIVER = r"""
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>
extern "C" {
void* rc_create(int32_t, const int32_t*, const double*, int32_t, int32_t, const double*, const double*,
                const double*, const double*, const double*, const double*, const double*, const double*,
                const double*, const double*, int32_t);
void rc_sizes(void*, int64_t*, int64_t*);
void rc_T(void*, const double*, double, const double*, const double*, double*, double*);
void rc_free(void*);
}
static std::vector<double> rd(FILE* f, size_t n) { std::vector<double> v(n); for (auto& x : v) if (fscanf(f, "%lf", &x) != 1) exit(3); return v; }
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "r");
  int n, nx, nu, th;
  if (fscanf(f, "%d %d %d %d", &n, &nx, &nu, &th) != 4) return 2;
  std::vector<int32_t> anc(n);
  for (auto& a : anc) if (fscanf(f, "%d", &a) != 1) return 3;
  auto prob = rd(f, n), A = rd(f, (size_t)n * nx * nx), B = rd(f, (size_t)n * nx * nu), Q = rd(f, (size_t)n * nx),
       R = rd(f, (size_t)n * nu), QN = rd(f, (size_t)n * nx), a = rd(f, n), xmin = rd(f, (size_t)n * nx),
       xmax = rd(f, (size_t)n * nx), umin = rd(f, (size_t)n * nu), umax = rd(f, (size_t)n * nu), x0 = rd(f, nx),
       al = rd(f, 1);
  void* h = rc_create(n, anc.data(), prob.data(), nx, nu, A.data(), B.data(), Q.data(), R.data(), QN.data(), a.data(),
                      xmin.data(), xmax.data(), umin.data(), umax.data(), th);
  int64_t nz = 0, ne = 0;
  rc_sizes(h, &nz, &ne);
  auto z = rd(f, nz), e = rd(f, ne);
  std::vector<double> zo(nz), eo(ne);
  rc_T(h, x0.data(), al[0], z.data(), e.data(), zo.data(), eo.data());
  for (auto v : zo) printf("%.17g\n", v);
  for (auto v : eo) printf("%.17g\n", v);
  rc_free(h);
  return 0;
}
"""


def test_sanitized_build_gives_the_same_T(tmp_path):
    """The C++ operator built with the address and undefined-behaviour
    sanitizers runs T without a finding (an out-of-bounds access fails the
    run) on shapes that stress its indexing -- horizon 1, nu > nx, a node
    with 17 children, chains -- with three threads, and gives the library
    build's T to 1e-13."""
    import os
    import shutil
    import subprocess
    from oracle import riccati_cpu
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    src = tmp_path / "drv.cpp"
    src.write_text(SAN_DRIVER)
    exe = tmp_path / "drv"
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fopenmp", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", str(src), riccati_cpu.SRC, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("sanitizer build unavailable: " + r.stderr[-200:])
    cases = {
        "two_nodes": W.with_tree(W.tree_from_branching([1])[0], seed=11, nx=3, nu=2),
        "N1_star": W.with_tree(W.tree_from_branching([5])[0], seed=12, nx=3, nu=2),
        "nu_gt_nx": W.random_tree(9, N=3, max_branch=4, nx=2, nu=5),
        "root_17_2": CASES["root_17_2"](),
        "chains": CASES["chains"](),
    }
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", OMP_NUM_THREADS="3")
    for name, d in cases.items():
        cp = CP(Problem(d))
        rng = np.random.default_rng(5)
        z = rng.standard_normal(cp.n_z)
        e = rng.standard_normal(cp.n_eta)
        parts = [f"{len(d['anc'])} {d['nx']} {d['nu']} 3", " ".join(map(str, np.asarray(d["anc"], int)))]
        for k in ("prob", "A", "B", "Q", "R", "QN", "a", "xmin", "xmax", "umin", "umax", "x0"):
            parts.append(" ".join(repr(float(v)) for v in np.asarray(d[k], float).ravel()))
        parts += [repr(float(cp.alpha)), " ".join(repr(float(v)) for v in z), " ".join(repr(float(v)) for v in e)]
        inp = tmp_path / f"{name}.txt"
        inp.write_text("\n".join(parts) + "\n")
        r = subprocess.run([str(exe), str(inp)], capture_output=True, text=True, env=env)
        assert r.returncode == 0, (name, r.stderr[-2000:])
        got = np.array([float(v) for v in r.stdout.split()])
        rc = RiccatiCPU(d, threads=3)
        zo, eo = rc.T(z, e, cp.alpha)
        rc.close()
        assert _rel(got, np.concatenate([zo, eo])) < 1e-13, name
