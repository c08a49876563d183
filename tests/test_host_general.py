"""Host logic of the general form (csrc/general.cpp, csrc/tree.cpp), on the
CPU: a small C++ driver built with g++ runs build_tree, build_offsets and
build_general on seeded data and prints what they computed; the test checks
it against numpy and the oracle's layout:
  * the per-node matrices in both device layouts equal the inputs, and the
    cost factors are upper triangular with F^T F = Q;
  * the certified (x, u) block norm is an upper bound of numpy's largest
    eigenvalue of Gamma^T Gamma + sum_c blockdiag(Q^c, R^c), within 1e-6;
  * each S2 projector equals I - M^+ M (numpy pseudoinverse) for
    M = [[E^T, -I, -I], [F^T, 0, 0]];
  * the z and eta offsets of a problem with conic risk measures equal the
    oracle layout's."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.problem import Problem
from paper_2212_01110_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
SANITIZE = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g"]
CSRC = os.path.join(HERE, "..", "paper_2212_01110_gb300", "csrc")
INC = os.path.join(HERE, "..", "include")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "general.h"
namespace spock {
static std::string g_err;
void set_error(const std::string& m) { g_err = m; }
int fail(int code, const std::string& m) { g_err = m; return code; }
}
using namespace spock;
static std::vector<double> rd(FILE* f, size_t n) { std::vector<double> v(n); for (auto& x : v) if (fscanf(f, "%lf", &x) != 1) exit(3); return v; }
static void pr(const char* k, const std::vector<double>& v) { printf("\"%s\": [", k); for (size_t i = 0; i < v.size(); ++i) printf(i ? ",%.17g" : "%.17g", v[i]); printf("],\n"); }
template <typename T> static void pri(const char* k, const std::vector<T>& v) { printf("\"%s\": [", k); for (size_t i = 0; i < v.size(); ++i) printf(i ? ",%lld" : "%lld", (long long)v[i]); printf("],\n"); }
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "r");
  int n, nx, nu, nc, ncN, dense, hasrisk;
  if (fscanf(f, "%d %d %d %d %d %d %d", &n, &nx, &nu, &nc, &ncN, &dense, &hasrisk) != 7) return 2;
  std::vector<int32_t> anc(n);
  for (auto& a : anc) if (fscanf(f, "%d", &a) != 1) return 3;
  auto prob = rd(f, n);
  const size_t q = dense ? (size_t)nx * nx : nx, r = dense ? (size_t)nu * nu : nu;
  auto Q = rd(f, n * q), R = rd(f, n * r), QN = rd(f, n * q), a = rd(f, n);
  auto Gx = rd(f, (size_t)n * nc * nx), Gu = rd(f, (size_t)n * nc * nu), cmin = rd(f, (size_t)n * nc), cmax = rd(f, (size_t)n * nc);
  auto GN = rd(f, (size_t)n * ncN * nx), cNmin = rd(f, (size_t)n * ncN), cNmax = rd(f, (size_t)n * ncN);
  std::vector<spock_risk> risk(n);
  std::vector<std::vector<double>> keep;
  for (int i = 0; i < n && hasrisk; ++i) {
    int ny, nnu, kp, m;
    if (fscanf(f, "%d %d %d %d", &ny, &nnu, &kp, &m) != 4) return 4;
    if (ny == 0) { risk[i] = spock_risk{0, 0, 0, nullptr, nullptr, nullptr}; continue; }
    keep.push_back(rd(f, ny)); const double* b = keep.back().data();
    keep.push_back(rd(f, (size_t)ny * m)); const double* E = keep.back().data();
    const double* F = nullptr;
    if (nnu) { keep.push_back(rd(f, (size_t)ny * nnu)); F = keep.back().data(); }
    risk[i] = spock_risk{ny, nnu, kp, b, E, F};
  }
  Tree t;
  if (build_tree(n, anc.data(), prob.data(), t) != SPOCK_OK) { printf("tree error\n"); return 5; }
  GenHost g; std::string err;
  int rc = build_general(t, nx, nu, dense != 0, Q.data(), R.data(), QN.data(), a.data(), hasrisk ? risk.data() : nullptr,
                         nc, Gx.data(), Gu.data(), cmin.data(), cmax.data(), ncN, GN.data(), cNmin.data(), cNmax.data(), 2, g, err);
  if (rc != SPOCK_OK) { printf("{\"rc\": %d}\n", rc); return 0; }   // as the library: nothing else is built
  Offsets o;
  build_offsets(t, nx, nu, nc, ncN, &g.ny_user, o);
  printf("{\"rc\": %d,\n", rc);
  pri("user_of", t.user_of);
  pri("ldims", std::vector<int>{g.d.ldc, g.d.ldxu, g.d.ldx, g.d.ldu, g.d.ldcn, g.d.cst});
  pr("gc", g.gc); pr("gt", g.gt); pr("fqc", g.fqc); pr("fqt", g.fqt); pr("frc", g.frc);
  pr("fnc", g.fnc); pr("gnc", g.gnc); pr("gnt", g.gnt); pr("clo", g.clo); pr("chi", g.chi);
  pr("rpi", g.rpi); pri("rpoff", g.rpoff); pri("rny", g.rny);
  pri("zx", o.zx); pri("zz2", o.zz2); pri("enl", o.enl); pri("enr", o.enr); pri("elf", o.elf);
  printf("\"n_z\": %lld, \"n_eta\": %lld, \"normL2_xu\": %.17g, \"normL2_ys\": %.17g}\n", (long long)o.n_z, (long long)o.n_eta, g.normL2_xu, g.normL2_ys);
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
    d = tmp_path_factory.mktemp("hostgen")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    cmd = [gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", INC, "-I", cuda_inc, str(src),
           os.path.join(CSRC, "general.cpp"), os.path.join(CSRC, "tree.cpp"), "-o", str(exe), "-lpthread"]
    # address and undefined-behaviour sanitizers where the toolchain has them:
    # an out-of-bounds write in the host code fails the run
    r = subprocess.run(cmd[:1] + SANITIZE + cmd[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def _run(driver, d, tmp_path):
    n, nx, nu = len(d["anc"]), d["nx"], d["nu"]
    dense = np.asarray(d["Q"]).ndim == 3
    nc, ncN = d["Gx"].shape[1], d["GN"].shape[1]
    risk = d.get("risk")
    parts = [f"{n} {nx} {nu} {nc} {ncN} {int(dense)} {int(risk is not None)}",
             " ".join(map(str, np.asarray(d["anc"], int)))]
    for k in ("prob", "Q", "R", "QN", "a", "Gx", "Gu", "cmin", "cmax", "GN", "cNmin", "cNmax"):
        parts.append(" ".join(repr(float(v)) for v in np.asarray(d[k], float).ravel()))
    if risk is not None:
        kids = np.bincount(np.asarray(d["anc"])[1:], minlength=n)
        for i, r in enumerate(risk):
            if r is None:
                parts.append(f"0 0 0 {kids[i]}")
                continue
            F = np.asarray(r["F"], float)
            nnu = F.shape[1] if F.ndim == 2 else 0
            parts.append(f"{len(r['b'])} {nnu} {r['kp']} {kids[i]}")
            parts.append(" ".join(repr(float(v)) for v in np.asarray(r["b"]).ravel()))
            parts.append(" ".join(repr(float(v)) for v in np.asarray(r["E"]).ravel()))
            if nnu:
                parts.append(" ".join(repr(float(v)) for v in F.ravel()))
    inp = tmp_path / "in.txt"
    inp.write_text("\n".join(parts) + "\n")
    r = subprocess.run([driver, str(inp)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.loads(r.stdout)


@pytest.mark.parametrize("nx,nu", [(5, 3), (2, 5)])
def test_matrices_factors_and_norm(driver, tmp_path, nx, nu):
    d = W.general_random(W.random_tree(3, N=3, max_branch=3, nx=nx, nu=nu), seed=1, extra_rows=3, extra_leaf_rows=2)
    out = _run(driver, d, tmp_path)
    assert out["rc"] == 0
    P = Problem(d)
    n, nx, nu, nc, ncN = P.tree.n, P.nx, P.nu, P.nc, P.ncN
    ldc, ldxu, ldx, ldu, ldcn, cst = out["ldims"]
    user_of = out["user_of"]
    gc, gt, fqc, fqt = (np.array(out[k]) for k in ("gc", "gt", "fqc", "fqt"))
    fnc, gnc, gnt, clo = (np.array(out[k]) for k in ("fnc", "gnc", "gnt", "clo"))
    nl = len(P.tree.nonleaf)
    for k in range(n):
        u = user_of[k]
        if k < nl:
            G = np.hstack([d["Gx"][u], d["Gu"][u]])
            Mc = gc[k * (nx + nu) * ldc:(k + 1) * (nx + nu) * ldc].reshape(nx + nu, ldc)[:, :nc].T
            Mt = gt[k * nc * ldxu:(k + 1) * nc * ldxu].reshape(nc, ldxu)[:, :nx + nu]
            np.testing.assert_array_equal(Mc, G)
            np.testing.assert_array_equal(Mt, G)
            np.testing.assert_array_equal(clo[k * cst:k * cst + nc], d["cmin"][u])
        else:
            Gn = gnc[k * nx * ldcn:(k + 1) * nx * ldcn].reshape(nx, ldcn)[:, :ncN].T
            np.testing.assert_array_equal(Gn, d["GN"][u])
            Gt = gnt[k * ncN * ldx:(k + 1) * ncN * ldx].reshape(ncN, ldx)[:, :nx]
            np.testing.assert_array_equal(Gt, d["GN"][u])
            Fn = fnc[k * nx * ldx:(k + 1) * nx * ldx].reshape(nx, ldx)[:, :nx].T
            np.testing.assert_allclose(Fn.T @ Fn, d["QN"][u], rtol=1e-12, atol=1e-12)
        if k > 0:
            F = fqc[k * nx * ldx:(k + 1) * nx * ldx].reshape(nx, ldx)[:, :nx].T
            Ft = fqt[k * nx * ldx:(k + 1) * nx * ldx].reshape(nx, ldx)[:, :nx]
            assert np.allclose(np.tril(F, -1), 0.0)
            np.testing.assert_array_equal(F, Ft)
            np.testing.assert_allclose(F.T @ F, d["Q"][u], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(F, np.linalg.cholesky(d["Q"][u]).T, rtol=1e-10, atol=1e-12)
    # certified block norm of the (x, u) / x column groups
    lam = 0.0
    for i in P.tree.nonleaf:
        G = np.hstack([P.Gx[i], P.Gu[i]])
        M = G.T @ G
        for c in P.tree.children[i]:
            M[:nx, :nx] += P.Qmat(c)
            M[nx:, nx:] += P.Rmat(c)
        lam = max(lam, np.linalg.eigvalsh(M)[-1])
    for j in P.tree.leaves:
        lam = max(lam, np.linalg.eigvalsh(P.GN[j].T @ P.GN[j] + P.QNmat(j))[-1])
    assert lam * (1 - 1e-12) <= out["normL2_xu"] <= lam * (1 + 1e-6)


RISK_CASES = {
    "tv_fig1": lambda: W.risk_measures(W.general_random(W.with_tree(W.fig1_tree(), seed=2, nx=3, nu=2), seed=3),
                                       "tv", radius=0.3),
    # z_2 block of 121 entries at the root (AV@R in conic form, 30 children)
    "avar_root_30": lambda: W.risk_measures(
        W.general_random(W.with_tree(W.tree_from_branching([30, 1])[0], seed=9, nx=3, nu=2), seed=4), "avar"),
    "mean_avar_nu_gt_nx": lambda: W.risk_measures(
        W.general_random(W.random_tree(9, N=3, max_branch=4, nx=2, nu=5), seed=5), "mean_avar"),
}


@pytest.mark.parametrize("name", sorted(RISK_CASES))
def test_risk_projectors_and_offsets(driver, tmp_path, name):
    d = RISK_CASES[name]()
    out = _run(driver, d, tmp_path)
    assert out["rc"] == 0
    P = Problem(d)
    lay = P.lay
    user_of = out["user_of"]
    rpi, rpoff = np.array(out["rpi"]), out["rpoff"]
    for k, u in enumerate(user_of):
        if k >= len(P.tree.nonleaf):
            continue
        b, E, F, kp = P.risk[u]
        m = E.shape[1]
        nz2 = b.size + 2 * m
        top = np.hstack([E.T, -np.eye(m), -np.eye(m)])
        M = np.vstack([top, np.hstack([F.T, np.zeros((F.shape[1], 2 * m))])]) if F.shape[1] else top
        ref = np.eye(nz2) - np.linalg.pinv(M) @ M
        got = rpi[rpoff[k]:rpoff[k] + nz2 * nz2].reshape(nz2, nz2).T
        np.testing.assert_allclose(got, ref, atol=1e-12)
        assert out["rny"][k] == b.size
        assert out["zz2"][k] == lay.y[u][0]
        assert out["enl"][k] == lay.e_y[u][0]
        assert out["zx"][k] == lay.x[u][0]
    for k, u in enumerate(user_of):
        if k > 0:
            assert out["enr"][k] == lay.e_qx[u][0]
        if k >= len(P.tree.nonleaf):
            assert out["elf"][k] == lay.e_lc[u][0]
    assert (out["n_z"], out["n_eta"]) == (lay.n_z, lay.n_eta)
    # (y, s) block norm: [[I, 0], [-b^T, 1]]
    ys = max((2 + b @ b + np.sqrt((b @ b) * (b @ b + 4))) / 2 for b, _, _, _ in P.risk.values())
    assert abs(out["normL2_ys"] - ys) <= 1e-12 * ys


def _bad_risk(kind):
    d = W.risk_measures(W.general_random(W.with_tree(W.fig1_tree(), seed=2, nx=3, nu=2), seed=3), "tv", radius=0.3)
    risk = [None if r is None else dict(r) for r in d["risk"]]
    i = next(k for k, r in enumerate(risk) if r is not None)
    r = risk[i]
    if kind == "kp_above_ny":
        r["kp"] = len(r["b"]) + 1
    elif kind == "rank_deficient_F":
        F = np.asarray(r["F"], float)
        r["F"] = np.hstack([F, F[:, :1]])           # a repeated column
    elif kind == "nan_b":
        r["b"] = np.asarray(r["b"], float).copy()
        r["b"][0] = np.nan
    return dict(d, risk=risk)


@pytest.mark.parametrize("kind,code", [("kp_above_ny", -1), ("rank_deficient_F", -1), ("nan_b", -4),
                                       ("too_large_z2", -1), ("indefinite_Q", -3), ("crossed_bounds", -1)])
def test_invalid_inputs_are_rejected_cleanly(driver, tmp_path, kind, code):
    """build_general returns the documented error for malformed risk
    measures, an S2 block above 160 entries, an indefinite cost matrix and
    crossed constraint bounds, with no out-of-bounds access on the way (the
    driver runs under the sanitizers)."""
    if kind in ("kp_above_ny", "rank_deficient_F", "nan_b"):
        d = _bad_risk(kind)
    elif kind == "too_large_z2":   # AV@R in conic form at a 60-child root: 121 + 120 entries
        d = W.risk_measures(W.general_random(W.with_tree(W.tree_from_branching([60, 1])[0], seed=9, nx=3, nu=2),
                                             seed=4), "avar")
    elif kind == "indefinite_Q":
        d = W.general_random(W.random_tree(3, N=3, max_branch=3, nx=4, nu=3), seed=1)
        d["Q"] = np.array(d["Q"], float)
        d["Q"][1] = -np.eye(4)
    else:
        d = W.general_random(W.random_tree(3, N=3, max_branch=3, nx=4, nu=3), seed=1)
        d["cmin"] = np.array(d["cmin"], float)
        d["cmin"][0, 0] = d["cmax"][0, 0] + 1.0
    out = _run(driver, d, tmp_path)
    assert out["rc"] == code


def test_threaded_construction_has_no_data_race(tmp_path):
    """build_general spreads the nodes over host threads (factors, block
    norms, S2 projectors); built with the thread sanitizer, no data race is
    reported on a polyhedral problem and on conic AV@R at a 30-child root."""
    gxx = shutil.which("g++")
    cuda_inc = next((p for p in ("/usr/local/cuda/include", "/usr/include") if
                     os.path.exists(os.path.join(p, "cuda_runtime.h"))), None)
    if not gxx or cuda_inc is None:
        pytest.skip("g++ or cuda_runtime.h not available")
    src = tmp_path / "driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "driver_tsan"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-I", CSRC, "-I", INC, "-I", cuda_inc,
                        str(src), os.path.join(CSRC, "general.cpp"), os.path.join(CSRC, "tree.cpp"), "-o", str(exe),
                        "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("thread sanitizer unavailable: " + r.stderr[-200:])
    for d in (W.general_random(W.large_tree(1, branching_stages=3, branch=4, N=4, nx=6, nu=3), seed=2),
              W.risk_measures(W.general_random(W.with_tree(W.tree_from_branching([30, 1])[0], seed=9, nx=3, nu=2),
                                               seed=4), "avar")):
        assert _run(str(exe), d, tmp_path)["rc"] == 0   # a sanitizer report exits non-zero
