// Host side of the general form (spock_problem_create_general): the
// per-node matrices of the rows of L in the device layouts, the upper
// Cholesky factors of dense cost matrices, and the (x, u) column-group block
// norms of L.
//
// Rows of L that read node k's (x^k, u^k) (definition of L):
//   Gamma^k (x^k, u^k)                         nc rows of k's nonleaf block
//   Q^c 1/2 x^k, R^c 1/2 u^k for each child c  rows of c's nonroot block
//   Gamma_N^k x^k, Q_N^k 1/2 x^k                rows of a leaf's block
// These rows read no other variable, so (x^k, u^k) is one column group of the
// block-diagonal permutation of L (remark after the definition of L) and its
// squared block norm is lambda_max(Gamma^T Gamma + sum_c blockdiag(Q^c, R^c))
// (F^T F = Q for the factor used in L), resp. lambda_max(Gamma_N^T Gamma_N +
// Q_N) at a leaf.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "general.h"

namespace spock {

namespace {

int32_t pad4(int32_t n) { return (n + 3) / 4 * 4; }

// Upper Cholesky factor F (F^T F = M, F upper triangular) of the symmetric
// n x n matrix M (row-major, upper triangle read).  False unless every pivot
// is positive and finite.
bool chol_upper(const double* M, int n, std::vector<double>& F) {
  F.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double dj = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) dj -= F[(size_t)k * n + j] * F[(size_t)k * n + j];
    if (!(dj > 0.0) || !std::isfinite(dj)) return false;
    const double fjj = std::sqrt(dj);
    F[(size_t)j * n + j] = fjj;
    for (int i = j + 1; i < n; ++i) {
      double v = M[(size_t)j * n + i];
      for (int k = 0; k < j; ++k) v -= F[(size_t)k * n + j] * F[(size_t)k * n + i];
      F[(size_t)j * n + i] = v / fjj;
    }
  }
  return true;
}

// Whether sigma I - M is positive definite (Cholesky succeeds), M symmetric.
bool shifted_posdef(const std::vector<double>& M, int n, double sigma, std::vector<double>& W) {
  W.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) W[(size_t)i * n + j] = (i == j ? sigma : 0.0) - M[(size_t)i * n + j];
  std::vector<double> F;
  return chol_upper(W.data(), n, F);
}

// An upper bound of the largest eigenvalue of the symmetric positive
// semidefinite M: a power-iteration estimate rho (at most 300 steps), raised
// until sigma I - M is positive definite (sigma = rho (1 + delta),
// delta = 1e-9, 4e-9, 1.6e-8, ...): within a factor 1 + 4 delta of the
// smallest certified bound.
double lambda_max_upper(const std::vector<double>& M, int n) {
  std::vector<double> v(n), w(n);
  for (int i = 0; i < n; ++i) v[i] = 1.0 + 0.01 * (double)((i * 7919) % 13);
  double rho = 0.0;
  for (int it = 0; it < 300; ++it) {
    double nv = 0.0;
    for (int i = 0; i < n; ++i) nv += v[i] * v[i];
    nv = std::sqrt(nv);
    if (!(nv > 0.0)) break;
    for (int i = 0; i < n; ++i) v[i] /= nv;
    double r = 0.0;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += M[(size_t)i * n + j] * v[j];
      w[i] = s;
      r += v[i] * s;
    }
    const bool done = it > 10 && std::fabs(r - rho) <= 1e-13 * std::fabs(r);
    rho = r;
    v.swap(w);
    if (done) break;
  }
  rho = std::max(rho, 0.0);
  std::vector<double> W;
  double delta = 1e-9;
  for (int tries = 0; tries < 40; ++tries) {
    const double sigma = rho * (1.0 + delta) + 1e-300;
    if (shifted_posdef(M, n, sigma, W)) return sigma;
    delta *= 4.0;
  }
  // Gershgorin bound (always valid)
  double g = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += std::fabs(M[(size_t)i * n + j]);
    g = std::max(g, s);
  }
  return g;
}

template <typename F>
void parallel_nodes(int n, int threads, F&& fn) {
  threads = std::max(1, std::min(threads, n / 64 + 1));
  std::atomic<int> next(0);
  auto work = [&]() {
    for (;;) {
      const int b = next.fetch_add(64);
      if (b >= n) return;
      for (int k = b; k < std::min(n, b + 64); ++k) fn(k);
    }
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < threads; ++i) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
}

// Stores the rows x cols matrix M (row-major) of node k in both layouts.
void put_both(const double* M, int rows, int cols, std::vector<double>& cm, int ld, std::vector<double>& tm,
              int ldT, size_t node) {
  double* c = &cm[node * (size_t)cols * ld];
  double* t = &tm[node * (size_t)rows * ldT];
  for (int r = 0; r < rows; ++r)
    for (int q = 0; q < cols; ++q) {
      c[(size_t)q * ld + r] = M[(size_t)r * cols + q];
      t[(size_t)r * ldT + q] = M[(size_t)r * cols + q];
    }
}

}  // namespace

// Risk measure of nonleaf node k (internal id, m children) in conic form:
// b, E (ny x m), F (ny x n_nu) and kp, from the caller's spock_risk or AV@R
// with parameter a (b = (p, 0, 1), E = [a I, -I, 1]^T, kp = 2 m; no
// projector: the kernels project on S2 by the closed form).  For a given
// risk measure the projector on S2 = ker M, M = [[E^T, -I, -I], [F^T, 0, 0]],
// is I - M^T (M M^T)^-1 M (nz2 x nz2, column-major).  False if M M^T is not
// positive definite.
static bool risk_node(const Tree& t, int k, const double* a, const spock_risk* risk, std::vector<double>& b,
                      int& kp, std::vector<double>& Pi) {
  const int m = t.ch_count[k], c0 = t.ch_begin[k];
  const int32_t u = t.user_of[k];
  int ny, nnu;
  std::vector<double> E, F;
  if (risk) {
    const spock_risk& r = risk[u];
    ny = r.ny;
    nnu = r.n_nu;
    kp = r.kp;
    b.assign(r.b, r.b + ny);
    E.assign(r.E, r.E + (size_t)ny * m);
    if (nnu > 0) F.assign(r.F, r.F + (size_t)ny * nnu);
  } else {
    ny = 2 * m + 1;
    nnu = 0;
    kp = 2 * m;
    b.assign(ny, 0.0);
    E.assign((size_t)ny * m, 0.0);
    for (int j = 0; j < m; ++j) {
      b[j] = t.prob[c0 + j];
      E[(size_t)j * m + j] = a[u];
      E[(size_t)(m + j) * m + j] = -1.0;
      E[(size_t)(2 * m) * m + j] = 1.0;
    }
    b[2 * m] = 1.0;
    Pi.clear();   // AV@R: the kernels use the closed form of the projection
    return true;
  }
  const int nz2 = ny + 2 * m, nr = m + nnu;
  std::vector<double> M((size_t)nr * nz2, 0.0);
  for (int j = 0; j < m; ++j) {
    for (int l = 0; l < ny; ++l) M[(size_t)j * nz2 + l] = E[(size_t)l * m + j];
    M[(size_t)j * nz2 + ny + j] = -1.0;
    M[(size_t)j * nz2 + ny + m + j] = -1.0;
  }
  for (int q = 0; q < nnu; ++q)
    for (int l = 0; l < ny; ++l) M[(size_t)(m + q) * nz2 + l] = F[(size_t)l * nnu + q];
  std::vector<double> G((size_t)nr * nr, 0.0), Fc;
  for (int i = 0; i < nr; ++i)
    for (int j = i; j < nr; ++j) {
      double s = 0.0;
      for (int l = 0; l < nz2; ++l) s += M[(size_t)i * nz2 + l] * M[(size_t)j * nz2 + l];
      G[(size_t)i * nr + j] = G[(size_t)j * nr + i] = s;
    }
  if (!chol_upper(G.data(), nr, Fc)) return false;
  // X = G^-1 M by two triangular solves per column (G = Fc^T Fc)
  std::vector<double> X(M);
  for (int col = 0; col < nz2; ++col) {
    for (int i = 0; i < nr; ++i) {   // Fc^T y = m_col
      double s = X[(size_t)i * nz2 + col];
      for (int k2 = 0; k2 < i; ++k2) s -= Fc[(size_t)k2 * nr + i] * X[(size_t)k2 * nz2 + col];
      X[(size_t)i * nz2 + col] = s / Fc[(size_t)i * nr + i];
    }
    for (int i = nr - 1; i >= 0; --i) {   // Fc x = y
      double s = X[(size_t)i * nz2 + col];
      for (int k2 = i + 1; k2 < nr; ++k2) s -= Fc[(size_t)i * nr + k2] * X[(size_t)k2 * nz2 + col];
      X[(size_t)i * nz2 + col] = s / Fc[(size_t)i * nr + i];
    }
  }
  Pi.assign((size_t)nz2 * nz2, 0.0);
  for (int c = 0; c < nz2; ++c)
    for (int r = 0; r < nz2; ++r) {
      double s = (r == c) ? 1.0 : 0.0;
      for (int i = 0; i < nr; ++i) s -= M[(size_t)i * nz2 + r] * X[(size_t)i * nz2 + c];
      Pi[(size_t)c * nz2 + r] = s;
    }
  return true;
}

int build_general(const Tree& t, int nx, int nu, bool dense, const double* Q, const double* R, const double* QN,
                  const double* a, const spock_risk* risk, int nc, const double* Gx, const double* Gu,
                  const double* cmin, const double* cmax, int ncN, const double* GN, const double* cNmin,
                  const double* cNmax, int threads, GenHost& o, std::string& err) {
  const int n = t.n, nl = t.n_nonleaf, nxu = nx + nu;
  GenDims& g = o.d;
  g.nc = nc;
  g.ncN = ncN;
  g.ldc = pad4(nc);
  g.ldxu = pad4(nxu);
  g.ldx = pad4(nx);
  g.ldu = pad4(nu);
  g.ldcn = pad4(ncN);
  g.cst = pad4(std::max(nc, ncN));
  const size_t nn = (size_t)n;
  o.gc.assign(nn * nxu * g.ldc, 0.0);
  o.gt.assign(nn * nc * g.ldxu, 0.0);
  o.fqc.assign(nn * nx * g.ldx, 0.0);
  o.fqt.assign(nn * nx * g.ldx, 0.0);
  o.frc.assign(nn * nu * g.ldu, 0.0);
  o.frt.assign(nn * nu * g.ldu, 0.0);
  o.fnc.assign(nn * nx * g.ldx, 0.0);
  o.fnt.assign(nn * nx * g.ldx, 0.0);
  o.gnc.assign(nn * nx * g.ldcn, 0.0);
  o.gnt.assign(nn * ncN * g.ldx, 0.0);
  o.clo.assign(nn * g.cst, 0.0);
  o.chi.assign(nn * g.cst, 0.0);
  std::vector<double> block_norm2(nn, 0.0);
  std::atomic<int> bad(0);   // 1: cost matrix not positive definite, 2: bounds
  // cost matrix M of node u (user id) of dimension dim: dense or diagonal
  auto cost = [&](const double* base, int dim, int32_t u, std::vector<double>& M) {
    M.assign((size_t)dim * dim, 0.0);
    if (dense) {
      const double* s = base + (size_t)u * dim * dim;
      for (int i = 0; i < dim; ++i)
        for (int j = i; j < dim; ++j) M[(size_t)i * dim + j] = M[(size_t)j * dim + i] = s[(size_t)i * dim + j];
    } else {
      for (int i = 0; i < dim; ++i) M[(size_t)i * dim + i] = base[(size_t)u * dim + i];
    }
  };
  parallel_nodes(n, threads, [&](int k) {
    const int32_t u = t.user_of[k];
    std::vector<double> M, F;
    const bool leaf = k >= nl;
    if (k > 0) {   // factors of the edge into k
      cost(Q, nx, u, M);
      if (!chol_upper(M.data(), nx, F)) { bad = 1; return; }
      put_both(F.data(), nx, nx, o.fqc, g.ldx, o.fqt, g.ldx, (size_t)k);
      cost(R, nu, u, M);
      if (!chol_upper(M.data(), nu, F)) { bad = 1; return; }
      put_both(F.data(), nu, nu, o.frc, g.ldu, o.frt, g.ldu, (size_t)k);
    }
    if (leaf) {
      cost(QN, nx, u, M);
      if (!chol_upper(M.data(), nx, F)) { bad = 1; return; }
      put_both(F.data(), nx, nx, o.fnc, g.ldx, o.fnt, g.ldx, (size_t)k);
      const double* G = GN + (size_t)u * ncN * nx;
      put_both(G, ncN, nx, o.gnc, g.ldcn, o.gnt, g.ldx, (size_t)k);
      for (int r = 0; r < ncN; ++r) {
        const double lo = cNmin[(size_t)u * ncN + r], hi = cNmax[(size_t)u * ncN + r];
        if (std::isnan(lo) || std::isnan(hi) || lo > hi) { bad = 2; return; }
        o.clo[(size_t)k * g.cst + r] = lo;
        o.chi[(size_t)k * g.cst + r] = hi;
      }
      // block of x^k: Gamma_N^T Gamma_N + Q_N
      std::vector<double> B((size_t)nx * nx, 0.0);
      for (int i = 0; i < nx; ++i)
        for (int j = 0; j < nx; ++j) {
          double s = M[(size_t)i * nx + j];
          for (int r = 0; r < ncN; ++r) s += G[(size_t)r * nx + i] * G[(size_t)r * nx + j];
          B[(size_t)i * nx + j] = s;
        }
      block_norm2[k] = lambda_max_upper(B, nx);
      return;
    }
    // nonleaf: Gamma^k = [Gx | Gu] (nc x (nx + nu)) and its bounds
    std::vector<double> G((size_t)nc * nxu);
    for (int r = 0; r < nc; ++r) {
      for (int q = 0; q < nx; ++q) G[(size_t)r * nxu + q] = Gx[((size_t)u * nc + r) * nx + q];
      for (int q = 0; q < nu; ++q) G[(size_t)r * nxu + nx + q] = Gu[((size_t)u * nc + r) * nu + q];
      const double lo = cmin[(size_t)u * nc + r], hi = cmax[(size_t)u * nc + r];
      if (std::isnan(lo) || std::isnan(hi) || lo > hi) { bad = 2; return; }
      o.clo[(size_t)k * g.cst + r] = lo;
      o.chi[(size_t)k * g.cst + r] = hi;
    }
    put_both(G.data(), nc, nxu, o.gc, g.ldc, o.gt, g.ldxu, (size_t)k);
    // block of (x^k, u^k): Gamma^T Gamma + sum_c blockdiag(Q^c, R^c)
    std::vector<double> B((size_t)nxu * nxu, 0.0);
    for (int i = 0; i < nxu; ++i)
      for (int j = 0; j < nxu; ++j) {
        double s = 0.0;
        for (int r = 0; r < nc; ++r) s += G[(size_t)r * nxu + i] * G[(size_t)r * nxu + j];
        B[(size_t)i * nxu + j] = s;
      }
    for (int c = t.ch_begin[k]; c < t.ch_begin[k] + t.ch_count[k]; ++c) {
      const int32_t uc = t.user_of[c];
      cost(Q, nx, uc, M);
      for (int i = 0; i < nx; ++i)
        for (int j = 0; j < nx; ++j) B[(size_t)i * nxu + j] += M[(size_t)i * nx + j];
      cost(R, nu, uc, M);
      for (int i = 0; i < nu; ++i)
        for (int j = 0; j < nu; ++j) B[(size_t)(nx + i) * nxu + nx + j] += M[(size_t)i * nu + j];
    }
    block_norm2[k] = lambda_max_upper(B, nxu);
  });
  if (bad == 1) {
    err = "a cost matrix (Q, R or Q_N) is not positive definite";
    return SPOCK_ERR_NOT_POSDEF;
  }
  if (bad == 2) {
    err = "constraint bounds: cmin > cmax or NaN";
    return SPOCK_ERR_INVALID_ARG;
  }
  o.normL2_xu = *std::max_element(block_norm2.begin(), block_norm2.end());
  // risk measures (sequential: small per-node work)
  o.rny.assign(nn, 0);
  o.rkp.assign(nn, 0);
  o.rboff.assign(nn, -1);
  o.rpoff.assign(nn, -1);
  o.ny_user.assign(nn, 0);
  o.rb.clear();
  o.rpi.clear();
  o.d.max_nz2 = 0;
  double best_ys = 0.0;
  for (int k = 0; k < nl; ++k) {
    const int32_t u = t.user_of[k];
    const int m = t.ch_count[k];
    if (risk) {
      const spock_risk& r = risk[u];
      if (r.ny < 1 || r.n_nu < 0 || r.kp < 0 || r.kp > r.ny || !r.b || !r.E || (r.n_nu > 0 && !r.F)) {
        err = "risk measure: need ny >= 1, 0 <= kp <= ny, n_nu >= 0 and b, E (and F) set";
        return SPOCK_ERR_INVALID_ARG;
      }
      bool fin = true;
      for (int l = 0; l < r.ny; ++l) fin = fin && std::isfinite(r.b[l]);
      for (int l = 0; l < r.ny * m; ++l) fin = fin && std::isfinite(r.E[l]);
      for (int l = 0; l < r.ny * r.n_nu; ++l) fin = fin && std::isfinite(r.F[l]);
      if (!fin) {
        err = "risk measure: non-finite b, E or F";
        return SPOCK_ERR_NUMERICAL;
      }
    } else if (!(a[u] >= 0.0 && a[u] <= 1.0)) {
      err = "AV@R parameter must be in [0, 1]";
      return SPOCK_ERR_INVALID_ARG;
    }
    std::vector<double> b, Pi;
    int kp = 0;
    if (!risk_node(t, k, a, risk, b, kp, Pi)) {
      err = "risk measure: [[E^T, -I, -I], [F^T, 0, 0]] must have full row rank";
      return SPOCK_ERR_INVALID_ARG;
    }
    const int ny = (int)b.size(), nz2 = ny + 2 * m;
    if (!Pi.empty() && nz2 > kMaxZ2) {
      err = "risk measure: ny + 2 m must not exceed 160 at a node";
      return SPOCK_ERR_INVALID_ARG;
    }
    o.rny[k] = ny;
    o.rkp[k] = kp;
    o.ny_user[u] = ny;
    o.rboff[k] = (int64_t)o.rb.size();
    o.rb.insert(o.rb.end(), b.begin(), b.end());
    while (o.rb.size() % 4) o.rb.push_back(0.0);
    if (!Pi.empty()) {   // a projector only for risk measures given in conic form
      o.rpoff[k] = (int64_t)o.rpi.size();
      o.rpi.insert(o.rpi.end(), Pi.begin(), Pi.end());
      while (o.rpi.size() % 4) o.rpi.push_back(0.0);
      o.d.max_nz2 = std::max(o.d.max_nz2, nz2);
    }
    // (y, s) block [[I, 0], [-b^T, 1]]: squared norm (2 + B + sqrt(B (B + 4))) / 2, B = ||b||^2
    double B2 = 0.0;
    for (double v : b) B2 += v * v;
    best_ys = std::max(best_ys, (2.0 + B2 + std::sqrt(B2 * (B2 + 4.0))) / 2.0);
  }
  o.normL2_ys = best_ys;
  return SPOCK_OK;
}

}  // namespace spock
